// Kernel argument blocks and launchers shared by the C-ABI layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spiir {

// A decimated band's summed output, added to the top band's sum after linear
// interpolation (multirate banks).  Rows are [D][T][len] complex64.
struct LowerBand {
    const float2 *z;
    int64_t len;               // band samples in this call
    int32_t R;                 // decimation factor (top-rate samples per band sample)
    int32_t shift;             // log2(R) when R is a power of two, else -1
    int32_t buf_off;           // this band's float2 offset in a template's prefetch buffer
    int32_t pad;
};
constexpr int kMaxLowerBands = 7;

// Arithmetic of the filter kernel (spiir_options.precision).
constexpr int kModePlain = 0;
constexpr int kModeCompensated = 1;
constexpr int kModeChunked = 2;
constexpr int kPreciseFcap = 4;   // filters per lane in the compensated / chunked kernels

// Plain FP32 filter kernel (one launch per bank or band).
struct K1Args {
    const float *xe;           // [D][xe_stride] strain: Dh history samples, then the call's
    int64_t xe_stride;         // floats per detector row (multiple of 4)
    int32_t n;                 // samples in this call (band rate)
    int32_t Tb, H, S, R, CS, C, W;
    int32_t fcap;              // filters-per-lane cap of the layout (selects the kernel)
    int32_t G;                 // lanes per template (16: two templates per warp)
    const int32_t *units;      // [n_units][2] (group, detector)
    const int32_t *group_F;    // [G]
    const int64_t *group_pbase;// [G]
    const int4 *warp_info;     // [G*W] (template or -1, first warp of it, its warps, 0)
    const float4 *params;      // [n_slots] (ar, ai, br, bi) kernel form
    const int2 *ringoff;       // [n_slots] (pos0, copy base)
    float2 *state;             // [D][n_slots] filter outputs, kernel form
    int64_t n_slots;
    float *z;                  // [D][T][z_len][2] or null
    int64_t z_len;             // samples per z row (>= n)
    int64_t T;
    float *peak_best;          // [D][T] running max |z|^2, or null (no peak)
    int64_t *peak_idx;         // [D][T]
    int64_t t0;                // absolute index of this call's first sample, added to
    const int64_t *t0_dev;     // ... *t0_dev when non-null (device-side stream counter,
                               //     so a captured graph's replays keep counting)
    int32_t *err;              // device error word
    uint64_t wait_limit_ns;    // bound on every mbarrier wait
    int32_t n_lower;
    int32_t low_len;           // float2 per template slot in the lower-band prefetch buffer           // lower bands added in the combine (0 = single rate)
    LowerBand lower[kMaxLowerBands];
    float2 *ckpt;              // [nc][D][n_slots] state after sample c*ckpt_blocks*Tb - 1
    float2 *sub16;             // [ceil(n/16)][D][n_slots] state before every 16-sample span
                               // (the adjoint's recompute points), or null; plain
                               // precision only (the segment-capable kernels write it)
                               // (c >= 1), kernel form; null = no checkpoints
    int32_t ckpt_blocks;       // blocks between checkpoints
    int32_t n_det;             // detectors (checkpoint row stride)
    int32_t mode;              // kModePlain / kModeCompensated / kModeChunked
    int32_t chunk;             // chunked: samples per chunk (divides Tb, multiple of 8)
    // time segments (plain mode): the grid is n_units x P, CTA b serves unit
    // b % n_units and segment b / n_units of n_seg samples
    int32_t n_units;           // (group, detector) units per segment
    int32_t n_seg;             // samples per segment (multiple of Tb; = n when P == 1)
    int32_t zero_init;         // segments start from zero state (the projection pass)
    const float2 *seg_init;    // [P][D][n_slots] start state of every segment (or null)
    float2 *seg_end;           // [P][D][n_slots] end states of the projection pass (or null)
    int64_t peak_seg_stride;   // per-segment peak entries, overwritten by their one
                               // writer (0: merge into one shared array)
    void *state_ext;           // compensated: float4 [D][n_slots] (re hi, re lo, im hi, im lo);
                               // chunked: double2 [D][n_slots] FP64 anchor
    const double2 *aT;         // chunked: [n_slots] a^chunk in FP64 (kernel form)
    // launches covering part of the segments: segments seg_first ..
    // seg_first + seg_count - 1 (seg_count 0: all of them)
    int32_t seg_first;
    int32_t seg_count;
    // chunked tensor-core form: the state before every kTcT-sample chunk of
    // the launched segment, [chunks][D][n_slots]; lanes restart from it at each
    // chunk start (null: not this form)
    const float2 *anchors;
    // persistent launch of the unsegmented plain kernel: a grid of the
    // resident CTAs takes units from this counter (zeroed by the launcher
    // before the launch); null = one CTA per unit
    int32_t *queue;
};
constexpr int kAnchorFcap = 8;   // filters per lane in the anchored kernel

// Adjoint (reverse-time) kernel of one zero-state filter call.  Its work
// unit is a task: kAdjRounds filter rounds (32 filters each) of one template
// warp of the forward layout; a CTA runs W tasks of one detector.
struct K6Args {
    const float *xe;           // [D][xe_stride]: Dh zeros, then the call's strain
    int64_t xe_stride;
    int32_t n;                 // samples
    int32_t Dh;                // history samples before x in xe (>= max delay)
    int32_t W, Cc;             // tasks (warps) per CTA, checkpoint interval (samples)
    const float2 *gz;          // [D][T][n] dL/dRe z + i dL/dIm z
    int64_t T;
    const int32_t *units;      // [n_units][2] (task group, detector)
    const int4 *tasks;         // [n_groups * W] (first slot of round 0, rounds, template of
                               //  lanes 0..15 (or all), template of lanes 16..31 or -1);
                               //  template -1 = empty task
    int32_t round_stride;      // slots between a warp's consecutive rounds (32 x layout W)
    int32_t G;                 // lanes per template of the forward layout
    const float4 *params;      // kernel form (odd lanes hold conj(a), (Im b, Re b))
    const int2 *ringoff;
    const float2 *ckpt;        // [nc][D][n_slots] from the forward pass
    const float2 *sub16;       // [ceil(n/16)][D][n_slots] state before every kAdjSub span
                               // from the forward pass (then no per-chunk recompute), or null
    int64_t n_slots;
    int32_t n_det;
    float *acc;                // [P][D][n_slots][6] (mu re, im, g_a re, im, g_b re, im)
    float2 *seeds;             // [P-1][D][n_slots] seeds of the input-gradient pass, or null
    float2 *sub;               // [P][n_units][W][kAdjRounds][Cc / kAdjSub][32] workspace
    // time segments of whole chunks: CTA b serves unit b % n_units over the
    // chunks of segment b / n_units, from mu at the segment's end (null: 0)
    int32_t n_units;
    int32_t cps;               // chunks per segment
    int32_t P;                 // segments
    const float2 *mu_end;      // [P][D][n_slots] natural form
};

// Input gradient of the adjoint, g_x[m] = sum_l Re(conj(nu_l[m]) b_l) with
// nu_l[m] = mu_l[m + d_l] = g_z[m + d_l] + conj(a_l) nu_l[m + 1]: every filter
// reads its template's g_z at its own delay and all filters meet at m.
struct K7Args {
    const float2 *gz;          // [D][T][n]
    int64_t T;
    int32_t n, Dh;             // samples; history (>= max delay)
    int32_t S, P;              // segment length (a multiple of 32), segments
    const int4 *tasks;         // the adjoint task list
    const int2 *units;         // [n_units] (first task, tasks): tasks of one template
                               //  (or one half-warp pair), at most kK7MaxWarps
    int32_t n_units, W;        // units; warps per CTA (tasks of the largest unit / tasks
                               //  per warp: 2, or 1 for half-warp templates)
    int32_t round_stride;
    int32_t G;
    const float4 *params;
    const int2 *ringoff;
    int64_t n_slots;
    int32_t n_det;
    const float2 *seeds;       // [P-1][D][n_slots] natural form: mu at the top of the
                               //  16-sample span holding (q + 1) S + d (reverse form), or
                               //  (tangent form, acc != null) mu at (q + 1) S + Dh
    float *gx;                 // [D][n], zeroed by the caller; CTAs add with atomics
    // tangent form: the input-gradient pass also sums g_b = sum_m nu[m] x[m]
    const float *xe;           // [D][xe_stride]: Dh zeros, then x
    int64_t xe_stride;
    float *acc;                // [P][D][n_slots][6]: entries 4, 5 (g_b) written; null =
                               //  reverse form
};
constexpr int kK7Chunk = 256;   // outputs per staged g_z window
constexpr int kK7MaxWarps = 8;
cudaError_t launch_k7(const K7Args &a, cudaStream_t s);

// Gradients of a and b in tangent (forward-mode) form, one filter per lane.
// Lanes follow the tangent order: filters grouped by template, each warp
// spanning at most two templates, lanes of a template ordered so that
// neighbours read strain at different banks.
struct KTArgs {
    const float *xe;           // [D][xe_stride]: Dh zeros, then the call's strain; rows
    int64_t xe_stride;         //  16-byte aligned and >= Dh + ceil(n / Tb) Tb long
    int32_t n, Dh, Tb;         // samples; history (>= max delay, multiple of 4); block
                               //  (multiple of 16)
    int32_t W;                 // warps per CTA
    const float2 *gz;          // [D][T][n]
    int64_t T;
    int32_t nf;                // filters per lane: 1, or 2 (a packed pair of one template)
    const int2 *lanes;         // [n_pos] position (warp nf + f) 32 + lane: filter f of the
                               //  lane, (slot, 0/1: the warp's first or second template);
                               //  slot -1 = empty
    const int2 *warp_tmpl;     // [n_pos / (32 nf)] the warp's two templates (-1: none)
    int64_t n_pos;             // positions, a multiple of 32 nf
    const float4 *params;      // kernel form (odd slots hold conj(a), (Im b, Re b))
    const int2 *ringoff;       // (Dh - d, .) per slot
    int64_t n_slots;
    float *acc;                // [D][n_slots][6]: (0, 0, g_a, g_b) of each slot's filter
    int32_t with_gb;           // 0: g_b left to the input-gradient pass (entries 4, 5
                               //  untouched)
};
int kt_smem_bytes(int Dh, int Tb, int W);
cudaError_t launch_kt(const KTArgs &a, int D, cudaStream_t s);
int k7_smem_bytes(int Dh, int W, int G);
constexpr int kAdjSub = 16;    // samples per recomputed span in the adjoint
constexpr int kAdjRounds = 2;  // filter rounds per adjoint task (independent chains per lane)

cudaError_t launch_k6(const K6Args &a, int64_t n_units, cudaStream_t s);
// Reverse projection for time-segmented adjoints: for segments
// q = 1..P-1, [q seg_len + off, (q + 1) seg_len + off) clipped to the call,
// the adjoint state at the segment's first sample from a zero state at its
// end, E[q][det][slot]; then mu_end[q] (the state at (q + 1) seg_len + off,
// zero at or past the call's end) for every q, carried backwards in FP64.
cudaError_t launch_adj_project(const float4 *params, const int32_t *slot_tmpl, const float2 *gz,
                               int64_t n_slots, int D, int64_t T, int64_t n, int64_t seg_len,
                               int64_t off, int P, float2 *E, float2 *mu_end, cudaStream_t s);
// smem bytes the adjoint kernel needs
int k6_smem_bytes(int Cc, int Dh);
// g_a[f] = sum_det acc[det][s].ga, g_b likewise, for every slot s holding filter f
cudaError_t launch_adj_finalize(const float *acc, const int64_t *slot_filter, int64_t n_slots,
                                int D, int P, float2 *ga, float2 *gb, cudaStream_t s);
// params[s] = kernel form of (a[f], b[f]) for every slot s holding filter f
cudaError_t launch_set_coefficients(const float2 *a, const float2 *b,
                                    const int64_t *slot_filter, int64_t n_slots,
                                    float4 *params, cudaStream_t s);

cudaError_t launch_k1(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
// Registers per thread of the unsegmented single-band plain kernel that a
// layout with this filters-per-lane cap launches (0 if unknown).
int k1_plain_regs(int fcap);

// Raise a kernel's dynamic shared-memory limit once per (kernel, device, size).
cudaError_t ensure_smem_limit(const void *kernel, int smem_bytes);

// Tensor-core projection of segment start states (spiir_tc.cu): chunks of
// kTcT samples, windows of kTcK = 2 kTcT strain samples per GEMM column.
constexpr int kTcT = 256;
constexpr int kTcK = 2 * kTcT;
constexpr int kTcSeeds = kTcK / 32;   // weight seeds per slot (one per 32 window samples)

struct TcArgs {
    const float2 *seed;        // [n_slots][kTcSeeds] weight seeds (launch_tc_seeds)
    const float4 *params;      // [n_slots] kernel-form (ar, ai, br, bi)
    const unsigned char *B;    // strain-window tiles of this call (tc_strain_bytes)
    const int2 *ringoff;       // (Dh - d, copy base) per slot
    const float2 *aT;          // a^kTcT per slot (kernel form)
    const float2 *state;       // [D][n_slots] state before the call
    float2 *seg_init;          // [P][D][n_slots] out: state at each segment start
    int64_t n_slots;
    int32_t D;
    int32_t Dh;
    int64_t n_cols;            // windows (GEMM columns) of this launch
    int32_t n_ntiles;          // set by the launcher: accumulator tiles
    int32_t n_btiles;          // set by the launcher: strain tiles per detector
    int32_t col0;              // window of column 0: c'' = col + col0 = -(Dh / kTcT) - 1
    int32_t c_last;            // last chunk the scan needs ((P - 1) * cps - 1)
    int32_t cps;               // chunks per segment
    int32_t *err;              // bit 8: a wait timed out
    uint64_t wait_limit_ns;
    // anchor mode (anchors != null): FP64 scan over chunks [c_first, c_end)
    float2 *anchors;           // [c_end - c_first][D][n_slots] state before each chunk
    double2 *s64;              // [D][n_slots] FP64 state, in: before c_first, out: after
    const double2 *aT64;       // a^kTcT per slot in FP64
    int32_t c_first;
    int32_t c_end;
    int32_t c_full;            // chunks below c_full are whole; they alone advance s64
};
int64_t tc_strain_bytes(int64_t n_cols, int D);
int tc_cols_per_tile();     // windows per column tile (TcArgs::n_ntiles counts these)
// Weight seeds ([n_slots][kTcSeeds]: V_l at the largest valid m of each
// 32-wide m-group, from which the projection generates its weight tiles)
// and a^kTcT (FP32 and FP64) for every slot of a band.
cudaError_t launch_tc_seeds(const float4 *params, const int2 *ringoff, int64_t n_slots, int Dh,
                            float2 *seed, float2 *aT, double2 *aT64, cudaStream_t s);
// Strain windows of the call staged in xe, split BF16, tile layout.
cudaError_t launch_tc_strain(const float *xe, int64_t xe_stride, int Dh, int64_t n, int D,
                             int64_t n_cols, int col0, unsigned char *B, cudaStream_t s);
// s64 = state (after a call that ended inside a chunk: the FP32 recompute of
// that partial chunk is the end state).
cudaError_t launch_state_to_fp64(const float2 *state, double2 *s64, int64_t count, cudaStream_t s);
// GEMM + chunk scan: seg_init for every segment (segment 0 = state), or in
// anchor mode the FP64-carried state before every chunk of [c_first, c_end).
cudaError_t launch_tc_project(const TcArgs &a, cudaStream_t s);

// Finalize running peaks into the caller's buffers (sqrt of |z|^2).
cudaError_t launch_peak_out(const float *best, const int64_t *idx, int64_t count,
                            float *out_abs, int64_t *out_idx, cudaStream_t s);

// The same, except that every entry reads (NaN, -1) when *err is nonzero (a
// bounded wait of the call gave up).
cudaError_t launch_peak_out_checked(const float *best, const int64_t *idx, int64_t count,
                                   const int32_t *err, float *out_abs, int64_t *out_idx,
                                   cudaStream_t s);

// Segment start states: for every (detector, slot), s_0 = state,
// s_{p+1} = a^n_seg s_p + seg_end[p] (FP64), seg_init[p] = s_p, p < P.
cudaError_t launch_segment_carry(const float4 *params, const float2 *state,
                                 const float2 *seg_end, float2 *seg_init, int64_t n_slots, int D,
                                 int P, int n_seg, cudaStream_t s);
// Running peaks merged over segments in time order (earlier wins ties); with
// t0 non-null the same launch advances the plan's sample counter by advance.
cudaError_t launch_peak_merge(const float *seg_best, const int64_t *seg_idx, int P,
                              int64_t count, float *best, int64_t *idx, int64_t *t0,
                              int64_t advance, cudaStream_t s);

// *t0 += n (device-side sample counter of a plan).
cudaError_t launch_advance(int64_t *t0, int64_t n, cudaStream_t s);

// best[i] = -1, idx[i] = -1.
cudaError_t launch_peak_reset(float *best, int64_t *idx, int64_t count, cudaStream_t s);

// xe[d][Dh + i] = x[d][R * i] for i < nb (decimation into a band's strain rows).
// band front end: x_b[k] = sum_{i<L} taps[i] x[R k - i] from xt = [H history | x]
constexpr int kFirMaxTaps = 512;
cudaError_t launch_fir_decimate(const float *xt, int64_t xt_stride, int H, int D, int R,
                               int64_t nb, const float *taps, int L, float *xe,
                               int64_t xe_stride, int64_t Dh, cudaStream_t s);
cudaError_t launch_decimate(const float *x, int64_t n, int D, int R, int64_t nb, float *xe,
                            int64_t xe_stride, int64_t Dh, cudaStream_t s);

// Self-test: wait on an mbarrier nothing will complete, with a bound; sets *err.
cudaError_t launch_bounded_wait_probe(int32_t *err, uint64_t limit_ns, cudaStream_t s);

// Network peak across detectors (spiir_network.cu): one CTA per template.
constexpr int kNetMaxD = 8;       // detectors
constexpr int kNetMaxWindow = 1024;
struct NetArgs {
    const float2 *z;              // [D][T][n]
    int32_t D;
    int64_t T, n;
    int32_t w[kNetMaxD];          // offsets allowed per detector (w[0] = 0)
    int32_t off_p[kNetMaxD];      // shared-memory word offsets (network_smem_words)
    int32_t off_g[kNetMaxD];
    float *rho;                   // [T]
    int64_t *t;                   // [T]
    int32_t *shift;               // [T][D] or null
    int32_t n_chunks;             // CTAs per template (time chunks; set by the launcher)
    int32_t chunk_tiles;          // tiles of 2048 outputs per chunk
};
// shared-memory words of a tile; fills the per-detector offsets
int network_smem_words(const int32_t *w, int D, int32_t *off_p, int32_t *off_g);
cudaError_t launch_network_peak(const NetArgs &a, cudaStream_t s);

// Chi^2 at each template's peak from its p group series (spiir_veto.cu)
cudaError_t launch_chi2_peak(const float2 *zg, int D, int64_t T, int p, int64_t n, float *peak,
                             int64_t *t, float *chi2, cudaStream_t s);

}  // namespace spiir
