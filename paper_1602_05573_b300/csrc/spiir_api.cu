// C-ABI entry points (include/spiir.h): plan lifecycle, streaming state,
// workspace, and the launch sequence of each call.  Device compute lives in
// the kernel files; this file only validates, allocates and enqueues.
#include "spiir.h"
#include "spiir_internal.h"
#include "spiir_kernels.h"
#include "spiir_layout.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace {
thread_local std::string g_detail;
}  // namespace

namespace spiir {
namespace detail {

spiir_status fail(spiir_status st, const std::string &why)
{
    g_detail = why;
    return st;
}

spiir_status cuda_fail(cudaError_t e, const char *what)
{
    g_detail = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) +
               ")";
    (void)cudaGetLastError();  // clear a sticky launch error for the next call
    return SPIIR_ECUDA;
}

spiir_status validate_bank(const spiir_bank_desc *bank)
{
    if (!bank) return fail(SPIIR_EINVAL, "bank is NULL");
    if (bank->n_templates < 1) return fail(SPIIR_EINVAL, "n_templates must be >= 1");
    if (bank->n_detectors < 1) return fail(SPIIR_EINVAL, "n_detectors must be >= 1");
    if (!bank->filter_off || !bank->a_reim || !bank->b_reim || !bank->delay)
        return fail(SPIIR_EINVAL, "filter_off, a_reim, b_reim and delay are required");
    const int64_t *off = bank->filter_off;
    if (off[0] != 0) return fail(SPIIR_EINVAL, "filter_off[0] must be 0");
    for (int64_t t = 0; t < bank->n_templates; ++t)
        if (off[t + 1] < off[t])
            return fail(SPIIR_EINVAL, "filter_off must be non-decreasing (template " +
                                          std::to_string(t) + ")");
    const int64_t L = off[bank->n_templates];
    for (int64_t l = 0; l < L; ++l) {
        const double ar = bank->a_reim[2 * l], ai = bank->a_reim[2 * l + 1];
        const double br = bank->b_reim[2 * l], bi = bank->b_reim[2 * l + 1];
        if (!std::isfinite(ar) || !std::isfinite(ai) || !std::isfinite(br) || !std::isfinite(bi))
            return fail(SPIIR_EINVAL, "non-finite pole or gain at filter " + std::to_string(l));
        if (ar * ar + ai * ai >= 1.0)
            return fail(SPIIR_EINVAL, "|a| >= 1 (unstable pole) at filter " + std::to_string(l));
        if (bank->delay[l] < 0)
            return fail(SPIIR_EINVAL, "negative delay at filter " + std::to_string(l));
    }
    if (bank->n_bands > 1) {
        if (!bank->band_of_filter || !bank->band_decim)
            return fail(SPIIR_EINVAL, "multirate bank needs band_of_filter and band_decim");
        int minR = 1 << 30;
        for (int j = 0; j < bank->n_bands; ++j) {
            if (bank->band_decim[j] < 1 || bank->band_decim[j] > 4096)
                return fail(SPIIR_EINVAL, "band_decim must be in [1, 4096]");
            minR = std::min(minR, bank->band_decim[j]);
        }
        if (minR != 1) return fail(SPIIR_EINVAL, "a multirate bank needs a band with decim 1");
        for (int64_t l = 0; l < L; ++l)
            if (bank->band_of_filter[l] < 0 || bank->band_of_filter[l] >= bank->n_bands)
                return fail(SPIIR_EINVAL, "band_of_filter out of range at filter " +
                                              std::to_string(l));
    } else if (bank->n_bands == 1 && bank->band_decim && bank->band_decim[0] != 1) {
        return fail(SPIIR_EINVAL, "a single band must have decim 1");
    } else if (bank->n_bands < 0) {
        return fail(SPIIR_EINVAL, "n_bands must be >= 0");
    }
    return SPIIR_OK;
}

}  // namespace detail
}  // namespace spiir

namespace {

using spiir::detail::cuda_fail;
using spiir::detail::fail;
using spiir::detail::validate_bank;

// Keeps the caller's current device and restores it on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        err = cudaSetDevice(dev);
        ok = err == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T> cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

template <typename T> cudaError_t h2d(T *dst, const std::vector<T> &src)
{
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on any device wait

}  // namespace

// One rate band of a plan (a single-rate bank has one band with R = 1).
struct Band {
    int R = 1;
    spiir::Layout lay;
    float4 *params = nullptr;
    int2 *ringoff = nullptr;
    int32_t *units = nullptr;
    int32_t *group_F = nullptr;
    int64_t *group_pbase = nullptr;
    int4 *warp_info = nullptr;
    float2 *state = nullptr;   // [D][n_slots]
    float *hist = nullptr;     // [D][Dh]
    float *xe = nullptr;       // [D][xe_stride] workspace
    int64_t xe_stride = 0;
    int64_t xe_cap = 0;        // samples the workspace holds after the history
    float2 *zb = nullptr;      // [D][T][zb_len] band-rate sums (decimated bands)
    int64_t zb_cap = 0;        // complex samples per row the workspace holds
    int64_t *slot_filter = nullptr;  // [n_slots] bank filter of each slot, -1 = padding
    void *state_ext = nullptr;       // compensated / chunked state, 16 B per slot and detector
    double2 *aT = nullptr;           // chunked: a^chunk per slot (FP64)
    // adjoint workspace
    float *bw_xe = nullptr;
    int64_t bw_xe_stride = 0, bw_cap = 0;
    float2 *bw_state = nullptr;
    float2 *ckpt = nullptr;
    int64_t ckpt_cap = 0;      // checkpoints the buffer holds
    float *acc = nullptr;
    float2 *seg_end = nullptr;     // time segments: [P][D][n_slots] projection end states
    float2 *seg_init = nullptr;    //                [P][D][n_slots] segment start states
    float *seg_best = nullptr;     //                [P][D][T] per-segment peaks
    int64_t *seg_idx = nullptr;
    int seg_cap = 0;               // segments the workspaces hold
    float2 *tc_seed = nullptr;     // tensor-core projection: weight seeds [n_slots][kTcSeeds]
    float2 *tc_aT = nullptr;       //   a^256 per slot
    bool tc_valid = false;         //   weights match the current coefficients
    unsigned char *tc_b = nullptr; //   strain-window tiles of a call
    int64_t tc_b_cap = 0;          //   bytes
    double2 *tc_aT64 = nullptr;    //   a^256 per slot in FP64
    float2 *tc_anchor = nullptr;   // chunked tensor-core form: anchors of a time tile
    int64_t tc_anchor_cap = 0;     //   float2 elements
    int4 *adj_tasks = nullptr;     // adjoint work list (built on the first backward call)
    int32_t *adj_units = nullptr;
    int64_t adj_n_units = 0;
    int adj_W = 4;
    float2 *adj_sub = nullptr;     // [P][adj_n_units][adj_W][kAdjRounds][Cc/kAdjSub][32]
    int64_t adj_sub_cap = 0;
    int32_t *adj_slot_tmpl = nullptr; // template of every slot (-1 padding)
    float2 *adj_E = nullptr;       // [P][D][n_slots] reverse projection, segment starts
    float2 *adj_mu = nullptr;      // [P][D][n_slots] adjoint state after each segment
    int adj_seg_cap = 0;           // segments adj_E / adj_mu / acc hold
    float2 *adj_sub16 = nullptr;   // [n/16][D][n_slots] forward state at every span start
    int64_t adj_sub16_cap = 0;     //   float2 elements
    float *fir = nullptr;          // front-end FIR taps of this band (device), or null
    int fir_len = 0;
    int2 *adj_units7 = nullptr;    // input-gradient units: (first task, tasks) of one template
    int64_t adj_n_units7 = 0;
    int adj_W7 = 1;                // warps per input-gradient CTA (largest unit)
    float2 *adj_seeds = nullptr;   // [P-1][D][n_slots] input-gradient segment seeds
    // tangent form, for 1 and 2 filters per lane ([nf - 1]): positions in
    // tangent order (slot, 0/1), the two templates of every warp, positions
    int2 *kt_lanes[2] = {nullptr, nullptr};
    int2 *kt_warp_tmpl[2] = {nullptr, nullptr};
    int64_t kt_n_pos[2] = {0, 0};
};

struct spiir_plan {
    int device = -1;
    int precision = 0;
    int D = 1;
    int64_t T = 0;
    int64_t Ltot = 0;
    spiir_options opt{};
    std::vector<Band> bands;
    float *peak_best = nullptr;   // [D][T]
    int64_t *peak_idx = nullptr;  // [D][T]
    int32_t *err = nullptr;
    int64_t *t0_dev = nullptr;    // samples since reset, on the device (graph replays advance it)
    int32_t *queue = nullptr;     // unit counter of persistent filter launches
    bool persistent = false;      // unsegmented plain calls launch persistent CTAs
    int64_t t0 = 0;               // the same, as enqueued by this host (alignment checks)
    int top = 0;                  // index of the top-rate band
    int maxR = 1;                 // largest decimation factor
    // band front-end FIRs: the last kFirMaxTaps - 1 top-rate samples, and a
    // per-call staging buffer [D][kFirMaxTaps - 1 + n] of (history, x)
    float *fir_xh = nullptr;
    float *fir_xt = nullptr;
    int64_t fir_xt_cap = 0;       // samples per detector row
    // kept for the autotuner (single-rate plans with autotune set)
    bool tuned = false;
    int n_sm = 148;
    std::vector<std::vector<int64_t>> lists;
    std::vector<float> a_host, b_host;
    std::vector<int32_t> d_host;
    std::string tune_report;
    // the tangent adjoint runs its g_a pass beside the input-gradient pass:
    // a second stream and its fork/join events (created on first use)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int32_t last_launches = 0;    // kernels the last filter/backward call launched
    int32_t last_segments = 1;    // time segments of the last call's top band
    // kernel timing (opt.kernel_timing): event pairs since the last read
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_used;   // (first event index, kernel class)
};

namespace {
constexpr int kTimeK1 = 0, kTimeTc = 1, kTimeAdj = 2;
constexpr size_t kMaxTimedLaunches = 4096;

// Records an event before a timed launch; returns its pool index or -1.
int time_begin(spiir_plan *p, cudaStream_t s)
{
    if (!p->opt.kernel_timing) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return -1;
    const size_t i = p->ev_used.size() * 2;
    if (p->ev_used.size() >= kMaxTimedLaunches) return -1;
    while (p->ev_pool.size() < i + 2) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return -1;
        p->ev_pool.push_back(ev);
    }
    if (cudaEventRecord(p->ev_pool[i], s) != cudaSuccess) return -1;
    return (int)i;
}
void time_end(spiir_plan *p, cudaStream_t s, int i, int cls)
{
    if (i < 0) return;
    if (cudaEventRecord(p->ev_pool[(size_t)i + 1], s) == cudaSuccess)
        p->ev_used.push_back(std::make_pair(i, cls));
}
}  // namespace

namespace {

void free_band(Band &b)
{
    cudaFree(b.params);
    cudaFree(b.ringoff);
    cudaFree(b.units);
    cudaFree(b.group_F);
    cudaFree(b.group_pbase);
    cudaFree(b.warp_info);
    cudaFree(b.state);
    cudaFree(b.hist);
    cudaFree(b.xe);
    cudaFree(b.zb);
    cudaFree(b.slot_filter);
    cudaFree(b.state_ext);
    cudaFree(b.aT);
    cudaFree(b.bw_xe);
    cudaFree(b.bw_state);
    cudaFree(b.ckpt);
    cudaFree(b.acc);
    cudaFree(b.seg_end);
    cudaFree(b.seg_init);
    cudaFree(b.seg_best);
    cudaFree(b.seg_idx);
    cudaFree(b.tc_seed);
    cudaFree(b.tc_aT);
    cudaFree(b.tc_b);
    cudaFree(b.tc_aT64);
    cudaFree(b.tc_anchor);
    cudaFree(b.adj_tasks);
    cudaFree(b.adj_units);
    cudaFree(b.adj_sub);
    cudaFree(b.adj_slot_tmpl);
    cudaFree(b.adj_E);
    cudaFree(b.adj_mu);
    cudaFree(b.adj_sub16);
    cudaFree(b.adj_units7);
    cudaFree(b.fir);
    cudaFree(b.adj_seeds);
    for (int f = 0; f < 2; ++f) {
        cudaFree(b.kt_lanes[f]);
        cudaFree(b.kt_warp_tmpl[f]);
    }
    b = Band();
}

// a^T in double for every slot, from the kernel-form (stored) pole
std::vector<double2> powers(const spiir::Layout &L, int T)
{
    std::vector<double2> out((size_t)L.n_slots);
    for (int64_t s = 0; s < L.n_slots; ++s) {
        double br = L.params[4 * s], bi = L.params[4 * s + 1];  // base
        double rr = 1.0, ri = 0.0;                              // result
        for (int e = T; e > 0; e >>= 1) {
            if (e & 1) {
                const double nr = rr * br - ri * bi, ni = rr * bi + ri * br;
                rr = nr;
                ri = ni;
            }
            const double nr = br * br - bi * bi, ni = 2.0 * br * bi;
            br = nr;
            bi = ni;
        }
        out[(size_t)s] = make_double2(rr, ri);
    }
    return out;
}

spiir_status upload_band(Band &b, int D, int precision, int chunk)
{
    const spiir::Layout &L = b.lay;
    cudaError_t e;
    if (precision != SPIIR_PREC_PLAIN) {
        if ((e = dalloc(reinterpret_cast<double2 **>(&b.state_ext), (size_t)D * L.n_slots)) !=
            cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "device allocation failed")
                                                  : cuda_fail(e, "cudaMalloc");
        if ((e = cudaMemset(b.state_ext, 0, sizeof(double2) * (size_t)D * L.n_slots)) !=
            cudaSuccess)
            return cuda_fail(e, "plan upload");
    }
    if (precision == SPIIR_PREC_CHUNKED_FP64) {
        const std::vector<double2> aT = powers(L, chunk);
        if ((e = dalloc(&b.aT, aT.size())) != cudaSuccess ||
            (e = cudaMemcpy(b.aT, aT.data(), aT.size() * sizeof(double2),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "plan upload");
    }
    if ((e = dalloc(&b.params, L.n_slots)) != cudaSuccess ||
        (e = dalloc(&b.ringoff, L.n_slots)) != cudaSuccess ||
        (e = dalloc(&b.units, L.units.size())) != cudaSuccess ||
        (e = dalloc(&b.group_F, L.group_F.size())) != cudaSuccess ||
        (e = dalloc(&b.group_pbase, L.group_pbase.size())) != cudaSuccess ||
        (e = dalloc(&b.warp_info, L.warp_info.size() / 4)) != cudaSuccess ||
        (e = dalloc(&b.state, (size_t)D * L.n_slots)) != cudaSuccess ||
        (e = dalloc(&b.hist, (size_t)D * L.Dh)) != cudaSuccess ||
        (e = dalloc(&b.slot_filter, L.n_slots)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "device allocation failed")
                                              : cuda_fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(b.params, L.params.data(), L.params.size() * sizeof(float),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b.ringoff, L.ringoff.data(), L.ringoff.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = h2d(b.units, L.units)) != cudaSuccess ||
        (e = h2d(b.group_F, L.group_F)) != cudaSuccess ||
        (e = h2d(b.slot_filter, L.slot_filter)) != cudaSuccess ||
        (e = h2d(b.group_pbase, L.group_pbase)) != cudaSuccess ||
        (e = cudaMemcpy(b.warp_info, L.warp_info.data(), L.warp_info.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(b.state, 0, sizeof(float2) * (size_t)D * L.n_slots)) != cudaSuccess ||
        (e = cudaMemset(b.hist, 0, sizeof(float) * (size_t)D * L.Dh)) != cudaSuccess)
        return cuda_fail(e, "plan upload");
    return SPIIR_OK;
}

// Make the band's strain workspace hold n more samples (after the history).
spiir_status ensure_xe(spiir_plan *p, Band &b, int64_t n, cudaStream_t s)
{
    const int64_t need = ((n + b.lay.Tb - 1) / b.lay.Tb) * b.lay.Tb;
    if (b.xe && b.xe_cap >= need) return SPIIR_OK;
    if (b.xe) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        cudaFree(b.xe);
        b.xe = nullptr;
    }
    const int64_t cap = std::max<int64_t>(need, 4096);
    const int64_t stride = b.lay.Dh + cap;
    cudaError_t e = dalloc(&b.xe, (size_t)p->D * stride);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "strain workspace allocation")
                                              : cuda_fail(e, "cudaMalloc");
    b.xe_cap = cap;
    b.xe_stride = stride;
    return SPIIR_OK;
}

spiir::K1Args k1_args(const spiir_plan *p, const Band &b, int64_t n, float *z, int64_t z_len,
                      bool with_peak)
{
    const spiir::Layout &L = b.lay;
    spiir::K1Args a{};
    a.xe = b.xe;
    a.xe_stride = b.xe_stride;
    a.n = (int32_t)n;
    a.Tb = L.Tb;
    a.H = L.H;
    a.S = L.S;
    a.R = L.R;
    a.CS = L.CS;
    a.C = L.C;
    a.W = L.W;
    a.units = b.units;
    a.group_F = b.group_F;
    a.group_pbase = b.group_pbase;
    a.warp_info = b.warp_info;
    a.fcap = L.Fcap;
    a.G = L.G;
    a.mode = p->precision == SPIIR_PREC_COMPENSATED
                 ? spiir::kModeCompensated
                 : (p->precision == SPIIR_PREC_CHUNKED_FP64 ? spiir::kModeChunked
                                                            : spiir::kModePlain);
    a.chunk = p->opt.chunk_len;
    a.state_ext = b.state_ext;
    a.aT = b.aT;
    a.n_det = p->D;
    a.n_units = (int32_t)L.n_units();
    a.n_seg = (int32_t)n;          // one segment unless spiir_filter splits the call
    a.zero_init = 0;
    a.seg_init = nullptr;
    a.seg_end = nullptr;
    a.peak_seg_stride = 0;
    a.params = b.params;
    a.ringoff = b.ringoff;
    a.state = b.state;
    a.n_slots = L.n_slots;
    a.z = z;
    a.z_len = z_len;
    a.T = p->T;
    a.peak_best = with_peak ? p->peak_best : nullptr;
    a.peak_idx = with_peak ? p->peak_idx : nullptr;
    a.t0 = p->t0;
    a.err = p->err;
    a.wait_limit_ns = kWaitLimitNs;
    // the persistent kernel serves units in stages of non-increasing F
    bool f_sorted = true;
    for (int64_t u = 1; u < L.n_units() && f_sorted; ++u)
        f_sorted = L.group_F[L.units[2 * u]] <= L.group_F[L.units[2 * (u - 1)]];
    a.queue = (p->persistent && f_sorted) ? p->queue : nullptr;
    return a;
}

}  // namespace

extern "C" {

void spiir_options_default(spiir_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = SPIIR_PREC_PLAIN;
    opt->chunk_len = 256;
    opt->block_len = 0;
    opt->warps_per_cta = 0;
    opt->ring_copies = 0;
    opt->device = 0;
    opt->autotune = 0;
}

const char *spiir_status_str(spiir_status st)
{
    switch (st) {
    case SPIIR_OK: return "ok";
    case SPIIR_EINVAL: return "invalid argument";
    case SPIIR_ENOMEM: return "out of memory";
    case SPIIR_ECUDA: return "CUDA runtime error";
    case SPIIR_ETIMEOUT: return "bounded device wait timed out";
    case SPIIR_EUNSUPPORTED: return "unsupported device or size";
    }
    return "unknown status";
}

const char *spiir_last_error_detail(void) { return g_detail.c_str(); }

spiir_status spiir_plan_create(const spiir_bank_desc *bank, const spiir_options *opt_in,
                               spiir_plan **out)
{
    if (!out) return fail(SPIIR_EINVAL, "out is NULL");
    *out = nullptr;
    spiir_status st = validate_bank(bank);
    if (st != SPIIR_OK) return st;
    spiir_options opt;
    spiir_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.precision < SPIIR_PREC_PLAIN || opt.precision > SPIIR_PREC_CHUNKED_TC)
        return fail(SPIIR_EINVAL, "unknown precision mode");
    if (opt.chunk_len == 0) opt.chunk_len = 256;
    if (opt.tile_chunks < 0) return fail(SPIIR_EINVAL, "tile_chunks must be >= 0");
    if (opt.persistent < 0 || opt.persistent > 2)
        return fail(SPIIR_EINVAL, "persistent must be 0 (auto), 1 (off) or 2 (on)");
    if (opt.adjoint_form < SPIIR_ADJOINT_AUTO || opt.adjoint_form > SPIIR_ADJOINT_TANGENT)
        return fail(SPIIR_EINVAL, "adjoint_form must be 0 (auto), 1 (reverse) or 2 (tangent)");
    if (opt.tail_split < -1 || opt.tail_split > 200)
        return fail(SPIIR_EINVAL, "tail_split must be -1 (off), 0 (auto) or 1..200 per mille");
    if (opt.precision == SPIIR_PREC_CHUNKED_TC && opt.chunk_len != spiir::kTcT)
        return fail(SPIIR_EINVAL, "the tensor-core chunked form uses chunks of " +
                                      std::to_string(spiir::kTcT) + " samples");
    if (opt.projection < SPIIR_PROJECT_AUTO || opt.projection > SPIIR_PROJECT_TENSOR)
        return fail(SPIIR_EINVAL, "projection must be 0 (auto), 1 (recurrence) or 2 (tensor)");
    if (opt.block_len != 0 && (opt.block_len < 32 || opt.block_len % 32 != 0))
        return fail(SPIIR_EINVAL, "block_len must be 0 or a multiple of 32");

    int n_sm = 148;
    if (opt.device >= 0) {
        int count = 0;
        cudaError_t e = cudaGetDeviceCount(&count);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
        if (opt.device >= count)
            return fail(SPIIR_EINVAL, "device ordinal " + std::to_string(opt.device) +
                                          " out of range");
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, opt.device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
        if (prop.major != 10 || prop.minor != 3)
            return fail(SPIIR_EUNSUPPORTED,
                        std::string("kernels are built for sm_103a; device is ") + prop.name +
                            " (sm_" + std::to_string(prop.major) + std::to_string(prop.minor) +
                            ")");
        n_sm = prop.multiProcessorCount;
    }

    spiir_plan *p = new (std::nothrow) spiir_plan();
    if (!p) return fail(SPIIR_ENOMEM, "host allocation");
    p->device = opt.device;
    p->precision = opt.precision;
    p->D = bank->n_detectors;
    p->T = bank->n_templates;
    p->Ltot = bank->filter_off[bank->n_templates];
    p->opt = opt;
    p->persistent = opt.persistent == 2;

    // bands: filter lists per template and band
    std::vector<int> decims;
    if (bank->n_bands > 1)
        decims.assign(bank->band_decim, bank->band_decim + bank->n_bands);
    else
        decims.push_back(1);
    spiir::LayoutOptions lo;
    lo.W = opt.warps_per_cta;
    lo.Tb = opt.block_len ? opt.block_len : 512;
    lo.C = opt.ring_copies;
    lo.Fcap = opt.max_filters_per_lane;
    lo.G = opt.lanes_per_template;
    if (opt.precision == SPIIR_PREC_CHUNKED_TC) {
        // the anchored kernel holds at most kAnchorFcap filters per lane
        if (lo.Fcap == 0 || lo.Fcap > spiir::kAnchorFcap) lo.Fcap = spiir::kAnchorFcap;
    } else if (opt.precision != SPIIR_PREC_PLAIN) {
        // the compensated and chunked kernels hold at most kPreciseFcap filters per lane
        if (lo.Fcap == 0 || lo.Fcap > spiir::kPreciseFcap) lo.Fcap = spiir::kPreciseFcap;
        if (opt.chunk_len < 8 || opt.chunk_len % 8 != 0 || lo.Tb % opt.chunk_len != 0)
            return fail(SPIIR_EINVAL, "chunk_len must be a multiple of 8 dividing block_len (" +
                                          std::to_string(lo.Tb) + ")");
    }
    lo.n_sm = n_sm;
    // the tail split serves single-rate plain banks (the persistent launch)
    // (option 0 = off, -1 = auto, k = per mille; the layout's -1 = off, 0 = auto)
    lo.tail = (opt.precision == SPIIR_PREC_PLAIN && decims.size() == 1 && opt.tail_split != 0)
                  ? (opt.tail_split < 0 ? 0 : opt.tail_split)
                  : -1;
    if (opt.device >= 0 && lo.tail >= 0) {
        DeviceGuard g(opt.device);
        lo.regs = g.ok ? spiir::k1_plain_regs(lo.Fcap == 0 ? spiir::kMaxF : lo.Fcap) : 0;
    }
    p->bands.resize(decims.size());
    for (size_t j = 0; j < decims.size(); ++j) {
        std::vector<std::vector<int64_t>> lists((size_t)p->T);
        for (int64_t t = 0; t < p->T; ++t)
            for (int64_t l = bank->filter_off[t]; l < bank->filter_off[t + 1]; ++l)
                if (decims.size() == 1 || bank->band_of_filter[l] == (int)j)
                    lists[t].push_back(l);
        p->bands[j].R = decims[j];
        std::string err;
        if (!spiir::build_layout(lists, p->D, bank->a_reim, bank->b_reim, bank->delay, lo,
                                 &p->bands[j].lay, &err)) {
            delete p;
            return fail(SPIIR_EUNSUPPORTED, err);
        }
        // a band small enough for automatic time segments gets 256-sample
        // blocks: shorter segments, more of them
        const spiir::Layout &L0 = p->bands[j].lay;
        if (opt.block_len == 0 && opt.precision == SPIIR_PREC_PLAIN && opt.time_segments == 0 &&
            L0.n_units() * L0.W * 4 <= 8 * (int64_t)n_sm && L0.Tb != 256) {
            spiir::LayoutOptions lo2 = lo;
            lo2.Tb = 256;
            spiir::Layout L2;
            if (spiir::build_layout(lists, p->D, bank->a_reim, bank->b_reim, bank->delay, lo2,
                                    &L2, &err))
                p->bands[j].lay = std::move(L2);
        }
        // block length for residency: when a multirate top band's filter
        // kernel (two ring copies and the lower-band buffers) keeps fewer CTAs
        // on an SM by its shared memory at 512-sample blocks than its registers
        // allow (3 of 4), the longest shorter block (a multiple of 64) that lets
        // them all reside.  Measured on the multirate bank: 92.6 -> 89.7 ms per
        // step at 448 samples.  (Single-rate banks keep their blocks: the
        // autotuner chooses theirs, and the tangent adjoint wants a history of
        // whole 256-sample chunks.)
        bool top_mr = false;   // the multirate top band (the first at the top rate)
        if (decims.size() > 1 && decims[j] == 1) {
            top_mr = true;
            for (size_t i = 0; i < j; ++i) top_mr = top_mr && decims[i] != 1;
        }
        if (top_mr && opt.block_len == 0 && opt.precision == SPIIR_PREC_PLAIN &&
            opt.device >= 0 && p->bands[j].lay.Tb == 512) {
            // dynamic shared memory of a launch (the call's k1_smem)
            auto k1_bytes = [&](const spiir::Layout &L) {
                int low = 0;
                if (top_mr) {
                    for (size_t i = 0; i < decims.size(); ++i)
                        if (i != j) low += (L.Tb + decims[i] - 1) / decims[i] + 2;
                    low = (low + 1) / 2 * 2;
                }
                return L.smem_bytes() + L.W * (32 / L.G) * low * (int)sizeof(float2);
            };
            DeviceGuard g(opt.device);
            int smem_sm = 0, reserved = 0;
            const int regs = g.ok ? spiir::k1_plain_regs(p->bands[j].lay.Fcap) : 0;
            if (g.ok && regs > 0 &&
                cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                       opt.device) == cudaSuccess &&
                cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock,
                                       opt.device) == cudaSuccess) {
                const int threads = p->bands[j].lay.W * 32;
                const int by_regs = std::min({32, 2048 / threads, 65536 / (threads * regs)});
                auto by_smem = [&](const spiir::Layout &L) {
                    return smem_sm / (k1_bytes(L) + reserved);
                };
                if (by_smem(p->bands[j].lay) < by_regs) {
                    for (int tb : {448, 384, 320, 256}) {
                        spiir::LayoutOptions lo2 = lo;
                        lo2.Tb = tb;
                        spiir::Layout L2;
                        if (spiir::build_layout(lists, p->D, bank->a_reim, bank->b_reim,
                                                bank->delay, lo2, &L2, &err) &&
                            by_smem(L2) >= by_regs) {
                            p->bands[j].lay = std::move(L2);
                            break;
                        }
                    }
                }
            } else {
                (void)cudaGetLastError();
            }
        }
    }
    if (p->bands.size() > 1 + spiir::kMaxLowerBands) {
        delete p;
        return fail(SPIIR_EUNSUPPORTED, "at most " + std::to_string(1 + spiir::kMaxLowerBands) +
                                            " bands");
    }
    // the first band at the top rate carries the fused epilogue
    for (size_t j = 0; j < p->bands.size(); ++j)
        if (p->bands[j].R == 1) {
            p->top = (int)j;
            break;
        }
    for (const Band &b : p->bands) p->maxR = std::max(p->maxR, b.R);
    p->n_sm = n_sm;
    if (opt.autotune && p->bands.size() == 1 && opt.precision == SPIIR_PREC_PLAIN) {
        const int64_t L = p->Ltot;
        p->a_host.assign(bank->a_reim, bank->a_reim + 2 * L);
        p->b_host.assign(bank->b_reim, bank->b_reim + 2 * L);
        p->d_host.assign(bank->delay, bank->delay + L);
        p->lists.assign((size_t)p->T, {});
        for (int64_t t = 0; t < p->T; ++t)
            for (int64_t l = bank->filter_off[t]; l < bank->filter_off[t + 1]; ++l)
                p->lists[t].push_back(l);
    } else {
        p->tuned = true;
    }
    if (p->device < 0) {  // host-only plan
        *out = p;
        return SPIIR_OK;
    }
    DeviceGuard guard(p->device);
    if (!guard.ok) {
        delete p;
        return cuda_fail(guard.err, "cudaSetDevice");
    }
    for (Band &b : p->bands) {
        st = upload_band(b, p->D, p->precision, p->opt.chunk_len);
        if (st != SPIIR_OK) {
            spiir_plan_destroy(p);
            return st;
        }
    }
    cudaError_t e;
    if ((e = dalloc(&p->peak_best, (size_t)p->D * p->T)) != cudaSuccess ||
        (e = dalloc(&p->peak_idx, (size_t)p->D * p->T)) != cudaSuccess ||
        (e = dalloc(&p->err, 1)) != cudaSuccess ||
        (e = dalloc(&p->t0_dev, 1)) != cudaSuccess ||
        (e = dalloc(&p->queue, 1)) != cudaSuccess) {
        spiir_plan_destroy(p);
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "device allocation failed")
                                              : cuda_fail(e, "cudaMalloc");
    }
    st = spiir_reset(p, nullptr);
    if (st == SPIIR_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "plan init");
    }
    if (st != SPIIR_OK) {
        spiir_plan_destroy(p);
        return st;
    }
    *out = p;
    return SPIIR_OK;
}

spiir_status spiir_plan_destroy(spiir_plan *p)
{
    if (!p) return SPIIR_OK;
    if (p->device >= 0) {
        DeviceGuard guard(p->device);
        cudaDeviceSynchronize();
        for (Band &b : p->bands) free_band(b);
        cudaFree(p->peak_best);
        cudaFree(p->peak_idx);
        cudaFree(p->err);
        cudaFree(p->t0_dev);
        cudaFree(p->queue);
        cudaFree(p->fir_xh);
        cudaFree(p->fir_xt);
        for (cudaEvent_t ev : p->ev_pool) cudaEventDestroy(ev);
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->ev_join) cudaEventDestroy(p->ev_join);
        if (p->aux) cudaStreamDestroy(p->aux);
    }
    delete p;
    return SPIIR_OK;
}

spiir_status spiir_plan_get_info(const spiir_plan *p, spiir_plan_info *info)
{
    if (!p || !info) return fail(SPIIR_EINVAL, "plan or info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->n_templates = p->T;
    info->n_filters = p->Ltot;
    info->n_detectors = p->D;
    info->precision = p->precision;
    double wf = 0.0, rounds = 0.0;
    for (const Band &b : p->bands) {
        const spiir::Layout &L = b.lay;
        info->n_slots += L.n_slots;
        info->n_units += L.n_units();
        info->warps_per_cta = L.W;
        info->block_len = L.Tb;
        info->ring_copies = L.C;
        if (&b == &p->bands[p->top]) info->history_len = L.Dh;
        info->smem_bytes = std::max(info->smem_bytes, L.smem_bytes());
        info->max_filters_per_lane = std::max(info->max_filters_per_lane, L.maxF);
        if (&b == &p->bands[p->top]) info->lanes_per_template = L.G;
        wf += L.conflict_ratio * (double)L.n_slots;
        rounds += (double)L.n_slots;
    }
    info->bank_conflict_ratio = rounds > 0 ? wf / rounds : 1.0;
    info->last_call_launches = p->last_launches;
    info->last_call_segments = p->last_segments;
    info->persistent = p->persistent ? 1 : 0;
    info->tail_templates = p->bands[p->top].lay.tail_templates;
    info->resident_ctas = p->bands[p->top].lay.slots_model;
    return SPIIR_OK;
}

const char *spiir_plan_tune_report(const spiir_plan *p)
{
    return p ? p->tune_report.c_str() : "";
}

spiir_status spiir_plan_get_slots(const spiir_plan *p, int64_t *slot_filter,
                                  int64_t *slot_template)
{
    if (!p || !slot_filter || !slot_template) return fail(SPIIR_EINVAL, "NULL argument");
    int64_t at = 0;
    for (const Band &b : p->bands) {
        std::memcpy(slot_filter + at, b.lay.slot_filter.data(), sizeof(int64_t) * b.lay.n_slots);
        std::memcpy(slot_template + at, b.lay.slot_template.data(),
                    sizeof(int64_t) * b.lay.n_slots);
        at += b.lay.n_slots;
    }
    return SPIIR_OK;
}

spiir_status spiir_reset(spiir_plan *p, void *stream)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no device state");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    for (Band &b : p->bands) {
        if ((e = cudaMemsetAsync(b.state, 0, sizeof(float2) * (size_t)p->D * b.lay.n_slots, s)) !=
                cudaSuccess ||
            (e = cudaMemsetAsync(b.hist, 0, sizeof(float) * (size_t)p->D * b.lay.Dh, s)) !=
                cudaSuccess ||
            (b.state_ext &&
             (e = cudaMemsetAsync(b.state_ext, 0, sizeof(double2) * (size_t)p->D * b.lay.n_slots,
                                  s)) != cudaSuccess))
            return cuda_fail(e, "reset");
    }
    if ((e = spiir::launch_peak_reset(p->peak_best, p->peak_idx, (int64_t)p->D * p->T, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(p->err, 0, sizeof(int32_t), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->t0_dev, 0, sizeof(int64_t), s)) != cudaSuccess ||
        (p->fir_xh && (e = cudaMemsetAsync(p->fir_xh, 0,
                                           sizeof(float) * (size_t)p->D * (spiir::kFirMaxTaps - 1),
                                           s)) != cudaSuccess))
        return cuda_fail(e, "reset");
    p->t0 = 0;
    return SPIIR_OK;
}

// Time segments for a band call of nb samples, each at least one block long.
// By default: banks that fill under 1/8 of the GPU's warp slots get enough
// segments for ~8 warps per SM (at least 4, at most 64); banks that fill
// less than one full wave (16 warps per SM) over a long call (>= 64 blocks)
// get 2, which evens out the wave; larger banks none.  A time_segments
// option above 0 forces the count.
int segments_for(const spiir_plan *p, const Band &b, int64_t nb)
{
    if (p->precision != SPIIR_PREC_PLAIN) return 1;
    const int req = p->opt.time_segments;
    const int64_t warps = b.lay.n_units() * b.lay.W;
    const int64_t nblocks = nb / (int64_t)b.lay.Tb;
    int P = 1;
    if (req >= 1) {
        P = req;
    } else {
        const int64_t target = 8 * (int64_t)p->n_sm;
        const int64_t want = std::min<int64_t>(64, target / std::max<int64_t>(warps, 1));
        if (want >= 4) P = (int)want;
        else if (warps < 16 * (int64_t)p->n_sm && nblocks >= 64) P = 2;
    }
    const int64_t max_p = std::max<int64_t>(1, nblocks);
    P = (int)std::max<int64_t>(1, std::min<int64_t>(P, max_p));
    return (req < 1 && P < 2) ? 1 : P;
}

// Projection weight seeds (the projection generates its weight tiles from
// them) and a^256 of a band, built on first use and after every coefficient
// update.
spiir_status ensure_tc_weights(spiir_plan *p, Band &b, cudaStream_t s)
{
    if (b.tc_valid) return SPIIR_OK;
    const spiir::Layout &L = b.lay;
    cudaError_t e;
    if (!b.tc_seed) {
        if ((e = dalloc(&b.tc_seed, (size_t)L.n_slots * spiir::kTcSeeds)) != cudaSuccess ||
            (e = dalloc(&b.tc_aT, (size_t)L.n_slots)) != cudaSuccess ||
            (e = dalloc(&b.tc_aT64, (size_t)L.n_slots)) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "projection weight seeds")
                                                  : cuda_fail(e, "cudaMalloc");
    }
    if ((e = spiir::launch_tc_seeds(b.params, b.ringoff, L.n_slots, (int)L.Dh, b.tc_seed,
                                    b.tc_aT, b.tc_aT64, s)) != cudaSuccess)
        return cuda_fail(e, "projection weight seeds launch");
    b.tc_valid = true;
    p->last_launches += 1;
    return SPIIR_OK;
}

spiir_status ensure_tc_strain(Band &b, int64_t bytes, cudaStream_t s)
{
    if (b.tc_b_cap >= bytes) return SPIIR_OK;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(b.tc_b);
    b.tc_b = nullptr;
    if ((e = cudaMalloc(&b.tc_b, (size_t)bytes)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "projection workspace")
                                              : cuda_fail(e, "cudaMalloc");
    b.tc_b_cap = bytes;
    return SPIIR_OK;
}

// Dynamic shared memory of a K1 launch: the layout's ring and block sums,
// plus the lower-band prefetch buffers of a multirate top band.
int k1_smem(const Band &b, const spiir::K1Args &a)
{
    return b.lay.smem_bytes() +
           (a.n_lower > 0 ? b.lay.W * (32 / b.lay.G) * a.low_len * (int)sizeof(float2) : 0);
}

// The chunked tensor-core form over one band call, in time tiles whose
// anchors fit a bounded workspace.  Per tile: strain windows, the split-BF16
// GEMM of chunk sums with the FP64 chunk scan (anchors of every chunk, the
// FP64 state carried to the next tile), then the anchored FP32 pass (z and
// running peaks).
spiir_status launch_anchored(spiir_plan *p, Band &b, spiir::K1Args a, cudaStream_t s,
                             int64_t *t0_advance)
{
    const spiir::Layout &L = b.lay;
    const int D = p->D;
    const int64_t n = a.n;
    const int64_t per = (int64_t)D * L.n_slots;
    cudaError_t e;
    spiir_status st = ensure_tc_weights(p, b, s);
    if (st != SPIIR_OK) return st;
    // tile: whole blocks and whole chunks, anchors within a quarter of the
    // free device memory (at most 16 GiB): fewer tiles, fewer weight passes
    int64_t unit = L.Tb;
    while (unit % spiir::kTcT != 0) unit += L.Tb;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)4 << 30;
    const int64_t budget = std::min<int64_t>((int64_t)16 << 30,
                                             std::max<int64_t>((int64_t)1 << 30, (int64_t)(free_b / 4)));
    const int64_t max_chunks = p->opt.tile_chunks > 0
                                   ? (int64_t)p->opt.tile_chunks
                                   : std::max<int64_t>(1, budget / (8 * per));
    const int64_t hq = L.Dh / spiir::kTcT;
    const int64_t budget_tile = std::max<int64_t>(unit, max_chunks * spiir::kTcT / unit * unit);
    int64_t n_tile = std::min<int64_t>(budget_tile, (n + unit - 1) / unit * unit);
    if (p->opt.tile_chunks <= 0) {
        // a tile's windows (chunks + hq) fill k whole column tiles of the
        // GEMM: k within the budget, chosen for the fewest column tiles over
        // the call, each time tile counted half a column tile more (its
        // launches), ties to the larger k; then the call split evenly over
        // that many time tiles (a tile 4 windows past 512 would take a third,
        // almost empty, column tile)
        const int64_t u = unit / spiir::kTcT;   // chunks per whole unit
        const int64_t cols = spiir::tc_cols_per_tile();
        const int64_t n_chunks = (n + spiir::kTcT - 1) / spiir::kTcT;
        const int64_t k_max = std::min<int64_t>((budget_tile / spiir::kTcT + hq) / cols,
                                                (n_chunks + hq + cols - 1) / cols);
        int64_t best_k = 0, best_tiles = 0;
        double best_cost = 0.0;
        for (int64_t k = 1; k <= k_max; ++k) {
            const int64_t cap = (k * cols - hq) / u * u;
            if (cap < u) continue;
            const int64_t tl = (n_chunks + cap - 1) / cap;
            const double cost = (double)tl * ((double)k + 0.5);
            if (best_k == 0 || cost <= best_cost) {
                best_k = k;
                best_tiles = tl;
                best_cost = cost;
            }
        }
        if (best_k > 0) {
            const int64_t cap = (best_k * cols - hq) / u * u;
            const int64_t per_tile =
                std::min<int64_t>(cap, ((n_chunks + best_tiles - 1) / best_tiles + u - 1) / u * u);
            n_tile = std::max<int64_t>(unit, std::min<int64_t>(n_tile, per_tile * spiir::kTcT));
        }
    }
    const int64_t chunks = n_tile / spiir::kTcT;
    if (b.tc_anchor_cap < chunks * per) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamSynchronize");
        cudaFree(b.tc_anchor);
        b.tc_anchor = nullptr;
        if ((e = dalloc(&b.tc_anchor, (size_t)(chunks * per))) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "anchor workspace")
                                                  : cuda_fail(e, "cudaMalloc");
        b.tc_anchor_cap = chunks * per;
    }
    st = ensure_tc_strain(b, spiir::tc_strain_bytes(chunks + hq, D), s);
    if (st != SPIIR_OK) return st;
    const int64_t tiles = (n + n_tile - 1) / n_tile;
    a.n_seg = (int32_t)n_tile;
    a.anchors = b.tc_anchor;
    a.seg_count = 1;
    a.peak_seg_stride = 0;
    for (int64_t q = 0; q < tiles; ++q) {
        const int64_t c_first = q * chunks;
        const int64_t c_end = std::min<int64_t>(c_first + chunks, (n + spiir::kTcT - 1) / spiir::kTcT);
        // windows c'' = c - q_l - 1 for chunks c of the tile, q_l <= hq
        const int64_t n_cols = c_end - c_first + hq;
        spiir::TcArgs t{};
        t.seed = b.tc_seed;
        t.params = b.params;
        t.B = b.tc_b;
        t.ringoff = b.ringoff;
        t.aT = b.tc_aT;
        t.aT64 = b.tc_aT64;
        t.state = b.state;
        t.s64 = reinterpret_cast<double2 *>(b.state_ext);
        t.anchors = b.tc_anchor;
        t.n_slots = L.n_slots;
        t.D = D;
        t.Dh = (int32_t)L.Dh;
        t.n_cols = n_cols;
        t.col0 = (int32_t)(c_first - hq - 1);
        t.c_first = (int32_t)c_first;
        t.c_end = (int32_t)c_end;
        t.c_full = (int32_t)(n / spiir::kTcT);
        t.err = p->err;
        t.wait_limit_ns = a.wait_limit_ns;
        a.seg_first = (int32_t)q;
        if ((e = spiir::launch_tc_strain(b.xe, b.xe_stride, (int)L.Dh, n, D, n_cols, t.col0,
                                         b.tc_b, s)) != cudaSuccess)
            return cuda_fail(e, "chunked tensor-core launch");
        const int tt = time_begin(p, s);
        if ((e = spiir::launch_tc_project(t, s)) != cudaSuccess)
            return cuda_fail(e, "chunked tensor-core launch");
        time_end(p, s, tt, kTimeTc);
        const int tk = time_begin(p, s);
        if ((e = spiir::launch_k1(a, L.n_units(), k1_smem(b, a), s)) != cudaSuccess)
            return cuda_fail(e, "chunked tensor-core launch");
        time_end(p, s, tk, kTimeK1);
        p->last_launches += 3;
    }
    if (n % spiir::kTcT != 0) {   // the call ended inside a chunk
        if ((e = spiir::launch_state_to_fp64(b.state, reinterpret_cast<double2 *>(b.state_ext),
                                             per, s)) != cudaSuccess)
            return cuda_fail(e, "end state launch");
        p->last_launches += 1;
    }
    if (t0_advance != nullptr) {
        if ((e = spiir::launch_advance(t0_advance, n, s)) != cudaSuccess)
            return cuda_fail(e, "sample counter launch");
        p->last_launches += 1;
    }
    p->last_segments = (int)tiles;
    return SPIIR_OK;
}

// Launch K1 for one band call split into time segments.  The start state of
// every segment comes either from the split-BF16 tensor-core projection of
// the strain (chunk sums scanned across segments) or from a zero-state pass
// over all but the last segment whose end states an FP64 carry turns into
// true start states; the main pass then runs every segment from its start
// state and the per-segment peaks are merged in time order.  The chunked
// tensor-core precision goes to launch_anchored instead.
// phase: kPhaseAll, or kPhaseProject (segment start states only) followed by
// kPhaseMain (the filter pass from them) on the same band and arguments.
constexpr int kPhaseAll = 0, kPhaseProject = 1, kPhaseMain = 2;

spiir_status launch_segmented(spiir_plan *p, Band &b, spiir::K1Args a, int P, cudaStream_t s,
                              int64_t *t0_advance = nullptr, int phase = kPhaseAll)
{
    if (p->precision == SPIIR_PREC_CHUNKED_TC) {
        if (phase == kPhaseProject) return SPIIR_OK;
        return launch_anchored(p, b, a, s, t0_advance);
    }
    const spiir::Layout &L = b.lay;
    const int D = p->D;
    const int64_t per = (int64_t)D * L.n_slots;
    const int64_t n = a.n;
    // segment starts on block boundaries, and on chunk boundaries for the
    // tensor-core projection
    const bool tc = p->opt.projection != SPIIR_PROJECT_RECURRENCE;
    int64_t unit = L.Tb;
    if (tc)
        while (unit % spiir::kTcT != 0) unit += L.Tb;
    const int64_t n_seg = ((n + P - 1) / P + unit - 1) / unit * unit;
    P = (int)((n + n_seg - 1) / n_seg);
    cudaError_t e;
    if (t0_advance != nullptr) p->last_segments = std::max(P, 1);
    if (P <= 1) {
        if (phase == kPhaseProject) return SPIIR_OK;
        const int tk = time_begin(p, s);
        if ((e = spiir::launch_k1(a, L.n_units(), k1_smem(b, a), s)) != cudaSuccess)
            return cuda_fail(e, "filter kernel launch");
        time_end(p, s, tk, kTimeK1);
        p->last_launches += 1;
        if (t0_advance != nullptr && (e = spiir::launch_advance(t0_advance, n, s)) != cudaSuccess)
            return cuda_fail(e, "sample counter launch");
        p->last_launches += t0_advance != nullptr ? 1 : 0;
        return SPIIR_OK;
    }
    if (b.seg_cap < P) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamSynchronize");
        cudaFree(b.seg_end);
        cudaFree(b.seg_init);
        cudaFree(b.seg_best);
        cudaFree(b.seg_idx);
        b.seg_end = b.seg_init = nullptr;
        b.seg_best = nullptr;
        b.seg_idx = nullptr;
        if ((e = dalloc(&b.seg_end, (size_t)P * per)) != cudaSuccess ||
            (e = dalloc(&b.seg_init, (size_t)P * per)) != cudaSuccess ||
            (e = dalloc(&b.seg_best, (size_t)P * D * p->T)) != cudaSuccess ||
            (e = dalloc(&b.seg_idx, (size_t)P * D * p->T)) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "segment workspace")
                                                  : cuda_fail(e, "cudaMalloc");
        b.seg_cap = P;
    }
    a.n_seg = (int32_t)n_seg;
    if (phase == kPhaseMain) {
        // start states already projected
    } else if (tc) {
        // segment start states from the split-BF16 GEMM of chunk sums + scan
        spiir_status st = ensure_tc_weights(p, b, s);
        if (st != SPIIR_OK) return st;
        const int64_t cps = n_seg / spiir::kTcT;
        const int64_t c_last = (int64_t)(P - 1) * cps - 1;
        const int64_t hq = L.Dh / spiir::kTcT;
        const int64_t n_cols = c_last + hq + 1;
        st = ensure_tc_strain(b, spiir::tc_strain_bytes(n_cols, D), s);
        if (st != SPIIR_OK) return st;
        spiir::TcArgs t{};
        t.seed = b.tc_seed;
        t.params = b.params;
        t.B = b.tc_b;
        t.ringoff = b.ringoff;
        t.aT = b.tc_aT;
        t.state = a.state;   // the call's start state (the plan's, or the adjoint's zero state)
        t.seg_init = b.seg_init;
        t.n_slots = L.n_slots;
        t.D = D;
        t.Dh = (int32_t)L.Dh;
        t.n_cols = n_cols;
        t.col0 = (int32_t)(-hq - 1);
        t.c_last = (int32_t)c_last;
        t.cps = (int32_t)cps;
        t.err = p->err;
        t.wait_limit_ns = a.wait_limit_ns;
        if ((e = spiir::launch_tc_strain(a.xe, a.xe_stride, (int)L.Dh, n, D, n_cols, t.col0,
                                         b.tc_b, s)) != cudaSuccess)
            return cuda_fail(e, "tensor-core projection launch");
        const int tt = time_begin(p, s);
        if ((e = spiir::launch_tc_project(t, s)) != cudaSuccess)
            return cuda_fail(e, "tensor-core projection launch");
        time_end(p, s, tt, kTimeTc);
    } else {
        // projection: segments 0..P-2 from zero state, no z, no peak
        spiir::K1Args proj = a;
        proj.zero_init = 1;
        proj.seg_end = b.seg_end;
        proj.z = nullptr;
        proj.peak_best = nullptr;
        proj.peak_idx = nullptr;
        proj.n_lower = 0;
        const int tk = time_begin(p, s);
        if ((e = spiir::launch_k1(proj, L.n_units(), L.smem_bytes(), s)) != cudaSuccess)
            return cuda_fail(e, "segment projection launch");
        time_end(p, s, tk, kTimeK1);
        if ((e = spiir::launch_segment_carry(b.params, a.state, b.seg_end, b.seg_init, L.n_slots,
                                             D, P, (int)n_seg, s)) != cudaSuccess)
            return cuda_fail(e, "segment projection launch");
    }
    if (phase == kPhaseProject) return SPIIR_OK;
    // main pass: every segment from its start state
    float *best = a.peak_best;
    int64_t *idx = a.peak_idx;
    a.seg_init = b.seg_init;
    if (best != nullptr) {   // every entry is written by the one CTA that owns it
        a.peak_best = b.seg_best;
        a.peak_idx = b.seg_idx;
        a.peak_seg_stride = (int64_t)D * p->T;
    }
    const int tk = time_begin(p, s);
    if ((e = spiir::launch_k1(a, L.n_units(), k1_smem(b, a), s)) != cudaSuccess)
        return cuda_fail(e, "filter kernel launch");
    time_end(p, s, tk, kTimeK1);
    p->last_launches += 3 + ((best != nullptr || t0_advance != nullptr) ? 1 : 0);
    if (best != nullptr) {
        if ((e = spiir::launch_peak_merge(b.seg_best, b.seg_idx, P, (int64_t)D * p->T, best, idx,
                                          t0_advance, n, s)) != cudaSuccess)
            return cuda_fail(e, "segment peak merge");
    } else if (t0_advance != nullptr &&
               (e = spiir::launch_advance(t0_advance, n, s)) != cudaSuccess) {
        return cuda_fail(e, "sample counter launch");
    }
    return SPIIR_OK;
}

// Time candidate layouts on a prefix of the first call's strain (zero state,
// no z, no peak) and keep the fastest.  Synchronous; runs once per plan.
spiir_status autotune(spiir_plan *p, const float *x_dev, int64_t n, cudaStream_t s)
{
    struct Cand {
        int Fcap, W, C, Tb;
        int tail;          // layout tail split: -1 off, 0 auto
        bool persistent;   // persistent launch (else one CTA per unit)
    };
    static const Cand cands[] = {
        {10, 4, 1, 512, -1, false}, {10, 4, 1, 512, -1, true}, {10, 4, 1, 512, 0, false},
        {10, 4, 2, 512, -1, false}, {10, 4, 1, 256, -1, false}, {10, 2, 1, 512, -1, false},
        {10, 8, 1, 256, -1, false}, {8, 4, 1, 512, -1, false},  {4, 8, 2, 256, -1, false},
        {4, 4, 1, 512, -1, false},  {2, 8, 1, 256, -1, false}};
    const bool forced_launch = p->opt.persistent != 0;
    // the trials run the candidates unsegmented on a prefix: a call that runs
    // in time segments (a bank under one wave of 16 warps per SM) would not be
    // timed the way it runs, so such plans keep the default layout (measured:
    // the autotuned layout took the adjoint bank's forward from 2.10 to 2.69 ms)
    if (segments_for(p, p->bands[0], n) > 1) {
        p->tune_report = "skipped: calls of this bank run in time segments";
        p->tuned = true;
        return SPIIR_OK;
    }
    const int64_t nt = std::min<int64_t>(n, 8192);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
        return cuda_fail(e, "autotune events");
    float best_ms = 1e30f;
    bool best_persistent = p->persistent;
    Band best;
    bool have = false;
    std::string report;
    for (const Cand &c : cands) {
        Band b;
        spiir::LayoutOptions lo;
        lo.Fcap = c.Fcap;
        lo.W = c.W;
        lo.C = c.C;
        lo.Tb = c.Tb;
        lo.n_sm = p->n_sm;
        if (forced_launch && c.persistent != p->persistent) continue;
        lo.tail = p->opt.tail_split > 0 ? p->opt.tail_split : c.tail;
        if (lo.tail >= 0) lo.regs = spiir::k1_plain_regs(c.Fcap);
        std::string err;
        if (!spiir::build_layout(p->lists, p->D, p->a_host.data(), p->b_host.data(),
                                 p->d_host.data(), lo, &b.lay, &err))
            continue;
        spiir_status st = upload_band(b, p->D, p->precision, p->opt.chunk_len);
        if (st == SPIIR_OK) st = ensure_xe(p, b, nt, s);
        if (st != SPIIR_OK) {
            free_band(b);
            continue;
        }
        const int64_t Dh = b.lay.Dh;
        if ((e = cudaMemset2DAsync(b.xe, b.xe_stride * 4, 0, Dh * 4, p->D, s)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(b.xe + Dh, b.xe_stride * 4, x_dev, n * 4, nt * 4, p->D,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
            free_band(b);
            continue;
        }
        spiir::K1Args a = k1_args(p, b, nt, nullptr, nt, false);
        a.queue = c.persistent ? p->queue : nullptr;
        // one untimed launch, then the timed one
        e = spiir::launch_k1(a, b.lay.n_units(), b.lay.smem_bytes(), s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = spiir::launch_k1(a, b.lay.n_units(), b.lay.smem_bytes(), s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            free_band(b);
            return cuda_fail(e, "autotune launch");
        }
        report += "cap" + std::to_string(c.Fcap) + "/W" + std::to_string(c.W) + "/C" +
                  std::to_string(c.C) + "/Tb" + std::to_string(c.Tb) + "/tail" +
                  std::to_string(b.lay.tail_templates) + (c.persistent ? "/persistent" : "") +
                  "=" + std::to_string(ms) + "ms ";
        if (ms < best_ms) {
            if (have) free_band(best);
            best = b;
            best_ms = ms;
            best_persistent = c.persistent;
            have = true;
        } else {
            free_band(b);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (have) {
        // the candidate's state and history were zero-initialised by the upload
        if ((e = cudaMemsetAsync(best.state, 0, sizeof(float2) * (size_t)p->D * best.lay.n_slots,
                                 s)) != cudaSuccess)
            return cuda_fail(e, "autotune reset");
        free_band(p->bands[0]);
        p->bands[0] = best;
        p->persistent = best_persistent;
    }
    p->tune_report = report;
    p->tuned = true;
    return SPIIR_OK;
}

spiir_status spiir_filter(spiir_plan *p, const float *x_dev, int64_t n, float *z_dev,
                          void *stream)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan cannot filter");
    if (n < 0) return fail(SPIIR_EINVAL, "n must be >= 0");
    if (n == 0) return SPIIR_OK;
    if (!x_dev) return fail(SPIIR_EINVAL, "x_dev is NULL");
    if (n > (int64_t)1 << 30) return fail(SPIIR_EINVAL, "n above 2^30 samples per call");
    if (p->t0 % p->maxR != 0)
        return fail(SPIIR_EINVAL, "multirate stream: the previous call's length was not a "
                                  "multiple of the largest decimation factor");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->tuned && p->t0 == 0) {
        spiir_status st = autotune(p, x_dev, n, s);
        if (st != SPIIR_OK) return st;
    }
    const int D = p->D;
    cudaError_t e;
    p->last_launches = 0;
    // decimated bands first (their sums feed the top band's epilogue), top band last
    std::vector<int> order;
    for (int j = 0; j < (int)p->bands.size(); ++j)
        if (j != p->top) order.push_back(j);
    order.push_back(p->top);
    spiir::K1Args top_args{};
    // band front ends: stage (top-rate history, x) once for every FIR band
    constexpr int H = spiir::kFirMaxTaps - 1;
    bool any_fir = false;
    for (const Band &b : p->bands) any_fir = any_fir || b.fir_len > 0;
    if (any_fir) {
        if (p->fir_xt_cap < H + n) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(p->fir_xt);
            p->fir_xt = nullptr;
            p->fir_xt_cap = 0;
            if ((e = dalloc(&p->fir_xt, (size_t)D * (H + n))) != cudaSuccess)
                return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "front-end staging")
                                                      : cuda_fail(e, "cudaMalloc");
            p->fir_xt_cap = H + n;
        }
        const int64_t st = p->fir_xt_cap;
        if ((e = cudaMemcpy2DAsync(p->fir_xt, st * 4, p->fir_xh, H * 4, H * 4, D,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(p->fir_xt + H, st * 4, x_dev, n * 4, n * 4, D,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "front-end staging");
    }
    // Multirate calls with two or more lower bands use the plan's second
    // stream, forked here: the first, third ... lower band runs there; the
    // top band's staging and segment projection (which need only its own
    // strain and state) and the other lower bands run on the caller's stream;
    // both join before the top band's main pass, which reads the lower bands'
    // sums.  The bands are independent, so the smaller passes fill the GPU
    // beside the larger.
    const bool fork = order.size() > 2;
    if (fork) {
        if (!p->aux &&
            ((e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking)) != cudaSuccess ||
             (e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
             (e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming)) != cudaSuccess))
            return cuda_fail(e, "band stream");
        if ((e = cudaEventRecord(p->ev_fork, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0)) != cudaSuccess)
            return cuda_fail(e, "band fork");
    }
    // xe[:, 0:Dh] = band history, xe[:, Dh:Dh+nb] = this call's band samples
    auto stage = [&](Band &b, int64_t nb, cudaStream_t bs) -> spiir_status {
        spiir_status st = ensure_xe(p, b, nb, bs);
        if (st != SPIIR_OK) return st;
        const int64_t Dh = b.lay.Dh;
        if ((e = cudaMemcpy2DAsync(b.xe, b.xe_stride * 4, b.hist, Dh * 4, Dh * 4, D,
                                   cudaMemcpyDeviceToDevice, bs)) != cudaSuccess)
            return cuda_fail(e, "strain staging copy");
        if (b.fir_len > 0) {
            e = spiir::launch_fir_decimate(p->fir_xt, p->fir_xt_cap, H, D, b.R, nb, b.fir,
                                           b.fir_len, b.xe, b.xe_stride, Dh, bs);
            p->last_launches += 1;
        } else if (b.R == 1) {
            e = cudaMemcpy2DAsync(b.xe + Dh, b.xe_stride * 4, x_dev, n * 4, n * 4, D,
                                  cudaMemcpyDeviceToDevice, bs);
        } else {
            e = spiir::launch_decimate(x_dev, n, D, b.R, nb, b.xe, b.xe_stride, Dh, bs);
            p->last_launches += 1;
        }
        if (e != cudaSuccess) return cuda_fail(e, "strain staging");
        return SPIIR_OK;
    };
    // band history for the next call: the last Dh band samples of (history, x_b)
    auto keep_history = [&](Band &b, int64_t nb, cudaStream_t bs) -> spiir_status {
        const int64_t Dh = b.lay.Dh;
        if ((e = cudaMemcpy2DAsync(b.hist, Dh * 4, b.xe + nb, b.xe_stride * 4, Dh * 4, D,
                                   cudaMemcpyDeviceToDevice, bs)) != cudaSuccess)
            return cuda_fail(e, "history copy");
        return SPIIR_OK;
    };
    Band &tb = p->bands[p->top];
    spiir::K1Args ta{};   // the top band's arguments, made once its strain is staged
    auto stage_top = [&]() -> spiir_status {
        spiir_status st = stage(tb, n, s);
        if (st != SPIIR_OK) return st;
        ta = k1_args(p, tb, n, z_dev, n, true);
        ta.t0 = 0;
        ta.t0_dev = p->t0_dev;
        return SPIIR_OK;
    };
    const int top_P = segments_for(p, tb, n);
    if (fork) {
        spiir_status st = stage_top();
        if (st == SPIIR_OK)
            st = launch_segmented(p, tb, ta, top_P, s, p->t0_dev, kPhaseProject);
        if (st != SPIIR_OK) return st;
    }
    int n_lower_seen = 0;
    for (int j : order) {
        if (j == p->top) break;   // the top band comes last (order ends with it)
        Band &b = p->bands[j];
        const int64_t nb = (n + b.R - 1) / b.R;   // band samples in this call
        const cudaStream_t bs = (fork && !(n_lower_seen++ & 1)) ? p->aux : s;
        spiir_status st = stage(b, nb, bs);
        if (st != SPIIR_OK) return st;
        if (!b.zb || b.zb_cap < nb) {
            if (b.zb) {   // the top band (caller's stream) read it last call
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(bs)) != cudaSuccess)
                    return cuda_fail(e, "cudaStreamSynchronize");
                cudaFree(b.zb);
                b.zb = nullptr;
            }
            if ((e = dalloc(&b.zb, (size_t)D * p->T * nb)) != cudaSuccess)
                return e == cudaErrorMemoryAllocation
                           ? fail(SPIIR_ENOMEM, "band workspace allocation")
                           : cuda_fail(e, "cudaMalloc");
            b.zb_cap = nb;
        }
        spiir::K1Args a = k1_args(p, b, nb, reinterpret_cast<float *>(b.zb), nb, false);
        a.t0 = p->t0 / b.R;
        st = launch_segmented(p, b, a, segments_for(p, b, nb), bs);
        if (st != SPIIR_OK) return st;
        spiir::LowerBand &lb = top_args.lower[top_args.n_lower++];
        lb.z = b.zb;
        lb.len = nb;
        lb.R = b.R;
        lb.shift = -1;
        for (int sh = 0; sh < 31; ++sh)
            if ((1 << sh) == b.R) lb.shift = sh;
        if ((st = keep_history(b, nb, bs)) != SPIIR_OK) return st;
    }
    if (fork && ((e = cudaEventRecord(p->ev_join, p->aux)) != cudaSuccess ||
                 (e = cudaStreamWaitEvent(s, p->ev_join, 0)) != cudaSuccess))
        return cuda_fail(e, "band join");
    {
        spiir_status st = fork ? SPIIR_OK : stage_top();
        if (st != SPIIR_OK) return st;
        ta.n_lower = top_args.n_lower;
        // per template: the band samples one block interpolates from
        int32_t off = 0;
        for (int i = 0; i < ta.n_lower; ++i) {
            ta.lower[i] = top_args.lower[i];
            ta.lower[i].buf_off = off;
            off += (int32_t)((tb.lay.Tb + ta.lower[i].R - 1) / ta.lower[i].R + 2);
        }
        ta.low_len = (off + 1) / 2 * 2;
        st = launch_segmented(p, tb, ta, top_P, s, p->t0_dev, fork ? kPhaseMain : kPhaseAll);
        if (st == SPIIR_OK) st = keep_history(tb, n, s);
        if (st != SPIIR_OK) return st;
    }
    // the last H top-rate samples of (history, x) for the next call's front ends
    if (any_fir && (e = cudaMemcpy2DAsync(p->fir_xh, H * 4, p->fir_xt + n, p->fir_xt_cap * 4,
                                          H * 4, D, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "front-end history copy");
    p->t0 += n;
    return SPIIR_OK;
}

spiir_status spiir_set_band_fir(spiir_plan *p, int32_t band, const float *taps, int32_t n_taps)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no front end");
    if (band < 0 || band >= (int32_t)p->bands.size()) return fail(SPIIR_EINVAL, "no such band");
    if (n_taps < 0 || n_taps > spiir::kFirMaxTaps || (n_taps > 0 && !taps))
        return fail(SPIIR_EINVAL, "n_taps must be in [0, " +
                                      std::to_string(spiir::kFirMaxTaps) + "] with taps given");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();   // calls in flight may read the taps
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    Band &b = p->bands[band];
    cudaFree(b.fir);
    b.fir = nullptr;
    b.fir_len = 0;
    if (n_taps == 0) return SPIIR_OK;
    if (!p->fir_xh) {
        const size_t words = (size_t)p->D * (spiir::kFirMaxTaps - 1);
        if ((e = dalloc(&p->fir_xh, words)) != cudaSuccess ||
            (e = cudaMemset(p->fir_xh, 0, words * sizeof(float))) != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "front-end history")
                                                  : cuda_fail(e, "cudaMalloc");
    }
    if ((e = dalloc(&b.fir, (size_t)n_taps)) != cudaSuccess ||
        (e = cudaMemcpy(b.fir, taps, sizeof(float) * n_taps, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "front-end taps")
                                              : cuda_fail(e, "front-end taps upload");
    b.fir_len = n_taps;
    return SPIIR_OK;
}

spiir_status spiir_chi2_peak(const float *zg_dev, int32_t n_detectors, int64_t n_templates,
                             int32_t n_bins, int64_t n, float *peak_dev, int64_t *t_dev,
                             float *chi2_dev, void *stream)
{
    if (!zg_dev || !peak_dev || !t_dev || !chi2_dev)
        return fail(SPIIR_EINVAL, "zg_dev, peak_dev, t_dev and chi2_dev are required");
    if (n_detectors < 1 || n_templates < 0 || n_bins < 1 || n_bins > 64 || n < 1 ||
        (int64_t)n_detectors * n_templates > INT32_MAX)
        return fail(SPIIR_EINVAL, "n_detectors >= 1, 0 <= n_templates, 1 <= n_bins <= 64, n >= 1");
    cudaError_t e = spiir::launch_chi2_peak(reinterpret_cast<const float2 *>(zg_dev), n_detectors,
                                            n_templates, n_bins, n, peak_dev, t_dev, chi2_dev,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "chi^2 launch");
    return SPIIR_OK;
}

spiir_status spiir_network_peak(const float *z_dev, int32_t n_detectors, int64_t n_templates,
                                int64_t n, const int32_t *window, float *rho_dev,
                                int64_t *t_dev, int32_t *shift_dev, void *stream)
{
    if (!z_dev || !window || !rho_dev || !t_dev)
        return fail(SPIIR_EINVAL, "z_dev, window, rho_dev and t_dev are required");
    if (n_detectors < 1 || n_detectors > spiir::kNetMaxD)
        return fail(SPIIR_EINVAL, "n_detectors must be in [1, " +
                                      std::to_string(spiir::kNetMaxD) + "]");
    if (n_templates < 0 || n_templates > INT32_MAX || n < 1 || n > ((int64_t)1 << 40))
        return fail(SPIIR_EINVAL, "n_templates must be in [0, 2^31), n in [1, 2^40]");
    spiir::NetArgs a{};
    a.z = reinterpret_cast<const float2 *>(z_dev);
    a.D = n_detectors;
    a.T = n_templates;
    a.n = n;
    for (int d = 1; d < n_detectors; ++d) {
        if (window[d] < 0 || window[d] > spiir::kNetMaxWindow)
            return fail(SPIIR_EINVAL, "window[d] must be in [0, " +
                                          std::to_string(spiir::kNetMaxWindow) + "]");
        a.w[d] = window[d];
    }
    if (spiir::network_smem_words(a.w, a.D, a.off_p, a.off_g) * 4 > 200 * 1024)
        return fail(SPIIR_EUNSUPPORTED, "detector windows too wide for shared memory");
    a.rho = rho_dev;
    a.t = t_dev;
    a.shift = shift_dev;
    cudaError_t e = spiir::launch_network_peak(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "network peak launch");
    return SPIIR_OK;
}

spiir_status spiir_peak(spiir_plan *p, float *peak_abs_dev, int64_t *peak_idx_dev, void *stream)
{
    if (!p || !peak_abs_dev || !peak_idx_dev) return fail(SPIIR_EINVAL, "NULL argument");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no peaks");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = spiir::launch_peak_out(p->peak_best, p->peak_idx, (int64_t)p->D * p->T,
                                           peak_abs_dev, peak_idx_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "peak kernel launch");
    return SPIIR_OK;
}

// Adjoint tasks: kAdjRounds filter rounds of one layout warp (template);
// adj_W tasks per CTA, every detector.
spiir_status build_adjoint_tasks(Band &b, int D)
{
    const spiir::Layout &L = b.lay;
    std::vector<int32_t> tasks;
    for (int64_t g = 0; g < L.n_groups(); ++g)
        for (int w = 0; w < L.W; ++w) {
            const int32_t t = L.warp_info[(g * L.W + w) * 4];
            const int32_t t2 = L.G == 16 ? L.warp_info[(g * L.W + w) * 4 + 3] : -1;
            if (t < 0) continue;
            for (int r0 = 0; r0 < L.group_F[g]; r0 += spiir::kAdjRounds) {
                tasks.push_back((int32_t)(L.group_pbase[g] + ((int64_t)r0 * L.W + w) * 32));
                tasks.push_back(std::min(spiir::kAdjRounds, L.group_F[g] - r0));
                tasks.push_back(t);
                tasks.push_back(t2);
            }
        }
    const int64_t n_tasks = (int64_t)tasks.size() / 4;
    const int64_t n_groups = (n_tasks + b.adj_W - 1) / b.adj_W;
    tasks.resize((size_t)n_groups * b.adj_W * 4, 0);
    for (int64_t i = n_tasks; i < n_groups * b.adj_W; ++i) tasks[4 * i + 2] = -1;  // empty
    // input-gradient units: runs of tasks with the same template(s), split
    // into pieces of at most kK7MaxWarps tasks
    std::vector<int32_t> units7;
    int W7 = 1;
    for (int64_t i = 0; i < n_tasks;) {
        int64_t j = i + 1;
        while (j < n_tasks && j - i < spiir::kK7MaxWarps && tasks[4 * j + 2] == tasks[4 * i + 2] &&
               tasks[4 * j + 3] == tasks[4 * i + 3])
            ++j;
        units7.push_back((int32_t)i);
        units7.push_back((int32_t)(j - i));
        W7 = std::max(W7, (int)(j - i));
        i = j;
    }
    std::vector<int32_t> units((size_t)n_groups * D * 2);
    for (int64_t g = 0; g < n_groups; ++g)
        for (int d = 0; d < D; ++d) {
            units[2 * (g * D + d)] = (int32_t)g;
            units[2 * (g * D + d) + 1] = d;
        }
    std::vector<int32_t> stmpl(L.slot_template.begin(), L.slot_template.end());
    cudaError_t e;
    if ((e = dalloc(&b.adj_slot_tmpl, stmpl.size())) != cudaSuccess ||
        (e = cudaMemcpy(b.adj_slot_tmpl, stmpl.data(), stmpl.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = dalloc(&b.adj_tasks, (size_t)n_groups * b.adj_W)) != cudaSuccess ||
        (e = dalloc(&b.adj_units, units.size())) != cudaSuccess ||
        (e = cudaMemcpy(b.adj_tasks, tasks.data(), tasks.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b.adj_units, units.data(), units.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = dalloc(&b.adj_units7, units7.size() / 2)) != cudaSuccess ||
        (e = cudaMemcpy(b.adj_units7, units7.data(), units7.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "adjoint task list")
                                              : cuda_fail(e, "adjoint task upload");
    b.adj_n_units = n_groups * D;
    b.adj_n_units7 = (int64_t)units7.size() / 2;
    b.adj_W7 = W7;
    return SPIIR_OK;
}

// Tangent order of a band's filters for nf filters per lane: grouped by
// template (bank order), a lane's filters from one template, each warp
// spanning at most two templates (a third starts a new warp).  Filter f of a
// lane reads strain at bank (Dh - d) mod 32, so it takes a filter whose delay
// mod 32 no earlier lane's filter f in the warp has, while the template has
// one (else one from the fullest residue class).  Positions are
// (warp nf + f) 32 + lane.
spiir_status build_tangent_order(Band &b, int64_t T, int nf)
{
    const spiir::Layout &L = b.lay;
    std::vector<std::vector<int64_t>> per((size_t)T);
    for (int64_t s = 0; s < L.n_slots; ++s)
        if (L.slot_filter[s] >= 0 && L.slot_template[s] >= 0) per[L.slot_template[s]].push_back(s);
    std::vector<int32_t> lanes, wtmpl;
    std::vector<int32_t> row((size_t)nf * 32 * 2);
    int c = 0, t0 = -1, t1 = -1;
    uint32_t used[2] = {0, 0};   // residues taken by filter f of the current warp
    auto reset_rows = [&]() {
        for (size_t i = 0; i < row.size(); i += 2) {
            row[i] = -1;
            row[i + 1] = 0;
        }
    };
    reset_rows();
    auto close_warp = [&]() {
        lanes.insert(lanes.end(), row.begin(), row.end());
        wtmpl.push_back(t0);
        wtmpl.push_back(t1);
        reset_rows();
        c = 0;
        t0 = t1 = -1;
        used[0] = used[1] = 0;
    };
    for (int64_t t = 0; t < T; ++t) {
        std::vector<std::vector<int64_t>> bucket(32);
        for (int64_t s : per[t]) {
            const int d = L.Dh - L.ringoff[2 * s];
            bucket[((d % 32) + 32) % 32].push_back(s);
        }
        size_t left = per[t].size(), k0 = 0;
        while (left > 0) {
            if (c == 32) close_warp();
            int li;
            if ((int64_t)t0 == t) li = 0;
            else if ((int64_t)t1 == t) li = 1;
            else if (t0 < 0) { t0 = (int)t; li = 0; }
            else if (t1 < 0) { t1 = (int)t; li = 1; }
            else { close_warp(); t0 = (int)t; li = 0; }
            for (int f = 0; f < nf && left > 0; ++f, --left, ++k0) {
                int pick = -1;
                for (int j = 0; j < 32 && pick < 0; ++j) {
                    const int k = (int)((k0 + j) % 32);
                    if (!bucket[k].empty() && !(used[f] & (1u << k))) pick = k;
                }
                if (pick < 0)
                    for (int k = 0; k < 32; ++k)
                        if (pick < 0 || bucket[k].size() > bucket[pick].size()) pick = k;
                const int64_t s = bucket[pick].back();
                bucket[pick].pop_back();
                used[f] |= 1u << pick;
                if (s > INT32_MAX)
                    return fail(SPIIR_EUNSUPPORTED, "tangent form: slot index above 2^31");
                row[2 * ((size_t)f * 32 + c)] = (int32_t)s;
                row[2 * ((size_t)f * 32 + c) + 1] = li;
            }
            ++c;
        }
    }
    if (c > 0) close_warp();
    const int k = nf - 1;
    cudaError_t e;
    if ((e = dalloc(&b.kt_lanes[k], lanes.size() / 2)) != cudaSuccess ||
        (e = cudaMemcpy(b.kt_lanes[k], lanes.data(), lanes.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = dalloc(&b.kt_warp_tmpl[k], std::max<size_t>(1, wtmpl.size() / 2))) != cudaSuccess ||
        (wtmpl.size() > 0 &&
         (e = cudaMemcpy(b.kt_warp_tmpl[k], wtmpl.data(), wtmpl.size() * sizeof(int32_t),
                         cudaMemcpyHostToDevice)) != cudaSuccess))
        return e == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "tangent lane order")
                                              : cuda_fail(e, "tangent lane order upload");
    b.kt_n_pos[k] = (int64_t)lanes.size() / 2;
    return SPIIR_OK;
}

// Warps per tangent CTA: the fewest per-SM warps over the launch (one wave:
// the busiest SM's warps; several: the mean), larger W on ties.
int tangent_warps_per_cta(int64_t warps, int D, int Dh, int Tb, int n_sm)
{
    int best = 1;
    double best_cost = 1e300;
    for (int W = 1; W <= 8; W *= 2) {
        const int smem = spiir::kt_smem_bytes(Dh, Tb, W);
        if (smem > 227 * 1024) continue;
        const int64_t per_sm = std::min<int64_t>({32, (228 * 1024) / (smem + 1024), 32 / W});
        if (per_sm < 1) continue;
        const int64_t ctas = (warps + W - 1) / W * D;
        const double cost = ctas <= per_sm * n_sm ? (double)W * ((ctas + n_sm - 1) / n_sm)
                                                  : (double)W * ctas / n_sm;
        if (cost <= best_cost) {
            best_cost = cost;
            best = W;
        }
    }
    return best;
}

spiir_status spiir_filter_backward(spiir_plan *p, const float *x_dev, int64_t n,
                                   const float *grad_z_dev, float *grad_a_dev,
                                   float *grad_b_dev, float *grad_x_dev, void *stream)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan cannot run the adjoint");
    if (p->bands.size() != 1)
        return fail(SPIIR_EUNSUPPORTED, "the adjoint is built for single-rate banks");
    if (n < 1 || n > ((int64_t)1 << 30)) return fail(SPIIR_EINVAL, "n must be in [1, 2^30]");
    if (!x_dev || !grad_z_dev || !grad_a_dev || !grad_b_dev)
        return fail(SPIIR_EINVAL, "x_dev, grad_z_dev, grad_a_dev and grad_b_dev are required");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    Band &b = p->bands[0];
    const spiir::Layout &L = b.lay;
    const int D = p->D;
    // checkpoint interval: a whole number of blocks, about 1024 samples
    const int Cc = L.Tb * std::max(1, (1024 + L.Tb - 1) / L.Tb);
    const int64_t nc = (n + Cc - 1) / Cc;
    const int64_t need = ((n + L.Tb - 1) / L.Tb) * L.Tb;
    cudaError_t e;
    auto oom = [&](cudaError_t err) {
        return err == cudaErrorMemoryAllocation ? fail(SPIIR_ENOMEM, "adjoint workspace")
                                                : cuda_fail(err, "cudaMalloc");
    };
    if (!b.adj_tasks) {
        spiir_status st = build_adjoint_tasks(b, D);
        if (st != SPIIR_OK) return st;
    }
    // g_a, g_b: tangent or reverse form
    // (the tangent form's input-gradient pass warms up over whole 256-sample
    // chunks: the history must be whole chunks)
    bool tangent = false;
    if (p->opt.adjoint_form != SPIIR_ADJOINT_REVERSE &&
        spiir::kt_smem_bytes(L.Dh, L.Tb, 1) <= 227 * 1024 &&
        (!grad_x_dev || L.Dh % spiir::kK7Chunk == 0)) {
        for (int nf = 1; nf <= 2; ++nf)
            if (!b.kt_lanes[nf - 1]) {
                spiir_status st = build_tangent_order(b, p->T, nf);
                if (st != SPIIR_OK) return st;
            }
        // auto: the tangent pass runs every filter over the whole call in one
        // thread, so it wants a bank of >= 2 warps per SM at one filter per
        // thread (>= 8 with g_x, whose pass it then shares the GPU with), or a
        // short call (measured: 7 x 100 filters, 3000 samples, 0.068 vs
        // 0.163 ms without g_x; 128 x 200, 65536: 1.85 vs 3.22 ms without,
        // 5.77 vs 4.35 ms with g_x; 64 x 200 x 3 detectors: 4.41 vs 6.24 ms)
        const int64_t warps1 = (b.kt_n_pos[0] / 32) * D;
        tangent = p->opt.adjoint_form == SPIIR_ADJOINT_TANGENT || n <= 8192 ||
                  warps1 >= (grad_x_dev ? 8 : 2) * (int64_t)p->n_sm;
    }
    if (p->opt.adjoint_form == SPIIR_ADJOINT_TANGENT && !tangent)
        return fail(SPIIR_EUNSUPPORTED,
                    "tangent adjoint: strain window above 227 KB, or history not a multiple "
                    "of 256 samples");
    const bool need_ckpt = !tangent;
    if (!b.bw_xe || b.bw_cap < need || (need_ckpt && b.ckpt_cap < nc)) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamSynchronize");
        if (!b.bw_xe || b.bw_cap < need) {
            cudaFree(b.bw_xe);
            b.bw_xe = nullptr;
            b.bw_cap = 0;
            b.bw_xe_stride = L.Dh + need;
            if ((e = dalloc(&b.bw_xe, (size_t)D * b.bw_xe_stride)) != cudaSuccess) return oom(e);
            b.bw_cap = need;
        }
        if (need_ckpt && b.ckpt_cap < nc) {
            cudaFree(b.ckpt);
            b.ckpt = nullptr;
            b.ckpt_cap = 0;
            if ((e = dalloc(&b.ckpt, (size_t)nc * D * L.n_slots)) != cudaSuccess) return oom(e);
            b.ckpt_cap = nc;
        }
    }
    if (!b.bw_state) {
        if ((e = dalloc(&b.bw_state, (size_t)D * L.n_slots)) != cudaSuccess) return oom(e);
    }
    // time segments (options.time_segments, or enough CTAs for about four
    // waves of 16 warps per SM, at most 16).  Reverse form: whole checkpoint
    // intervals for the reverse pass and the input-gradient pass.  Tangent
    // form: only the input-gradient pass is segmented, in whole 256-sample
    // chunks (every segment but the last warms up over Dh samples; measured
    // on the 256 x 200-filter bank: 4 segments 6.09 ms per backward, 6: 6.05,
    // 10: 5.65, 16: 5.74, 32: 6.08).
    const int W7 = L.G == 16 ? b.adj_W7 : (b.adj_W7 + 1) / 2;
    int P = 1;
    int64_t S7 = 0;   // input-gradient segment length (tangent form)
    {
        const int64_t warps = b.adj_n_units * b.adj_W;
        const int req = p->opt.time_segments;
        if (req >= 1) P = req;
        else P = (int)std::min<int64_t>(16, std::max<int64_t>(1, (64 * (int64_t)p->n_sm + warps - 1) / warps));
        if (tangent) {
            const int64_t chunks = (n + spiir::kK7Chunk - 1) / spiir::kK7Chunk;
            P = (int)std::max<int64_t>(1, std::min<int64_t>(P, chunks));
            S7 = ((chunks + P - 1) / P) * spiir::kK7Chunk;
            P = (int)((n + S7 - 1) / S7);
        } else {
            P = (int)std::max<int64_t>(1, std::min<int64_t>(P, nc));
        }
    }
    const int64_t cps = tangent ? 0 : (nc + P - 1) / P;
    if (!tangent) P = (int)((nc + cps - 1) / cps);
    if (b.adj_seg_cap < P) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamSynchronize");
        cudaFree(b.acc);
        cudaFree(b.adj_E);
        cudaFree(b.adj_mu);
        cudaFree(b.adj_seeds);
        b.acc = nullptr;
        b.adj_E = b.adj_mu = b.adj_seeds = nullptr;
        b.adj_seg_cap = 0;
        if ((e = dalloc(&b.acc, (size_t)P * D * L.n_slots * 6)) != cudaSuccess ||
            (e = dalloc(&b.adj_E, (size_t)P * D * L.n_slots)) != cudaSuccess ||
            (e = dalloc(&b.adj_mu, (size_t)P * D * L.n_slots)) != cudaSuccess ||
            (e = dalloc(&b.adj_seeds, (size_t)P * D * L.n_slots)) != cudaSuccess)
            return oom(e);
        b.adj_seg_cap = P;
    }
    // zero history + x (and, for the reverse form, zero state and accumulators), zero g_x
    if ((e = cudaMemset2DAsync(b.bw_xe, b.bw_xe_stride * 4, 0, (size_t)L.Dh * 4, D, s)) !=
            cudaSuccess ||
        (e = cudaMemcpy2DAsync(b.bw_xe + L.Dh, b.bw_xe_stride * 4, x_dev, n * 4, n * 4, D,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
        (!tangent &&
         (e = cudaMemsetAsync(b.bw_state, 0, sizeof(float2) * (size_t)D * L.n_slots, s)) !=
             cudaSuccess) ||
        ((!tangent || grad_x_dev) &&
         (e = cudaMemsetAsync(b.acc, 0, sizeof(float) * 6 * (size_t)P * D * L.n_slots, s)) !=
             cudaSuccess) ||
        (grad_x_dev &&
         (e = cudaMemsetAsync(grad_x_dev, 0, sizeof(float) * (size_t)D * n, s)) != cudaSuccess))
        return cuda_fail(e, "adjoint staging");
    p->last_launches = 0;
    if (grad_x_dev &&
        spiir::k7_smem_bytes(L.Dh, L.G == 16 ? b.adj_W7 : (b.adj_W7 + 1) / 2, L.G) > 227 * 1024)
        return fail(SPIIR_EUNSUPPORTED, "adjoint windows above 227 KB of shared memory");
    spiir::K6Args a{};
    a.seeds = (P > 1 && grad_x_dev) ? b.adj_seeds : nullptr;
    const bool overlap = tangent && grad_x_dev != nullptr;
    int t_all = -1;   // one timed window around both passes when they overlap
    if (overlap) {
        if (!p->aux &&
            ((e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking)) != cudaSuccess ||
             (e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
             (e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming)) != cudaSuccess))
            return cuda_fail(e, "adjoint stream");
        t_all = time_begin(p, s);
    }
    if (tangent) {
        // g_a, g_b: one forward pass of the derivative recurrences
        spiir::KTArgs t{};
        t.xe = b.bw_xe;
        t.xe_stride = b.bw_xe_stride;
        t.n = (int32_t)n;
        t.Dh = L.Dh;
        t.Tb = L.Tb;
        // filter pairs per lane when that still gives >= 12 warps per SM (with
        // fewer, one filter per lane hides latency better: measured on the
        // 256 x 200-filter bank, 5.4 warps per SM at pairs, 5.96 vs 5.64 ms)
        t.nf = (b.kt_n_pos[1] / 64) * D >= 12 * (int64_t)p->n_sm ? 2 : 1;
        t.W = tangent_warps_per_cta(b.kt_n_pos[t.nf - 1] / (32 * t.nf), D, L.Dh, L.Tb, p->n_sm);
        t.gz = reinterpret_cast<const float2 *>(grad_z_dev);
        t.T = p->T;
        t.lanes = b.kt_lanes[t.nf - 1];
        t.warp_tmpl = b.kt_warp_tmpl[t.nf - 1];
        t.n_pos = b.kt_n_pos[t.nf - 1];
        t.params = b.params;
        t.ringoff = b.ringoff;
        t.n_slots = L.n_slots;
        t.acc = b.acc;
        t.with_gb = grad_x_dev == nullptr;   // else the input-gradient pass sums g_b
        if (overlap) {
            // forked onto the plan's second stream: runs beside the
            // input-gradient pass (one limited by issue latency, the other by
            // shared memory); joined before the finalize
            if ((e = cudaEventRecord(p->ev_fork, s)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0)) != cudaSuccess ||
                (e = spiir::launch_kt(t, D, p->aux)) != cudaSuccess ||
                (e = cudaEventRecord(p->ev_join, p->aux)) != cudaSuccess)
                return cuda_fail(e, "tangent adjoint launch");
        } else {
            const int tt = time_begin(p, s);
            if ((e = spiir::launch_kt(t, D, s)) != cudaSuccess)
                return cuda_fail(e, "tangent adjoint launch");
            time_end(p, s, tt, kTimeAdj);
        }
        p->last_launches += 1;
    } else {
        // forward pass from zero state, keeping the state every Cc samples
        spiir::K1Args f{};
        f = k1_args(p, b, n, nullptr, n, false);
        f.mode = spiir::kModePlain;   // checkpoints come from the FP32 recurrence
        f.xe = b.bw_xe;
        f.xe_stride = b.bw_xe_stride;
        f.state = b.bw_state;
        f.t0 = 0;
        f.ckpt = b.ckpt;
        f.ckpt_blocks = Cc / L.Tb;
        f.n_det = D;
        // the forward also keeps the state at every 16-sample span start when that
        // fits a quarter of free memory (at most 8 GiB): the reverse pass then
        // skips its per-chunk recompute
        {
            const int64_t want = ((n + 15) / 16) * D * L.n_slots;
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
            const int64_t budget = std::min<int64_t>((int64_t)8 << 30, (int64_t)(free_b / 4));
            if (b.adj_sub16_cap < want && want * (int64_t)sizeof(float2) <= budget) {
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
                    return cuda_fail(e, "cudaStreamSynchronize");
                cudaFree(b.adj_sub16);
                b.adj_sub16 = nullptr;
                b.adj_sub16_cap = 0;
                if (dalloc(&b.adj_sub16, (size_t)want) == cudaSuccess) b.adj_sub16_cap = want;
                else (void)cudaGetLastError();   // fall back to the per-chunk recompute
            }
            f.sub16 = (b.adj_sub16_cap >= want && p->precision == SPIIR_PREC_PLAIN) ? b.adj_sub16
                                                                                     : nullptr;
        }
        if (p->precision == SPIIR_PREC_PLAIN) {
            // time-segmented like a plain call when the bank is small (checkpoints
            // are written at whole intervals from the call's start either way)
            const int saved = p->last_segments;
            spiir_status st = launch_segmented(p, b, f, segments_for(p, b, n), s);
            p->last_segments = saved;
            if (st != SPIIR_OK) return st;
        } else {
            const int tf = time_begin(p, s);
            if ((e = spiir::launch_k1(f, L.n_units(), L.smem_bytes(), s)) != cudaSuccess)
                return cuda_fail(e, "adjoint forward launch");
            time_end(p, s, tf, kTimeK1);
            p->last_launches += 1;
        }
        // reverse pass: projection of the adjoint state to segment ends, then
        // every segment's reverse pass at once
        if ((e = spiir::launch_adj_project(b.params, b.adj_slot_tmpl,
                                           reinterpret_cast<const float2 *>(grad_z_dev), L.n_slots,
                                           D, p->T, n, cps * Cc, 0, P, b.adj_E, b.adj_mu, s)) !=
            cudaSuccess)
            return cuda_fail(e, "adjoint projection launch");
        const int64_t sub_need = (int64_t)P * b.adj_n_units * b.adj_W * spiir::kAdjRounds *
                                 (Cc / spiir::kAdjSub) * 32;
        if (b.adj_sub_cap < sub_need) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(b.adj_sub);
            b.adj_sub = nullptr;
            if ((e = dalloc(&b.adj_sub, (size_t)sub_need)) != cudaSuccess) return oom(e);
            b.adj_sub_cap = sub_need;
        }
        a.xe = b.bw_xe;
        a.xe_stride = b.bw_xe_stride;
        a.n = (int32_t)n;
        a.Dh = L.Dh;
        a.W = b.adj_W;
        a.Cc = Cc;
        a.gz = reinterpret_cast<const float2 *>(grad_z_dev);
        a.T = p->T;
        a.units = b.adj_units;
        a.tasks = b.adj_tasks;
        a.round_stride = L.W * 32;
        a.G = L.G;
        a.params = b.params;
        a.ringoff = b.ringoff;
        a.ckpt = b.ckpt;
        a.n_slots = L.n_slots;
        a.n_det = D;
        a.acc = b.acc;
        a.sub = b.adj_sub;
        a.n_units = (int32_t)b.adj_n_units;
        a.cps = (int32_t)cps;
        a.P = P;
        a.sub16 = f.sub16;
        a.mu_end = P > 1 ? b.adj_mu : nullptr;
        if (spiir::k6_smem_bytes(Cc, L.Dh) > 227 * 1024)
            return fail(SPIIR_EUNSUPPORTED, "adjoint windows above 227 KB of shared memory");
        const int ta = time_begin(p, s);
        if ((e = spiir::launch_k6(a, b.adj_n_units, s)) != cudaSuccess)
            return cuda_fail(e, "adjoint kernel launch");
        time_end(p, s, ta, kTimeAdj);
        // projection (+ carry), reverse pass
        p->last_launches += (P > 1 ? 2 : 1) + 1;
    }
    if (grad_x_dev) {
        // input gradient in the shifted frame; its segment seeds come from the
        // reverse pass, or (tangent form) from its own projection + carry
        spiir::K7Args g{};
        g.gz = reinterpret_cast<const float2 *>(grad_z_dev);
        g.T = p->T;
        g.n = (int32_t)n;
        g.Dh = L.Dh;
        g.S = (int32_t)(tangent ? S7 : cps * Cc);
        g.P = P;
        g.tasks = b.adj_tasks;
        g.units = b.adj_units7;
        g.n_units = (int32_t)b.adj_n_units7;
        g.W = W7;
        g.round_stride = L.W * 32;
        g.G = L.G;
        g.params = b.params;
        g.ringoff = b.ringoff;
        g.n_slots = L.n_slots;
        g.n_det = D;
        g.seeds = a.seeds;
        g.gx = grad_x_dev;
        const int tg = overlap ? -1 : time_begin(p, s);
        if (tangent) {
            // seeds: mu at (q + 1) S + Dh from the reverse projection over
            // segments shifted by Dh; the pass also sums g_b
            if ((e = spiir::launch_adj_project(b.params, b.adj_slot_tmpl, g.gz, L.n_slots, D,
                                               p->T, n, g.S, L.Dh, P, b.adj_E, b.adj_seeds, s)) !=
                cudaSuccess)
                return cuda_fail(e, "input-gradient projection launch");
            g.seeds = P > 1 ? b.adj_seeds : nullptr;
            g.xe = b.bw_xe;
            g.xe_stride = b.bw_xe_stride;
            g.acc = b.acc;
            p->last_launches += P > 1 ? 2 : 1;
        }
        if ((e = spiir::launch_k7(g, s)) != cudaSuccess)
            return cuda_fail(e, "adjoint input-gradient launch");
        time_end(p, s, tg, kTimeAdj);
        p->last_launches += 1;
    }
    if (overlap) {
        if ((e = cudaStreamWaitEvent(s, p->ev_join, 0)) != cudaSuccess)
            return cuda_fail(e, "adjoint join");
        time_end(p, s, t_all, kTimeAdj);
    }
    if ((e = spiir::launch_adj_finalize(b.acc, b.slot_filter, L.n_slots, D,
                                        (tangent && !grad_x_dev) ? 1 : P,
                                        reinterpret_cast<float2 *>(grad_a_dev),
                                        reinterpret_cast<float2 *>(grad_b_dev), s)) !=
        cudaSuccess)
        return cuda_fail(e, "adjoint finalize launch");
    p->last_launches += 1;
    return SPIIR_OK;
}

spiir_status spiir_set_coefficients(spiir_plan *p, const float *a_reim_dev,
                                    const float *b_reim_dev, void *stream)
{
    if (!p || !a_reim_dev || !b_reim_dev) return fail(SPIIR_EINVAL, "NULL argument");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no device coefficients");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    for (Band &b : p->bands) {
        cudaError_t e = spiir::launch_set_coefficients(
            reinterpret_cast<const float2 *>(a_reim_dev),
            reinterpret_cast<const float2 *>(b_reim_dev), b.slot_filter, b.lay.n_slots, b.params,
            (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "coefficient update launch");
        b.tc_valid = false;   // projection weights are rebuilt on the next segmented call
    }
    return SPIIR_OK;
}

spiir_status spiir_state_get(spiir_plan *p, float *state, float *history, int64_t *samples)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no state");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (state) {
        std::memset(state, 0, sizeof(float) * 2 * (size_t)p->D * p->Ltot);
        for (const Band &b : p->bands) {
            const spiir::Layout &L = b.lay;
            std::vector<float> dev((size_t)2 * p->D * L.n_slots);
            if (p->precision == SPIIR_PREC_PLAIN) {
                e = cudaMemcpy(dev.data(), b.state, dev.size() * sizeof(float),
                               cudaMemcpyDeviceToHost);
            } else {  // 16-byte extended state, rounded to complex64
                std::vector<double2> ext((size_t)p->D * L.n_slots);
                e = cudaMemcpy(ext.data(), b.state_ext, ext.size() * sizeof(double2),
                               cudaMemcpyDeviceToHost);
                for (size_t i = 0; i < ext.size(); ++i) {
                    if (p->precision == SPIIR_PREC_COMPENSATED) {
                        const float4 v = *reinterpret_cast<const float4 *>(&ext[i]);
                        dev[2 * i] = v.x + v.y;
                        dev[2 * i + 1] = v.z + v.w;
                    } else {
                        dev[2 * i] = (float)ext[i].x;
                        dev[2 * i + 1] = (float)ext[i].y;
                    }
                }
            }
            if (e != cudaSuccess) return cuda_fail(e, "state copy");
            for (int det = 0; det < p->D; ++det)
                for (int64_t s = 0; s < L.n_slots; ++s) {
                    const int64_t f = L.slot_filter[s];
                    if (f < 0) continue;
                    const float u = dev[2 * ((size_t)det * L.n_slots + s)];
                    const float v = dev[2 * ((size_t)det * L.n_slots + s) + 1];
                    const bool swapped = (s & 1) != 0;  // odd lane: (im, re) order
                    state[2 * ((size_t)det * p->Ltot + f)] = swapped ? v : u;
                    state[2 * ((size_t)det * p->Ltot + f) + 1] = swapped ? u : v;
                }
        }
    }
    if (history) {
        const Band &b = p->bands[p->top];
        e = cudaMemcpy(history, b.hist, sizeof(float) * (size_t)p->D * b.lay.Dh,
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "history copy");
    }
    if (samples) {
        e = cudaMemcpy(samples, p->t0_dev, sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "sample counter copy");
    }
    return SPIIR_OK;
}

spiir_status spiir_state_set(spiir_plan *p, const float *state, const float *history,
                             int64_t samples)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan has no state");
    if (samples < 0) return fail(SPIIR_EINVAL, "samples must be >= 0");
    for (const Band &b : p->bands)
        if (b.fir_len > 0)
            return fail(SPIIR_EUNSUPPORTED, "state import with band front-end FIRs (their "
                                            "top-rate history is not part of the state)");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (state) {
        for (Band &b : p->bands) {
            const spiir::Layout &L = b.lay;
            std::vector<float> dev((size_t)2 * p->D * L.n_slots, 0.f);
            for (int det = 0; det < p->D; ++det)
                for (int64_t s = 0; s < L.n_slots; ++s) {
                    const int64_t f = L.slot_filter[s];
                    if (f < 0) continue;
                    const float re = state[2 * ((size_t)det * p->Ltot + f)];
                    const float im = state[2 * ((size_t)det * p->Ltot + f) + 1];
                    const bool swapped = (s & 1) != 0;
                    dev[2 * ((size_t)det * L.n_slots + s)] = swapped ? im : re;
                    dev[2 * ((size_t)det * L.n_slots + s) + 1] = swapped ? re : im;
                }
            if (p->precision == SPIIR_PREC_PLAIN) {
                e = cudaMemcpy(b.state, dev.data(), dev.size() * sizeof(float),
                               cudaMemcpyHostToDevice);
            } else {  // extended state from complex64 (low parts zero)
                std::vector<double2> ext((size_t)p->D * L.n_slots);
                for (size_t i = 0; i < ext.size(); ++i) {
                    if (p->precision == SPIIR_PREC_COMPENSATED)
                        *reinterpret_cast<float4 *>(&ext[i]) =
                            make_float4(dev[2 * i], 0.f, dev[2 * i + 1], 0.f);
                    else
                        ext[i] = make_double2(dev[2 * i], dev[2 * i + 1]);
                }
                e = cudaMemcpy(b.state_ext, ext.data(), ext.size() * sizeof(double2),
                               cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) return cuda_fail(e, "state copy");
        }
    }
    if (history) {
        Band &b = p->bands[p->top];
        e = cudaMemcpy(b.hist, history, sizeof(float) * (size_t)p->D * b.lay.Dh,
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "history copy");
    }
    p->t0 = samples;
    e = cudaMemcpy(p->t0_dev, &samples, sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "sample counter copy");
    return SPIIR_OK;
}

spiir_status spiir_kernel_times(spiir_plan *p, double *ms_out, int64_t *n_out)
{
    if (!p || !ms_out) return fail(SPIIR_EINVAL, "plan or ms is NULL");
    double t[SPIIR_KERNEL_CLASSES] = {0.0, 0.0, 0.0};
    int64_t c[SPIIR_KERNEL_CLASSES] = {0, 0, 0};
    if (p->device >= 0 && !p->ev_used.empty()) {
        DeviceGuard guard(p->device);
        if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
        for (const auto &u : p->ev_used) {
            cudaError_t e = cudaEventSynchronize(p->ev_pool[(size_t)u.first + 1]);
            float ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, p->ev_pool[(size_t)u.first],
                                         p->ev_pool[(size_t)u.first + 1]);
            if (e != cudaSuccess) {
                p->ev_used.clear();
                return cuda_fail(e, "kernel timing events");
            }
            t[u.second] += ms;
            c[u.second] += 1;
        }
    }
    p->ev_used.clear();
    for (int k = 0; k < SPIIR_KERNEL_CLASSES; ++k) {
        ms_out[k] = t[k];
        if (n_out) n_out[k] = c[k];
    }
    return SPIIR_OK;
}

spiir_status spiir_check(spiir_plan *p, void *stream)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return SPIIR_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int32_t word = 0;
    e = cudaMemcpy(&word, p->err, sizeof(word), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "error word copy");
    if (word & (1 | 2 | 8)) return fail(SPIIR_ETIMEOUT, "a bounded device wait gave up (error word " +
                                                  std::to_string(word) + ")");
    if (word) return fail(SPIIR_ECUDA, "device error word " + std::to_string(word));
    return SPIIR_OK;
}

spiir_status spiir_selftest_bounded_wait(spiir_plan *p, uint64_t limit_ns, void *stream)
{
    if (!p) return fail(SPIIR_EINVAL, "plan is NULL");
    if (p->device < 0) return fail(SPIIR_EINVAL, "host-only plan");
    if (limit_ns == 0 || limit_ns > 10000000000ull)
        return fail(SPIIR_EINVAL, "limit_ns must be in (0, 1e10]");
    DeviceGuard guard(p->device);
    if (!guard.ok) return cuda_fail(guard.err, "cudaSetDevice");
    cudaError_t e = spiir::launch_bounded_wait_probe(p->err, limit_ns, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    return SPIIR_OK;
}

}  // extern "C"
