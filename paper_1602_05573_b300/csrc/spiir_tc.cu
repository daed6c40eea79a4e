// Tensor-core projection of segment start states (split-BF16 tcgen05 GEMM +
// chunk scan) for time-segmented filter calls.
//
// A call split into time segments needs every filter's state at each
// segment start.  With chunks of T = 256 samples, the zero-state response of
// filter l over chunk c is (section "GPU accelerated SPIIR method",
// subsection "SPIIR method": the single-pole recurrence summed in closed form)
//     S_l(c) = sum_{j<T} a_l^{T-1-j} b_l x[cT + j - d_l],
// and the states follow the chunk recurrence s_l(c+1) = a_l^T s_l(c) + S_l(c).
// Writing d_l = q_l T + r_l, S_l(c) = G_l(c - q_l - 1) with the delay-free
// window product
//     G_l(c'') = sum_{m<2T} V_l[m] x[c''T + m],
//     V_l[m]   = a_l^{2T-1-r_l-m} b_l  for T - r_l <= m < 2T - r_l, else 0,
// which for all filters and windows is one dense GEMM: rows (Re V_l, Im V_l),
// K = 2T, one column per window.  It runs on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, BF16 operands, FP32 accumulate in TMEM) with each
// operand split in two BF16 parts, hi + lo, and three products
// hi*hi + hi*lo + lo*hi (~2^-16 relative per term).  The epilogue warps read
// their accumulator rows from TMEM and run the chunk recurrence over the
// columns in order, in FP32 (the recurrence contracts by |a|^T per chunk, so
// rounding does not grow along it), writing the state at each segment start.
//
// Both operands sit in shared memory in the tensor cores' layout (K-major,
// no swizzle: 8-row x 16-byte core matrices, K-direction core stride 128 B,
// row-group stride 1024 B, 128 x 64 tiles of 16 KB).  The strain windows
// are staged in HBM in that layout by tc_strain_kernel and arrive by 1-D TMA
// bulk copies; the weights are never stored: per stage, generator warps
// build the CTA's 128 x 64 weight tile from a per-slot table of starting
// powers (a^p b for the smallest power p of each 32-wide m-group, FP64
// rounded once), walking down in m with one complex FP32 multiply by a per
// sample (at most 31 steps from a seed, ~2e-6 relative worst case, below
// the ~8e-6 of the split-BF16 representation), and split each value in
// BF16 hi/lo.  One CTA serves 128 GEMM rows (64 filter slots) of one
// detector for the whole call, 256 windows per accumulator (N = 256):
// warp 4 issues the copies (two stages) and the MMAs, warps 5-8 generate
// the weight tiles, warps 0-3 own TMEM lanes 0-127 and scan.
#include "spiir_kernels.h"
#include "spiir_ptx.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cstdint>

namespace spiir {

namespace {

constexpr int kRowsTile = 128;                  // GEMM rows per CTA (64 slots x re/im)
constexpr int kColsTile = 256;                  // windows per strain tile in HBM
constexpr int kKBlk = 64;                       // K per staged block
constexpr int kKBlocks = kTcK / kKBlk;          // 8
constexpr uint32_t kTileBytes = 128u * kKBlk * 2u;   // 16 KB: 128 rows x 64 BF16 (A)
constexpr uint32_t kBTileBytes = (uint32_t)kColsTile * kKBlk * 2u;   // B: 256 rows x 64
// pipeline stages of (A, B) tiles: 192 KB of shared memory either way
template <int NT> __host__ __device__ constexpr int stages_for() { return NT == 128 ? 3 : 2; }
constexpr int kMaxStages = 3;
constexpr int kEpiThreads = 128;

// byte offset of element (row, k) inside a 128 x 64 tile
__host__ __device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bf16_val(uint16_t b)
{
    return __bfloat162float(__ushort_as_bfloat16(b));
}
// v = hi + lo with hi, lo in BF16
__device__ __forceinline__ void split_bf16(float v, uint16_t &hi, uint16_t &lo)
{
    hi = bf16_bits(v);
    lo = bf16_bits(v - bf16_val(hi));
}
// the same split of two values at once: hi and lo words hold (v0, v1) as
// BF16 pairs, v0 in the low half
__device__ __forceinline__ void split_bf16x2(float v0, float v1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
    hi = *reinterpret_cast<const uint32_t *>(&h2);
    const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(v0 - h0, v1 - h1);
    lo = *reinterpret_cast<const uint32_t *>(&l2);
}

// ---- float-float (hi + lo) arithmetic on the FP32 pipe ---------------------
// Error-free transformations (Knuth's two-sum, the FMA two-product) keep the
// carried state to ~2^-44 relative at FP32-pipe speed; B300's FP64 pipe is
// a small fraction of its FP32 rate.
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_from(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ ff ff_renorm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ff_renorm(p, e);
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    return ff_renorm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }

// ---- weight seeds: per slot and 32-wide m-group, V_l at the group's largest
// valid m.  V_l[m] = a^(2T-1-r-m) b for T - r <= m < 2T - r (r = d mod T),
// else 0 (kernel form: odd lanes hold conj(a) and (Im b, Re b), which the
// projection keeps).  One thread per (slot, group): a^p by binary powering in
// FP64, times b, rounded once; the group-0 thread also writes a^T.
constexpr int kSeedGroup = 32;                  // m per seed (one walk)

__host__ __device__ __forceinline__ void cpow64(double ar, double ai, int e, double &rr,
                                                double &ri)
{
    double br = ar, bi = ai;
    rr = 1.0;
    ri = 0.0;
    for (; e > 0; e >>= 1) {
        if (e & 1) {
            const double t = rr * br - ri * bi;
            ri = rr * bi + ri * br;
            rr = t;
        }
        const double t = br * br - bi * bi;
        bi = 2.0 * br * bi;
        br = t;
    }
}

__global__ void tc_seeds_kernel(const float4 *params, const int2 *ringoff, int64_t n_slots,
                                int Dh, float2 *seed, float2 *aT, double2 *aT64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots * kTcSeeds) return;
    const int64_t s = i / kTcSeeds;
    const int g = (int)(i % kTcSeeds);
    const float4 p = params[s];
    const int r = (Dh - ringoff[s].x) % kTcT;
    const int m_hi = min(g * kSeedGroup + kSeedGroup - 1, 2 * kTcT - r - 1);
    const int m_lo = max(g * kSeedGroup, kTcT - r);
    float2 v = make_float2(0.f, 0.f);
    if (m_lo <= m_hi) {
        double rr, ri;
        cpow64(p.x, p.y, 2 * kTcT - 1 - r - m_hi, rr, ri);
        v = make_float2((float)(rr * p.z - ri * p.w), (float)(rr * p.w + ri * p.z));
    }
    seed[i] = v;
    if (g == 0) {   // a^T, FP64 then rounded once
        double rr, ri;
        cpow64(p.x, p.y, kTcT, rr, ri);
        aT[s] = make_float2((float)rr, (float)ri);
        aT64[s] = make_double2(rr, ri);
    }
}

// ---- strain windows: B[col][m] = x[(col + col0) T + m], split in BF16 ------
// xe holds [Dh history | n call samples] per detector (call sample k at
// Dh + k); samples outside [-Dh, n) read as zero.
__global__ void tc_strain_kernel(const float *xe, int64_t xe_stride, int Dh, int64_t n, int D,
                                 int64_t n_cols_pad, int col0, unsigned char *B)
{
    const int64_t per_det = n_cols_pad * (kTcK / 8);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per_det * D) return;
    const int det = (int)(i / per_det);
    const int64_t col = (i % per_det) / (kTcK / 8);
    const int m0 = (int)(i % (kTcK / 8)) * 8;
    const int64_t k0 = (col + col0) * (int64_t)kTcT + m0;   // call sample of m0
    const float *row = xe + (int64_t)det * xe_stride + Dh;
    uint16_t h[8], l[8];
    for (int j = 0; j < 8; ++j) {
        const int64_t k = k0 + j;
        const float v = (k >= -(int64_t)Dh && k < n) ? row[k] : 0.f;
        split_bf16(v, h[j], l[j]);
    }
    const int64_t nt = col / kColsTile;
    const int rl = (int)(col % kColsTile);
    const int kb = m0 / kKBlk, kl = m0 % kKBlk;
    const int64_t n_ntiles = n_cols_pad / kColsTile;
    unsigned char *base =
        B + (((int64_t)det * n_ntiles + nt) * kKBlocks + kb) * 2 * (int64_t)kBTileBytes;
    uint4 v;
    v.x = h[0] | ((uint32_t)h[1] << 16); v.y = h[2] | ((uint32_t)h[3] << 16);
    v.z = h[4] | ((uint32_t)h[5] << 16); v.w = h[6] | ((uint32_t)h[7] << 16);
    *reinterpret_cast<uint4 *>(base + tile_off(rl, kl)) = v;
    v.x = l[0] | ((uint32_t)l[1] << 16); v.y = l[2] | ((uint32_t)l[3] << 16);
    v.z = l[4] | ((uint32_t)l[5] << 16); v.w = l[6] | ((uint32_t)l[7] << 16);
    *reinterpret_cast<uint4 *>(base + kBTileBytes + tile_off(rl, kl)) = v;
}

// ---- tcgen05 helpers -------------------------------------------------------
// Shared-memory matrix descriptor, K-major without swizzle: start address,
// K-direction core-matrix stride (leading byte offset), row-group stride
// (stride byte offset), descriptor version 1 (bits 46-48 = 0b001).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24.
template <int NT> __host__ __device__ constexpr uint32_t idesc_for()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
           ((uint32_t)(kRowsTile >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// ---- projection: GEMM tile loop + chunk scan ---------------------------------
// ANCH = false: FP32 scan from the call's start state, states written at the
// segment starts (segmented plain calls).  ANCH = true: float-float scan
// (~2^-44 relative, FP64-class) from the carried FP64 state over chunks
// [c_first, c_end), the state before every chunk written as its anchor
// (rounded to FP32) and the state after the last written back in FP64 (the
// chunked tensor-core precision form).
// NT: windows per accumulator (N of the MMA): 256, or 128 for calls with few
// windows (the strain tiles in HBM are 256 wide; a 128-wide column tile is
// one half of one).
// Generator thread t of the CTA's M-tile mt: slot 64 mt + (t & 63), the
// 32-wide half (t >> 6) of each K-block.  V at m = 32 g + 31 - i (i = 0..31
// from the group's top) is seed a^(i - i0) for the valid m (i >= i0, the
// seed's position); four independent chains, one per i mod 4, each start at
// seed a^e (e = 0..3, the chain's first valid position) and step by a^4, so
// a walk is 8 dependent complex multiplies, not 32.  Values are written as
// BF16 hi/lo into the stage's A tiles (rows 2 s and 2 s + 1 = Re and Im),
// two per packed conversion.
struct WeightGen {
    int64_t slot;
    int sl, h, r;
    bool valid;
    float ar, ai, a2r, a2i, a3r, a3i, a4r, a4i;   // a^1..a^4 (kernel form), FP64 rounded once

    __device__ __forceinline__ void init(const TcArgs &A, int64_t mt, int t)
    {
        sl = t & 63;
        h = t >> 6;
        slot = mt * (kRowsTile / 2) + sl;
        valid = slot < A.n_slots;
        r = 0;
        ar = ai = a2r = a2i = a3r = a3i = a4r = a4i = 0.f;
        if (valid) {
            const float4 p = A.params[slot];
            r = (A.Dh - A.ringoff[slot].x) % kTcT;
            double pr, pi;
            ar = p.x;
            ai = p.y;
            cpow64(p.x, p.y, 2, pr, pi);
            a2r = (float)pr;
            a2i = (float)pi;
            cpow64(p.x, p.y, 3, pr, pi);
            a3r = (float)pr;
            a3i = (float)pi;
            cpow64(p.x, p.y, 4, pr, pi);
            a4r = (float)pr;
            a4i = (float)pi;
        }
    }
    // seed of generator thread t's slot in M-tile mt, K-block kb
    static __device__ __forceinline__ float2 seed_at(const TcArgs &A, int64_t mt, int t, int kb)
    {
        const int64_t sl = mt * (kRowsTile / 2) + (t & 63);
        return sl < A.n_slots ? A.seed[sl * kTcSeeds + 2 * kb + (t >> 6)] : make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void gen(int kb, float2 sd, unsigned char *stage) const
    {
        const int g = 2 * kb + h;
        int m_lo = 1, m_hi = 0;   // valid m of this group (empty by default)
        if (valid) {
            m_hi = min(g * kSeedGroup + kSeedGroup - 1, 2 * kTcT - r - 1);
            m_lo = max(g * kSeedGroup, kTcT - r);
        }
        const int i0 = g * kSeedGroup + kSeedGroup - 1 - m_hi;   // >= 0 when valid
        // seed a^e, e = 0..3
        const float s1r = __fmaf_rn(sd.x, ar, -__fmul_rn(sd.y, ai)), s1i = __fmaf_rn(sd.x, ai, __fmul_rn(sd.y, ar));
        const float s2r = __fmaf_rn(sd.x, a2r, -__fmul_rn(sd.y, a2i)), s2i = __fmaf_rn(sd.x, a2i, __fmul_rn(sd.y, a2r));
        const float s3r = __fmaf_rn(sd.x, a3r, -__fmul_rn(sd.y, a3i)), s3i = __fmaf_rn(sd.x, a3i, __fmul_rn(sd.y, a3r));
        float cr[4], ci[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = (k - i0) & 3;
            cr[k] = e == 0 ? sd.x : e == 1 ? s1r : e == 2 ? s2r : s3r;
            ci[k] = e == 0 ? sd.y : e == 1 ? s1i : e == 2 ? s2i : s3i;
        }
        const int row = 2 * sl;
        const int k0 = h * kSeedGroup;   // k of m = 32 g inside the K-block
        // eight k at a time, from the top of the group down
#pragma unroll
        for (int q = kSeedGroup / 8 - 1; q >= 0; --q) {
            float vr[8], vi[8];
#pragma unroll
            for (int j = 7; j >= 0; --j) {
                const int m = g * kSeedGroup + 8 * q + j;
                const int k = 3 - (j & 3);   // chain of position i = 31 - 8 q - j
                vr[j] = 0.f;
                vi[j] = 0.f;
                if (m >= m_lo && m <= m_hi) {
                    vr[j] = cr[k];
                    vi[j] = ci[k];
                    const float nr = __fmaf_rn(cr[k], a4r, -__fmul_rn(ci[k], a4i));
                    ci[k] = __fmaf_rn(cr[k], a4i, __fmul_rn(ci[k], a4r));
                    cr[k] = nr;
                }
            }
            uint32_t hr[4], lr[4], hi_[4], li[4];
#pragma unroll
            for (int p2 = 0; p2 < 4; ++p2) {
                split_bf16x2(vr[2 * p2], vr[2 * p2 + 1], hr[p2], lr[p2]);
                split_bf16x2(vi[2 * p2], vi[2 * p2 + 1], hi_[p2], li[p2]);
            }
            const int kl = k0 + 8 * q;
            *reinterpret_cast<uint4 *>(stage + tile_off(row, kl)) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
            *reinterpret_cast<uint4 *>(stage + kTileBytes + tile_off(row, kl)) =
                make_uint4(lr[0], lr[1], lr[2], lr[3]);
            *reinterpret_cast<uint4 *>(stage + tile_off(row + 1, kl)) =
                make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
            *reinterpret_cast<uint4 *>(stage + kTileBytes + tile_off(row + 1, kl)) =
                make_uint4(li[0], li[1], li[2], li[3]);
        }
    }
};

constexpr int kGenThreads = 128;
constexpr int kProjThreads = kEpiThreads + 32 + kGenThreads;

template <bool ANCH, int NT>
__global__ void __launch_bounds__(kProjThreads, 1) tc_project_kernel(const TcArgs A)
{
    constexpr uint32_t kBT = (uint32_t)NT * kKBlk * 2u;          // one B component
    constexpr uint32_t kSB = 2u * kTileBytes + 2u * kBT;          // stage bytes
    constexpr uint32_t kIdesc = idesc_for<NT>();
    constexpr int kStages = stages_for<NT>();
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[3 * kMaxStages + 4];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int det = blockIdx.y;
    // persistent CTAs: M-tiles blockIdx.x, + gridDim.x, ...; the column tiles
    // of consecutive M-tiles run back to back (tile u = i n_ntiles + nt of
    // the CTA's i-th M-tile), so one M-tile's last scan overlaps the next
    // one's MMAs
    const int64_t mtiles = (2 * A.n_slots + kRowsTile - 1) / kRowsTile;
    const int n_local = blockIdx.x < mtiles
                            ? (int)((mtiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    const uint32_t full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[kStages]);
    // generated weight tile of a stage written (all generator threads)
    const uint32_t wfull0 = smem_addr(&bars[2 * kStages + 4]);
    // two TMEM accumulators: the MMAs of column tile nt + 1 run while the
    // epilogue reads tile nt
    const uint32_t acc_full0 = smem_addr(&bars[2 * kStages]);
    const uint32_t acc_empty0 = smem_addr(&bars[2 * kStages + 2]);
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(empty0 + 8 * st, 1);
            mbar_init(wfull0 + 8 * st, kGenThreads);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full0 + 8 * b, 1);
            mbar_init(acc_empty0 + 8 * b, kEpiThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_addr(&tmem_slot)),
            "r"(2 * NT)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int n_ntiles = A.n_ntiles;
    const int total = n_local * n_ntiles * kKBlocks;   // K-blocks of this CTA
    auto mt_of = [&](int u) { return (int64_t)blockIdx.x + (int64_t)(u / n_ntiles) * gridDim.x; };
    bool ok = true;

    if (warp > 4) {
        // weight generators: stage it % kStages gets K-block it % kKBlocks once
        // the MMAs that read the stage before (block it - kStages) are done
        const int t = tid - kEpiThreads - 32;
        WeightGen wg;
        int64_t cur_mt = -1;
        float2 sd = total > 0 ? WeightGen::seed_at(A, mt_of(0), t, 0) : make_float2(0.f, 0.f);
        for (int it = 0; it < total; ++it) {
            const int st = it % kStages;
            const int64_t mt = mt_of(it / kKBlocks);
            if (mt != cur_mt) {
                wg.init(A, mt, t);
                cur_mt = mt;
            }
            // the next K-block's seed, loaded while this one is generated
            const float2 sd_next =
                it + 1 < total ? WeightGen::seed_at(A, mt_of((it + 1) / kKBlocks), t, (it + 1) % kKBlocks)
                               : sd;
            if (it >= kStages &&
                !mbar_wait(empty0 + 8 * st, (uint32_t)((it / kStages - 1) & 1), A.wait_limit_ns)) {
                atomicOr(A.err, 8);
                break;
            }
            wg.gen(it % kKBlocks, sd, smem + st * kSB);
            // generic-proxy writes, read next by the tensor cores (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(wfull0 + 8 * st);
            sd = sd_next;
        }
    } else if (warp == 4) {
        if (lane == 0) {
            // producer + MMA issue, two stages
            const unsigned char *bt =
                A.B + (int64_t)det * A.n_btiles * kKBlocks * 2 * kBTileBytes;
            auto fill = [&](int it) {
                const int st = it % kStages;
                const int nt = (it / kKBlocks) % n_ntiles, kb = it % kKBlocks;
                const uint32_t dst = smem_addr(smem) + st * kSB;
                const uint32_t full = full0 + 8 * st;
                mbar_expect_tx(full, 2u * kBT);
                // the strain tile holding windows [nt * NT, nt * NT + NT)
                const int64_t col0 = (int64_t)nt * NT;
                const unsigned char *src =
                    bt + ((col0 / kColsTile) * kKBlocks + kb) * 2 * kBTileBytes;
                if (NT == kColsTile) {
                    bulk_g2s(dst + 2 * kTileBytes, src, 2 * kBTileBytes, full);
                } else {   // rows of the half tile are the first or second kBT bytes
                    const uint32_t off = (uint32_t)((col0 % kColsTile) / NT) * kBT;
                    bulk_g2s(dst + 2 * kTileBytes, src + off, kBT, full);
                    bulk_g2s(dst + 2 * kTileBytes + kBT, src + kBTileBytes + off, kBT, full);
                }
            };
            // blocks it+1 .. it+kStages-1 are copied while the MMAs of block it
            // run; a stage is refilled once the MMAs that read it (block it-1)
            // have finished
            for (int f = 0; f < kStages - 1 && f < total; ++f) fill(f);
            for (int it = 0; it < total && ok; ++it) {
                const int st = it % kStages;
                const int u = it / kKBlocks, kb = it % kKBlocks;   // accumulator tile, K-block
                ok = mbar_wait(full0 + 8 * st, (uint32_t)((it / kStages) & 1), A.wait_limit_ns) &&
                     mbar_wait(wfull0 + 8 * st, (uint32_t)((it / kStages) & 1), A.wait_limit_ns);
                if (ok && kb == 0 && u >= 2)   // epilogue has read tile u - 2 (same TMEM)
                    ok = mbar_wait(acc_empty0 + 8 * (u & 1), (uint32_t)(((u - 2) >> 1) & 1),
                                   A.wait_limit_ns);
                if (!ok) break;
                tc_fence_after();
                const uint32_t s0 = smem_addr(smem) + st * kSB;
                const uint32_t acc = tmem + (uint32_t)((u & 1) * NT);
#pragma unroll
                for (int kk = 0; kk < kKBlk / 16; ++kk) {
                    const uint32_t adv = kk * 256u;   // 16 K = two core matrices
                    const uint64_t ah = umma_desc(s0 + adv), al = umma_desc(s0 + kTileBytes + adv);
                    const uint64_t bh = umma_desc(s0 + 2 * kTileBytes + adv);
                    const uint64_t bl = umma_desc(s0 + 2 * kTileBytes + kBT + adv);
                    umma_bf16(acc, ah, bh, kIdesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    umma_bf16(acc, ah, bl, kIdesc, 1u);
                    umma_bf16(acc, al, bh, kIdesc, 1u);
                }
                umma_commit(empty0 + 8 * st);          // stage free once these MMAs finish
                if (kb == kKBlocks - 1) umma_commit(acc_full0 + 8 * (u & 1));
                if (it + kStages - 1 < total) {
                    const int nx = it + kStages - 1, sx = nx % kStages;
                    if (nx >= kStages)
                        ok = mbar_wait(empty0 + 8 * sx, (uint32_t)((nx / kStages - 1) & 1),
                                       A.wait_limit_ns);
                    if (ok) fill(nx);
                }
            }
            if (!ok) atomicOr(A.err, 8);
        }
    } else {
        // epilogue: row = TMEM lane; rows 2s, 2s+1 are Re and Im of slot s
        const int row = warp * 32 + lane;
        const int comp = row & 1;
        for (int mi = 0; mi < n_local && ok; ++mi) {
        const int64_t mt = mt_of(mi * n_ntiles);
        const int64_t slot = mt * (kRowsTile / 2) + (row >> 1);
        const bool valid = slot < A.n_slots;
        const int64_t ds = (int64_t)det * A.n_slots + slot;
        float2 aT = make_float2(0.f, 0.f), s = make_float2(0.f, 0.f);
        ff aTr = {0.f, 0.f}, aTi = {0.f, 0.f};
        ff mine = {0.f, 0.f};   // ANCH: this thread's component of the carried state
        int q = 0;
        if (valid) {
            q = (A.Dh - A.ringoff[slot].x) / kTcT;
            if (ANCH) {
                const double2 a64 = A.aT64[slot];
                aTr = ff_from(a64.x);
                aTi = ff_from(a64.y);
                const double2 s64 = A.s64[ds];
                mine = ff_from(comp ? s64.y : s64.x);
            } else {
                aT = A.aT[slot];
                s = A.state[ds];
                if (comp == 0) A.seg_init[ds] = s;
            }
        }
        // global column col carries chunk c = col + cq of this row
        const int cq = A.col0 + q + 1;
        // the columns whose chunks this row's scan uses, [col_lo, col_hi), and
        // their union over the warp: 16-column groups outside it are skipped
        int col_lo = ANCH ? A.c_first - cq : -cq;
        int col_hi = ANCH ? A.c_end - cq : A.c_last + 1 - cq;
        if (!valid) {
            col_lo = INT_MAX;
            col_hi = INT_MIN;
        }
        const int w_lo = __reduce_min_sync(0xffffffffu, col_lo);
        const int w_hi = __reduce_max_sync(0xffffffffu, col_hi);
        // ANCH, two chunks per step: s(c+2) = A^2 s(c) + (A g(c) + g(c+1)),
        // A = a^T.  Per thread, the complex product's own component is
        // P_r x_mine + sigma P_i x_other (sigma = -1 for Re, +1 for Im).
        ff A2r = {0.f, 0.f}, sA2i = {0.f, 0.f}, saTi = {0.f, 0.f};
        float ar32 = 0.f, ai32 = 0.f;
        if (ANCH) {
            A2r = ff_add(ff_mul(aTr, aTr), ff_neg(ff_mul(aTi, aTi)));
            const ff p = ff_mul(aTr, aTi);
            const ff A2i = {2.f * p.h, 2.f * p.l};
            sA2i = comp ? A2i : ff_neg(A2i);
            saTi = comp ? aTi : ff_neg(aTi);
            ar32 = __fadd_rn(aTr.h, aTr.l);
            ai32 = __fadd_rn(aTi.h, aTi.l);
        }
        // non-ANCH: the next chunk after which a segment starts, and its index
        int nxt = A.cps - 1, seg_b = 1;
        // ANCH with odd cq: the last column of a group waits for its pair
        const int par = cq & 1;
        float pend = 0.f;
        int pend_c = A.c_end;   // no chunk (>= c_end)
        // one chunk: the anchor (state before chunk c), then the state advances
        // (ANCH: rows with en false only take part in the shuffles)
        auto step1 = [&](float g, int c, bool en = true) {
            if (ANCH) {
                // each thread advances its own component; the other one comes
                // from the partner lane (Re <-> Im)
                const ff other = {__shfl_xor_sync(0xffffffffu, mine.h, 1),
                                  __shfl_xor_sync(0xffffffffu, mine.l, 1)};
                if (en && valid && c >= A.c_first && c < A.c_end) {
                    const ff sr = comp ? other : mine, si = comp ? mine : other;
                    if (comp == 0)
                        A.anchors[(int64_t)(c - A.c_first) * A.D * A.n_slots + ds] =
                            make_float2(__fadd_rn(sr.h, sr.l), __fadd_rn(si.h, si.l));
                    if (c < A.c_full) {   // a partial last chunk only gets its anchor
                        // Re: aTr sr - aTi si + g;  Im: aTr si + aTi sr + g
                        const ff t = ff_add(ff_mul(aTr, mine), ff_mul(saTi, other));
                        mine = ff_add(t, ff{g, 0.f});
                    }
                }
            } else {
                const float other = __shfl_xor_sync(0xffffffffu, g, 1);
                const float gr = comp ? other : g, gi = comp ? g : other;
                if (valid && c >= 0 && c <= A.c_last) {
                    const float nr = fmaf(aT.x, s.x, fmaf(-aT.y, s.y, gr));
                    const float ni = fmaf(aT.x, s.y, fmaf(aT.y, s.x, gi));
                    s = make_float2(nr, ni);
                    if (c == nxt) {   // segment seg_b starts after chunk c
                        if (comp == 0) A.seg_init[((int64_t)seg_b * A.D + det) * A.n_slots + slot] = s;
                        nxt += A.cps;
                        ++seg_b;
                    }
                }
            }
        };
        for (int nt = 0; nt < n_ntiles; ++nt) {
            const int u = mi * n_ntiles + nt;
            ok = mbar_wait(acc_full0 + 8 * (u & 1), (uint32_t)((u >> 1) & 1), A.wait_limit_ns) &&
                 ok;
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int c0 = 0; c0 < NT; c0 += 16) {
                const int gcol = nt * NT + c0;
                if (gcol + 16 <= w_lo || gcol >= w_hi) continue;   // warp-uniform
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                    "%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) +
                          (uint32_t)((u & 1) * NT + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (ANCH) {
                    // pairs start at even chunks of the call: at even columns
                    // for even cq, odd columns (the first with the previous
                    // group's last) for odd cq
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float ga = par ? (k == 0 ? pend : __uint_as_float(v[2 * k - 1 + (k == 0)]))
                                             : __uint_as_float(v[2 * k]);
                        const float gb = par ? __uint_as_float(v[2 * k]) : __uint_as_float(v[2 * k + 1]);
                        const int c = gcol + 2 * k - par + cq;
                        // both chunks anchored and advanced: one paired step.  A
                        // row's pairs depend on its chunk parity alone (not on its
                        // warp), so a call split at even chunks repeats them exactly
                        const bool two = valid && c >= A.c_first && c + 1 < A.c_end &&
                                         c + 1 < A.c_full;
                        const bool all_two = __all_sync(0xffffffffu, two || !valid);
                        const float oga = __shfl_xor_sync(0xffffffffu, ga, 1);
                        const ff o = {__shfl_xor_sync(0xffffffffu, mine.h, 1),
                                      __shfl_xor_sync(0xffffffffu, mine.l, 1)};
                        // this thread's component of A g(c) + g(c+1)
                        const ff h = ff_add(ff_add(ff_mul(aTr, ff{ga, 0.f}),
                                                   ff_mul(saTi, ff{oga, 0.f})),
                                            ff{gb, 0.f});
                        if (two && comp == 0) {
                            // anchors of chunks c (the carried state, rounded)
                            // and c + 1 (A s + g(c), in FP32 from the rounded state)
                            const float r = __fadd_rn(mine.h, mine.l), i = __fadd_rn(o.h, o.l);
                            float2 *an = A.anchors + (int64_t)(c - A.c_first) * A.D * A.n_slots + ds;
                            an[0] = make_float2(r, i);
                            an[(int64_t)A.D * A.n_slots] =
                                make_float2(fmaf(ar32, r, fmaf(-ai32, i, ga)),
                                            fmaf(ar32, i, fmaf(ai32, r, oga)));
                        }
                        const ff paired = ff_add(ff_add(ff_mul(A2r, mine), ff_mul(sA2i, o)), h);
                        if (!all_two) {   // rows at a range edge: one chunk at a time
                            step1(ga, c, !two);
                            step1(gb, c + 1, !two);
                        }
                        if (two) mine = paired;
                    }
                    pend = __uint_as_float(v[15]);
                    pend_c = gcol + 15 + cq;
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) step1(__uint_as_float(v[j]), gcol + j + cq);
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty0 + 8 * (u & 1));
        }
        if (ANCH) {   // the last column of an odd-cq row, then the carried FP64 state
            if (ok) step1(par ? pend : 0.f, par ? pend_c : A.c_end);
            const float oh = __shfl_xor_sync(0xffffffffu, mine.h, 1);
            const float ol = __shfl_xor_sync(0xffffffffu, mine.l, 1);
            if (ok && valid && comp == 0)
                A.s64[ds] = make_double2((double)mine.h + (double)mine.l, (double)oh + (double)ol);
        }
        }   // M-tiles
        if (!ok && lane == 0) atomicOr(A.err, 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * NT)
                     : "memory");
}

__global__ void state_to_fp64_kernel(const float2 *state, double2 *s64, int64_t count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) s64[i] = make_double2(state[i].x, state[i].y);
}

}  // namespace

cudaError_t launch_state_to_fp64(const float2 *state, double2 *s64, int64_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    state_to_fp64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(state, s64, count);
    return cudaGetLastError();
}

int64_t tc_strain_bytes(int64_t n_cols, int D)
{
    const int64_t ntiles = (n_cols + kColsTile - 1) / kColsTile;
    return (int64_t)D * ntiles * kKBlocks * 2 * (int64_t)kBTileBytes;
}

int tc_cols_per_tile() { return kColsTile; }

cudaError_t launch_tc_seeds(const float4 *params, const int2 *ringoff, int64_t n_slots, int Dh,
                            float2 *seed, float2 *aT, double2 *aT64, cudaStream_t s)
{
    const int64_t threads = n_slots * kTcSeeds;
    if (threads == 0) return cudaSuccess;
    tc_seeds_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(params, ringoff, n_slots,
                                                                       Dh, seed, aT, aT64);
    return cudaGetLastError();
}

cudaError_t launch_tc_strain(const float *xe, int64_t xe_stride, int Dh, int64_t n, int D,
                             int64_t n_cols, int col0, unsigned char *B, cudaStream_t s)
{
    const int64_t n_cols_pad = (n_cols + kColsTile - 1) / kColsTile * kColsTile;
    const int64_t threads = (int64_t)D * n_cols_pad * (kTcK / 8);
    if (threads == 0) return cudaSuccess;
    tc_strain_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(xe, xe_stride, Dh, n, D,
                                                                        n_cols_pad, col0, B);
    return cudaGetLastError();
}

template <bool ANCH, int NT> cudaError_t launch_project_nt(TcArgs a, int64_t mtiles, cudaStream_t s)
{
    constexpr int smem = stages_for<NT>() * (int)(2u * kTileBytes + 2u * (uint32_t)NT * kKBlk * 2u);
    const void *k = reinterpret_cast<const void *>(tc_project_kernel<ANCH, NT>);
    cudaError_t e = ensure_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    a.n_ntiles = (int32_t)((a.n_cols + NT - 1) / NT);
    a.n_btiles = (int32_t)((a.n_cols + kColsTile - 1) / kColsTile);
    // one resident CTA per SM (its shared memory), the M-tiles dealt round robin
    int dev = 0, n_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const int64_t gx = std::min<int64_t>(mtiles, std::max<int64_t>(1, n_sm / std::max(1, a.D)));
    tc_project_kernel<ANCH, NT><<<dim3((unsigned)gx, (unsigned)a.D), kProjThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tc_project(const TcArgs &a, cudaStream_t s)
{
    const int64_t mtiles = (2 * a.n_slots + kRowsTile - 1) / kRowsTile;
    if (mtiles == 0 || a.n_cols <= 0) return cudaSuccess;
    const bool narrow = a.n_cols <= 128;   // one half tile: half the strain bytes per stage
    if (a.anchors != nullptr)
        return narrow ? launch_project_nt<true, 128>(a, mtiles, s)
                      : launch_project_nt<true, 256>(a, mtiles, s);
    return narrow ? launch_project_nt<false, 128>(a, mtiles, s)
                  : launch_project_nt<false, 256>(a, mtiles, s);
}

}  // namespace spiir
