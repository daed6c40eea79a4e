// Network peak across detectors (coincidence of the detectors' SNR series).
//
// The SPIIR filter gives each (detector, template) its own SNR series z; a
// signal reaches the detectors at times that differ by at most the light
// travel time between them (the review's multi-messenger section localises
// a source from exactly these arrival-time differences).  Per template this
// pass forms, with detector 0 as the reference,
//     s(t) = |z_0(t)|^2 + sum_{d>=1} max_{|u| <= w_d, 0 <= t+u < n} |z_d(t+u)|^2
// and returns the first t maximising s, rho = sqrt(s(t*)) and, per detector
// d >= 1, the first offset u (from -w_d upward) reaching the maximum at t*.
// The values decide integers, so they are formed exactly as stated:
// |z|^2 = re*re + im*im with separately rounded products (no contraction),
// the detector terms added in detector order, a correctly rounded sqrt.
//
// Mapping: a CTA takes one template over a run of tiles of 2048 outputs
// (a time chunk), streams the D rows of z for each tile (detector d >= 1
// with a halo of w_d on each side; tiles inside the series without bounds
// checks) and keeps |z|^2 in shared memory; each thread then takes R = 8 or
// 16 consecutive outputs (chosen per call from the windows), forms every
// detector's window maximum for them (windows of R to 129 samples: all R
// windows share the run's last sample, so one suffix and one prefix scan
// give them; shorter windows: the same in runs of 8, or directly up to 7
// samples; wider than 129: doubling levels built by the CTA first), sums
// the detectors and keeps its running best.  The CTA reduces (largest
// value, earliest t).  With one chunk per template it then finds the
// offsets at t* from z directly.  With several (so that the grid fills the
// SMs in many full waves rather than a few waves with a part-empty last
// one), each CTA folds its best into a 64-bit key per template by atomicMax
// (value bits in an unsigned order above the complemented t, so the larger
// value and then the earlier t wins, exactly the single-CTA order), and a
// second kernel turns the key into rho, t and the offsets.  The pass reads
// z once (plus the halos): it is bound by HBM bandwidth.
#include "spiir_kernels.h"

#include <climits>
#include <cmath>
#include <cstdint>


namespace spiir {

namespace {

constexpr int kNetTile = 2048;       // outputs per shared-memory pass
constexpr int kNetScanMax = 64;      // wider windows go by doubling
constexpr int kNetMaxThreads = 256;

__device__ __forceinline__ float mag2(float2 v)
{
    return __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
}

// (value, index) pair order of the reductions: larger value first, then the
// smaller index
__device__ __forceinline__ bool better(float v, int64_t i, float bv, int64_t bi)
{
    return v > bv || (v == bv && i < bi);
}

// CTA-wide best (value, index); every thread gets the result
__device__ void cta_best(float &v, int64_t &i, float *sv, int64_t *si)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, v, o);
        const int64_t oi = __shfl_down_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (better(sv[w], si[w], sv[0], si[0])) {
                sv[0] = sv[w];
                si[0] = si[w];
            }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();   // sv, si are reused by the next call
}

// Key of a (value, t) pair for the chunked reduction: the float's bits
// mapped to an unsigned order (negatives: every bit flipped; otherwise the
// sign bit set) above 0xffffffff - t (t < 2^32), so a larger key means a
// larger value, or the same value at an earlier t.  Key 0 is below every
// pair's key.
__device__ __forceinline__ unsigned long long net_key(float v, int64_t t)
{
    uint32_t u = __float_as_uint(v);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned long long)(0xffffffffu - (uint32_t)t);
}

__device__ __forceinline__ void net_unkey(unsigned long long k, float &v, int64_t &t)
{
    uint32_t u = (uint32_t)(k >> 32);
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    v = __uint_as_float(u);
    t = (int64_t)(0xffffffffu - (uint32_t)(k & 0xffffffffu));
}

// Shared-memory word of sample i of a detector's |z|^2 array for runs of R
// outputs per thread: one pad word every R samples, so the 32 lanes of a
// warp, each at the start of its own run (stride R + 1 words), hit 32
// different banks.
template <int R>
__device__ __forceinline__ int pidx(int i) { return i + i / R; }

// Wide windows (w > kNetScanMax): the maxima over 2, 4, 8, ... samples by
// doubling, m_2s[i] = max(m_s[i], m_s[i + s]), ping-ponged between p and g
// up to the largest s <= L = 2w + 1 (one parallel pass of the CTA per
// level); a window [i, i + 2w] is then max(m_s[i], m_s[i + L - s]).
template <int R>
__device__ void net_doubling(float *p, float *g, int w)
{
    const int L = 2 * w + 1, M = kNetTile + 2 * w;
    float *src = p, *dst = g;
    for (int sp = 1; 2 * sp <= L; sp *= 2) {
        for (int i = threadIdx.x; i + 2 * sp <= M; i += kNetTile / R)
            dst[pidx<R>(i)] = fmaxf(src[pidx<R>(i)], src[pidx<R>(i + sp)]);
        __syncthreads();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
}

// Window maxima m[k] of RR consecutive outputs i0 .. i0 + RR - 1 (windows
// [i, i + 2w] of the halo'd array, 2w >= RR - 1).  Every window of the run
// holds the pivot q = i0 + RR - 1: suffix maxima from each output to q,
// prefix maxima from q to each window's end.
template <int R, int RR>
__device__ __forceinline__ void net_pivot_run(const float *p, int w, int i0, float *m)
{
#pragma unroll
    for (int k = RR - 1; k >= 0; --k)
        m[k] = k == RR - 1 ? p[pidx<R>(i0 + k)] : fmaxf(p[pidx<R>(i0 + k)], m[k + 1]);
    // the middle of the prefix in four independent chains (loads issue
    // ahead of the maxima; max is exact, so the order does not matter).
    // i0 and RR are multiples of 8 and pads fall every 8 or 16 samples, so
    // each aligned group of 8 samples is 8 consecutive words: one address
    // per group.
    float r4[4] = {p[pidx<R>(i0 + RR - 1)], -INFINITY, -INFINITY, -INFINITY};
    int j = RR;
    for (; j + 8 <= 2 * w; j += 8) {
        const float *b = p + pidx<R>(i0 + j);
#pragma unroll
        for (int q = 0; q < 8; ++q) r4[q & 3] = fmaxf(r4[q & 3], b[q]);
    }
    for (; j < 2 * w; ++j) r4[0] = fmaxf(r4[0], p[pidx<R>(i0 + j)]);
    float run = fmaxf(fmaxf(r4[0], r4[1]), fmaxf(r4[2], r4[3]));
#pragma unroll
    for (int k = 0; k < RR; ++k) {
        run = fmaxf(run, p[pidx<R>(i0 + k + 2 * w)]);
        m[k] = fmaxf(m[k], run);
    }
}

// Window maxima of the thread's R consecutive outputs, added to s[].
template <int R>
__device__ __forceinline__ void net_add_window(const float *p, const float *g, int w, int i0,
                                               float (&s)[R])
{
    float m[R];
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) m[k] = p[pidx<R>(i0 + k)];
    } else if (2 * w + 1 < 8) {
        // narrow: each window directly (<= 7 samples)
#pragma unroll
        for (int k = 0; k < R; ++k) {
            float v = p[pidx<R>(i0 + k)];
            for (int j = 1; j <= 2 * w; ++j) v = fmaxf(v, p[pidx<R>(i0 + k + j)]);
            m[k] = v;
        }
    } else if (R > 8 && 2 * w + 1 < R) {
        // windows of 9..15 samples in runs of 16: two pivot runs of 8
        if constexpr (R > 8) {
            net_pivot_run<R, 8>(p, w, i0, m);
            net_pivot_run<R, 8>(p, w, i0 + 8, m + 8);
        }
    } else if (w <= kNetScanMax) {
        net_pivot_run<R, R>(p, w, i0, m);
    } else {
        const int L = 2 * w + 1;
        int sp = 1, lev = 0;   // largest power of two <= L, and its doubling level
        while (2 * sp <= L) {
            sp *= 2;
            ++lev;
        }
        const float *r = (lev & 1) ? g : p;
#pragma unroll
        for (int k = 0; k < R; ++k)
            m[k] = fmaxf(r[pidx<R>(i0 + k)], r[pidx<R>(i0 + k + L - sp)]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) s[k] = __fadd_rn(s[k], m[k]);
}

// Per detector d >= 1 the first offset u (from -w_d upward) reaching d's
// window maximum at best_t; the CTA's threads split each window.
__device__ void net_shifts(const NetArgs &A, int64_t tau, int64_t best_t, float *red_v,
                           int64_t *red_i)
{
    const int tid = threadIdx.x;
    const int64_t n = A.n;
    if (tid == 0) A.shift[tau * A.D] = 0;
    for (int d = 1; d < A.D; ++d) {
        const int w = A.w[d];
        const float2 *row = A.z + ((int64_t)d * A.T + tau) * n;
        float v = -INFINITY;
        int64_t u_best = (int64_t)w + 1;
        for (int u = -w + tid; u <= w; u += (int)blockDim.x) {
            const int64_t pos = best_t + u;
            const float m = (pos >= 0 && pos < n) ? mag2(row[pos]) : -INFINITY;
            if (better(m, u, v, u_best)) {
                v = m;
                u_best = u;
            }
        }
        cta_best(v, u_best, red_v, red_i);
        if (tid == 0) A.shift[tau * A.D + d] = (int32_t)u_best;
    }
}

// R consecutive outputs per thread, kNetTile / R threads per CTA.
template <int R>
__global__ void __launch_bounds__(kNetTile / R) network_peak_kernel(const NetArgs A)
{
    constexpr int kThreads = kNetTile / R;
    static_assert(kThreads % R == 0, "padded words advance by a constant per thread stride");
    extern __shared__ float sm[];
    __shared__ float red_v[kThreads / 32];
    __shared__ int64_t red_i[kThreads / 32];
    const int64_t tau = blockIdx.x / A.n_chunks;
    const int chunk = (int)(blockIdx.x % A.n_chunks);
    const int tid = threadIdx.x;
    const int64_t n = A.n;
    constexpr int tile = kNetTile;
    const int64_t t_begin = (int64_t)chunk * A.chunk_tiles * tile;
    const int64_t t_end = t_begin + (int64_t)A.chunk_tiles * tile < n
                              ? t_begin + (int64_t)A.chunk_tiles * tile : n;
    float best = -INFINITY;
    int64_t best_t = t_begin;

    for (int64_t t0 = t_begin; t0 < t_end; t0 += tile) {
        // |z|^2 of every detector (positions outside the series: -inf)
        for (int d = 0; d < A.D; ++d) {
            const int w = d ? A.w[d] : 0;
            const int M = tile + 2 * w;
            const float2 *row = A.z + ((int64_t)d * A.T + tau) * n;
            float *p = sm + A.off_p[d];
            // kThreads is a multiple of R, so the padded word advances by a
            // constant kStep per kThreads samples
            constexpr int kStep = kThreads + kThreads / R;
            if (t0 - w >= 0 && t0 - w + M <= n) {
                // interior tile: every position inside the series
                const float2 *src = row + (t0 - w);
                int wi = pidx<R>(tid);
#pragma unroll 8
                for (int i = tid; i < M; i += kThreads, wi += kStep) p[wi] = mag2(src[i]);
            } else {
                int wi = pidx<R>(tid);
#pragma unroll 8
                for (int i = tid; i < M; i += kThreads, wi += kStep) {
                    const int64_t pos = t0 - w + i;
                    p[wi] = (pos >= 0 && pos < n) ? mag2(row[pos]) : -INFINITY;
                }
            }
        }
        __syncthreads();
        for (int d = 1; d < A.D; ++d)
            if (A.w[d] > kNetScanMax) net_doubling<R>(sm + A.off_p[d], sm + A.off_g[d], A.w[d]);
        // thread: outputs t0 + i0 .. t0 + i0 + R - 1 (past the series: -inf)
        const int i0 = tid * R;
        float s[R];
#pragma unroll
        for (int k = 0; k < R; ++k) s[k] = sm[A.off_p[0] + pidx<R>(i0 + k)];
        for (int d = 1; d < A.D; ++d)
            net_add_window<R>(sm + A.off_p[d], sm + A.off_g[d], A.w[d], i0, s);
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (s[k] > best) {   // a thread's outputs come in increasing t
                best = s[k];
                best_t = t0 + i0 + k;
            }
        __syncthreads();   // the next tile overwrites shared memory
    }
    cta_best(best, best_t, red_v, red_i);
    if (A.n_chunks > 1) {
        // the key array is the caller's t output (8 bytes per template)
        if (tid == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(A.t) + tau, net_key(best, best_t));
        return;
    }
    if (tid == 0) {
        A.rho[tau] = __fsqrt_rn(best);
        A.t[tau] = best_t;
    }
    if (A.shift != nullptr) net_shifts(A, tau, best_t, red_v, red_i);
}

// Chunked reduction's end: one CTA per template decodes the key into rho and
// t, then finds the offsets at t*.
__global__ void __launch_bounds__(kNetMaxThreads) network_finish_kernel(const NetArgs A)
{
    __shared__ float red_v[kNetMaxThreads / 32];
    __shared__ int64_t red_i[kNetMaxThreads / 32];
    __shared__ int64_t t_star;
    const int64_t tau = blockIdx.x;
    if (threadIdx.x == 0) {
        float v;
        int64_t t;
        net_unkey(reinterpret_cast<const unsigned long long *>(A.t)[tau], v, t);
        t_star = t;
        A.rho[tau] = __fsqrt_rn(v);
    }
    __syncthreads();
    const int64_t best_t = t_star;
    if (threadIdx.x == 0) A.t[tau] = best_t;
    if (A.shift != nullptr) net_shifts(A, tau, best_t, red_v, red_i);
}

// Outputs per thread for these windows.  Shared-memory loads per output of
// the window maxima, summed over detectors d >= 1: runs of 8 cost about
// (2w + 9) / 8 for w >= 4 (2w + 1 below), runs of 16 about (2w + 17) / 16
// but, with the same shared memory per CTA and half the threads, 32 warps
// per SM instead of 48 and a slower load phase.  Measured on 4096 templates x 3 detectors x 65536 samples: runs
// of 8 are faster up to windows 40/40 (22.25 loads per output; 1.307 vs
// 1.419 ms) and 10/64 (20.75; 1.267 vs 1.313 ms), runs of 16 from 48/48
// (26.25; 1.294 vs 1.376 ms; 64/64: 1.312 vs 1.578 ms).  Windows past the
// scan limit go by doubling, whose CTA-wide levels want the wider CTA.
constexpr double kNetR16Loads = 24.0;

int net_run_len(const int32_t *w, int D)
{
    double loads = 0.0;
    for (int d = 1; d < D; ++d) {
        if (w[d] > kNetScanMax) return 8;
        loads += w[d] >= 4 ? (2.0 * w[d] + 9.0) / 8.0 : 2.0 * w[d] + 1.0;
    }
    return loads > kNetR16Loads ? 16 : 8;
}

}  // namespace

int network_smem_words(const int32_t *w, int D, int32_t *off_p, int32_t *off_g)
{
    const int R = net_run_len(w, D);
    int at = 0;
    for (int d = 0; d < D; ++d) {
        const int wd = d ? w[d] : 0;
        const int M = kNetTile + 2 * wd, words = M + M / R + 1;   // padded, see pidx
        off_p[d] = at;
        at += words;
        off_g[d] = at;
        if (wd > kNetScanMax) at += words;   // the doubling's second buffer
    }
    return at;
}

template <int R>
static cudaError_t launch_network_r(NetArgs a, int smem, cudaStream_t s)
{
    constexpr int kThreads = kNetTile / R;
    const void *kern = reinterpret_cast<const void *>(network_peak_kernel<R>);
    cudaError_t e = ensure_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    // time chunks per template: at least 8 waves of the resident CTAs, then
    // the count (up to twice that) whose last wave is fullest (1-2% faster
    // than one CTA per template on 4096 templates).  The chunked reduction
    // keys t in 32 bits, so longer series keep one CTA per template.
    const int64_t tiles = (a.n + kNetTile - 1) / kNetTile;
    int64_t C = 1, ct = tiles;
    if (tiles > 1 && a.n <= (int64_t)0xffffffff) {
        int dev = 0, n_sm = 0, resident = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &resident, network_peak_kernel<R>, kThreads, smem)) != cudaSuccess)
            return e;
        const int64_t slots = (int64_t)n_sm * (resident > 0 ? resident : 1);
        int64_t c0 = (8 * slots + a.T - 1) / a.T;
        c0 = c0 < 1 ? 1 : (c0 > tiles ? tiles : c0);
        double best_eff = -1.0;
        for (int64_t c = c0; c <= 2 * c0 && c <= tiles; ++c) {
            const int64_t per = (tiles + c - 1) / c, cc = (tiles + per - 1) / per;
            const double waves = (double)(a.T * cc) / (double)slots;
            const double eff = waves / std::ceil(waves);
            if (eff > best_eff + 1e-9 && a.T * cc <= INT32_MAX) {
                best_eff = eff;
                C = cc;
                ct = per;
            }
        }
    }
    // grid sizes: a.T * C CTAs (the chunk search keeps it <= INT32_MAX) and,
    // for C == 1, a.T itself, which must then fit a grid dimension as well
    if (a.T > INT32_MAX || a.T * C > INT32_MAX) return cudaErrorInvalidConfiguration;
    a.n_chunks = (int32_t)C;
    a.chunk_tiles = (int32_t)ct;
    if (C > 1 && (e = cudaMemsetAsync(a.t, 0, (size_t)a.T * sizeof(int64_t), s)) != cudaSuccess)
        return e;
    network_peak_kernel<R><<<(unsigned)(a.T * C), kThreads, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess || C == 1) return e;
    network_finish_kernel<<<(unsigned)a.T, kNetMaxThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_network_peak(const NetArgs &a, cudaStream_t s)
{
    if (a.T <= 0 || a.n <= 0) return cudaSuccess;
    int32_t off_p[kNetMaxD], off_g[kNetMaxD];
    const int words = network_smem_words(a.w, a.D, off_p, off_g);
    const int smem = words * (int)sizeof(float);
    for (int d = 0; d < a.D; ++d)
        if (off_p[d] != a.off_p[d] || off_g[d] != a.off_g[d]) return cudaErrorInvalidValue;
    return net_run_len(a.w, a.D) == 16 ? launch_network_r<16>(a, smem, s)
                                       : launch_network_r<8>(a, smem, s);
}

}  // namespace spiir
