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
// Mapping: one CTA per template streams its D rows of z in tiles of 2048
// outputs (detector d >= 1 with a halo of w_d on each side) and keeps |z|^2
// in shared memory; each thread then takes 8 consecutive outputs, forms
// every detector's window maximum for them (windows up to 129 samples: all 8
// windows share the run's last sample, so one suffix and one prefix scan
// give them; wider windows: doubling levels built by the CTA first), sums
// the detectors and keeps its running best.  The CTA then reduces (largest
// value, earliest t) and finds the offsets at t* from z directly.  The pass
// reads z once (plus the halos): it is bound by HBM bandwidth.
#include "spiir_kernels.h"

#include <cmath>
#include <cstdint>

namespace spiir {

namespace {

constexpr int kNetThreads = 256;
constexpr int kNetR = 8;                         // consecutive outputs per thread
constexpr int kNetTile = kNetThreads * kNetR;    // outputs per shared-memory pass
constexpr int kNetScanMax = 64;                  // wider windows go by doubling

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

// Shared-memory word of sample i of a detector's |z|^2 array: one pad word
// every 8 samples, so the 32 lanes of a warp, each at the start of its own
// run of 8 outputs (stride 8 samples = 9 words), hit 32 different banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }

// Wide windows (w > kNetScanMax): the maxima over 2, 4, 8, ... samples by
// doubling, m_2s[i] = max(m_s[i], m_s[i + s]), ping-ponged between p and g
// up to the largest s <= L = 2w + 1 (one parallel pass of the CTA per
// level); a window [i, i + 2w] is then max(m_s[i], m_s[i + L - s]).
__device__ void net_doubling(float *p, float *g, int w, int tile)
{
    const int L = 2 * w + 1, M = tile + 2 * w;
    float *src = p, *dst = g;
    for (int sp = 1; 2 * sp <= L; sp *= 2) {
        for (int i = threadIdx.x; i + 2 * sp <= M; i += kNetThreads)
            dst[pidx(i)] = fmaxf(src[pidx(i)], src[pidx(i + sp)]);
        __syncthreads();
        float *tmp = src;
        src = dst;
        dst = tmp;
    }
}

// Window maxima of kNetR consecutive outputs i0 .. i0 + 7 (windows
// [i, i + 2w] of the halo'd array), added to s[].
__device__ __forceinline__ void net_add_window(const float *p, const float *g, int w, int i0,
                                               float (&s)[kNetR])
{
    float m[kNetR];
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < kNetR; ++k) m[k] = p[pidx(i0 + k)];
    } else if (2 * w + 1 < kNetR) {
        // narrow: each window directly (<= 7 samples)
#pragma unroll
        for (int k = 0; k < kNetR; ++k) {
            float v = p[pidx(i0 + k)];
            for (int j = 1; j <= 2 * w; ++j) v = fmaxf(v, p[pidx(i0 + k + j)]);
            m[k] = v;
        }
    } else if (w <= kNetScanMax) {
        // every window of the run holds the pivot q = i0 + 7: suffix maxima
        // from each output to q, prefix maxima from q to each window's end
#pragma unroll
        for (int k = kNetR - 1; k >= 0; --k)
            m[k] = k == kNetR - 1 ? p[pidx(i0 + k)] : fmaxf(p[pidx(i0 + k)], m[k + 1]);
        // the middle of the prefix in four independent chains (loads issue
        // ahead of the maxima; max is exact, so the order does not matter)
        float r4[4] = {p[pidx(i0 + kNetR - 1)], -INFINITY, -INFINITY, -INFINITY};
        int j = kNetR;
#pragma unroll 2
        for (; j + 4 <= 2 * w; j += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) r4[q] = fmaxf(r4[q], p[pidx(i0 + j + q)]);
        }
        for (; j < 2 * w; ++j) r4[0] = fmaxf(r4[0], p[pidx(i0 + j)]);
        float run = fmaxf(fmaxf(r4[0], r4[1]), fmaxf(r4[2], r4[3]));
#pragma unroll
        for (int k = 0; k < kNetR; ++k) {
            run = fmaxf(run, p[pidx(i0 + k + 2 * w)]);
            m[k] = fmaxf(m[k], run);
        }
    } else {
        const int L = 2 * w + 1;
        int sp = 1, lev = 0;   // largest power of two <= L, and its doubling level
        while (2 * sp <= L) {
            sp *= 2;
            ++lev;
        }
        const float *r = (lev & 1) ? g : p;
#pragma unroll
        for (int k = 0; k < kNetR; ++k) m[k] = fmaxf(r[pidx(i0 + k)], r[pidx(i0 + k + L - sp)]);
    }
#pragma unroll
    for (int k = 0; k < kNetR; ++k) s[k] = __fadd_rn(s[k], m[k]);
}

__global__ void __launch_bounds__(kNetThreads) network_peak_kernel(const NetArgs A)
{
    extern __shared__ float sm[];
    __shared__ float red_v[kNetThreads / 32];
    __shared__ int64_t red_i[kNetThreads / 32];
    const int64_t tau = blockIdx.x;
    const int tid = threadIdx.x;
    const int64_t n = A.n;
    constexpr int tile = kNetTile;
    float best = -INFINITY;
    int64_t best_t = 0;

    for (int64_t t0 = 0; t0 < n; t0 += tile) {
        // |z|^2 of every detector (positions outside the series: -inf)
        for (int d = 0; d < A.D; ++d) {
            const int w = d ? A.w[d] : 0;
            const int M = tile + 2 * w;
            const float2 *row = A.z + ((int64_t)d * A.T + tau) * n;
            float *p = sm + A.off_p[d];
#pragma unroll 8
            for (int i = tid; i < M; i += kNetThreads) {
                const int64_t pos = t0 - w + i;
                p[pidx(i)] = (pos >= 0 && pos < n) ? mag2(row[pos]) : -INFINITY;
            }
        }
        __syncthreads();
        for (int d = 1; d < A.D; ++d)
            if (A.w[d] > kNetScanMax) net_doubling(sm + A.off_p[d], sm + A.off_g[d], A.w[d], tile);
        // thread: outputs t0 + i0 .. t0 + i0 + 7 (past the series: -inf)
        const int i0 = tid * kNetR;
        float s[kNetR];
#pragma unroll
        for (int k = 0; k < kNetR; ++k) s[k] = sm[A.off_p[0] + pidx(i0 + k)];
        for (int d = 1; d < A.D; ++d)
            net_add_window(sm + A.off_p[d], sm + A.off_g[d], A.w[d], i0, s);
#pragma unroll
        for (int k = 0; k < kNetR; ++k)
            if (s[k] > best) {   // a thread's outputs come in increasing t
                best = s[k];
                best_t = t0 + i0 + k;
            }
        __syncthreads();   // the next tile overwrites shared memory
    }
    cta_best(best, best_t, red_v, red_i);
    if (tid == 0) {
        A.rho[tau] = __fsqrt_rn(best);
        A.t[tau] = best_t;
    }
    if (A.shift == nullptr) return;
    if (tid == 0) A.shift[tau * A.D] = 0;
    // offsets at t*: the first u reaching detector d's window maximum
    for (int d = 1; d < A.D; ++d) {
        const int w = A.w[d];
        const float2 *row = A.z + ((int64_t)d * A.T + tau) * n;
        float v = -INFINITY;
        int64_t u_best = (int64_t)w + 1;
        for (int u = -w + tid; u <= w; u += kNetThreads) {
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

}  // namespace

int network_smem_words(const int32_t *w, int D, int32_t *off_p, int32_t *off_g)
{
    int at = 0;
    for (int d = 0; d < D; ++d) {
        const int wd = d ? w[d] : 0;
        const int M = kNetTile + 2 * wd, words = M + (M >> 3) + 1;   // padded, see pidx
        off_p[d] = at;
        at += words;
        off_g[d] = at;
        if (wd > kNetScanMax) at += words;   // the doubling's second buffer
    }
    return at;
}

cudaError_t launch_network_peak(const NetArgs &a, cudaStream_t s)
{
    if (a.T <= 0 || a.n <= 0) return cudaSuccess;
    int32_t off_p[kNetMaxD], off_g[kNetMaxD];
    const int words = network_smem_words(a.w, a.D, off_p, off_g);
    const int smem = words * (int)sizeof(float);
    for (int d = 0; d < a.D; ++d)
        if (off_p[d] != a.off_p[d] || off_g[d] != a.off_g[d]) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void *>(network_peak_kernel), smem);
    if (e != cudaSuccess) return e;
    network_peak_kernel<<<(unsigned)a.T, kNetThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace spiir
