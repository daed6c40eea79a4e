// Adjoint (vector-Jacobian product) of the SPIIR filter bank for sm_103a.
//
// For a real loss L of the SNR series z (section "GPU accelerated SPIIR
// method", subsection "SPIIR method": z[k] = sum_l y_l[k],
// y_l[k] = a_l y_l[k-1] + b_l x[k-d_l]), given g_z[k] = dL/dRe z + i dL/dIm z,
// each filter's adjoint state runs backwards in time,
//     mu_l[k] = g_z[k] + conj(a_l) mu_l[k+1],          mu_l[n] = 0,
// and the gradients (same convention) are
//     g_a_l  = sum_k mu_l[k] conj(y_l[k-1]),
//     g_b_l  = sum_k mu_l[k] x[k-d_l],
//     g_x[m] = sum_l Re(conj(mu_l[m+d_l]) b_l).
// The reverse pass needs y_l[k-1] at every k.  Recomputing y backwards
// through 1/a_l is unstable, so the forward kernel stores the state every Cc
// samples and this kernel, for each chunk in reverse order, recomputes the
// chunk forward from its checkpoint (pass A, keeping the state every
// kAdjSub samples in shared memory) and then, for each kAdjSub-sample span in
// reverse, recomputes the span into registers (pass B) and runs the adjoint
// over it.
//
// Mapping: one CTA per (group of W templates, detector), as in the forward
// kernel; lane i of a warp walks the warp's filter rounds one at a time (mu,
// g_a and g_b of each filter live in global memory between chunks, so
// registers do not grow with the filter count).  The strain window of a
// chunk is staged in shared memory; g_z of the template is read by lanes
// 0..kAdjSub-1 once per span and broadcast with shuffles; g_x is scattered
// into a shared ring with shared-memory atomics (the layout places a round's
// 32 delays on 32 different banks) and added to global memory per chunk.
#include "spiir_kernels.h"

#include <cstdint>

namespace spiir {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(256) k6_adjoint(const K6Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int Dw = A.Dh + A.Cc;                          // strain window per chunk
    float *xs = reinterpret_cast<float *>(smem);         // [Dw]
    float *gxs = xs + Dw;                                // [Dw]
    float2 *sub = reinterpret_cast<float2 *>(gxs + Dw);  // [W][Cc / kAdjSub][32]
    const int nsub_max = A.Cc / kAdjSub;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = A.units[2 * blockIdx.x];
    const int det = A.units[2 * blockIdx.x + 1];
    const int F = A.group_F[g];
    const int4 wi = A.warp_info[(int64_t)g * A.W + warp];
    const int tmpl = wi.x;
    const bool active = tmpl >= 0;
    const int64_t pb = A.group_pbase[g];
    const int n = A.n;
    const int nc = (n + A.Cc - 1) / A.Cc;
    const float *xrow = A.xe + (int64_t)det * A.xe_stride;
    const float2 *grow = active ? A.gz + ((int64_t)det * A.T + tmpl) * n : nullptr;
    float2 *wsub = sub + (int64_t)warp * nsub_max * 32;
    float *acc_det = A.acc + (int64_t)det * A.n_slots * 6;

    for (int c = nc - 1; c >= 0; --c) {
        const int kc = c * A.Cc;
        const int cv = min(A.Cc, n - kc);
        // strain x[kc - Dh + i] = xe[kc + i] (xe holds Dh zeros before x)
        for (int i = threadIdx.x; i < Dw; i += blockDim.x) {
            xs[i] = i < A.Dh + cv ? xrow[kc + i] : 0.f;
            gxs[i] = 0.f;
        }
        __syncthreads();
        if (active) {
            const int nsub = (cv + kAdjSub - 1) / kAdjSub;
            for (int r = 0; r < F; ++r) {
                const int64_t s = pb + ((int64_t)r * A.W + warp) * 32 + lane;
                const float4 p = A.params[s];
                const bool odd = (lane & 1) != 0;   // stored as conj(a), (Im b, Re b)
                const float ar = p.x, ai = odd ? -p.y : p.y;
                const float br = odd ? p.w : p.z, bi = odd ? p.z : p.w;
                const int xo = A.ringoff[s].x;   // Dh - d: xs index of x[kc - d]
                float *acc = acc_det + s * 6;
                float mr = acc[0], mi = acc[1];
                float gar = acc[2], gai = acc[3], gbr = acc[4], gbi = acc[5];
                // state y[kc - 1]
                float yr = 0.f, yi = 0.f;
                if (c > 0) {
                    const float2 ck = A.ckpt[((int64_t)c * A.n_det + det) * A.n_slots + s];
                    yr = odd ? ck.y : ck.x;
                    yi = odd ? ck.x : ck.y;
                }
                // pass A: forward over the chunk, state kept every kAdjSub samples
                for (int q = 0; q < nsub; ++q) {
                    wsub[q * 32 + lane] = make_float2(yr, yi);
                    const int k0 = q * kAdjSub;
#pragma unroll
                    for (int t = 0; t < kAdjSub; ++t) {
                        if (k0 + t < cv) {
                            const float x = xs[xo + k0 + t];
                            const float nr = fmaf(ar, yr, fmaf(-ai, yi, br * x));
                            const float ni = fmaf(ar, yi, fmaf(ai, yr, bi * x));
                            yr = nr;
                            yi = ni;
                        }
                    }
                }
                // pass B: spans in reverse; y[k-1] recomputed into registers
                for (int q = nsub - 1; q >= 0; --q) {
                    const int k0 = q * kAdjSub;
                    float pr[kAdjSub], pi[kAdjSub];   // y[k0 + t - 1]
                    {
                        const float2 y0 = wsub[q * 32 + lane];
                        float ur = y0.x, ui = y0.y;
#pragma unroll
                        for (int t = 0; t < kAdjSub; ++t) {
                            pr[t] = ur;
                            pi[t] = ui;
                            if (t + 1 < kAdjSub) {
                                const float x = xs[xo + k0 + t];
                                const float nr = fmaf(ar, ur, fmaf(-ai, ui, br * x));
                                const float ni = fmaf(ar, ui, fmaf(ai, ur, bi * x));
                                ur = nr;
                                ui = ni;
                            }
                        }
                    }
                    float2 gl = make_float2(0.f, 0.f);
                    if (lane < kAdjSub && k0 + lane < cv) gl = grow[kc + k0 + lane];
#pragma unroll
                    for (int t = kAdjSub - 1; t >= 0; --t) {
                        const float Gr = __shfl_sync(kFull, gl.x, t);
                        const float Gi = __shfl_sync(kFull, gl.y, t);
                        if (k0 + t < cv) {
                            // mu <- g_z + conj(a) mu
                            const float nr = Gr + fmaf(ar, mr, ai * mi);
                            const float ni = Gi + fmaf(ar, mi, -ai * mr);
                            mr = nr;
                            mi = ni;
                            // g_a += mu conj(y[k-1]),  g_b += mu x[k-d]
                            gar = fmaf(mr, pr[t], fmaf(mi, pi[t], gar));
                            gai = fmaf(mi, pr[t], fmaf(-mr, pi[t], gai));
                            const float x = xs[xo + k0 + t];
                            gbr = fmaf(mr, x, gbr);
                            gbi = fmaf(mi, x, gbi);
                            if (A.gx != nullptr)
                                atomicAdd(&gxs[xo + k0 + t], fmaf(mr, br, mi * bi));
                        }
                    }
                }
                acc[0] = mr;
                acc[1] = mi;
                acc[2] = gar;
                acc[3] = gai;
                acc[4] = gbr;
                acc[5] = gbi;
            }
        }
        __syncthreads();
        if (A.gx != nullptr) {
            // g_x[kc - Dh + i] gets this chunk's contributions
            float *gxrow = A.gx + (int64_t)det * n;
            for (int i = threadIdx.x; i < A.Dh + cv; i += blockDim.x) {
                const int m = kc - A.Dh + i;
                const float v = gxs[i];
                if (m >= 0 && v != 0.f) atomicAdd(&gxrow[m], v);
            }
        }
        __syncthreads();
    }
}

__global__ void adj_finalize(const float *acc, const int64_t *slot_filter, int64_t n_slots,
                             int D, float2 *ga, float2 *gb)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int64_t f = slot_filter[s];
    if (f < 0) return;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    for (int d = 0; d < D; ++d) {
        const float *p = acc + ((int64_t)d * n_slots + s) * 6;
        a.x += p[2];
        a.y += p[3];
        b.x += p[4];
        b.y += p[5];
    }
    ga[f] = a;
    gb[f] = b;
}

__global__ void set_coefficients(const float2 *a, const float2 *b, const int64_t *slot_filter,
                                 int64_t n_slots, float4 *params)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int64_t f = slot_filter[s];
    if (f < 0) return;
    const float2 av = a[f], bv = b[f];
    // odd lanes hold their filter in (im, re) order: conj(a), (Im b, Re b)
    params[s] = (s & 1) ? make_float4(av.x, -av.y, bv.y, bv.x)
                        : make_float4(av.x, av.y, bv.x, bv.y);
}

}  // namespace

int k6_smem_bytes(int W, int Cc, int Dh)
{
    return (int)(2 * sizeof(float) * (Dh + Cc) + sizeof(float2) * W * (Cc / kAdjSub) * 32);
}

cudaError_t launch_k6(const K6Args &a, int64_t n_units, cudaStream_t s)
{
    if (n_units <= 0 || a.n <= 0) return cudaSuccess;
    const int smem = k6_smem_bytes(a.W, a.Cc, a.Dh);
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void *>(k6_adjoint), smem);
    if (e != cudaSuccess) return e;
    k6_adjoint<<<(unsigned)n_units, a.W * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_finalize(const float *acc, const int64_t *slot_filter, int64_t n_slots,
                                int D, float2 *ga, float2 *gb, cudaStream_t s)
{
    if (n_slots <= 0) return cudaSuccess;
    adj_finalize<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(acc, slot_filter, n_slots, D,
                                                                    ga, gb);
    return cudaGetLastError();
}

cudaError_t launch_set_coefficients(const float2 *a, const float2 *b,
                                    const int64_t *slot_filter, int64_t n_slots,
                                    float4 *params, cudaStream_t s)
{
    if (n_slots <= 0) return cudaSuccess;
    set_coefficients<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(a, b, slot_filter,
                                                                        n_slots, params);
    return cudaGetLastError();
}

}  // namespace spiir
