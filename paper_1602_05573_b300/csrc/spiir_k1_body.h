// The filter kernel K1 (see spiir_k1.cu for its design): the per-lane
// arithmetic policies, the CTA work unit and the kernel templates, shared
// by the translation units that instantiate them (one per filters-per-lane
// cap, one for the precision forms) so that they compile in parallel.
// Everything here has internal linkage; each unit instantiates only the
// kernels it launches.
#pragma once

#include "spiir_kernels.h"
#include "spiir_layout.h"
#include "spiir_ptx.h"

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

namespace spiir {

// CTAs of `k` resident on the device at once (defined in spiir_k1.cu)
cudaError_t resident_ctas(const void *k, int threads, int smem_bytes, int *out);

namespace {

constexpr unsigned kFull = 0xffffffffu;



// Bytes one strain block brings into the ring (every copy, plus the mirror
// of slot 0 placed after the ring so windows never wrap).
__device__ __forceinline__ uint32_t block_bytes(const K1Args &A, int64_t eblk)
{
    const uint32_t one = (uint32_t)A.Tb * 4u * (uint32_t)A.C;
    return (eblk % A.S) == 0 ? 2u * one : one;
}

// Issue the copies of strain block eblk (xe samples [eblk*Tb, (eblk+1)*Tb)).
__device__ __forceinline__ void issue_block(const K1Args &A, const float *xrow, float *ring,
                                            int64_t eblk, uint32_t bar)
{
    const int slot = (int)(eblk % A.S);
    const float *src = xrow + eblk * A.Tb;
    const uint32_t bytes = (uint32_t)A.Tb * 4u;
    for (int c = 0; c < A.C; ++c) {
        float *dst = ring + (int64_t)c * A.CS + (int64_t)slot * A.Tb;
        bulk_g2s(smem_addr(dst), src, bytes, bar);
        if (slot == 0) bulk_g2s(smem_addr(dst + A.R), src, bytes, bar);
    }
}

// ---- cross-lane sum of 8 samples -----------------------------------------
// zr/zi: this lane's partial sums (its filters) for 8 consecutive samples.
// Even lanes hold (re, im), odd lanes (im, re).  After the exchange, lane i
// (and lane i^16) holds component (i & 1) of sample s(i) summed over the
// warp; lanes 0..15 write the 8 complex sums to out[0..15].  In half-warp
// mode the last (lane 16) exchange is skipped and each half writes its own
// template's sums to out[half * Tb * 2 + ...].
__device__ __forceinline__ void warp_sum8(const float (&zr)[kTS], const float (&zi)[kTS],
                                          int lane, float *out, bool half, int Tb)
{
    float v[kTS];
#pragma unroll
    for (int j = 0; j < kTS; ++j) v[j] = zr[j] + __shfl_xor_sync(kFull, zi[j], 1);
    const bool b1 = (lane & 2) != 0, b2 = (lane & 4) != 0, b3 = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b1 ? v[i] : v[i + 4];
        const float keep = b1 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(kFull, send, 2);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b2 ? v[i] : v[i + 2];
        const float keep = b2 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(kFull, send, 4);
    }
    {
        const float send = b3 ? v[0] : v[1];
        const float keep = b3 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(kFull, send, 8);
    }
    const int s = (b1 ? 4 : 0) + (b2 ? 2 : 0) + (b3 ? 1 : 0);
    if (half) {
        // lanes 0..15 and 16..31 serve different templates: each half holds
        // its template's 8 complex sums; write them to the half's buffer
        out[(lane >> 4) * Tb * 2 + 2 * s + (lane & 1)] = v[0];
    } else {
        v[0] += __shfl_xor_sync(kFull, v[0], 16);
        if (lane < 16) out[2 * s + (lane & 1)] = v[0];
    }
}

// ---- the first warp of a template: add its warps' sums, store, peak ------
// Multirate banks: each lower band's sum is brought to this (top) rate by
// linear interpolation between band samples i = k / R and i + 1 (held at the
// call's last band sample), z_up = (1 - f) z_b[i] + f z_b[i + 1], f = (k mod R)/R,
// and added before the store and the peak.  The band samples a block needs
// were prefetched into `low` (this template's buffer) when the block began.
__device__ __forceinline__ int band_index(const LowerBand &lb, int k)
{
    return lb.shift >= 0 ? (k >> lb.shift) : k / lb.R;
}

// Asynchronous copies (no register round trip) of the band samples block
// [k0, k0 + nv) interpolates from, into this template's prefetch buffer.
__device__ __forceinline__ void prefetch_lower(const K1Args &A, float2 *low, int det, int tmpl,
                                               int lane, int k0, int nv)
{
    for (int b = 0; b < A.n_lower; ++b) {
        const LowerBand &lb = A.lower[b];
        const int lo = band_index(lb, k0);
        const int hi = min(band_index(lb, k0 + nv - 1) + 1, (int)lb.len - 1);
        const float2 *row = lb.z + ((int64_t)det * A.T + tmpl) * lb.len;
        for (int e = lane; e <= hi - lo; e += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                             smem_addr(low + lb.buf_off + e)),
                         "l"(row + lo + e)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <bool LOW>
__device__ __forceinline__ void combine_block(const K1Args &A, const float2 *zb, int first,
                                              int nw, const float2 *low, int lane, int k0,
                                              int nv, float *zrow, float &best, int &bidx)
{
    const int n_lower = LOW ? A.n_lower : 0;
    if (n_lower > 0) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
    }
    // z store and running peak of sample i (|z|^2 = re*re + im*im, no
    // contraction: reproducible on the host)
    auto store_peak = [&](float2 acc, int i) {
        if (zrow != nullptr) reinterpret_cast<float2 *>(zrow)[k0 + i] = acc;
        const float p = __fadd_rn(__fmul_rn(acc.x, acc.x), __fmul_rn(acc.y, acc.y));
        if (p > best) {
            best = p;
            bidx = k0 + i;
        }
    };
    // One or two lower bands whose decimation factors divide 32 (and so the
    // block start k0): lane i always takes samples i mod 32 of the block, so
    // each band's interpolation weight is fixed per lane and its band sample
    // advances by 32 / R per step; set up once here instead of per sample.
    // The arithmetic of each term is that of the general loop below.
    if (LOW && n_lower >= 1 && n_lower <= 2) {
        bool fast = true;
        for (int b = 0; b < n_lower; ++b)
            fast = fast && A.lower[b].shift >= 0 && A.lower[b].R <= 32 &&
                   (k0 & (A.lower[b].R - 1)) == 0;
        if (fast) {
            const LowerBand &l0 = A.lower[0], &l1 = A.lower[n_lower - 1];
            const bool two = n_lower == 2;
            // band sample of this lane's first output, relative to the block's
            const int r0 = lane >> l0.shift, r1 = lane >> l1.shift;
            const int st0 = 32 >> l0.shift, st1 = 32 >> l1.shift;
            const int lo0 = k0 >> l0.shift, lo1 = k0 >> l1.shift;
            const int last0 = (int)l0.len - 1 - lo0, last1 = (int)l1.len - 1 - lo1;
            const float f0 = (float)(lane & (l0.R - 1)) / (float)l0.R;
            const float f1 = (float)(lane & (l1.R - 1)) / (float)l1.R;
            const float g0 = 1.0f - f0, g1 = 1.0f - f1;
            const float2 *b0 = low + l0.buf_off, *b1 = low + l1.buf_off;
            // the acc of sample i (band samples q0, q1 of this lane)
            auto acc_at = [&](int i, int q0, int q1) {
                float2 acc = zb[(int64_t)first * A.Tb + i];
                for (int w = 1; w < nw; ++w) {
                    const float2 o = zb[(int64_t)(first + w) * A.Tb + i];
                    acc.x += o.x;
                    acc.y += o.y;
                }
                {
                    const float2 u = b0[q0], v = b0[q0 + 1 <= last0 ? q0 + 1 : last0];
                    acc.x += fmaf(f0, v.x, g0 * u.x);
                    acc.y += fmaf(f0, v.y, g0 * u.y);
                }
                if (two) {
                    const float2 u = b1[q1], v = b1[q1 + 1 <= last1 ? q1 + 1 : last1];
                    acc.x += fmaf(f1, v.x, g1 * u.x);
                    acc.y += fmaf(f1, v.y, g1 * u.y);
                }
                return acc;
            };
            // four samples' loads before their stores and peak updates (in
            // sample order, so the first index still wins ties)
            int i = lane, q0 = r0, q1 = r1;
            for (; i + 96 < nv; i += 128, q0 += 4 * st0, q1 += 4 * st1) {
                float2 acc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = acc_at(i + 32 * u, q0 + u * st0, q1 + u * st1);
#pragma unroll
                for (int u = 0; u < 4; ++u) store_peak(acc[u], i + 32 * u);
            }
            for (; i < nv; i += 32, q0 += st0, q1 += st1) store_peak(acc_at(i, q0, q1), i);
            return;
        }
    }
    auto acc_at = [&](int i) {
        float2 acc = zb[(int64_t)first * A.Tb + i];
        for (int w = 1; w < nw; ++w) {
            const float2 o = zb[(int64_t)(first + w) * A.Tb + i];
            acc.x += o.x;
            acc.y += o.y;
        }
        for (int b = 0; b < n_lower; ++b) {
            const LowerBand &lb = A.lower[b];
            const int k = k0 + i;
            const int lo = band_index(lb, k0);
            const int ib = band_index(lb, k);
            const int ib1 = ib + 1 < lb.len ? ib + 1 : (int)lb.len - 1;
            const int rem = lb.shift >= 0 ? (k & (lb.R - 1)) : k % lb.R;
            const float f = (float)rem / (float)lb.R;
            const float2 u = low[lb.buf_off + ib - lo], v = low[lb.buf_off + ib1 - lo];
            acc.x += fmaf(f, v.x, (1.0f - f) * u.x);
            acc.y += fmaf(f, v.y, (1.0f - f) * u.y);
        }
        return acc;
    };
    // four samples' loads before their stores and peak updates (in sample
    // order, so the first index still wins ties)
    int i = lane;
    for (; i + 96 < nv; i += 128) {
        float2 acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = acc_at(i + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) store_peak(acc[u], i + 32 * u);
    }
    for (; i < nv; i += 32) store_peak(acc_at(i), i);
}

// ---- arithmetic policies: one lane's F filters --------------------------
// Each policy keeps its filters' coefficients and state in registers and
// advances them 8 samples at a time, returning this lane's per-sample sums.
// ad[r] is the shared-memory byte address of the strain sample filter r
// reads at the step's first sample; sample t of the step is at ad[r] + 4 t.
// step8 runs FULL = true for 8 whole samples, false for a ragged tail of
// `valid` samples (the state stays put past the tail).

// Plain FP32: two filters per packed FP32x2 instruction (8 packed ops per
// filter pair and sample), an odd filter in scalar FP32.
template <int F> struct PackedLanes {
    static constexpr int kF = F;
    static constexpr int NP = F / 2;
    static constexpr bool ODD = (F & 1) != 0;
    static constexpr int NPA = NP > 0 ? NP : 1;
    uint64_t AR[NPA], AI[NPA], NAI[NPA], BR[NPA], BI[NPA], YR[NPA], YI[NPA];
    float ar1 = 0.f, ai1 = 0.f, br1 = 0.f, bi1 = 0.f, yr1 = 0.f, yi1 = 0.f;

    __device__ __forceinline__ void load(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                         const float2 *sin)
    {
        float4 p[F];
        float2 st[F];
#pragma unroll
        for (int r = 0; r < F; ++r) {
            const int64_t s = pb + ((int64_t)r * A.W + warp) * 32 + lane;
            p[r] = A.params[s];
            st[r] = sin != nullptr ? sin[(int64_t)det * A.n_slots + s] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            AR[q] = pk(p[2 * q].x, p[2 * q + 1].x);
            AI[q] = pk(p[2 * q].y, p[2 * q + 1].y);
            NAI[q] = pk(-p[2 * q].y, -p[2 * q + 1].y);
            BR[q] = pk(p[2 * q].z, p[2 * q + 1].z);
            BI[q] = pk(p[2 * q].w, p[2 * q + 1].w);
            YR[q] = pk(st[2 * q].x, st[2 * q + 1].x);
            YI[q] = pk(st[2 * q].y, st[2 * q + 1].y);
        }
        if (ODD) {
            ar1 = p[F - 1].x;
            ai1 = p[F - 1].y;
            br1 = p[F - 1].z;
            bi1 = p[F - 1].w;
            yr1 = st[F - 1].x;
            yi1 = st[F - 1].y;
        }
    }
    __device__ __forceinline__ float2 state_of(int r) const
    {
        float lo, hi, ilo, ihi;
        if (ODD && r == F - 1) return make_float2(yr1, yi1);
        upk(YR[r / 2], lo, hi);
        upk(YI[r / 2], ilo, ihi);
        return (r & 1) ? make_float2(hi, ihi) : make_float2(lo, ilo);
    }
    template <bool FULL>
    __device__ __forceinline__ void step8(const uint32_t (&ad)[F], int valid, float (&zr)[kTS],
                                          float (&zi)[kTS])
    {
#pragma unroll
        for (int t = 0; t < kTS; ++t) {
            if (!FULL && t >= valid) {  // ragged tail: state stays put
                zr[t] = 0.f;
                zi[t] = 0.f;
                continue;
            }
            uint64_t ZR = 0, ZI = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const uint64_t X = pk(lds_f32(ad[2 * q] + 4u * t), lds_f32(ad[2 * q + 1] + 4u * t));
                // each pair of consecutive products shares one operand (X,
                // YR, YI), which the operand reuse of the register file can
                // serve without a second read (measured 0.7% faster than the
                // order without shared operands)
                uint64_t TR = mul2(BR[q], X);   // br x
                uint64_t TI = mul2(BI[q], X);   // bi x
                TR = fma2(AR[q], YR[q], TR);    // + ar yr
                TI = fma2(AI[q], YR[q], TI);    // + ai yr
                TI = fma2(AR[q], YI[q], TI);    // + ar yi
                TR = fma2(NAI[q], YI[q], TR);   // - ai yi
                YR[q] = TR;
                YI[q] = TI;
                if (q == 0) {
                    ZR = YR[0];
                    ZI = YI[0];
                } else {
                    ZR = add2(ZR, YR[q]);
                    ZI = add2(ZI, YI[q]);
                }
            }
            float sr = 0.f, si = 0.f;
            if (NP > 0) {
                float lo, hi;
                upk(ZR, lo, hi);
                sr = lo + hi;
                upk(ZI, lo, hi);
                si = lo + hi;
            }
            if (ODD) {
                const float x1 = lds_f32(ad[F - 1] + 4u * t);
                const float nr = fmaf(ar1, yr1, fmaf(-ai1, yi1, br1 * x1));
                const float ni = fmaf(ar1, yi1, fmaf(ai1, yr1, bi1 * x1));
                yr1 = nr;
                yi1 = ni;
                sr = NP > 0 ? sr + yr1 : yr1;
                si = NP > 0 ? si + yi1 : yi1;
            }
            zr[t] = sr;
            zi[t] = si;
        }
    }
    __device__ __forceinline__ void begin(const K1Args &, int) {}
    __device__ __forceinline__ void after8(const K1Args &, int) {}
    __device__ __forceinline__ void finish(const K1Args &, int) {}
    __device__ __forceinline__ void store(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                          float2 *sout)
    {
        if (sout == nullptr) return;
#pragma unroll
        for (int r = 0; r < F; ++r)
            sout[(int64_t)det * A.n_slots + pb + ((int64_t)r * A.W + warp) * 32 + lane] =
                state_of(r);
    }
};

// Compensated: each filter's state is a float-float pair (hi + lo, about 48
// significant bits).  The rounding that builds up over the ~1/(1-|a|) steps
// of a pole near the unit circle is that of the state update a y, so its
// two leading products a_re y_hi, a_im y_hi are taken exactly (two-product by
// FMA) and summed exactly (two-sum); the terms a y_lo and b x enter the low
// word rounded once (their rounding does not grow relative to |y|: the
// input's share of y is |b x| against |y| ~ |b x| / sqrt(1 - |a|^2)).  Pairs
// of filters run as packed FP32x2 (the pole is held negated as well, so that
// each product's exact error is one FMA); an odd filter runs in scalar FP32.
// 21 packed instructions per filter-update (42 lane operations).
template <int F> struct CompLanes {
    static constexpr int kF = F;
    static constexpr int NP = F / 2;
    static constexpr bool ODD = (F & 1) != 0;
    static constexpr int NPA = NP > 0 ? NP : 1;
    uint64_t AR[NPA], NAR[NPA], AI[NPA], NAI[NPA], BR[NPA], BI[NPA];
    uint64_t YRH[NPA], YRL[NPA], YIH[NPA], YIL[NPA];
    float ar1 = 0.f, ai1 = 0.f, br1 = 0.f, bi1 = 0.f;
    float yrh1 = 0.f, yrl1 = 0.f, yih1 = 0.f, yil1 = 0.f;

    __device__ __forceinline__ void load(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                         const float2 *)
    {
        const float4 *st = reinterpret_cast<const float4 *>(A.state_ext);
        float4 p[F], y[F];
#pragma unroll
        for (int r = 0; r < F; ++r) {
            const int64_t s = pb + ((int64_t)r * A.W + warp) * 32 + lane;
            p[r] = A.params[s];
            y[r] = st[(int64_t)det * A.n_slots + s];
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float4 u = p[2 * q], v = p[2 * q + 1];
            AR[q] = pk(u.x, v.x);
            NAR[q] = pk(-u.x, -v.x);
            AI[q] = pk(u.y, v.y);
            NAI[q] = pk(-u.y, -v.y);
            BR[q] = pk(u.z, v.z);
            BI[q] = pk(u.w, v.w);
            YRH[q] = pk(y[2 * q].x, y[2 * q + 1].x);
            YRL[q] = pk(y[2 * q].y, y[2 * q + 1].y);
            YIH[q] = pk(y[2 * q].z, y[2 * q + 1].z);
            YIL[q] = pk(y[2 * q].w, y[2 * q + 1].w);
        }
        if (ODD) {
            ar1 = p[F - 1].x;
            ai1 = p[F - 1].y;
            br1 = p[F - 1].z;
            bi1 = p[F - 1].w;
            yrh1 = y[F - 1].x;
            yrl1 = y[F - 1].y;
            yih1 = y[F - 1].z;
            yil1 = y[F - 1].w;
        }
    }
    // (h, l) = float-float s + t + lo from the exact sum s + t of two leading
    // terms; |s| >= |lo| as a rule (the fast two-sum)
    __device__ __forceinline__ static void lead2(uint64_t p1, uint64_t p2, uint64_t lo,
                                                 uint64_t &h, uint64_t &l)
    {
        const uint64_t s = add2(p1, p2);
        const uint64_t bb = sub2(s, p1);
        const uint64_t t = add2(sub2(p1, sub2(s, bb)), sub2(p2, bb));   // p1 + p2 = s + t
        const uint64_t lw = add2(t, lo);
        h = add2(s, lw);
        l = sub2(lw, sub2(h, s));
    }
    template <bool FULL>
    __device__ __forceinline__ void step8(const uint32_t (&ad)[F], int valid, float (&zr)[kTS],
                                          float (&zi)[kTS])
    {
#pragma unroll
        for (int t = 0; t < kTS; ++t) {
            if (!FULL && t >= valid) {
                zr[t] = 0.f;
                zi[t] = 0.f;
                continue;
            }
            uint64_t ZR = 0, ZI = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const uint64_t X = pk(lds_f32(ad[2 * q] + 4u * t), lds_f32(ad[2 * q + 1] + 4u * t));
                // Re: ar yrh - ai yih exactly, + (br x + ar yrl - ai yil) once rounded
                const uint64_t p1 = mul2(AR[q], YRH[q]), e1 = fma2(NAR[q], YRH[q], p1);
                const uint64_t p2 = mul2(NAI[q], YIH[q]), e2 = fma2(AI[q], YIH[q], p2);
                const uint64_t lr = sub2(fma2(BR[q], X, fma2(AR[q], YRL[q], mul2(NAI[q], YIL[q]))),
                                         add2(e1, e2));
                // Im: ar yih + ai yrh exactly, + (bi x + ar yil + ai yrl) once rounded
                const uint64_t p3 = mul2(AR[q], YIH[q]), e3 = fma2(NAR[q], YIH[q], p3);
                const uint64_t p4 = mul2(AI[q], YRH[q]), e4 = fma2(NAI[q], YRH[q], p4);
                const uint64_t li = sub2(fma2(BI[q], X, fma2(AR[q], YIL[q], mul2(AI[q], YRL[q]))),
                                         add2(e3, e4));
                lead2(p1, p2, lr, YRH[q], YRL[q]);
                lead2(p3, p4, li, YIH[q], YIL[q]);
                ZR = q == 0 ? add2(YRH[q], YRL[q]) : add2(ZR, add2(YRH[q], YRL[q]));
                ZI = q == 0 ? add2(YIH[q], YIL[q]) : add2(ZI, add2(YIH[q], YIL[q]));
            }
            float sr = 0.f, si = 0.f;
            if (NP > 0) {
                float lo, hi;
                upk(ZR, lo, hi);
                sr = lo + hi;
                upk(ZI, lo, hi);
                si = lo + hi;
            }
            if (ODD) {
                const float x = lds_f32(ad[F - 1] + 4u * t);
                const float p1 = __fmul_rn(ar1, yrh1), e1 = __fmaf_rn(-ar1, yrh1, p1);
                const float p2 = __fmul_rn(-ai1, yih1), e2 = __fmaf_rn(ai1, yih1, p2);
                const float lr = __fsub_rn(__fmaf_rn(br1, x, __fmaf_rn(ar1, yrl1, __fmul_rn(-ai1, yil1))),
                                           __fadd_rn(e1, e2));
                const float p3 = __fmul_rn(ar1, yih1), e3 = __fmaf_rn(-ar1, yih1, p3);
                const float p4 = __fmul_rn(ai1, yrh1), e4 = __fmaf_rn(-ai1, yrh1, p4);
                const float li = __fsub_rn(__fmaf_rn(bi1, x, __fmaf_rn(ar1, yil1, __fmul_rn(ai1, yrl1))),
                                           __fadd_rn(e3, e4));
                float s, bb, tt, lw;
                s = __fadd_rn(p1, p2);
                bb = __fsub_rn(s, p1);
                tt = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
                lw = __fadd_rn(tt, lr);
                yrh1 = __fadd_rn(s, lw);
                yrl1 = __fsub_rn(lw, __fsub_rn(yrh1, s));
                s = __fadd_rn(p3, p4);
                bb = __fsub_rn(s, p3);
                tt = __fadd_rn(__fsub_rn(p3, __fsub_rn(s, bb)), __fsub_rn(p4, bb));
                lw = __fadd_rn(tt, li);
                yih1 = __fadd_rn(s, lw);
                yil1 = __fsub_rn(lw, __fsub_rn(yih1, s));
                sr = NP > 0 ? sr + __fadd_rn(yrh1, yrl1) : __fadd_rn(yrh1, yrl1);
                si = NP > 0 ? si + __fadd_rn(yih1, yil1) : __fadd_rn(yih1, yil1);
            }
            zr[t] = sr;
            zi[t] = si;
        }
    }
    __device__ __forceinline__ void begin(const K1Args &, int) {}
    __device__ __forceinline__ void after8(const K1Args &, int) {}
    __device__ __forceinline__ void finish(const K1Args &, int) {}
    __device__ __forceinline__ float4 word(int r) const
    {
        if (ODD && r == F - 1) return make_float4(yrh1, yrl1, yih1, yil1);
        float a0, a1, b0, b1, c0, c1, d0, d1;
        upk(YRH[r / 2], a0, a1);
        upk(YRL[r / 2], b0, b1);
        upk(YIH[r / 2], c0, c1);
        upk(YIL[r / 2], d0, d1);
        return (r & 1) ? make_float4(a1, b1, c1, d1) : make_float4(a0, b0, c0, d0);
    }
    __device__ __forceinline__ void store(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                          float2 *)
    {
        float4 *st = reinterpret_cast<float4 *>(A.state_ext);
#pragma unroll
        for (int r = 0; r < F; ++r)
            st[(int64_t)det * A.n_slots + pb + ((int64_t)r * A.W + warp) * 32 + lane] = word(r);
    }
    __device__ __forceinline__ float2 state_of(int r) const
    {
        const float4 w = word(r);
        return make_float2(w.x + w.y, w.z + w.w);
    }
};

// Chunked scan with an FP64 carry (chunks of A.chunk samples from the start
// of the call).  Per chunk each filter runs two FP32 recurrences on the same
// strain: y from the anchored state (its outputs feed z) and u from zero
// state (the chunk's input projection S = sum_j a^(T-1-j) b x[...]).  At the
// chunk end the anchor advances in FP64, s <- a^T s + S, and y restarts from
// s rounded to FP32, so FP32 error never builds up over more than one chunk.
template <int F> struct ChunkLanes {
    static constexpr int kF = F;
    float ar[F], ai[F], br[F], bi[F], yr[F], yi[F], ur[F], ui[F];
    double aTr[F], aTi[F], sr64[F], si64[F];

    __device__ __forceinline__ void load(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                         const float2 *)
    {
        const double2 *st = reinterpret_cast<const double2 *>(A.state_ext);
#pragma unroll
        for (int r = 0; r < F; ++r) {
            const int64_t s = pb + ((int64_t)r * A.W + warp) * 32 + lane;
            const float4 p = A.params[s];
            const double2 y = st[(int64_t)det * A.n_slots + s];
            const double2 t = A.aT[s];
            ar[r] = p.x;
            ai[r] = p.y;
            br[r] = p.z;
            bi[r] = p.w;
            sr64[r] = y.x;
            si64[r] = y.y;
            yr[r] = (float)y.x;
            yi[r] = (float)y.y;
            ur[r] = 0.f;
            ui[r] = 0.f;
            aTr[r] = t.x;
            aTi[r] = t.y;
        }
    }
    template <bool FULL>
    __device__ __forceinline__ void step8(const uint32_t (&ad)[F], int valid, float (&zr)[kTS],
                                          float (&zi)[kTS])
    {
#pragma unroll
        for (int t = 0; t < kTS; ++t) {
            if (!FULL && t >= valid) {
                zr[t] = 0.f;
                zi[t] = 0.f;
                continue;
            }
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int r = 0; r < F; ++r) {
                const float x = lds_f32(ad[r] + 4u * t);
                const float bx = br[r] * x, by = bi[r] * x;
                const float nr = fmaf(ar[r], yr[r], fmaf(-ai[r], yi[r], bx));
                const float ni = fmaf(ar[r], yi[r], fmaf(ai[r], yr[r], by));
                const float mr = fmaf(ar[r], ur[r], fmaf(-ai[r], ui[r], bx));
                const float mi = fmaf(ar[r], ui[r], fmaf(ai[r], ur[r], by));
                yr[r] = nr;
                yi[r] = ni;
                ur[r] = mr;
                ui[r] = mi;
                sr += nr;
                si += ni;
            }
            zr[t] = sr;
            zi[t] = si;
        }
    }
    __device__ __forceinline__ void carry()
    {
#pragma unroll
        for (int r = 0; r < F; ++r) {
            const double nr = fma(aTr[r], sr64[r], fma(-aTi[r], si64[r], (double)ur[r]));
            const double ni = fma(aTr[r], si64[r], fma(aTi[r], sr64[r], (double)ui[r]));
            sr64[r] = nr;
            si64[r] = ni;
            yr[r] = (float)nr;
            yi[r] = (float)ni;
            ur[r] = 0.f;
            ui[r] = 0.f;
        }
    }
    // kend: samples of the call processed so far
    __device__ __forceinline__ void begin(const K1Args &, int) {}
    __device__ __forceinline__ void after8(const K1Args &A, int kend)
    {
        if (kend % A.chunk == 0) carry();
    }
    // a call that ends inside a chunk keeps the FP32 state as its anchor
    __device__ __forceinline__ void finish(const K1Args &A, int n)
    {
        if (n % A.chunk != 0) {
#pragma unroll
            for (int r = 0; r < F; ++r) {
                sr64[r] = yr[r];
                si64[r] = yi[r];
            }
        }
    }
    __device__ __forceinline__ void store(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                          float2 *)
    {
        double2 *st = reinterpret_cast<double2 *>(A.state_ext);
#pragma unroll
        for (int r = 0; r < F; ++r)
            st[(int64_t)det * A.n_slots + pb + ((int64_t)r * A.W + warp) * 32 + lane] =
                make_double2(sr64[r], si64[r]);
    }
    __device__ __forceinline__ float2 state_of(int r) const { return make_float2(yr[r], yi[r]); }
};

// Chunked tensor-core form: plain FP32 lanes that restart, at every
// kTcT-sample chunk start, from the chunk's anchor (the FP64-carried state of
// the chunk scan, rounded once), so FP32 rounding never runs for more than
// kTcT steps.  The next chunk's anchors are loaded a whole chunk ahead.
template <int F> struct AnchorLanes : PackedLanes<F> {
    using Base = PackedLanes<F>;
    float2 nxt[F];
    const float2 *arow = nullptr;   // this lane's anchor of round 0, chunk 0
    int64_t rstride = 0, cstride = 0;
    int nch = 0, ci = 0;

    __device__ __forceinline__ void load(const K1Args &A, int64_t pb, int warp, int lane, int det,
                                         const float2 *)
    {
        Base::load(A, pb, warp, lane, det, A.anchors);   // chunk 0: the segment's start
        arow = A.anchors + (int64_t)det * A.n_slots + pb + (int64_t)warp * 32 + lane;
        rstride = (int64_t)A.W * 32;
        cstride = (int64_t)A.n_det * A.n_slots;
    }
    __device__ __forceinline__ void fetch()
    {
        if (ci < nch) {
#pragma unroll
            for (int r = 0; r < F; ++r) nxt[r] = arow[ci * cstride + r * rstride];
        }
    }
    __device__ __forceinline__ void begin(const K1Args &, int n)
    {
        nch = (n + kTcT - 1) / kTcT;
        ci = 1;
        fetch();
    }
    // e: samples of the segment done
    __device__ __forceinline__ void after8(const K1Args &, int e)
    {
        if (ci < nch && e == ci * kTcT) {
#pragma unroll
            for (int q = 0; q < Base::NP; ++q) {
                this->YR[q] = pk(nxt[2 * q].x, nxt[2 * q + 1].x);
                this->YI[q] = pk(nxt[2 * q].y, nxt[2 * q + 1].y);
            }
            if (Base::ODD) {
                this->yr1 = nxt[F - 1].x;
                this->yi1 = nxt[F - 1].y;
            }
            ++ci;
            fetch();
        }
    }
};

// ---- running peak of one template: warp max, then merge with the plan's --
// overwrite: the CTA is the only writer of this (segment, detector, template)
// entry, which then needs no reset before the launch.
__device__ __forceinline__ void warp_peak_merge(const K1Args &A, float *peak_best,
                                                int64_t *peak_idx, int det, int tmpl, int lane,
                                                float best, int bidx, bool overwrite)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(kFull, best, off);
        const int oi = __shfl_xor_sync(kFull, bidx, off);
        if (ob > best || (ob == best && oi >= 0 && (bidx < 0 || oi < bidx))) {
            best = ob;
            bidx = oi;
        }
    }
    if (lane == 0 && overwrite) {
        const int64_t i = (int64_t)det * A.T + tmpl;
        peak_best[i] = bidx >= 0 ? best : -1.0f;
        peak_idx[i] = bidx >= 0 ? (A.t0_dev != nullptr ? *A.t0_dev : 0) + A.t0 + bidx : -1;
    } else if (lane == 0 && bidx >= 0) {
        const int64_t i = (int64_t)det * A.T + tmpl;
        if (best > peak_best[i]) {
            peak_best[i] = best;
            peak_idx[i] = (A.t0_dev != nullptr ? *A.t0_dev : 0) + A.t0 + bidx;
        }
    }
}

// ---- one CTA work unit: W warps x one detector, whole call ----------------
// The state before the 16-sample span starting at call sample k (a multiple
// of 16): the adjoint's recompute points.
template <class LANES>
__device__ __forceinline__ void save_sub16(const K1Args &A, const LANES &L, int64_t pb, int warp,
                                           int lane, int det, int k)
{
    constexpr int F = LANES::kF;
    float2 *row = A.sub16 + ((int64_t)(k >> 4) * A.n_det + det) * A.n_slots;
#pragma unroll
    for (int r = 0; r < F; ++r) row[pb + ((int64_t)r * A.W + warp) * 32 + lane] = L.state_of(r);
}

// SEG: the CTA serves one time segment of the call; LOW: the call adds lower
// bands (multirate top band).  Both are compile-time so the plain single-band
// kernel carries neither's code.
// Phases of the CTA's two block barriers completed by earlier units (a
// persistent CTA serves many units on the same barriers): bar0 completes one
// phase per even block of a unit, bar1 one per odd block.
struct Phases {
    uint32_t p0 = 0, p1 = 0;
};

template <template <int> class LANES, int F, bool SEG, bool LOW, int U>
__device__ __forceinline__ bool run_unit(const K1Args &A, int g, int det, float *ring,
                                         float *zbuf, uint32_t bar0, uint32_t bar1, Phases &ph)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 wi = A.warp_info[(int64_t)g * A.W + warp];
    const int tmpl = wi.x;
    const bool half = A.G == 16;
    const int tmpl2 = half ? wi.w : -1;      // half-warp mode: template of lanes 16..31
    const int per_warp = half ? 2 : 1;       // template slots per warp
    // lower-band prefetch buffers follow the two block-sum buffers
    float2 *lowbuf = reinterpret_cast<float2 *>(zbuf + (int64_t)2 * A.W * per_warp * A.Tb * 2);
    const bool active = tmpl >= 0;
    const bool leader = active && wi.y == warp;
    const int64_t pb = A.group_pbase[g];
    // this CTA's time segment: call samples [s0, s0 + n) (SEG == false: the
    // whole call, and the segment arithmetic compiles away)
    const int seg = SEG ? A.seg_first + (int)(blockIdx.x / A.n_units) : 0;
    const int nseg_total = SEG ? (A.n + A.n_seg - 1) / A.n_seg : 1;
    const int s0 = SEG ? seg * A.n_seg : 0;
    const int n = SEG ? min(A.n_seg, A.n - s0) : A.n;
    const int sblk = s0 / A.Tb;              // first block of the segment
    const int nblk = (n + A.Tb - 1) / A.Tb;
    const float *xrow = A.xe + (int64_t)det * A.xe_stride + (int64_t)sblk * A.Tb;

    LANES<F> L;
    // per filter: shared byte address of its strain window (ring copy base +
    // ring position), advanced 32 bytes per 8-sample step and wrapped per block
    const uint32_t ring_u32 = smem_addr(ring);
    uint32_t ad[F];
#pragma unroll
    for (int r = 0; r < F; ++r) ad[r] = ring_u32;
    if (active) {
#pragma unroll
        for (int r = 0; r < F; ++r) {
            // xrow starts at the segment: the same ring phase as a whole call
            const int2 ro = A.ringoff[pb + ((int64_t)r * A.W + warp) * 32 + lane];
            ad[r] = ring_u32 + 4u * (uint32_t)(ro.y + ro.x);
        }
        // segments read their start state from seg_init (segment 0's is a copy
        // of the call's start state: the last segment overwrites A.state)
        const float2 *sin =
            !SEG ? A.state
                 : (A.zero_init ? nullptr : A.seg_init + (int64_t)seg * A.n_det * A.n_slots);
        L.load(A, pb, warp, lane, det, sin);
        L.begin(A, n);
    }
    float *zrow = (A.z != nullptr && leader)
                      ? A.z + ((int64_t)det * A.T + tmpl) * 2 * A.z_len
                      : nullptr;
    float *zrow2 = (A.z != nullptr && leader && tmpl2 >= 0)
                       ? A.z + ((int64_t)det * A.T + tmpl2) * 2 * A.z_len
                       : nullptr;
    float best = -1.0f, best2 = -1.0f;
    int bidx = -1, bidx2 = -1;

    // prologue: history blocks + block 0 on bar0, block 1 on bar1
    if (threadIdx.x == 0) {
        uint32_t bytes = 0;
        for (int64_t e = 0; e <= A.H; ++e) bytes += block_bytes(A, e);
        mbar_expect_tx(bar0, bytes);
        for (int64_t e = 0; e <= A.H; ++e) issue_block(A, xrow, ring, e, bar0);
        if (nblk > 1) {
            mbar_expect_tx(bar1, block_bytes(A, A.H + 1));
            issue_block(A, xrow, ring, A.H + 1, bar1);
        }
    }

    int failed_at = -1;
    for (int j = 0; j < nblk; ++j) {
        const uint32_t bar = (j & 1) ? bar1 : bar0;
        const bool ok =
            mbar_wait(bar, (uint32_t)(((j >> 1) + ((j & 1) ? ph.p1 : ph.p0)) & 1), A.wait_limit_ns);
        if (__syncthreads_or(!ok)) {
            failed_at = j;
            break;
        }
        const int k0 = s0 + j * A.Tb;              // call-relative sample index
        const int nv = min(A.Tb, n - j * A.Tb);
        // this block's sums: [W * per_warp template slots][Tb] complex
        float *zb = zbuf + (int64_t)((j & 1) * A.W * per_warp) * A.Tb * 2;
        if (LOW && leader && A.n_lower > 0) {   // lower-band samples for this block's combine
            prefetch_lower(A, lowbuf + (int64_t)(wi.y * per_warp) * A.low_len, det, tmpl, lane,
                           k0, nv);
            if (tmpl2 >= 0)
                prefetch_lower(A, lowbuf + (int64_t)(warp * 2 + 1) * A.low_len, det, tmpl2,
                               lane, k0, nv);
        }
        if (active) {
            float *zw = zb + (int64_t)warp * per_warp * A.Tb * 2;
            // few filters per lane (and registers to spare): U whole steps
            // before their U cross-lane sums, whose shuffle chains then overlap
            int sb = 0;
            if (U > 1) {
                for (; sb + U * kTS <= nv; sb += U * kTS) {
                    float zr[U][kTS], zi[U][kTS];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (SEG && A.sub16 != nullptr && ((sb + u * kTS) & 15) == 0)
                            save_sub16(A, L, pb, warp, lane, det, s0 + j * A.Tb + sb + u * kTS);
                        L.template step8<true>(ad, kTS, zr[u], zi[u]);
                        L.after8(A, j * A.Tb + sb + (u + 1) * kTS);
#pragma unroll
                        for (int r = 0; r < F; ++r) ad[r] += 4u * kTS;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        warp_sum8(zr[u], zi[u], lane, zw + 2 * (sb + u * kTS), half, A.Tb);
                }
            }
            for (; sb < nv; sb += kTS) {
                const int valid = nv - sb;
                if (SEG && A.sub16 != nullptr && (sb & 15) == 0)
                    save_sub16(A, L, pb, warp, lane, det, s0 + j * A.Tb + sb);
                float zr[kTS], zi[kTS];
                if (valid >= kTS)
                    L.template step8<true>(ad, valid, zr, zi);
                else
                    L.template step8<false>(ad, valid, zr, zi);
                warp_sum8(zr, zi, lane, zw + 2 * sb, half, A.Tb);
                L.after8(A, j * A.Tb + sb + min(valid, kTS));
#pragma unroll
                for (int r = 0; r < F; ++r) ad[r] += 4u * kTS;
            }
            // a whole block moved every window by Tb samples: wrap those that
            // left the ring (position within its copy >= R)
            const uint32_t cs4 = 4u * (uint32_t)A.CS, r4 = 4u * (uint32_t)A.R;
#pragma unroll
            for (int r = 0; r < F; ++r) {
                const uint32_t off = ad[r] - ring_u32;
                uint32_t c = 0;
                for (int cc = 1; cc < A.C; ++cc) c += off >= (uint32_t)cc * cs4 ? 1u : 0u;
                if (off - c * cs4 >= r4) ad[r] -= r4;
            }
            // checkpoint of the filter state (for the adjoint's recompute), at
            // whole multiples of the interval from the call's start
            const int gblk = sblk + j + 1;
            if (A.ckpt != nullptr && gblk % A.ckpt_blocks == 0 && (int64_t)gblk * A.Tb < A.n) {
                const int64_t c = gblk / A.ckpt_blocks;
                float2 *row = A.ckpt + (c * A.n_det + det) * A.n_slots;
#pragma unroll
                for (int r = 0; r < F; ++r)
                    row[pb + ((int64_t)r * A.W + warp) * 32 + lane] = L.state_of(r);
            }
        }
        // every warp is done with the ring slot the next copy overwrites, and
        // this block's per-warp sums are visible
        __syncthreads();
        if (threadIdx.x == 0 && j + 2 < nblk) {
            const int64_t e = (int64_t)A.H + j + 2;
            mbar_expect_tx(bar, block_bytes(A, e));
            issue_block(A, xrow, ring, e, bar);
        }
        if (leader) {
            combine_block<LOW>(A, reinterpret_cast<const float2 *>(zb), wi.y * per_warp, wi.z,
                          lowbuf + (int64_t)(wi.y * per_warp) * A.low_len, lane, k0, nv, zrow,
                          best, bidx);
            if (tmpl2 >= 0)
                combine_block<LOW>(A, reinterpret_cast<const float2 *>(zb), warp * 2 + 1, 1,
                              lowbuf + (int64_t)(warp * 2 + 1) * A.low_len, lane, k0, nv, zrow2,
                              best2, bidx2);
        }
    }
    if (failed_at >= 0) {
        if (threadIdx.x == 0) {
            atomicOr(A.err, 1);
            // let copies still in flight land before the CTA's memory is reused:
            // the block that timed out, and the one issued after it (bounded)
            const int j = failed_at;
            mbar_wait((j & 1) ? bar1 : bar0,
                      (uint32_t)(((j >> 1) + ((j & 1) ? ph.p1 : ph.p0)) & 1), A.wait_limit_ns);
            if (j + 1 < nblk)
                mbar_wait(((j + 1) & 1) ? bar1 : bar0,
                          (uint32_t)((((j + 1) >> 1) + (((j + 1) & 1) ? ph.p1 : ph.p0)) & 1),
                          A.wait_limit_ns);
        }
        return false;
    }
    ph.p0 += (uint32_t)((nblk + 1) / 2);
    ph.p1 += (uint32_t)(nblk / 2);
    if (!active) return true;
    L.finish(A, n);
    {
        float2 *sout = !SEG ? A.state
                            : (A.seg_end != nullptr
                                   ? A.seg_end + (int64_t)seg * A.n_det * A.n_slots
                                   : (seg == nseg_total - 1 ? A.state : nullptr));
        L.store(A, pb, warp, lane, det, sout);
    }
    // running peak: largest |z|^2, earliest index on ties
    if (leader && A.peak_best != nullptr) {
        const bool own = SEG && A.peak_seg_stride != 0;   // per-segment entries
        float *peak_best = A.peak_best + (own ? seg * A.peak_seg_stride : 0);
        int64_t *peak_idx = A.peak_idx + (own ? seg * A.peak_seg_stride : 0);
        warp_peak_merge(A, peak_best, peak_idx, det, tmpl, lane, best, bidx, own);
        if (tmpl2 >= 0)
            warp_peak_merge(A, peak_best, peak_idx, det, tmpl2, lane, best2, bidx2, own);
    }
    return true;
}

// Registers per thread follow the filters-per-lane cap: CTAs of up to 256
// threads, min resident CTAs chosen so the cap's register need fits (cap 10
// is held to 128 registers: two CTAs per SM beat the spill-free 170).
template <int FCAP> struct K1Bounds;
template <> struct K1Bounds<2> { static constexpr int kMinBlocks = 4; };
template <> struct K1Bounds<4> { static constexpr int kMinBlocks = 3; };
template <> struct K1Bounds<6> { static constexpr int kMinBlocks = 2; };
template <> struct K1Bounds<8> { static constexpr int kMinBlocks = 2; };
template <> struct K1Bounds<10> { static constexpr int kMinBlocks = 2; };

// Steps per cross-lane-sum batch for F filters per lane in a kernel compiled
// for FCAP (only the 128-register kernels have room for several; the time-
// segmented kernels, which carry more state, only for F <= 4).  Two steps
// per batch up to 10 filters per lane measured 0.8% faster on the batched
// bank than up to 8, despite a few spilled registers outside the loop.
__host__ __device__ constexpr int unroll_for(int FCAP, int F, bool SEG)
{
    return FCAP >= 6 ? (F <= 2 ? 4 : (F <= (SEG ? 4 : 10) ? 2 : 1)) : 1;
}

// The CTA's F is uniform, so every warp takes the same case.  Returns false
// when a bounded wait gave up (the CTA then stops).
template <template <int> class LANES, int FCAP, bool SEG, bool LOW>
__device__ __forceinline__ bool dispatch_f(const K1Args &A, int g, int det, float *ring,
                                           float *zbuf, uint32_t bar0, uint32_t bar1, Phases &ph)
{
    const int F = A.group_F[g];
#define SPIIR_K1_CASE(FF)                                                                     \
    if (FCAP >= FF && F == FF)                                                               \
        return run_unit<LANES, (FCAP >= FF ? FF : 1), SEG, LOW,                              \
                        unroll_for(FCAP, (FCAP >= FF ? FF : 1), SEG)>(A, g, det, ring, zbuf, \
                                                                      bar0, bar1, ph);
    SPIIR_K1_CASE(1)
    SPIIR_K1_CASE(2)
    SPIIR_K1_CASE(3)
    SPIIR_K1_CASE(4)
    SPIIR_K1_CASE(5)
    SPIIR_K1_CASE(6)
    SPIIR_K1_CASE(7)
    SPIIR_K1_CASE(8)
    SPIIR_K1_CASE(9)
    SPIIR_K1_CASE(10)
#undef SPIIR_K1_CASE
    if (threadIdx.x == 0) atomicOr(A.err, 4);
    return false;
}

// Persistent CTAs: the units come in order of non-increasing F (the
// layout sorts them so), so a CTA runs one stage per F, from the cap down,
// each looping over the units of its F; a stage's loop holds one
// instantiation of run_unit, and the stages follow each other without an
// enclosing loop (a loop around all of them keeps every instantiation's
// hoisted invariants live at once).  Returns the first unit not served.
template <int FCAP, bool LOW, int F>
__device__ __forceinline__ int run_stage(const K1Args &A, int u, float *ring, float *zbuf,
                                         uint32_t bar0, uint32_t bar1, Phases &ph, int *next,
                                         bool &ok)
{
    if constexpr (F <= FCAP) {
        while (ok && u < A.n_units && A.group_F[A.units[2 * u]] == F) {
            ok = run_unit<PackedLanes, F, false, LOW, unroll_for(FCAP, F, false)>(
                A, A.units[2 * u], A.units[2 * u + 1], ring, zbuf, bar0, bar1, ph);
            if (!ok) break;
            // every warp is done with the ring, the block sums and `next`
            __syncthreads();
            if (threadIdx.x == 0) *next = atomicAdd(A.queue, 1);
            __syncthreads();
            u = *next;
        }
    }
    return u;
}

__device__ __forceinline__ void cta_setup(unsigned char *smem, const K1Args &A, float *&ring,
                                          float *&zbuf, uint32_t &bar0, uint32_t &bar1)
{
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    ring = reinterpret_cast<float *>(smem + 128);
    zbuf = ring + (int64_t)A.C * A.CS;
    bar0 = smem_addr(&bars[0]);
    bar1 = smem_addr(&bars[1]);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// One CTA per unit: CTA b serves unit b (SEG: unit b % n_units of segment
// b / n_units).
template <int FCAP, bool SEG, bool LOW>
__global__ void __launch_bounds__(256, K1Bounds<FCAP>::kMinBlocks) k1_plain(const K1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring, *zbuf;
    uint32_t bar0, bar1;
    cta_setup(smem, A, ring, zbuf, bar0, bar1);
    Phases ph;
    const int u = SEG ? (int)(blockIdx.x % A.n_units) : (int)blockIdx.x;
    dispatch_f<PackedLanes, FCAP, SEG, LOW>(A, A.units[2 * u], A.units[2 * u + 1], ring, zbuf,
                                            bar0, bar1, ph);
}

// Persistent launch of the unsegmented plain kernel: a grid of at most the
// resident CTAs takes units in the layout's order (largest F first) from a
// global counter the launcher zeroes, so the CTAs that finish first take the
// next unit and the smallest units end the launch (see run_stage).
template <int FCAP, bool LOW>
__global__ void __launch_bounds__(256, K1Bounds<FCAP>::kMinBlocks)
    k1_persistent(const K1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring, *zbuf;
    uint32_t bar0, bar1;
    cta_setup(smem, A, ring, zbuf, bar0, bar1);
    Phases ph;
    __shared__ int next;
    if (threadIdx.x == 0) next = atomicAdd(A.queue, 1);
    __syncthreads();
    int u = next;
    bool ok = true;
    u = run_stage<FCAP, LOW, 10>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 9>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 8>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 7>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 6>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 5>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 4>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 3>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 2>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    u = run_stage<FCAP, LOW, 1>(A, u, ring, zbuf, bar0, bar1, ph, &next, ok);
    // a unit out of F order (or an F above the cap) is not served: flag it
    if (ok && u < A.n_units && threadIdx.x == 0) atomicOr(A.err, 4);
}

}  // namespace

template <typename Kernel>
cudaError_t launch_kernel(Kernel k, const K1Args &a, int64_t n_units, int smem_bytes,
                          cudaStream_t s, bool persistent = false)
{
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void *>(k), smem_bytes);
    if (e != cudaSuccess) return e;
    if (persistent && a.queue != nullptr) {
        int ctas = 0;
        if ((e = resident_ctas(reinterpret_cast<const void *>(k), a.W * 32, smem_bytes, &ctas)) !=
            cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(a.queue, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
        const int64_t grid = std::min<int64_t>(n_units, ctas);
        k<<<(unsigned)grid, a.W * 32, smem_bytes, s>>>(a);
        return cudaGetLastError();
    }
    K1Args g = a;
    g.queue = nullptr;   // grid mode: one CTA per unit (and segment)
    const int P = a.n_seg > 0 ? (a.n + a.n_seg - 1) / a.n_seg : 1;
    const int P_launch = a.seg_count > 0 ? a.seg_count
                         : a.seg_end != nullptr ? P - 1   // the projection skips the last
                                                : P;
    if (P_launch <= 0) return cudaSuccess;
    k<<<(unsigned)(n_units * P_launch), a.W * 32, smem_bytes, s>>>(g);
    return cudaGetLastError();
}

template <int FCAP>
cudaError_t launch_k1_cap(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s)
{
    // several time segments, or span starts to keep (only the segment-capable
    // kernels carry that code; one segment runs there as well)
    const bool seg = a.n_seg < a.n || a.sub16 != nullptr;
    if (a.n_lower > 0) {
        if (seg) return launch_kernel(k1_plain<FCAP, true, true>, a, n_units, smem_bytes, s);
        return a.queue != nullptr
                   ? launch_kernel(k1_persistent<FCAP, true>, a, n_units, smem_bytes, s, true)
                   : launch_kernel(k1_plain<FCAP, false, true>, a, n_units, smem_bytes, s);
    }
    if (seg) return launch_kernel(k1_plain<FCAP, true, false>, a, n_units, smem_bytes, s);
    return a.queue != nullptr
               ? launch_kernel(k1_persistent<FCAP, false>, a, n_units, smem_bytes, s, true)
               : launch_kernel(k1_plain<FCAP, false, false>, a, n_units, smem_bytes, s);
}

// per-cap launchers and kernel handles (spiir_k1_capN.cu) and the
// precision forms' launcher (spiir_k1_precise.cu)
cudaError_t launch_k1_cap_2(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
const void *k1_plain_kernel_2();
cudaError_t launch_k1_cap_4(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
const void *k1_plain_kernel_4();
cudaError_t launch_k1_cap_6(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
const void *k1_plain_kernel_6();
cudaError_t launch_k1_cap_8(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
const void *k1_plain_kernel_8();
cudaError_t launch_k1_cap_10(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);
const void *k1_plain_kernel_10();
cudaError_t launch_k1_precise(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);

}  // namespace spiir
