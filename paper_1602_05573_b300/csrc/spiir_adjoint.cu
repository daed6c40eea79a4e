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
// The reverse pass (k6_adjoint: g_a, g_b) needs y_l[k-1] at every k.
// Recomputing y backwards through 1/a_l is unstable, so the forward kernel
// stores the state every Cc samples (and, when memory allows, at every
// kAdjSub-sample span start); without the span starts this kernel, for each
// chunk in reverse order, recomputes the chunk forward from its checkpoint
// (pass A, keeping the state every kAdjSub samples in a workspace), then for
// each kAdjSub-sample span in reverse recomputes the span into registers
// (pass B) and runs the adjoint over it.
//
// Mapping: filters are independent in the adjoint, so the unit of work is a
// task of two filter rounds (32 filters each) of one template; lane i runs
// its two filters as one packed FP32x2 pair (every recurrence and gradient
// update is one fma/mul.rn.f32x2 for both) and keeps mu, g_a, g_b in
// registers.  Long calls run as time segments of whole checkpoint
// intervals, each from the adjoint state projected to its end.  A CTA runs
// W tasks of one detector and stages each chunk's strain window in shared
// memory; g_z of the template is read by lanes 0..15 once per span and
// broadcast with shuffles.  g_x comes from k7_adjoint_x (below), in the
// shifted frame where it is a sum, not a scatter.
#include "spiir_kernels.h"
#include "spiir_ptx.h"

#include <cstdint>

namespace spiir {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(256, 2) k6_adjoint(const K6Args A)
{
    // a lane's two filter rounds share FP32x2 registers: (round 0, round 1)
    static_assert(kAdjRounds == 2, "the reverse pass pairs its two rounds");
    static_assert(kAdjSub == 16, "the forward keeps span starts every 16 samples");
    constexpr int R = kAdjRounds;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Dw = A.Dh + A.Cc;                          // strain window per chunk
    float *xs = reinterpret_cast<float *>(smem);         // [Dw]
    const int nsub_max = A.Cc / kAdjSub;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = (int)(blockIdx.x / A.n_units);
    const int u = (int)(blockIdx.x % A.n_units);
    const int g = A.units[2 * u];
    const int det = A.units[2 * u + 1];
    const int4 task = A.tasks[(int64_t)g * A.W + warp];
    const bool half = A.G == 16;                      // lanes 16..31 serve task.w
    const bool active = task.z >= 0;
    const int tmpl = (half && lane >= 16) ? task.w : task.z;
    const int nr = task.y;                   // rounds in this task (<= R)
    const int n = A.n;
    const int nc = (n + A.Cc - 1) / A.Cc;
    const int c_lo = seg * A.cps;                     // this CTA's chunks [c_lo, c_hi)
    const int c_hi = min(nc, c_lo + A.cps);
    const float *xrow = A.xe + (int64_t)det * A.xe_stride;
    const float2 *grow = tmpl >= 0 ? A.gz + ((int64_t)det * A.T + tmpl) * n : nullptr;
    const int gsrc = half ? (lane & 16) : 0;          // lane holding this lane's g_z
    float2 *wsub = A.sub + ((int64_t)blockIdx.x * A.W + warp) * R * nsub_max * 32;
    float *acc_det = A.acc + ((int64_t)seg * A.n_det + det) * A.n_slots * 6;

    // this lane's filters: slot of round i = task.x + i * round_stride + lane
    int64_t slot[R];
    float ar[R], ai[R], br[R], bi[R], m0r[R], m0i[R];
    int xo[R];
    const bool odd = (lane & 1) != 0;   // stored as conj(a), (Im b, Re b)
#pragma unroll
    for (int i = 0; i < R; ++i) {
        slot[i] = active ? (int64_t)task.x + (int64_t)i * A.round_stride + lane : 0;
        ar[i] = ai[i] = br[i] = bi[i] = m0r[i] = m0i[i] = 0.f;
        xo[i] = 0;
        if (active && i < nr) {
            const float4 p = A.params[slot[i]];
            ar[i] = p.x;
            ai[i] = odd ? -p.y : p.y;
            br[i] = odd ? p.w : p.z;
            bi[i] = odd ? p.z : p.w;
            xo[i] = A.ringoff[slot[i]].x;   // Dh - d: xs index of x[kc - d]
            if (A.mu_end != nullptr) {      // adjoint state after the segment
                const float2 m =
                    A.mu_end[((int64_t)seg * A.n_det + det) * A.n_slots + slot[i]];
                m0r[i] = m.x;
                m0i[i] = m.y;
            }
        }
    }
    const uint64_t AR = pk(ar[0], ar[1]), AI = pk(ai[0], ai[1]), NAI = pk(-ai[0], -ai[1]);
    const uint64_t BR = pk(br[0], br[1]), BI = pk(bi[0], bi[1]);
    uint64_t MR = pk(m0r[0], m0r[1]), MI = pk(m0i[0], m0i[1]);
    // seeds of the input-gradient pass: segment q' of that pass starts from
    // mu at k_t = (q' + 1) S + d, which lies in this segment when
    // q' = seg - d / S - 1; the state at the top of the 16-sample span holding
    // k_t is kept (-1: no target here)
    const int S = A.cps * A.Cc;
    int span_t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int d = A.Dh - xo[i];
        const int q = seg - d / S - 1;
        const int kt = seg * S + d % S;
        span_t[i] = (A.seeds != nullptr && active && i < nr && q >= 0 && q + 1 < A.P && kt < n)
                        ? (kt & ~(kAdjSub - 1)) : -1;
    }
    // g_a = sum mu conj(y[k-1]): Re in GAR, Im = GAI1 - GAI2; g_b = sum mu x
    uint64_t GAR = 0, GAI1 = 0, GAI2 = 0, GBR = 0, GBI = 0;

    for (int c = c_hi - 1; c >= c_lo; --c) {
        const int kc = c * A.Cc;
        const int cv = min(A.Cc, n - kc);
        // strain x[kc - Dh + i] = xe[kc + i] (xe holds Dh zeros before x)
        for (int i = threadIdx.x; i < Dw; i += blockDim.x) xs[i] = i < A.Dh + cv ? xrow[kc + i] : 0.f;
        __syncthreads();
        if (active) {
            const int nsub = (cv + kAdjSub - 1) / kAdjSub;
            const bool have_sub = A.sub16 != nullptr;   // the forward kept every span's start
            float yr0 = 0.f, yi0 = 0.f, yr1 = 0.f, yi1 = 0.f;   // state y[kc - 1]
            if (c > 0 && !have_sub) {
                const float2 *row = A.ckpt + ((int64_t)c * A.n_det + det) * A.n_slots;
                const float2 c0 = row[slot[0]];
                yr0 = odd ? c0.y : c0.x;
                yi0 = odd ? c0.x : c0.y;
                if (nr > 1) {
                    const float2 c1 = row[slot[1]];
                    yr1 = odd ? c1.y : c1.x;
                    yi1 = odd ? c1.x : c1.y;
                }
            }
            uint64_t YR = pk(yr0, yr1), YI = pk(yi0, yi1);
            // pass A: forward over the chunk, state kept every kAdjSub samples
            for (int q = 0; q < (have_sub ? 0 : nsub); ++q) {
                {
                    float a0, a1, b0, b1;
                    upk(YR, a0, a1);
                    upk(YI, b0, b1);
                    wsub[((int64_t)q * R + 0) * 32 + lane] = make_float2(a0, b0);
                    wsub[((int64_t)q * R + 1) * 32 + lane] = make_float2(a1, b1);
                }
                const int k0 = q * kAdjSub;
#pragma unroll
                for (int t = 0; t < kAdjSub; ++t) {
                    if (k0 + t < cv) {
                        const uint64_t X = pk(xs[xo[0] + k0 + t], xs[xo[1] + k0 + t]);
                        uint64_t TR = mul2(BR, X), TI = mul2(BI, X);
                        TR = fma2(NAI, YI, TR);   // br x - ai yi
                        TI = fma2(AI, YR, TI);    // bi x + ai yr
                        YR = fma2(AR, YR, TR);
                        YI = fma2(AR, YI, TI);
                    }
                }
            }
            // pass B: spans in reverse; y[k-1] recomputed into registers
            for (int q = nsub - 1; q >= 0; --q) {
                const int k0 = q * kAdjSub;
#pragma unroll
                for (int i = 0; i < R; ++i)
                    if (span_t[i] == kc + k0) {   // mu at kc + k0 + 16
                        float r0, r1, i0, i1;
                        upk(MR, r0, r1);
                        upk(MI, i0, i1);
                        const int qs = seg - (A.Dh - xo[i]) / S - 1;
                        A.seeds[((int64_t)qs * A.n_det + det) * A.n_slots + slot[i]] =
                            i == 0 ? make_float2(r0, i0) : make_float2(r1, i1);
                    }
                uint64_t PR[kAdjSub], PI[kAdjSub];   // y[k0 + t - 1], both rounds
                {
                    float2 s0, s1;
                    if (have_sub) {   // kernel form from the forward: odd lanes (im, re)
                        const float2 *row =
                            A.sub16 + ((int64_t)((kc + k0) >> 4) * A.n_det + det) * A.n_slots;
                        const float2 c0 = row[slot[0]];
                        const float2 c1 = nr > 1 ? row[slot[1]] : make_float2(0.f, 0.f);
                        s0 = odd ? make_float2(c0.y, c0.x) : c0;
                        s1 = odd ? make_float2(c1.y, c1.x) : c1;
                    } else {
                        s0 = wsub[((int64_t)q * R + 0) * 32 + lane];
                        s1 = wsub[((int64_t)q * R + 1) * 32 + lane];
                    }
                    uint64_t UR = pk(s0.x, s1.x), UI = pk(s0.y, s1.y);
#pragma unroll
                    for (int t = 0; t < kAdjSub; ++t) {
                        PR[t] = UR;
                        PI[t] = UI;
                        if (t + 1 < kAdjSub) {
                            const uint64_t X = pk(xs[xo[0] + k0 + t], xs[xo[1] + k0 + t]);
                            uint64_t TR = mul2(BR, X), TI = mul2(BI, X);
                            TR = fma2(NAI, UI, TR);
                            TI = fma2(AI, UR, TI);
                            UR = fma2(AR, UR, TR);
                            UI = fma2(AR, UI, TI);
                        }
                    }
                }
                // lanes gsrc + t hold g_z[k0 + t] of their half's template
                float2 gl = make_float2(0.f, 0.f);
                const int tl = lane & 15;
                if ((half || lane < 16) && grow != nullptr && k0 + tl < cv)
                    gl = grow[kc + k0 + tl];
                // one reverse step.  Steps past the call's end (the last span
                // of a call of n % 16 != 0) run on g_z = 0 from mu = 0 (the
                // last segment starts from zero): mu stays exactly 0 and every
                // update they make adds zero.
#pragma unroll
                for (int t = kAdjSub - 1; t >= 0; --t) {
                    const float Gr = __shfl_sync(kFull, gl.x, gsrc + t);
                    const float Gi = __shfl_sync(kFull, gl.y, gsrc + t);
                    // mu <- g_z + conj(a) mu
                    const uint64_t NMR = fma2(AR, MR, fma2(AI, MI, pk(Gr, Gr)));
                    const uint64_t NMI = fma2(AR, MI, fma2(NAI, MR, pk(Gi, Gi)));
                    MR = NMR;
                    MI = NMI;
                    // g_a += mu conj(y[k-1]),  g_b += mu x[k-d]
                    GAR = fma2(MR, PR[t], fma2(MI, PI[t], GAR));
                    GAI1 = fma2(MI, PR[t], GAI1);
                    GAI2 = fma2(MR, PI[t], GAI2);
                    const uint64_t X = pk(xs[xo[0] + k0 + t], xs[xo[1] + k0 + t]);
                    GBR = fma2(MR, X, GBR);
                    GBI = fma2(MI, X, GBI);
                    // keeps the compiler from hoisting later steps' loads
                    // into registers (128 per thread at two CTAs per SM)
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }
    if (active) {
        float v[6][R];
        upk(MR, v[0][0], v[0][1]);
        upk(MI, v[1][0], v[1][1]);
        upk(GAR, v[2][0], v[2][1]);
        float i1[R], i2[R];
        upk(GAI1, i1[0], i1[1]);
        upk(GAI2, i2[0], i2[1]);
        v[3][0] = i1[0] - i2[0];
        v[3][1] = i1[1] - i2[1];
        upk(GBR, v[4][0], v[4][1]);
        upk(GBI, v[5][0], v[5][1]);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (i >= nr) continue;
            float *acc = acc_det + slot[i] * 6;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] = v[k][i];
        }
    }
}

// Input gradient (the g_x part of the adjoint).  In the shifted frame
// nu_l[m] = mu_l[m + d_l] every filter reads its template's g_z at its own
// delay and all filters of the bank meet at the same output m, so the sum
// over filters is a reduction, not a scatter.  A CTA serves one unit (the
// tasks of one template, or one half-warp pair of templates) of one detector
// over one time segment [q S, (q + 1) S), in reverse.  Per chunk of kK7Chunk
// outputs it stages the template's g_z window [mc, mc + kK7Chunk + Dh) as
// re and im planes; lane i runs its two filters as one FP32x2 pair,
//     nu <- g_z[m + d] + conj(a) nu,    c = Re(conj(nu) b)  (both summed),
// and writes c for 32 consecutive outputs into a 32 x 32 warp tile, XOR
// swizzled so that the writes (one row) and the reads (lane j sums row j)
// both hit 32 banks.  The warps' sums meet in a fixed order and go to g_x
// with one atomic per output and CTA.
//
// Segment q < P - 1 starts from nu[(q + 1) S] = mu[(q + 1) S + d].
// TAN = false: the reverse pass kept mu at the top of the 16-sample span
// holding (q + 1) S + d; at most 16 reverse steps on g_z from there give it.
// TAN = true (the tangent form, which has no reverse pass): A.seeds holds
// mu at the common time B = (q + 1) S + Dh (the reverse projection over
// segments shifted by Dh).  The CTA first runs Dh warm-up steps
// m = B - 1 .. (q + 1) S from zero state with g_z read as zero from B on,
// which gives nu[(q + 1) S] but for the seed's share, then adds that share,
//     nu[(q + 1) S] += conj(a)^(Dh - d) mu[B].
// With TAN the CTA also sums g_b = sum_m nu[m] x[m] (x is the detector's
// strain, the same for every filter at output m) into A.acc.
template <int NP, bool TAN>
__global__ void __launch_bounds__(kK7MaxWarps * 32, 3) k7_adjoint_x(const K7Args A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int R = kAdjRounds;
    const int n_win = A.G == 16 ? 2 : 1;
    // g_z ring: window [mc, mc + Wd) of the chunk at output mc, sample j at
    // position j mod Wd, the first 32 positions mirrored after the end so a
    // 32-step run never wraps; each chunk after the first brings only its
    // kK7Chunk new samples
    const int Wd = kK7Chunk + A.Dh;                 // window length
    const int PL = Wd + 32;                         // plane stride (ring + mirror)
    float *win = reinterpret_cast<float *>(smem);   // [n_win][2][PL]: re plane, im plane
    float *tile = win + n_win * 2 * PL;             // [W][32][32]
    float *part = tile + A.W * 1024;                // [W][kK7Chunk]
    float *xsh = part + A.W * kK7Chunk;             // [kK7Chunk] strain of the chunk (TAN)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = A.n_units * A.n_det;
    const int seg = (int)(blockIdx.x / per);
    const int u = (int)(blockIdx.x % per) / A.n_det, det = (int)(blockIdx.x % per) % A.n_det;
    const int2 unit = A.units[u];
    const int n_warps = (unit.y + NP - 1) / NP;     // warps with tasks
    const bool active = warp < n_warps;
    const int4 head = A.tasks[unit.x];               // the unit's template(s)
    const int n = A.n;
    const int mlo = seg * A.S, mhi = min(n, mlo + A.S);
    const bool warm = TAN && seg + 1 < A.P;
    const int gend = warm ? min(n, mhi + A.Dh) : n; // g_z reads as zero from here on
    const int wsel = (A.G == 16 && lane >= 16) ? 1 : 0;
    const int tmpl = wsel ? head.w : head.z;
    const float2 *grow = A.gz + ((int64_t)det * A.T + (tmpl >= 0 ? tmpl : 0)) * n;
    const float *pr = win + wsel * 2 * PL;

    // slot of round i of task kk at this lane
    auto slot_at = [&](int kk, int i) -> int64_t {
        return (int64_t)A.tasks[kk].x + (int64_t)i * A.round_stride + lane;
    };
    // pair p of this lane: the two rounds of task unit.x + NP warp + p
    uint64_t AR[NP], AI[NP], NAI[NP], BR[NP], BI[NP], NR[NP], NI[NP], GBR[NP], GBI[NP];
    int dd[NP][R];   // delays (ring offsets of the window reads)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int k = NP * warp + p;
        const bool on = active && k < unit.y;
        const int4 task = A.tasks[unit.x + (on ? k : 0)];
        const int nr = on ? task.y : 0;
        float ar[R], ai[R], br[R], bi[R], nu_r[R], nu_i[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            ar[i] = ai[i] = br[i] = bi[i] = nu_r[i] = nu_i[i] = 0.f;
            dd[p][i] = 0;
            if (i >= nr) continue;
            const int64_t slot = slot_at(unit.x + k, i);
            const bool odd = (slot & 1) != 0;   // stored as conj(a), (Im b, Re b)
            const float4 q = A.params[slot];
            ar[i] = q.x;
            ai[i] = odd ? -q.y : q.y;
            br[i] = odd ? q.w : q.z;
            bi[i] = odd ? q.z : q.w;
            const int d = A.Dh - A.ringoff[slot].x;
            dd[p][i] = d;
            // start state nu[(q + 1) S] = mu[(q + 1) S + d] (zero past the call)
            const int kt = mhi + d;
            if (!TAN && seg + 1 < A.P && kt < n && tmpl >= 0) {
                const float2 m0 = A.seeds[((int64_t)seg * A.n_det + det) * A.n_slots + slot];
                float mr = m0.x, mi = m0.y;
                for (int j = (kt & ~(kAdjSub - 1)) + kAdjSub - 1; j >= kt; --j) {
                    const float2 g = j < n ? grow[j] : make_float2(0.f, 0.f);
                    const float tr = fmaf(ar[i], mr, fmaf(ai[i], mi, g.x));
                    const float ti = fmaf(ar[i], mi, fmaf(-ai[i], mr, g.y));
                    mr = tr;
                    mi = ti;
                }
                nu_r[i] = mr;
                nu_i[i] = mi;
            }
        }
        AR[p] = pk(ar[0], ar[1]);
        AI[p] = pk(ai[0], ai[1]);
        NAI[p] = pk(-ai[0], -ai[1]);
        BR[p] = pk(br[0], br[1]);
        BI[p] = pk(bi[0], bi[1]);
        NR[p] = pk(nu_r[0], nu_r[1]);
        NI[p] = pk(nu_i[0], nu_i[1]);
        GBR[p] = 0;
        GBI[p] = 0;
    }
    float *wt = tile + warp * 1024;
    float *gxrow = A.gx + (int64_t)det * n;
    // x[0 .. n) of this detector (TAN)
    const float *xrow = TAN ? A.xe + (int64_t)det * A.xe_stride + A.Dh : nullptr;

    // g_z samples [j0, j1) into the ring, zero from gend on
    auto fill = [&](int j0, int j1) {
        for (int w = 0; w < n_win; ++w) {
            const int t = w ? head.w : head.z;
            const float2 *row = A.gz + ((int64_t)det * A.T + (t >= 0 ? t : 0)) * n;
            float *dr = win + w * 2 * PL;
            for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
                const float2 v = (t >= 0 && j < gend) ? row[j] : make_float2(0.f, 0.f);
                const int q = j % Wd;
                dr[q] = v.x;
                dr[PL + q] = v.y;
                if (q < 32) {
                    dr[Wd + q] = v.x;
                    dr[PL + Wd + q] = v.y;
                }
            }
        }
    };
    bool first_chunk = true;
    auto stage = [&](int mc) {   // the window of the chunk at output mc
        if (first_chunk) fill(mc, mc + Wd);
        else fill(mc, mc + kK7Chunk);   // the previous chunk was at mc + kK7Chunk
        first_chunk = false;
    };
    // ring positions of the 32-step run from output m0 up, per pair and round
    int ob[NP][R];
    auto run_at = [&](int m0) {
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int i = 0; i < R; ++i) ob[p][i] = (m0 + dd[p][i]) % Wd;
    };
    // one reverse step of pair p at output m0 + t of the current run
    auto step = [&](int p, int t) {
        const uint64_t GR = pk(pr[ob[p][0] + t], pr[ob[p][1] + t]);
        const uint64_t GI = pk(pr[PL + ob[p][0] + t], pr[PL + ob[p][1] + t]);
        const uint64_t nR = fma2(AR[p], NR[p], fma2(AI[p], NI[p], GR));
        const uint64_t nI = fma2(AR[p], NI[p], fma2(NAI[p], NR[p], GI));
        NR[p] = nR;
        NI[p] = nI;
    };

    if (warm) {
        // warm-up over outputs [mhi, mhi + Dh), no output
        for (int c = A.Dh / kK7Chunk - 1; c >= 0; --c) {
            const int mc = mhi + c * kK7Chunk;
            stage(mc);
            __syncthreads();
            if (active)
                for (int blk = kK7Chunk / 32 - 1; blk >= 0; --blk) {
                    run_at(mc + blk * 32);
#pragma unroll
                    for (int t = 31; t >= 0; --t) {
#pragma unroll
                        for (int p = 0; p < NP; ++p) step(p, t);
                    }
                }
            __syncthreads();
        }
        // the seed's share: nu += conj(a)^(Dh - d) mu[B]
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int k = NP * warp + p;
            if (!active || k >= unit.y || tmpl < 0) continue;
            const int4 task = A.tasks[unit.x + k];
            float nr_[R], ni_[R], ar_[R], ai_[R];
            upk(NR[p], nr_[0], nr_[1]);
            upk(NI[p], ni_[0], ni_[1]);
            upk(AR[p], ar_[0], ar_[1]);
            upk(AI[p], ai_[0], ai_[1]);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (i >= task.y) continue;
                const int64_t slot = slot_at(unit.x + k, i);
                const float2 m0 = A.seeds[((int64_t)seg * A.n_det + det) * A.n_slots + slot];
                // conj(a)^e, e = Dh - d, by binary powering
                float br_ = ar_[i], bi_ = -ai_[i], pr_ = 1.f, pi_ = 0.f;
                for (int e = A.ringoff[slot].x; e > 0; e >>= 1) {
                    if (e & 1) {
                        const float t = pr_ * br_ - pi_ * bi_;
                        pi_ = pr_ * bi_ + pi_ * br_;
                        pr_ = t;
                    }
                    const float t = br_ * br_ - bi_ * bi_;
                    bi_ = 2.f * br_ * bi_;
                    br_ = t;
                }
                nr_[i] += pr_ * m0.x - pi_ * m0.y;
                ni_[i] += pr_ * m0.y + pi_ * m0.x;
            }
            NR[p] = pk(nr_[0], nr_[1]);
            NI[p] = pk(ni_[0], ni_[1]);
        }
    }

    const int n_chunks = (mhi - mlo + kK7Chunk - 1) / kK7Chunk;
    for (int c = n_chunks - 1; c >= 0; --c) {
        const int mc = mlo + c * kK7Chunk;
        const int cv = min(kK7Chunk, mhi - mc);
        stage(mc);
        if (TAN)
            for (int i = threadIdx.x; i < kK7Chunk; i += blockDim.x)
                xsh[i] = mc + i < n ? xrow[mc + i] : 0.f;
        __syncthreads();
        if (active) {
            // steps at m >= n (the top block of the call's last chunk) run on
            // g_z = 0 from nu = 0 and give zeros
            for (int blk = (cv + 31) / 32 - 1; blk >= 0; --blk) {
                const int mb = blk * 32;
                run_at(mc + mb);
#pragma unroll
                for (int t = 31; t >= 0; --t) {
                    float c = 0.f;
                    const float xv = TAN ? xsh[mb + t] : 0.f;
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        step(p, t);
                        float c0, c1;
                        upk(fma2(NR[p], BR[p], mul2(NI[p], BI[p])), c0, c1);
                        c += c0 + c1;
                        if (TAN) {
                            const uint64_t X = pk(xv, xv);
                            GBR[p] = fma2(NR[p], X, GBR[p]);
                            GBI[p] = fma2(NI[p], X, GBI[p]);
                        }
                    }
                    wt[t * 32 + (lane ^ t)] = c;
                }
                __syncwarp();
                // lane j: the warp's sum at output mb + j, in four chains
                float s4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int e = 0; e < 32; ++e) s4[e & 3] += wt[lane * 32 + (e ^ lane)];
                part[warp * kK7Chunk + mb + lane] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cv; i += blockDim.x) {
            float v = 0.f;
            for (int w = 0; w < n_warps; ++w) v += part[w * kK7Chunk + i];
            if (v != 0.f) atomicAdd(&gxrow[mc + i], v);
        }
        __syncthreads();
    }
    if (TAN && active) {
        // this segment's share of g_b = sum_m nu[m] x[m], natural form
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int k = NP * warp + p;
            if (k >= unit.y) continue;
            const int4 task = A.tasks[unit.x + k];
            float r[R], im[R];
            upk(GBR[p], r[0], r[1]);
            upk(GBI[p], im[0], im[1]);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (i >= task.y) continue;
                const int64_t slot = slot_at(unit.x + k, i);
                float *acc = A.acc + (((int64_t)seg * A.n_det + det) * A.n_slots + slot) * 6;
                acc[4] = r[i];
                acc[5] = im[i];
            }
        }
    }
}

// Gradients of a and b in tangent form.  y_l is linear in b_l and starts
// from zero, so y_l = b_l u_l with the unit-gain response
//     u_l[k] = a_l u_l[k-1] + x[k-d_l]                      (= dy_l[k]/db_l),
// and dy_l[k]/da_l = y_l[k-1] + a_l dy_l[k-1]/da_l = b_l v_l[k] with
//     v_l[k] = a_l v_l[k-1] + u_l[k-1].
// With g_z[k] = dL/dRe z + i dL/dIm z the gradients (PyTorch convention) are
//     g_b_l = sum_k g_z[k] conj(u_l[k]),   g_a_l = conj(b_l) sum_k g_z[k] conj(v_l[k]),
// the adjoint formulas sum_k mu_l[k] x[k-d_l] and sum_k mu_l[k] conj(y_l[k-1])
// with the order of summation exchanged (mu_l[k] = sum_{j>=k} conj(a_l)^(j-k) g_z[j]).
// One forward pass in time: no checkpoints, no recompute and no reverse
// recurrence; 16 FP32 operations per filter-update (u 4, v 4, the two sums
// 8), or 12 with GB = false, when the input-gradient pass sums g_b instead
// (sum_m nu[m] x[m] there costs 2).
//
// NF filters per lane (NF = 1: scalar FFMA; NF = 2: two filters of one
// template as a packed FP32x2 pair, half the instructions and one g_z read
// for both); no time segments (the bank must fill the GPU by itself).  A CTA
// of W warps serves W x 32 lanes of the tangent order on one detector: the strain window
// of each Tb-sample block (Dh history + Tb) is copied into shared memory by
// cp.async, double buffered; each warp stages its (at most two) templates'
// g_z 16 samples at a time (one load per lane, fetched two sub-blocks ahead)
// and every lane reads its template's row.  Sums restart every block and are
// added into block-level totals (rounding grows with the block, not the call).
template <int NF, bool GB>
__global__ void __launch_bounds__(256) kt_tangent(const KTArgs A)
{
    static_assert(NF == 1 || NF == 2, "one filter per lane, or a packed FP32x2 pair");
    extern __shared__ __align__(16) unsigned char smem[];
    const int Wd = A.Dh + A.Tb;
    float *xs = reinterpret_cast<float *>(smem);                     // [2][Wd]
    float2 *gbw = reinterpret_cast<float2 *>(xs + 2 * Wd);           // [W][36]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int det = blockIdx.y;
    const int64_t wg = (int64_t)blockIdx.x * A.W + warp;
    const bool wact = wg * 32 * NF < A.n_pos;                         // warp-uniform
    // filter f of this lane at position (wg NF + f) 32 + lane; both of one template
    int2 ln[NF];
    float ar[NF], ai[NF], br[NF], bi[NF];
    int xo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        ln[f] = wact ? A.lanes[(wg * NF + f) * 32 + lane] : make_int2(-1, 0);
        ar[f] = ai[f] = br[f] = bi[f] = 0.f;
        xo[f] = 0;
        if (ln[f].x >= 0) {
            const float4 p = A.params[ln[f].x];
            const bool odd = (ln[f].x & 1) != 0;   // stored as conj(a), (Im b, Re b)
            ar[f] = p.x;
            ai[f] = odd ? -p.y : p.y;
            br[f] = odd ? p.w : p.z;
            bi[f] = odd ? p.z : p.w;
            xo[f] = A.ringoff[ln[f].x].x;          // Dh - d
        }
    }
    const int2 wt = wact ? A.warp_tmpl[wg] : make_int2(-1, -1);
    // lane j stages sample (j & 15) of template (j >> 4) of its warp
    const int st = (lane >> 4) ? wt.y : wt.x;
    const float2 *grow = st >= 0 ? A.gz + ((int64_t)det * A.T + st) * A.n : nullptr;
    float2 *gb = gbw + warp * 36;
    const int gput = (lane >> 4) * 18 + (lane & 15);   // rows 18 apart: different banks
    const float2 *gr = gb + (ln[0].y ? 18 : 0);
    const float *xrow = A.xe + (int64_t)det * A.xe_stride;
    const int n = A.n, Tb = A.Tb;
    const int nblk = (n + Tb - 1) / Tb;

    // window of block j: xs[i] = xe[j Tb + i] = x[j Tb + i - Dh]
    auto issue = [&](int j) {
        const float *src = xrow + (int64_t)j * Tb;
        const uint32_t dst = smem_addr(xs + (j & 1) * Wd);
        for (int i = 4 * (int)threadIdx.x; i < Wd; i += 4 * (int)blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 4u * i),
                         "l"(src + i)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // state and sums; NF = 2 keeps the pair packed (lo = filter 0, hi = filter 1)
    uint64_t AR = 0, AI = 0, NAI = 0, UR = 0, UI = 0, VR = 0, VI = 0;
    float ur = 0.f, ui = 0.f, vr = 0.f, vi = 0.f;
    if (NF == 2) {
        AR = pk(ar[0], ar[NF - 1]);
        AI = pk(ai[0], ai[NF - 1]);
        NAI = pk(-ai[0], -ai[NF - 1]);
    }
    const float nai = -ai[0];
    float Tbr[NF], Tbi[NF], Tar[NF], Tai[NF];   // totals of the two sums
#pragma unroll
    for (int f = 0; f < NF; ++f) Tbr[f] = Tbi[f] = Tar[f] = Tai[f] = 0.f;
    // g_z of the next two sub-blocks, loaded two sub-blocks ahead of use
    float2 gnext = make_float2(0.f, 0.f), gnext2 = make_float2(0.f, 0.f);
    if (grow != nullptr && (lane & 15) < n) gnext = grow[lane & 15];
    if (grow != nullptr && 16 + (lane & 15) < n) gnext2 = grow[16 + (lane & 15)];
    issue(0);
    for (int j = 0; j < nblk; ++j) {
        if (j + 1 < nblk) {
            issue(j + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float *w0 = xs + (j & 1) * Wd + xo[0];
        const float *w1 = xs + (j & 1) * Wd + xo[NF - 1];
        const int k0 = j * Tb;
        const int nv = min(Tb, n - k0);
        // sum_k g_z conj(u): re = Gr ur + Gi ui, im = Gi ur - Gr ui (two chains);
        // likewise with v
        float sbr = 0.f, sbi1 = 0.f, sbi2 = 0.f, sar = 0.f, sai1 = 0.f, sai2 = 0.f;
        uint64_t SBR = 0, SBI1 = 0, SBI2 = 0, SAR = 0, SAI1 = 0, SAI2 = 0;
        auto step = [&](int t, float2 g) {
            if (NF == 1) {
                const float x = w0[t];
                const float nvr = fmaf(ar[0], vr, fmaf(nai, vi, ur));   // v <- a v + u
                const float nvi = fmaf(ar[0], vi, fmaf(ai[0], vr, ui));
                const float nur = fmaf(ar[0], ur, fmaf(nai, ui, x));    // u <- a u + x
                const float nui = fmaf(ar[0], ui, ai[0] * ur);
                ur = nur;
                ui = nui;
                vr = nvr;
                vi = nvi;
                if (GB) {
                    sbr = fmaf(g.x, ur, fmaf(g.y, ui, sbr));
                    sbi1 = fmaf(g.y, ur, sbi1);
                    sbi2 = fmaf(g.x, ui, sbi2);
                }
                sar = fmaf(g.x, vr, fmaf(g.y, vi, sar));
                sai1 = fmaf(g.y, vr, sai1);
                sai2 = fmaf(g.x, vi, sai2);
            } else {
                const uint64_t X = pk(w0[t], w1[t]);
                const uint64_t GR = pk(g.x, g.x), GI = pk(g.y, g.y);
                const uint64_t NVR = fma2(AR, VR, fma2(NAI, VI, UR));
                const uint64_t NVI = fma2(AR, VI, fma2(AI, VR, UI));
                const uint64_t NUR = fma2(AR, UR, fma2(NAI, UI, X));
                const uint64_t NUI = fma2(AR, UI, mul2(AI, UR));
                UR = NUR;
                UI = NUI;
                VR = NVR;
                VI = NVI;
                if (GB) {
                    SBR = fma2(GR, UR, fma2(GI, UI, SBR));
                    SBI1 = fma2(GI, UR, SBI1);
                    SBI2 = fma2(GR, UI, SBI2);
                }
                SAR = fma2(GR, VR, fma2(GI, VI, SAR));
                SAI1 = fma2(GI, VR, SAI1);
                SAI2 = fma2(GR, VI, SAI2);
            }
        };
        if (wact) {
            for (int sb = 0; sb < nv; sb += 16) {
                gb[gput] = gnext;
                __syncwarp();
                gnext = gnext2;
                {
                    const int k = k0 + sb + 32 + (lane & 15);
                    gnext2 = (grow != nullptr && k < n) ? grow[k] : make_float2(0.f, 0.f);
                }
                if (sb + 16 <= nv) {
#pragma unroll
                    for (int t = 0; t < 16; ++t) step(sb + t, gr[t]);
                } else {
                    for (int t = 0; t < nv - sb; ++t) step(sb + t, gr[t]);
                }
                __syncwarp();
            }
        }
        if (NF == 1) {
            Tbr[0] += sbr;
            Tbi[0] += sbi1 - sbi2;
            Tar[0] += sar;
            Tai[0] += sai1 - sai2;
        } else {
            float lo, hi, lo2, hi2;
            upk(SBR, lo, hi);
            Tbr[0] += lo;
            Tbr[NF - 1] += hi;
            upk(SBI1, lo, hi);
            upk(SBI2, lo2, hi2);
            Tbi[0] += lo - lo2;
            Tbi[NF - 1] += hi - hi2;
            upk(SAR, lo, hi);
            Tar[0] += lo;
            Tar[NF - 1] += hi;
            upk(SAI1, lo, hi);
            upk(SAI2, lo2, hi2);
            Tai[0] += lo - lo2;
            Tai[NF - 1] += hi - hi2;
        }
        __syncthreads();   // every warp is done with this buffer before it is refilled
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (ln[f].x < 0) continue;
        float *acc = A.acc + ((int64_t)det * A.n_slots + ln[f].x) * 6;
        acc[0] = 0.f;
        acc[1] = 0.f;
        acc[2] = br[f] * Tar[f] + bi[f] * Tai[f];   // conj(b) sum g_z conj(v)
        acc[3] = br[f] * Tai[f] - bi[f] * Tar[f];
        if (GB) {
            acc[4] = Tbr[f];
            acc[5] = Tbi[f];
        }
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
    for (int d = 0; d < D; ++d) {   // D here counts (segment, detector) rows
        const float *p = acc + ((int64_t)d * n_slots + s) * 6;
        a.x += p[2];
        a.y += p[3];
        b.x += p[4];
        b.y += p[5];
    }
    ga[f] = a;
    gb[f] = b;
}

// E[q] for q = 1..P-1: the adjoint state a segment's own g_z leaves at its
// start, mu <- g_z + conj(a) mu run backwards over the segment from zero.
// One thread per (segment, detector, 4 slots): the 4 slots sit in one
// 32-slot round, so they share one template and one g_z row; they run as two
// packed FP32x2 pairs, and g_z is loaded a group of 16 samples ahead.
constexpr int kProjSlots = 4;
constexpr int kProjAhead = 16;

__global__ void __launch_bounds__(128) adj_project_kernel(
    const float4 *params, const int32_t *slot_tmpl, const float2 *gz, int64_t n_slots, int D,
    int64_t T, int64_t n, int64_t seg_len, int64_t off, int P, float2 *E)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per4 = (int64_t)D * n_slots / kProjSlots;
    if (i >= (int64_t)(P - 1) * per4) return;
    const int q = 1 + (int)(i / per4);
    const int64_t ds0 = (i % per4) * kProjSlots;   // first (detector, slot) of the four
    const int det = (int)(ds0 / n_slots);
    const int64_t s0 = ds0 % n_slots;
    int tmpl = -1;
    float ar[kProjSlots], ai[kProjSlots];
#pragma unroll
    for (int k = 0; k < kProjSlots; ++k) {
        const int t = slot_tmpl[s0 + k];
        tmpl = max(tmpl, t);   // padding slots are -1, the others share one template
        const float4 p = params[s0 + k];
        ar[k] = p.x;
        ai[k] = ((s0 + k) & 1) ? -p.y : p.y;   // odd slots store conj(a)
    }
    uint64_t MR0 = 0, MI0 = 0, MR1 = 0, MI1 = 0;
    if (tmpl >= 0) {
        const uint64_t AR0 = pk(ar[0], ar[1]), AI0 = pk(ai[0], ai[1]);
        const uint64_t NAI0 = pk(-ai[0], -ai[1]);
        const uint64_t AR1 = pk(ar[2], ar[3]), AI1 = pk(ai[2], ai[3]);
        const uint64_t NAI1 = pk(-ai[2], -ai[3]);
        const float2 *g = gz + ((int64_t)det * T + tmpl) * n;
        const int64_t j0 = (int64_t)q * seg_len + off, j1 = min(n, j0 + seg_len);
        auto step = [&](float2 G1) {
            const uint64_t GR = pk(G1.x, G1.x), GI = pk(G1.y, G1.y);
            const uint64_t nr0 = fma2(AR0, MR0, fma2(AI0, MI0, GR));
            const uint64_t ni0 = fma2(AR0, MI0, fma2(NAI0, MR0, GI));
            const uint64_t nr1 = fma2(AR1, MR1, fma2(AI1, MI1, GR));
            const uint64_t ni1 = fma2(AR1, MI1, fma2(NAI1, MR1, GI));
            MR0 = nr0;
            MI0 = ni0;
            MR1 = nr1;
            MI1 = ni1;
        };
        int64_t j = j1;
        // whole groups of kProjAhead samples from the segment's end, each
        // group's g_z loaded while the previous group runs; then the rest
        if (j - kProjAhead >= j0) {
            float2 Gc[kProjAhead], Gn[kProjAhead];
#pragma unroll
            for (int t = 0; t < kProjAhead; ++t) Gc[t] = g[j - 1 - t];
            for (; j - kProjAhead >= j0; j -= kProjAhead) {
                const bool more = j - 2 * kProjAhead >= j0;
#pragma unroll
                for (int t = 0; t < kProjAhead; ++t)
                    Gn[t] = more ? g[j - kProjAhead - 1 - t] : make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < kProjAhead; ++t) step(Gc[t]);
#pragma unroll
                for (int t = 0; t < kProjAhead; ++t) Gc[t] = Gn[t];
            }
        }
        for (; j > j0; --j) step(g[j - 1]);
    }
    float mr[kProjSlots], mi[kProjSlots];
    upk(MR0, mr[0], mr[1]);
    upk(MI0, mi[0], mi[1]);
    upk(MR1, mr[2], mr[3]);
    upk(MI1, mi[2], mi[3]);
    float2 *e = E + (int64_t)q * D * n_slots + ds0;
#pragma unroll
    for (int k = 0; k < kProjSlots; ++k)
        e[k] = slot_tmpl[s0 + k] >= 0 ? make_float2(mr[k], mi[k]) : make_float2(0.f, 0.f);
}

// conj(a)^len in FP64 by binary powering
__device__ void conj_pow(double ar, double ai, int64_t len, double &rr, double &ri)
{
    double br = ar, bi = -ai;
    rr = 1.0;
    ri = 0.0;
    for (int64_t e = len; e > 0; e >>= 1) {
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

// mu_end[P-1] = 0; mu_end[q] = E[q+1] + conj(a)^len(q+1) mu_end[q+1] (FP64),
// len(q) = the samples of [q seg_len + off, (q + 1) seg_len + off) inside the
// call: seg_len, except for the one segment the call's end cuts (and 0 past it)
__global__ void adj_carry_kernel(const float4 *params, const float2 *E, int64_t n_slots, int D,
                                 int64_t n, int64_t seg_len, int64_t off, int P, float2 *mu_end)
{
    const int64_t ds = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)D * n_slots;
    if (ds >= per) return;
    const int64_t s = ds % n_slots;
    const float4 p = params[s];
    const double ar = p.x, ai = (s & 1) ? -(double)p.y : (double)p.y;
    double fr, fi, lr, li;   // powers for a whole segment and for the cut one
    conj_pow(ar, ai, seg_len, fr, fi);
    int64_t cut = -1;        // the segment holding the call's end, and its length
    for (int q = 1; q < P; ++q) {
        const int64_t j0 = (int64_t)q * seg_len + off;
        if (j0 < n && j0 + seg_len > n) cut = q;
    }
    if (cut >= 0) conj_pow(ar, ai, n - (cut * seg_len + off), lr, li);
    double mr = 0.0, mi = 0.0;
    mu_end[(int64_t)(P - 1) * per + ds] = make_float2(0.f, 0.f);
    for (int q = P - 2; q >= 0; --q) {
        const bool last = q + 1 == cut;
        const double rr = last ? lr : fr, ri = last ? li : fi;
        const float2 e = E[(int64_t)(q + 1) * per + ds];
        const double nr = (double)e.x + rr * mr - ri * mi;
        const double ni = (double)e.y + rr * mi + ri * mr;
        mr = nr;
        mi = ni;
        mu_end[(int64_t)q * per + ds] = make_float2((float)mr, (float)mi);
    }
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

int k6_smem_bytes(int Cc, int Dh) { return (int)(sizeof(float) * (Dh + Cc)); }

cudaError_t launch_k6(const K6Args &a, int64_t n_units, cudaStream_t s)
{
    if (n_units <= 0 || a.n <= 0 || a.cps <= 0 || a.n_units != n_units)
        return n_units <= 0 || a.n <= 0 ? cudaSuccess : cudaErrorInvalidValue;
    const int smem = k6_smem_bytes(a.Cc, a.Dh);
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void *>(k6_adjoint), smem);
    if (e != cudaSuccess) return e;
    const int64_t nc = (a.n + a.Cc - 1) / a.Cc;
    if ((nc + a.cps - 1) / a.cps != a.P) return cudaErrorInvalidValue;
    k6_adjoint<<<(unsigned)(n_units * a.P), a.W * 32, smem, s>>>(a);
    return cudaGetLastError();
}

int k7_smem_bytes(int Dh, int W, int G)
{
    return (int)(sizeof(float) * ((G == 16 ? 2 : 1) * 2 * (kK7Chunk + Dh + 32) + W * 1024 +
                                  W * kK7Chunk + kK7Chunk));
}

template <bool TAN>
cudaError_t launch_k7_form(const K7Args &a, cudaStream_t s)
{
    const int smem = k7_smem_bytes(a.Dh, a.W, a.G);
    // two tasks per warp (two independent chains per lane), one for half-warp
    // templates (a unit is then a single task)
    const void *fn = a.G == 16 ? reinterpret_cast<const void *>(k7_adjoint_x<1, TAN>)
                               : reinterpret_cast<const void *>(k7_adjoint_x<2, TAN>);
    cudaError_t e = ensure_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((int64_t)a.P * a.n_units * a.n_det);
    if (a.G == 16)
        k7_adjoint_x<1, TAN><<<grid, a.W * 32, smem, s>>>(a);
    else
        k7_adjoint_x<2, TAN><<<grid, a.W * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_k7(const K7Args &a, cudaStream_t s)
{
    if (a.n_units <= 0 || a.n <= 0) return cudaSuccess;
    const bool tan = a.acc != nullptr;
    // segments of whole 32-output blocks (whole chunks for the warm-up): only
    // the call's last block runs past its end (on zero input)
    if (a.W < 1 || a.W > kK7MaxWarps || a.S % 32 != 0 || (a.P > 1 && a.seeds == nullptr) ||
        (tan && (a.xe == nullptr || a.Dh % kK7Chunk != 0 || a.S % kK7Chunk != 0)))
        return cudaErrorInvalidValue;
    return tan ? launch_k7_form<true>(a, s) : launch_k7_form<false>(a, s);
}

int kt_smem_bytes(int Dh, int Tb, int W)
{
    return (int)(sizeof(float) * 2 * (Dh + Tb) + sizeof(float2) * 36 * W);
}

cudaError_t launch_kt(const KTArgs &a, int D, cudaStream_t s)
{
    if (a.n_pos <= 0 || a.n <= 0 || D <= 0) return cudaSuccess;
    if (a.W < 1 || a.W > 8 || (a.nf != 1 && a.nf != 2) || a.n_pos % (32 * a.nf) != 0 ||
        a.Tb % 16 != 0 || a.Dh % 4 != 0 ||
        a.xe_stride % 4 != 0 || (reinterpret_cast<uintptr_t>(a.xe) & 15) != 0)
        return cudaErrorInvalidValue;
    const int smem = kt_smem_bytes(a.Dh, a.Tb, a.W);
    const void *fn =
        a.nf == 2 ? (a.with_gb ? reinterpret_cast<const void *>(kt_tangent<2, true>)
                               : reinterpret_cast<const void *>(kt_tangent<2, false>))
                  : (a.with_gb ? reinterpret_cast<const void *>(kt_tangent<1, true>)
                               : reinterpret_cast<const void *>(kt_tangent<1, false>));
    cudaError_t e = ensure_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
    const int64_t warps = a.n_pos / (32 * a.nf);
    const dim3 grid((unsigned)((warps + a.W - 1) / a.W), (unsigned)D);
    if (a.nf == 2) {
        if (a.with_gb) kt_tangent<2, true><<<grid, a.W * 32, smem, s>>>(a);
        else kt_tangent<2, false><<<grid, a.W * 32, smem, s>>>(a);
    } else {
        if (a.with_gb) kt_tangent<1, true><<<grid, a.W * 32, smem, s>>>(a);
        else kt_tangent<1, false><<<grid, a.W * 32, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_finalize(const float *acc, const int64_t *slot_filter, int64_t n_slots,
                                int D, int P, float2 *ga, float2 *gb, cudaStream_t s)
{
    if (n_slots <= 0) return cudaSuccess;
    // the accumulator rows of all segments and detectors are summed alike
    adj_finalize<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(acc, slot_filter, n_slots,
                                                                    D * P, ga, gb);
    return cudaGetLastError();
}

cudaError_t launch_adj_project(const float4 *params, const int32_t *slot_tmpl, const float2 *gz,
                               int64_t n_slots, int D, int64_t T, int64_t n, int64_t seg_len,
                               int64_t off, int P, float2 *E, float2 *mu_end, cudaStream_t s)
{
    const int64_t per = (int64_t)D * n_slots;
    if (per <= 0 || P < 1) return cudaSuccess;
    if (P > 1) {
        if (n_slots % kProjSlots != 0) return cudaErrorInvalidValue;
        const int64_t th = (int64_t)(P - 1) * per / kProjSlots;
        adj_project_kernel<<<(unsigned)((th + 127) / 128), 128, 0, s>>>(
            params, slot_tmpl, gz, n_slots, D, T, n, seg_len, off, P, E);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    adj_carry_kernel<<<(unsigned)((per + 63) / 64), 64, 0, s>>>(params, E, n_slots, D, n, seg_len,
                                                                 off, P, mu_end);
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
