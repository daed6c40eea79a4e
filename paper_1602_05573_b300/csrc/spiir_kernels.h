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
    int32_t pad;
};
constexpr int kMaxLowerBands = 7;

// Plain FP32 filter kernel (one launch per bank or band).
struct K1Args {
    const float *xe;           // [D][xe_stride] strain: Dh history samples, then the call's
    int64_t xe_stride;         // floats per detector row (multiple of 4)
    int32_t n;                 // samples in this call (band rate)
    int32_t Tb, H, S, R, CS, C, W;
    int32_t fcap;              // filters-per-lane cap of the layout (selects the kernel)
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
    int64_t t0;                // absolute index of this call's first sample
    int32_t *err;              // device error word
    uint64_t wait_limit_ns;    // bound on every mbarrier wait
    int32_t n_lower;           // lower bands added in the combine (0 = single rate)
    LowerBand lower[kMaxLowerBands];
};

cudaError_t launch_k1(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s);

// Finalize running peaks into the caller's buffers (sqrt of |z|^2).
cudaError_t launch_peak_out(const float *best, const int64_t *idx, int64_t count,
                            float *out_abs, int64_t *out_idx, cudaStream_t s);

// best[i] = -1, idx[i] = -1.
cudaError_t launch_peak_reset(float *best, int64_t *idx, int64_t count, cudaStream_t s);

// xe[d][Dh + i] = x[d][R * i] for i < nb (decimation into a band's strain rows).
cudaError_t launch_decimate(const float *x, int64_t n, int D, int R, int64_t nb, float *xe,
                            int64_t xe_stride, int64_t Dh, cudaStream_t s);

// Self-test: wait on an mbarrier nothing will complete, with a bound; sets *err.
cudaError_t launch_bounded_wait_probe(int32_t *err, uint64_t limit_ns, cudaStream_t s);

}  // namespace spiir
