// spiir_filter_noalloc: a one-shot filter call that allocates no device
// memory.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree -- for
// example a process whose device memory is owned by another allocator (a
// framework's caching pool, a fixed real-time budget), code that runs while
// allocation is forbidden or would stall a low-latency pipeline, or a host
// that pre-plans every byte.  spiir_plan_create allocates its parameter
// layout and workspace with cudaMalloc, so those callers cannot use a plan.
//
// This entry point runs the same plain kernel as spiir_filter, on the same
// layout, but keeps every piece of its scratch (packed parameters, filter
// state, staged strain, running peaks, error word) in one file-scope
// __device__ array of kNoallocScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.  The caller passes the
// bank (host), the strain, and the output buffers (device).
#include "spiir.h"
#include "spiir_internal.h"
#include "spiir_kernels.h"
#include "spiir_layout.h"

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;  // 32 MiB per device
}

// The scratch.  In host code this name is only a stand-in for the symbol;
// the device address comes from cudaGetSymbolAddress (noalloc_scratch_on).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

using spiir::detail::cuda_fail;
using spiir::detail::fail;

constexpr int kMaxDevices = 64;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
std::mutex g_mu;
unsigned char *g_scratch[kMaxDevices] = {};

// Device address of the scratch array on device `dev` (which is current),
// looked up once per device.
spiir_status noalloc_scratch_on(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(SPIIR_EUNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch[dev];
    return SPIIR_OK;
}

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" spiir_status spiir_filter_noalloc(const spiir_bank_desc *bank, const float *x_dev,
                                             int64_t n, float *z_dev, float *peak_abs_dev,
                                             int64_t *peak_idx_dev, void *stream)
{
    spiir_status st = spiir::detail::validate_bank(bank);
    if (st != SPIIR_OK) return st;
    if (bank->n_bands > 1)
        return fail(SPIIR_EUNSUPPORTED, "spiir_filter_noalloc takes single-rate banks only");
    if (n < 1 || n > ((int64_t)1 << 30)) return fail(SPIIR_EINVAL, "n must be in [1, 2^30]");
    if (!x_dev || !peak_abs_dev || !peak_idx_dev)
        return fail(SPIIR_EINVAL, "x_dev, peak_abs_dev and peak_idx_dev are required");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int major = 0, minor = 0, n_sm = 0;
    if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    if (major != 10 || minor != 3)
        return fail(SPIIR_EUNSUPPORTED, "kernels are built for sm_103a");

    // the same layout a default plan would use (host memory only)
    const int64_t T = bank->n_templates;
    const int D = bank->n_detectors;
    std::vector<std::vector<int64_t>> lists((size_t)T);
    for (int64_t t = 0; t < T; ++t)
        for (int64_t l = bank->filter_off[t]; l < bank->filter_off[t + 1]; ++l)
            lists[t].push_back(l);
    spiir::LayoutOptions lo;
    lo.n_sm = n_sm;
    spiir::Layout L;
    std::string err;
    if (!spiir::build_layout(lists, D, bank->a_reim, bank->b_reim, bank->delay, lo, &L, &err))
        return fail(SPIIR_EUNSUPPORTED, err);

    // carve the scratch
    const int64_t G = L.n_groups();
    const int64_t stride = L.Dh + ((n + L.Tb - 1) / L.Tb) * L.Tb;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const size_t o_params = take(sizeof(float4) * (size_t)L.n_slots);
    const size_t o_ringoff = take(sizeof(int2) * (size_t)L.n_slots);
    const size_t o_units = take(sizeof(int32_t) * L.units.size());
    const size_t o_groupF = take(sizeof(int32_t) * (size_t)G);
    const size_t o_pbase = take(sizeof(int64_t) * (size_t)G);
    const size_t o_winfo = take(sizeof(int32_t) * L.warp_info.size());
    const size_t o_state = take(sizeof(float2) * (size_t)D * L.n_slots);
    const size_t o_xe = take(sizeof(float) * (size_t)D * stride);
    const size_t o_best = take(sizeof(float) * (size_t)D * T);
    const size_t o_idx = take(sizeof(int64_t) * (size_t)D * T);
    const size_t o_err = take(sizeof(int32_t));
    if (off > kNoallocScratchBytes)
        return fail(SPIIR_EINVAL, "spiir_filter_noalloc: this bank and length need " +
                                      std::to_string(off) + " bytes of scratch; the static "
                                      "scratch holds " +
                                      std::to_string(kNoallocScratchBytes) +
                                      " bytes (use a plan for larger problems)");

    unsigned char *base = nullptr;
    st = noalloc_scratch_on(dev, &base);
    if (st != SPIIR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    auto *params = reinterpret_cast<float4 *>(base + o_params);
    auto *ringoff = reinterpret_cast<int2 *>(base + o_ringoff);
    auto *units = reinterpret_cast<int32_t *>(base + o_units);
    auto *groupF = reinterpret_cast<int32_t *>(base + o_groupF);
    auto *pbase = reinterpret_cast<int64_t *>(base + o_pbase);
    auto *winfo = reinterpret_cast<int4 *>(base + o_winfo);
    auto *state = reinterpret_cast<float2 *>(base + o_state);
    auto *xe = reinterpret_cast<float *>(base + o_xe);
    auto *best = reinterpret_cast<float *>(base + o_best);
    auto *bidx = reinterpret_cast<int64_t *>(base + o_idx);
    auto *errw = reinterpret_cast<int32_t *>(base + o_err);

    // Upload the layout (pageable host copies are staged before the call
    // returns, so the host vectors may go out of scope afterwards), then
    // clear everything that must start at zero: the previous call's state,
    // strain history, peaks and error word are still in the array.
    if ((e = cudaMemcpyAsync(params, L.params.data(), L.params.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(ringoff, L.ringoff.data(), L.ringoff.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(units, L.units.data(), L.units.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(groupF, L.group_F.data(), L.group_F.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(pbase, L.group_pbase.data(), L.group_pbase.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(winfo, L.warp_info.data(), L.warp_info.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(state, 0, sizeof(float2) * (size_t)D * L.n_slots, s)) !=
            cudaSuccess ||
        (e = cudaMemset2DAsync(xe, stride * sizeof(float), 0, L.Dh * sizeof(float), D, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(errw, 0, sizeof(int32_t), s)) != cudaSuccess ||
        (e = spiir::launch_peak_reset(best, bidx, (int64_t)D * T, s)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(xe + L.Dh, stride * sizeof(float), x_dev, n * sizeof(float),
                               n * sizeof(float), D, cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
        return cuda_fail(e, "spiir_filter_noalloc staging");

    spiir::K1Args a{};
    a.xe = xe;
    a.xe_stride = stride;
    a.n = (int32_t)n;
    a.Tb = L.Tb;
    a.H = L.H;
    a.S = L.S;
    a.R = L.R;
    a.CS = L.CS;
    a.C = L.C;
    a.W = L.W;
    a.units = units;
    a.group_F = groupF;
    a.group_pbase = pbase;
    a.warp_info = winfo;
    a.fcap = L.Fcap;
    a.G = L.G;
    a.n_units = (int32_t)L.n_units();
    a.n_seg = (int32_t)n;
    a.params = params;
    a.ringoff = ringoff;
    a.state = state;
    a.n_slots = L.n_slots;
    a.z = z_dev;
    a.z_len = n;
    a.T = T;
    a.peak_best = best;
    a.peak_idx = bidx;
    a.t0 = 0;
    a.err = errw;
    a.wait_limit_ns = kWaitLimitNs;
    if ((e = spiir::launch_k1(a, L.n_units(), L.smem_bytes(), s)) != cudaSuccess)
        return cuda_fail(e, "spiir_filter_noalloc kernel launch");
    // the error word is in the scratch and the call never waits for its
    // work, so a bounded wait that gave up shows in the peaks: all (NaN, -1)
    if ((e = spiir::launch_peak_out_checked(best, bidx, (int64_t)D * T, errw, peak_abs_dev,
                                            peak_idx_dev, s)) != cudaSuccess)
        return cuda_fail(e, "spiir_filter_noalloc peak launch");
    return SPIIR_OK;
}
