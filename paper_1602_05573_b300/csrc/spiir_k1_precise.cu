// The filter kernel's precision forms (compensated, chunked FP64 carry,
// anchored for the chunked tensor-core form) and their launcher.
#include "spiir_k1_body.h"

namespace spiir {

namespace {

__global__ void __launch_bounds__(256, 2) k1_compensated(const K1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring, *zbuf;
    uint32_t bar0, bar1;
    cta_setup(smem, A, ring, zbuf, bar0, bar1);
    const int u = blockIdx.x % A.n_units;
    Phases ph;
    dispatch_f<CompLanes, kPreciseFcap, false, true>(A, A.units[2 * u], A.units[2 * u + 1], ring,
                                                     zbuf, bar0, bar1, ph);
}

__global__ void __launch_bounds__(256, 2) k1_chunked(const K1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring, *zbuf;
    uint32_t bar0, bar1;
    cta_setup(smem, A, ring, zbuf, bar0, bar1);
    const int u = blockIdx.x % A.n_units;
    Phases ph;
    dispatch_f<ChunkLanes, kPreciseFcap, false, true>(A, A.units[2 * u], A.units[2 * u + 1], ring,
                                                      zbuf, bar0, bar1, ph);
}

__global__ void __launch_bounds__(256, 2) k1_anchored(const K1Args A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring, *zbuf;
    uint32_t bar0, bar1;
    cta_setup(smem, A, ring, zbuf, bar0, bar1);
    const int u = (int)(blockIdx.x % A.n_units);
    Phases ph;
    dispatch_f<AnchorLanes, kAnchorFcap, true, true>(A, A.units[2 * u], A.units[2 * u + 1], ring,
                                                     zbuf, bar0, bar1, ph);
}

}  // namespace

cudaError_t launch_k1_precise(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s)
{
    if (a.anchors != nullptr) {
        if (a.fcap > kAnchorFcap || a.n_seg <= 0) return cudaErrorInvalidValue;
        return launch_kernel(k1_anchored, a, n_units, smem_bytes, s);
    }
    if (a.fcap > kPreciseFcap) return cudaErrorInvalidValue;
    return launch_kernel(a.mode == kModeCompensated ? k1_compensated : k1_chunked, a,
                         n_units, smem_bytes, s);
}

}  // namespace spiir
