// Filter kernels compiled for at most 8 filters per lane (k1_plain,
// k1_persistent): their launcher and kernel handle.
#include "spiir_k1_body.h"

namespace spiir {

cudaError_t launch_k1_cap_8(const K1Args &a, int64_t n_units, int smem_bytes, cudaStream_t s)
{
    return launch_k1_cap<8>(a, n_units, smem_bytes, s);
}

const void *k1_plain_kernel_8()
{
    return reinterpret_cast<const void *>(k1_plain<8, false, false>);
}

}  // namespace spiir
