// Helpers shared by the C-ABI translation units (error reporting, bank
// validation).  Not part of the public ABI.
#pragma once

#include "spiir.h"

#include <cuda_runtime.h>

#include <string>

namespace spiir {
namespace detail {

// Record a one-line reason for spiir_last_error_detail() and return st.
spiir_status fail(spiir_status st, const std::string &why);
// Record a CUDA error (name and message) and return SPIIR_ECUDA.
spiir_status cuda_fail(cudaError_t e, const char *what);
// Check a bank description; returns SPIIR_OK or SPIIR_EINVAL with a reason.
spiir_status validate_bank(const spiir_bank_desc *bank);

}  // namespace detail
}  // namespace spiir
