// Variable-length partitioning (§3.2.2) with the choice of split (k_var.cu).
#pragma once

#include "leco_internal.cuh"

namespace leco {

// seeded: each chunk's split grows from its seed both ways (§3.2.2, selecting good starting
// positions) instead of from the chunk's first value
cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, bool seeded, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st);

}  // namespace leco
