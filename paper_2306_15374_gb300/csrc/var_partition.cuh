// Variable-length partitioning (§3.2.2) with the choice of split (k_var.cu).
#pragma once

#include "leco_internal.cuh"

namespace leco {

// seeded: each chunk's split grows from its seed both ways (§3.2.2, selecting good starting
// positions) instead of from the chunk's first value
cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, bool seeded, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st);

// as var_partition; rec_out (when non-null) receives a new pool allocation of m records with the
// full fit of every final partition under `model` (constant or linear), exactly as the encoder's fit
// writes them (bit offset 0): the encoder then needs no fit of its own
cudaError_t var_partition_fit(const void* values, int dtype, uint64_t n, double tau, uint32_t cap, int model,
                              bool seeded, uint64_t* starts_out, uint64_t* m_out, Record** rec_out, cudaStream_t st);

// lenbits[p] = (starts[p+1] - starts[p]) * b_p from fitted records, and the widest b into *max_b
cudaError_t launch_lenbits(const Record* rec, const uint64_t* starts, uint64_t m, uint64_t* lenbits, uint32_t* max_b,
                           cudaStream_t st);

}  // namespace leco
