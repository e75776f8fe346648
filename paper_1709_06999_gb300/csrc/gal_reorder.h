// Z-order reordering of an observation's points (gal_data_create_sorted_*).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace gal {

// Order of M points (u, v on the host) along a Z-order (Morton) curve of the
// uv plane: each axis is quantised to 16 bits over [-rho, rho], rho the
// largest finite |(u, v)|, and the two 16-bit cells are bit-interleaved into
// one 32-bit key.  Points with a non-finite coordinate come last.  The sort is
// a stable least-significant-digit radix sort, so equal keys keep their input
// order and the result is the same on every run.  perm[i] is the input index
// of the i-th point.  Throws std::bad_alloc if the host buffers cannot be had.
template <typename T>
void z_order(const T* u, const T* v, int64_t M, std::vector<int64_t>& perm);

// out_k[i] = in_k[perm[i]] for the five arrays of an observation, i < M.
template <typename T>
cudaError_t permute5(const int64_t* perm, int64_t M, const T* const in[5], T* const out[5],
                     int blocks, cudaStream_t st);

}  // namespace gal
