// Z-order reordering of an observation's points: the order on the host, the
// gather of the five arrays on the device.  The chi-square is a sum over the
// points (Eq. chap6.eq:def.chi.square), so any order gives the same value up
// to rounding; points that are close in the uv plane sample neighbouring
// cells of the spectrum, and stored next to each other they let a gather read
// the cells of a window that only fits in L2 from far fewer cache lines.
#include "gal_reorder.h"

#include <cmath>
#include <utility>

namespace gal {

namespace {

uint32_t spread16(uint32_t x) {  // bit b of x to bit 2b
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

uint32_t cell16(double x, double rho, double scale) {
  const double q = std::floor((x + rho) * scale);
  return q <= 0.0 ? 0u : (q >= 65535.0 ? 65535u : (uint32_t)q);
}

template <typename T>
__global__ void permute5_kernel(const int64_t* __restrict__ perm, int64_t M, const T* __restrict__ a0,
                                const T* __restrict__ a1, const T* __restrict__ a2,
                                const T* __restrict__ a3, const T* __restrict__ a4,
                                T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2,
                                T* __restrict__ o3, T* __restrict__ o4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = perm[i];
    o0[i] = a0[k];
    o1[i] = a1[k];
    o2[i] = a2[k];
    o3[i] = a3[k];
    o4[i] = a4[k];
  }
}

}  // namespace

template <typename T>
void z_order(const T* u, const T* v, int64_t M, std::vector<int64_t>& perm) {
  double rho = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    const double a = (double)u[i], b = (double)v[i];
    if (std::isfinite(a) && std::isfinite(b)) rho = std::fmax(rho, std::sqrt(a * a + b * b));
  }
  const double scale = rho > 0.0 ? 65535.0 / (2.0 * rho) : 0.0;
  std::vector<uint32_t> key((size_t)M), key2((size_t)M);
  std::vector<int64_t> idx2((size_t)M);
  perm.resize((size_t)M);
  for (int64_t i = 0; i < M; ++i) {
    const double a = (double)u[i], b = (double)v[i];
    key[i] = (std::isfinite(a) && std::isfinite(b))
                 ? spread16(cell16(a, rho, scale)) | (spread16(cell16(b, rho, scale)) << 1)
                 : 0xFFFFFFFFu;
    perm[i] = i;
  }
  // four stable counting passes over the key bytes, lowest first
  for (int shift = 0; shift < 32; shift += 8) {
    int64_t count[257] = {};
    for (int64_t i = 0; i < M; ++i) ++count[((key[i] >> shift) & 0xFFu) + 1];
    for (int b = 0; b < 256; ++b) count[b + 1] += count[b];
    for (int64_t i = 0; i < M; ++i) {
      const int64_t d = count[(key[i] >> shift) & 0xFFu]++;
      key2[d] = key[i];
      idx2[d] = perm[i];
    }
    key.swap(key2);
    perm.swap(idx2);
  }
}

template <typename T>
cudaError_t permute5(const int64_t* perm, int64_t M, const T* const in[5], T* const out[5],
                     int blocks, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  int64_t need = (M + 255) / 256;
  const int grid = (int)(need < blocks ? need : blocks);
  permute5_kernel<T><<<grid < 1 ? 1 : grid, 256, 0, st>>>(perm, M, in[0], in[1], in[2], in[3],
                                                           in[4], out[0], out[1], out[2], out[3],
                                                           out[4]);
  return cudaGetLastError();
}

template void z_order<float>(const float*, const float*, int64_t, std::vector<int64_t>&);
template void z_order<double>(const double*, const double*, int64_t, std::vector<int64_t>&);
template cudaError_t permute5<float>(const int64_t*, int64_t, const float* const[5],
                                     float* const[5], int, cudaStream_t);
template cudaError_t permute5<double>(const int64_t*, int64_t, const double* const[5],
                                      double* const[5], int, cudaStream_t);

}  // namespace gal
