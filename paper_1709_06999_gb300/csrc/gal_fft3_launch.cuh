// Launchers of the compile-time-length row and column passes: one kernel
// instantiation per transform length, chosen by a switch on log2 of it.
#pragma once

#include <type_traits>

#include "gal_kernels.cuh"

namespace gal {

// Image rows of the one length row_fft3_ldg_kernel serves (float, 4096
// pixels, radix 16) take that kernel, in single calls and batches alike.
template <typename T, int LG, bool SWEEP, int V> constexpr bool row_ldg_shape() {
  return std::is_same<T, float>::value && !SWEEP && LG == kRowLdgLG && V == 16;
}
// its persistent grid: the resident blocks of the device, shared by the
// `n` requests of a launch (grid row y = request), at most one row each
template <auto Kern> int row_ldg_grid(int n) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kern, RowLdgShape::TT,
                                                    RowLdgShape::smem) != cudaSuccess)
    return 0;
  if (per_sm < 1) per_sm = 1;
  int x = (per_sm * current_device_sms() + n - 1) / n;
  return x > RowLdgShape::N ? RowLdgShape::N : x;
}

// A row pass with a beam follows beam_table_kernel in the stream and is
// launched as its programmatic dependent (BEAM kernels wait for the tables).
template <typename T, int LG, bool SWEEP, bool BEAM, int V = FftV<T>::V>
cudaError_t launch_row3_kern(const Jobs<RowJob<T>, 1>& jb, const cplx_t<T>* twc, int* err,
                             cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LG, N = 2 * M;
  if constexpr (row_ldg_shape<T, LG, SWEEP, V>()) {  // float rows of 4096 pixels
    constexpr auto kern = row_fft3_ldg_kernel<1, BEAM>;
    cudaError_t e = ensure_smem_attr<kern>(RowLdgShape::smem);
    if (e) return e;
    const int grid = row_ldg_grid<kern>(1);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if constexpr (BEAM)
      return launch_dependent(kern, dim3(grid), dim3(RowLdgShape::TT), RowLdgShape::smem, st, jb, twc);
    kern<<<grid, RowLdgShape::TT, RowLdgShape::smem, st>>>(jb, twc);
    return cudaGetLastError();
  } else {
    using SH = Shape3<T, M, N, 128, V>;
    constexpr auto kern = row_fft3_kernel<T, LG, !SWEEP, SWEEP, 1, BEAM, 128, 2, V>;
    const size_t smem = 128 + (size_t)(SWEEP ? 2 : 3) * SH::G * SH::RS * sizeof(C);
    cudaError_t e = ensure_smem_attr<kern>(smem);
    if (e) return e;
    int grid = N / SH::G;
    if constexpr (!SWEEP) {  // persistent blocks over the TMA row ring
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::threads, smem);
      if (e) return e;
      if (per_sm < 1) per_sm = 1;
      if (grid > per_sm * current_device_sms()) grid = per_sm * current_device_sms();
    }
    if constexpr (BEAM)
      return launch_dependent(kern, dim3(grid), dim3(SH::threads), smem, st, jb, twc, err);
    kern<<<grid, SH::threads, smem, st>>>(jb, twc, err);
    return cudaGetLastError();
  }
}

// the radix-8 float passes exist for image sides up to kAltRadixMaxSide
template <typename T, int N> constexpr bool has_alt_radix() {
  return sizeof(T) == 4 && N <= kAltRadixMaxSide && N / 2 >= kAltRadix;
}

template <typename T, int LG, bool SWEEP>
cudaError_t launch_row3(const T* image, const T* I, const SweepParams& sp, const void* tw,
                        void* F1, const double* rho2, double S, int* err, const T* beam,
                        cudaStream_t st, int radix) {
  using C = cplx_t<T>;
  const C* twc = static_cast<const C*>(tw);
  Jobs<RowJob<T>, 1> jb;
  jb.j[0] = RowJob<T>{image, I, SWEEP ? sweep_cast<T>(sp) : SweepT<T>{}, static_cast<C*>(F1),
                      rho2, S, beam};
  if constexpr (has_alt_radix<T, (2 << LG)>()) {
    if (radix == kAltRadix) {
      if (beam) return launch_row3_kern<T, LG, SWEEP, true, kAltRadix>(jb, twc, err, st);
      return launch_row3_kern<T, LG, SWEEP, false, kAltRadix>(jb, twc, err, st);
    }
  }
  if (beam) return launch_row3_kern<T, LG, SWEEP, true>(jb, twc, err, st);
  return launch_row3_kern<T, LG, SWEEP, false>(jb, twc, err, st);
}

template <typename T, int LG, int V = FftV<T>::V>
cudaError_t launch_col3_kern(const void* F1, void* Gw, const void* tw, const double* rho2, double S,
                             int kc_hint, bool full, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int N = 1 << LG;
  using SH = ColShape3<T, N, V>;
  constexpr auto kern = col_fft3_kernel<T, LG, 1, V>;
  const size_t smem = (size_t)2 * SH::G * SH::RS * sizeof(C);
  const cudaError_t e = ensure_smem_attr<kern>(smem);
  if (e) return e;
  const int P = full ? N : N / 2 + 1;  // most window columns
  const int kc = kc_hint > 0 && kc_hint <= P ? kc_hint : P;
  int col_blocks = (kc + SH::G - 1) / SH::G;
  const int cap = 2 * current_device_sms();
  if (col_blocks > cap) col_blocks = cap;
  Jobs<ColJob<T>, 1> jb;
  jb.j[0] = ColJob<T>{static_cast<const C*>(F1), static_cast<C*>(Gw), rho2, S, full ? 1 : 0};
  return launch_dependent(kern, dim3(col_blocks), dim3(SH::threads), smem, st, jb,
                          static_cast<const C*>(tw));
}

template <typename T, int LG>
cudaError_t launch_col3(const void* F1, void* Gw, const void* tw, const double* rho2, double S,
                        int kc_hint, bool full, cudaStream_t st, int radix) {
  if constexpr (has_alt_radix<T, (1 << LG)>()) {
    if (radix == kAltRadix)
      return launch_col3_kern<T, LG, kAltRadix>(F1, Gw, tw, rho2, S, kc_hint, full, st);
  }
  return launch_col3_kern<T, LG>(F1, Gw, tw, rho2, S, kc_hint, full, st);
}

template <typename T, int LG>
cudaError_t row3_switch(int lg, const T* image, const T* I, const SweepParams& sp,
                        const void* tw, void* F1, const double* rho2, double S, int* err,
                        const T* beam, cudaStream_t st, int radix) {
  if constexpr (LG > 12) {
    return cudaErrorNotSupported;
  } else {
    if (lg == LG) {
      if (I) return launch_row3<T, LG, true>(image, I, sp, tw, F1, rho2, S, err, beam, st, radix);
      return launch_row3<T, LG, false>(image, I, sp, tw, F1, rho2, S, err, beam, st, radix);
    }
    return row3_switch<T, LG + 1>(lg, image, I, sp, tw, F1, rho2, S, err, beam, st, radix);
  }
}

// largest column length with both ping-pong buffers in shared memory:
// 8192 float2 (2 x 8704 x 8 B) but 4096 double2 (8192 would need 295 KB)
template <typename T> constexpr int col3_max_lg() { return sizeof(T) == 4 ? 13 : 12; }

template <typename T, int LG>
cudaError_t col3_switch(int lg, const void* F1, void* Gw, const void* tw, const double* rho2,
                        double S, int kc_hint, bool full, cudaStream_t st, int radix) {
  if constexpr (LG > col3_max_lg<T>()) {
    return cudaErrorNotSupported;
  } else {
    if (lg == LG) return launch_col3<T, LG>(F1, Gw, tw, rho2, S, kc_hint, full, st, radix);
    return col3_switch<T, LG + 1>(lg, F1, Gw, tw, rho2, S, kc_hint, full, st, radix);
  }
}

inline int ilog2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

template <typename T>
cudaError_t row_fft3(const T* image, const T* I, const SweepParams& sp, int N, const void* tw,
                     void* F1, const double* rho2, double S, int* err, const T* beam,
                     cudaStream_t st, int radix) {
  constexpr int LG0 = ilog2c(FftV<T>::V);
  return row3_switch<T, LG0>(ilog2i(N / 2), image, I, sp, tw, F1, rho2, S, err, beam, st, radix);
}

template <typename T>
cudaError_t col_fft3(const void* F1, void* Gw, int N, const void* tw, const double* rho2, double S,
                     int kc_hint, bool full, cudaStream_t st, int radix) {
  constexpr int LG0 = ilog2c(FftV<T>::V);
  return col3_switch<T, LG0>(ilog2i(N), F1, Gw, tw, rho2, S, kc_hint, full, st, radix);
}

}  // namespace gal
