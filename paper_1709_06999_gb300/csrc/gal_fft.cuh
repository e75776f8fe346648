// In-place shared-memory Stockham FFT (forward, unnormalised, e^{-2 pi i k n / L}).
//
// A group of T = L/8 threads transforms one length-L sequence held in shared
// memory.  Every stage of radix R (8, or one leading stage of 4 or 2) is the
// self-sorting Stockham step: butterfly b reads the R values at b + r L/R,
// scales value r by W_{Ns R}^{r (b mod Ns)}, applies the radix-R DFT in
// registers and writes value r to (b div Ns) Ns R + (b mod Ns) + r Ns, where
// Ns is the product of the radices of the earlier stages.  Each thread owns 8
// values per stage (8/R butterflies), so a stage is: load to registers,
// barrier, compute, store, barrier.  Output is in natural order.
//
// Twiddles come from a table W_{Ntab}^k, k < Ntab, generated once in FP64 and
// rounded to the working precision; `tws` = Ntab / L.
#pragma once

#include "gal_common.cuh"

namespace gal {

template <typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// forward 4-point DFT, in place, natural order
template <typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C d0 = cadd(a0, a2), d2 = csub(a0, a2);
  const C d1 = cadd(a1, a3), d3 = cmul_mi(csub(a1, a3));
  a0 = cadd(d0, d1);
  a2 = csub(d0, d1);
  a1 = cadd(d2, d3);
  a3 = csub(d2, d3);
}

// forward 8-point DFT, in place, natural order: split into even outputs
// (4-point DFT of a_n + a_{n+4}) and odd outputs (4-point DFT of
// (a_n - a_{n+4}) W_8^n).
template <typename C> __device__ __forceinline__ void dft8(C* a) {
  using R = decltype(a[0].x);
  const R h = (R)0.70710678118654752440084436210484903928;
  C b0 = cadd(a[0], a[4]), b4 = csub(a[0], a[4]);
  C b1 = cadd(a[1], a[5]), b5 = csub(a[1], a[5]);
  C b2 = cadd(a[2], a[6]), b6 = csub(a[2], a[6]);
  C b3 = cadd(a[3], a[7]), b7 = csub(a[3], a[7]);
  b5 = mkc((b5.x + b5.y) * h, (b5.y - b5.x) * h);      // * W8^1 = (1 - i)/sqrt2
  b6 = cmul_mi(b6);                                      // * W8^2 = -i
  b7 = mkc((b7.y - b7.x) * h, -(b7.x + b7.y) * h);     // * W8^3 = (-1 - i)/sqrt2
  dft4(b0, b1, b2, b3);
  dft4(b4, b5, b6, b7);
  a[0] = b0; a[2] = b1; a[4] = b2; a[6] = b3;
  a[1] = b4; a[3] = b5; a[5] = b6; a[7] = b7;
}

template <int R, typename C> __device__ __forceinline__ void dftR(C* a) {
  if constexpr (R == 2) {
    dft2(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4(a[0], a[1], a[2], a[3]);
  } else {
    dft8(a);
  }
}

// One Stockham stage of radix R on the group's sequence s[0..L).  All threads
// of the block must call it (it contains __syncthreads).
template <int R, typename C>
__device__ __forceinline__ void stockham_stage(C* s, int L, int Ns, int t, int T,
                                               const C* __restrict__ tw, int tws) {
  constexpr int NB = 8 / R;
  C v[8];
  const int LR = L / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = s[b + r * LR];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * T;
    const int k = b & (Ns - 1);
    if (Ns > 1) {
      const int step = (L / (Ns * R)) * tws * k;
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], __ldg(tw + r * step));
    }
    dftR<R>(&v[q * R]);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[base + r * Ns] = v[q * R + r];
  }
  __syncthreads();
}

// Forward FFT of length L (power of two, L >= 2) of s[0..L), in place.  The
// group has T = max(1, L/8) threads; t in [0, T).  Must be called by every
// thread of the block with the same L.
template <typename C>
__device__ __forceinline__ void fft_inplace(C* s, int L, int t, int T, const C* __restrict__ tw,
                                            int tws) {
  if (L < 8) {
    if (t == 0) {
      if (L == 2) {
        dft2(s[0], s[1]);
      } else if (L == 4) {
        dft4(s[0], s[1], s[2], s[3]);
      }
    }
    __syncthreads();
    return;
  }
  const int lg = 31 - __clz(L);
  int Ns = 1;
  if (lg % 3 == 1) {
    stockham_stage<2>(s, L, Ns, t, T, tw, tws);
    Ns = 2;
  } else if (lg % 3 == 2) {
    stockham_stage<4>(s, L, Ns, t, T, tw, tws);
    Ns = 4;
  }
  while (Ns < L) {
    stockham_stage<8>(s, L, Ns, t, T, tw, tws);
    Ns *= 8;
  }
}

}  // namespace gal
