// Radix-R DFTs in registers (R = 2, 4, 8, 16; forward, natural input order)
// for the compile-time-length Stockham passes of gal_fft3.cuh.  bfly16 runs
// as 4 x 4 and leaves output k in register bfly_out<16>(k).
#pragma once

#include <type_traits>

#include "gal_common.cuh"

namespace gal {

// ---- radix-R DFTs in registers (forward, natural order) -------------------
template <typename C> __device__ __forceinline__ void bfly2(C* a) {
  const C t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <typename C> __device__ __forceinline__ void bfly4(C& a0, C& a1, C& a2, C& a3) {
  const C d0 = cadd(a0, a2), d2 = csub(a0, a2);
  const C d1 = cadd(a1, a3), d3 = cmul_mi(csub(a1, a3));
  a0 = cadd(d0, d1);
  a2 = csub(d0, d1);
  a1 = cadd(d2, d3);
  a3 = csub(d2, d3);
}

template <typename C> __device__ __forceinline__ void bfly8(C* a) {
  using R = decltype(a[0].x);
  const R h = (R)0.70710678118654752440084436210484903928;
  C b0 = cadd(a[0], a[4]), b4 = csub(a[0], a[4]);
  C b1 = cadd(a[1], a[5]), b5 = csub(a[1], a[5]);
  C b2 = cadd(a[2], a[6]), b6 = csub(a[2], a[6]);
  C b3 = cadd(a[3], a[7]), b7 = csub(a[3], a[7]);
  b5 = mkc((b5.x + b5.y) * h, (b5.y - b5.x) * h);
  b6 = cmul_mi(b6);
  b7 = mkc((b7.y - b7.x) * h, -(b7.x + b7.y) * h);
  bfly4(b0, b1, b2, b3);
  bfly4(b4, b5, b6, b7);
  a[0] = b0; a[2] = b1; a[4] = b2; a[6] = b3;
  a[1] = b4; a[3] = b5; a[5] = b6; a[7] = b7;
}

// 16-point DFT as 4 x 4: DFT4 over n1 of x[4 n1 + n2] for each n2, twiddle
// by W16^(n2 k1), DFT4 over n2; output index k1 + 4 k2.
template <typename C> __device__ __forceinline__ void bfly16(C* a) {
  using R = decltype(a[0].x);
  const R h = (R)0.70710678118654752440084436210484903928;   // cos(pi/4)
  const R c1 = (R)0.92387953251128675612818318939678828682;  // cos(pi/8)
  const R s1 = (R)0.38268343236508977172845998403039886676;  // sin(pi/8)
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) bfly4(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  // after this, a[4 k1 + n2] holds y[n2][k1]
  // twiddles W16^(n2 k1), W16 = exp(-i pi / 8)
  auto w1 = [&](C x) { return mkc(x.x * c1 + x.y * s1, x.y * c1 - x.x * s1); };  // W16^1
  auto w2 = [&](C x) { return mkc((x.x + x.y) * h, (x.y - x.x) * h); };          // W16^2
  auto w3 = [&](C x) { return mkc(x.x * s1 + x.y * c1, x.y * s1 - x.x * c1); };  // W16^3
  auto w6 = [&](C x) { return mkc((x.y - x.x) * h, -(x.x + x.y) * h); };         // W16^6
  auto w9 = [&](C x) { return mkc(-x.x * c1 - x.y * s1, x.x * s1 - x.y * c1); }; // W16^9 = -W16^1
  a[4 * 1 + 1] = w1(a[5]);
  a[4 * 1 + 2] = w2(a[6]);
  a[4 * 1 + 3] = w3(a[7]);
  a[4 * 2 + 1] = w2(a[9]);
  a[4 * 2 + 2] = cmul_mi(a[10]);
  a[4 * 2 + 3] = w6(a[11]);
  a[4 * 3 + 1] = w3(a[13]);
  a[4 * 3 + 2] = w6(a[14]);
  a[4 * 3 + 3] = w9(a[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) bfly4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  // a[4 k1 + k2] now holds X[k1 + 4 k2]; callers address output r through
  // bfly_out<16>(r) instead of moving registers
}

// register holding output r of bflyR<R>
template <int R> __host__ __device__ constexpr int bfly_out(int r) {
  return R == 16 ? 4 * (r % 4) + r / 4 : r;
}

template <int R, typename C> __device__ __forceinline__ void bflyR(C* a) {
  if constexpr (R == 2) bfly2(a);
  else if constexpr (R == 4) bfly4(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) bfly8(a);
  else bfly16(a);
}

}  // namespace gal
