// Device helpers shared by the kernels: complex arithmetic, float-float
// (double-float) arithmetic, and the exact spectrum-pruning bounds.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace gal {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

__host__ __device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * (-i)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return mkc(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
// a + f (b - a), componentwise
template <typename C, typename T> __device__ __forceinline__ C clerp(C a, C b, T f) {
  return mkc(a.x + f * (b.x - a.x), a.y + f * (b.y - a.y));
}

// ---------------------------------------------------------------------------
// float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, about 48
// significant bits.  Error-free transformations: TwoSum (Knuth), FastTwoSum
// (Dekker), TwoProd through a fused multiply-add.  Used for the uv -> grid
// index and phase arguments of the single-precision path, which GB300's
// FP64 pipe (a small fraction of the FP32 rate) would otherwise bottleneck.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__host__ __device__ __forceinline__ ff ff_split(double d) {
  ff r;
  r.hi = (float)d;
  r.lo = (float)(d - (double)r.hi);
  return r;
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  ff r;
  r.hi = a * b;
  r.lo = fmaf(a, b, -r.hi);
  return r;
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  ff r;
  r.hi = a + b;
  const float bb = r.hi - a;
  r.lo = (a - (r.hi - bb)) + (b - bb);
  return r;
}
// requires |a| >= |b| or a == 0
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  ff r;
  r.hi = a + b;
  r.lo = b - (r.hi - a);
  return r;
}
// float times float-float
__device__ __forceinline__ ff ff_mul_f(float a, ff b) {
  ff p = ff_two_prod(a, b.hi);
  p.lo = fmaf(a, b.lo, p.lo);
  return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = ff_two_sum(a.hi, b);
  s.lo += a.lo;
  return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) {
  ff r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}

// ---------------------------------------------------------------------------
// Spectrum pruning.  A uv point at distance rho from the origin maps, for any
// position angle, to |u'|, |v'| <= rho, i.e. to grid offsets of at most
// e = rho * nxy * dxy cells from (v = 0, u = 0).  The bilinear stencil reads
// one node beyond the floor of the index, and the single-precision index
// carries a relative error near 1e-7, so a margin of 3 cells makes the window
// exact: every node any point can read lies in columns [0, Kc) and rows
// [r0, r0 + nrw) of the half spectrum (nxy rows, nxy/2+1 columns).
// ---------------------------------------------------------------------------
struct Bounds {
  int Kc;   // number of u columns kept (from u = 0)
  int r0;   // first kept row of the v-shifted spectrum
  int nrw;  // number of kept rows
};

__host__ __device__ __forceinline__ Bounds make_bounds(double rho2, double S, int N) {
  Bounds b;
  const int P = N / 2 + 1;
  const double e = sqrt(rho2) * S;
  if (!(e < (double)N)) {  // also catches NaN
    b.Kc = P;
    b.r0 = 0;
    b.nrw = N;
    return b;
  }
  const int k = (int)floor(e) + 3;
  b.Kc = k + 1 < P ? k + 1 : P;
  const int lo = N / 2 - k > 0 ? N / 2 - k : 0;
  const int hi = N / 2 + k < N - 1 ? N / 2 + k : N - 1;
  b.r0 = lo;
  b.nrw = hi - lo + 1;
  return b;
}

// Columns of the full-plane (complex-to-complex) window: u from -lo to hi
// cells, stored as window columns 0 .. W-1 (column lo is u = 0).  A pruned
// window keeps -(Kc-1) .. Kc-1 (every point stays two cells inside); the
// whole plane keeps the node range -N/2 .. N/2-1 of the shifted spectrum.
struct FullCols {
  int lo, hi, W;
};

__host__ __device__ __forceinline__ FullCols full_cols(const Bounds& b, int N) {
  FullCols f;
  f.lo = b.Kc >= N / 2 + 1 ? N / 2 : b.Kc - 1;
  f.hi = b.Kc - 1 < N / 2 - 1 ? b.Kc - 1 : N / 2 - 1;
  f.W = f.lo + f.hi + 1;
  return f;
}

// Bounds for the whole block: one thread evaluates them (FP64: GB300's FP64
// pipe is narrow, so no per-thread FP64 work) and shares them.  Every thread
// of the block must call it.
__device__ __forceinline__ Bounds block_bounds(const double* rho2, double S, int N) {
  __shared__ Bounds sb;
  if (threadIdx.x == 0) sb = make_bounds(*rho2, S, N);
  __syncthreads();
  return sb;
}

}  // namespace gal
