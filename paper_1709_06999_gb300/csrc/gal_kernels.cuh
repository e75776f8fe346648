// Kernels of the visibility / chi-square path and their host-side launchers.
//
//   twiddle_kernel   W_N^k table, computed in FP64 (sincospi) and rounded once
//   extent_kernel    max_k (u_k^2 + v_k^2)                       (Sect. 3.3 (i))
//   sweep_kernel     profile -> image                           (Sect. 2, App. D)
//   row_pass_kernel  fftshift + real-to-complex FFT of each row, optionally
//                    generating the row from the profile on the fly (Sect. 4)
//   col_pass_kernel  complex FFT down each kept column + fftshift along v
//   gather_kernel    rotate, index, Hermitian fold, bilinear, phase
//                    (Sect. 3.2, 3.3, App. D) and, fused, the chi-square
//                    (Eq. chap6.eq:def.chi.square) with a fixed-order reduction
#pragma once

#include "gal_common.cuh"
#include "gal_fft.cuh"
#include "gal_internal.h"

namespace gal {

// ---------------------------------------------------------------------------
// twiddles: tw[k] = exp(-2 pi i k / N), k = 0 .. N-1
// ---------------------------------------------------------------------------
template <typename T>
__global__ void twiddle_kernel(cplx_t<T>* __restrict__ tw, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)N, &s, &c);
  tw[k] = mkc((T)c, (T)s);
}

// ---------------------------------------------------------------------------
// uv extent: *rho2 = max(*rho2, max_k u_k^2 + v_k^2) (NaN points ignored).
// Non-negative doubles order like their bit patterns, so atomicMax on the
// 64-bit pattern is an exact maximum.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void extent_kernel(const T* __restrict__ u, const T* __restrict__ v, int64_t M,
                              double* __restrict__ rho2) {
  double m = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)u[k], b = (double)v[k];
    const double r = a * a + b * b;
    if (r > m) m = r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_down_sync(0xffffffffu, m, o);
    if (x > m) m = x;
  }
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = m;
  __syncthreads();
  if (warp == 0) {
    m = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_down_sync(0xffffffffu, m, o);
      if (x > m) m = x;
    }
    if (lane == 0 && m > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(rho2),
                (unsigned long long)__double_as_longlong(m));
  }
}

// ---------------------------------------------------------------------------
// sweep: one pixel of the profile image (unshifted pixel (i, j)).
// ---------------------------------------------------------------------------
template <typename T> struct SweepT {
  T Rmin, inv_dR, xscale, yscale, area;
  int nr;
};

template <typename T> __host__ __device__ inline SweepT<T> sweep_cast(const SweepParams& p) {
  SweepT<T> q;
  q.Rmin = (T)p.Rmin;
  q.inv_dR = (T)(1.0 / p.dR);
  q.xscale = (T)(p.dxy / cos(p.inc));
  q.yscale = (T)p.dxy;
  q.area = (T)(p.dxy * p.dxy);
  q.nr = p.nr;
  return q;
}

// Round-to-nearest arithmetic with no contraction, so that a pixel value does
// not depend on the kernel it is inlined into (the fused row pass and the
// stand-alone sweep produce bit-identical images).
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }

// Linear interpolation of I at r = |((N/2-j) dxy / cos inc, (N/2-i) dxy)|,
// zero outside [Rmin, Rmin + (nr-1) dR]; the centre pixel takes the linear
// extrapolation of the first two samples to r = 0; result times dxy^2.
template <typename T>
__device__ __forceinline__ T sweep_pixel(const T* __restrict__ I, const SweepT<T>& p, int N, int i,
                                         int j) {
  const int h = N >> 1;
  if (i == h && j == h) {
    const T I0 = __ldg(I), I1 = __ldg(I + 1);
    return rn_mul(rn_sub(I0, rn_mul(rn_mul(p.Rmin, p.inv_dR), rn_sub(I1, I0))), p.area);
  }
  const T x = rn_mul((T)(h - j), p.xscale);
  const T y = rn_mul((T)(h - i), p.yscale);
  const T r = rn_sqrt(rn_add(rn_mul(x, x), rn_mul(y, y)));
  const T t = rn_mul(rn_sub(r, p.Rmin), p.inv_dR);
  if (!(t >= (T)0) || t > (T)(p.nr - 1)) return (T)0;
  int k = (int)t;
  if (k > p.nr - 2) k = p.nr - 2;
  const T f = rn_sub(t, (T)k);
  const T a = __ldg(I + k), b = __ldg(I + k + 1);
  return rn_mul(rn_add(a, rn_mul(f, rn_sub(b, a))), p.area);
}

template <typename T>
__global__ void sweep_kernel(const T* __restrict__ I, SweepT<T> p, int N, T* __restrict__ img) {
  const int64_t n = (int64_t)N * N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / N), j = (int)(q % N);
    img[q] = sweep_pixel(I, p, N, i, j);
  }
}

// ---------------------------------------------------------------------------
// Row pass.  F1 row i' (i' = 0..N-1) is the real-to-complex FFT of row i' of
// fftshift(image), i.e. of image row (i' + N/2) mod N with its two halves
// swapped; only the first Kc output bins are stored (pitch Kc).  The real row
// x is read as the complex sequence z_n = x_{2n} + i x_{2n+1} (M = N/2
// points), transformed, and unpacked with
//   X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W_N^k (Z_k - conj Z_{M-k}).
// With SWEEP the row is generated from the profile instead of read.
// ---------------------------------------------------------------------------
template <typename T, bool SWEEP>
__global__ void __launch_bounds__(1024) row_pass_kernel(const T* __restrict__ image, const T* __restrict__ I,
                                SweepT<T> sp, int N, const cplx_t<T>* __restrict__ tw,
                                cplx_t<T>* __restrict__ F1, const double* __restrict__ rho2,
                                double S) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int M = N >> 1;
  const int Tg = M >= 8 ? M / 8 : 1;
  const int g = threadIdx.x / Tg, t = threadIdx.x % Tg;
  const int rpb = blockDim.x / Tg;
  const int row = blockIdx.x * rpb + g;
  const bool active = row < N;
  C* s = sm + (size_t)g * M;
  const Bounds bd = make_bounds(*rho2, S, N);

  if (active) {
    const int irow = (row + M) & (N - 1);
    for (int n = t; n < M; n += Tg) {
      const int j = (2 * n + M) & (N - 1);
      C z;
      if constexpr (SWEEP) {
        z = mkc(sweep_pixel(I, sp, N, irow, j), sweep_pixel(I, sp, N, irow, j + 1));
      } else {
        z = *reinterpret_cast<const C*>(image + (size_t)irow * N + j);
      }
      s[n] = z;
    }
  }
  __syncthreads();
  fft_inplace(s, M, t, Tg, tw, 2);
  if (active) {
    C* out = F1 + (size_t)row * bd.Kc;
    using R = T;
    for (int k = t; k < bd.Kc; k += Tg) {
      const C a = s[k & (M - 1)];
      const C b = cconj(s[(M - k) & (M - 1)]);
      const C e = mkc((R)0.5 * (a.x + b.x), (R)0.5 * (a.y + b.y));
      const C d = mkc((R)0.5 * (a.x - b.x), (R)0.5 * (a.y - b.y));
      const C o = cmul(cmul_mi(d), __ldg(tw + k));
      out[k] = cadd(e, o);
    }
  }
}

// ---------------------------------------------------------------------------
// Column pass.  For each kept column c < Kc: complex FFT over the N rows of
// F1 (pitch Kc), then the v-axis fftshift: output row r holds frequency
// kv = (r + N/2) mod N.  Only rows r0 .. r0+nrw-1 are written, to the window
// Gw (nrw x Kc, pitch Kc).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) col_pass_kernel(const cplx_t<T>* __restrict__ F1, cplx_t<T>* __restrict__ Gw, int N,
                                const cplx_t<T>* __restrict__ tw, const double* __restrict__ rho2,
                                double S) {
  using C = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const Bounds bd = make_bounds(*rho2, S, N);
  const int Tg = N >= 8 ? N / 8 : 1;
  const int cpb = blockDim.x / Tg;
  const int c0 = blockIdx.x * cpb;
  if (c0 >= bd.Kc) return;  // uniform over the block
  const int g = threadIdx.x / Tg, t = threadIdx.x % Tg;
  const int ld = N + 1;  // padded column stride in shared memory
  for (int q = threadIdx.x; q < cpb * N; q += blockDim.x) {
    const int cl = q % cpb, i = q / cpb, c = c0 + cl;
    sm[(size_t)cl * ld + i] = c < bd.Kc ? F1[(size_t)i * bd.Kc + c] : mkc((T)0, (T)0);
  }
  __syncthreads();
  fft_inplace(sm + (size_t)g * ld, N, t, Tg, tw, 1);
  for (int q = threadIdx.x; q < cpb * bd.nrw; q += blockDim.x) {
    const int cl = q % cpb, rr = q / cpb, c = c0 + cl;
    if (c < bd.Kc) {
      const int kv = (bd.r0 + rr + N / 2) & (N - 1);
      Gw[(size_t)rr * bd.Kc + c] = sm[(size_t)cl * ld + kv];
    }
  }
}

// ---------------------------------------------------------------------------
// Gather: per uv point, rotation (Sect. 3.2), grid index with Hermitian fold
// (App. D), bilinear interpolation clamped to the node range (Sect. 3.3),
// phase factor exp(+2 pi i (u dRA + v dDec)) (Sect. 3.2, App. D sign; the
// offset rotates with the uv points, and the dot product is rotation
// invariant, so the unrotated u, v are used).
// ---------------------------------------------------------------------------

// position x = xh + xl clamped to [0, n-1]; cell c in [0, n-2], fraction f
__device__ __forceinline__ void cell_ff(float xh, float xl, int n, int& c, float& f) {
  float fl = floorf(xh);
  float fr = (xh - fl) + xl;
  if (fr < 0.f) {
    fl -= 1.f;
    fr += 1.f;
  } else if (fr >= 1.f) {
    fl += 1.f;
    fr -= 1.f;
  }
  if (fl < 0.f) {
    c = 0;
    f = 0.f;
  } else if (fl >= (float)(n - 1)) {
    c = n - 2;
    f = 1.f;
  } else {
    c = (int)fl;
    f = fr;
  }
}

__device__ __forceinline__ void cell_d(double x, int n, int& c, double& f) {
  x = fmin(fmax(x, 0.0), (double)(n - 1));
  double fl = floor(x);
  if (fl > (double)(n - 2)) fl = (double)(n - 2);
  c = (int)fl;
  f = x - fl;
}

template <typename T> struct GatherT;

template <> struct GatherT<float> {
  ff cpa, spa, S, phx, phy;
  float half;
  double Sd;
  int N, P;
  __host__ static GatherT make(const GatherParams& g) {
    GatherT r;
    r.Sd = g.S;
    r.cpa = ff_split(g.cpa);
    r.spa = ff_split(g.spa);
    r.S = ff_split(g.S);
    r.phx = ff_split(g.phx);
    r.phy = ff_split(g.phy);
    r.half = (float)(g.N / 2);
    r.N = g.N;
    r.P = g.N / 2 + 1;
    return r;
  }
};

template <> struct GatherT<double> {
  double cpa, spa, S, phx, phy, half;
  double Sd;
  int N, P;
  __host__ static GatherT make(const GatherParams& g) {
    GatherT r;
    r.Sd = g.S;
    r.cpa = g.cpa;
    r.spa = g.spa;
    r.S = g.S;
    r.phx = g.phx;
    r.phy = g.phy;
    r.half = (double)(g.N / 2);
    r.N = g.N;
    r.P = g.N / 2 + 1;
    return r;
  }
};

template <typename C>
__device__ __forceinline__ C window_bilinear(const C* __restrict__ Gw, const Bounds& bd, int r, int c,
                                             decltype(C().x) fr, decltype(C().x) fc,
                                             int* __restrict__ err) {
  int rr = r - bd.r0;
  if (rr < 0 || rr + 1 >= bd.nrw || c + 1 >= bd.Kc) {  // never taken: the window is exact
    atomicOr(err, 1);
    rr = min(max(rr, 0), bd.nrw - 2);
    c = min(c, bd.Kc - 2);
  }
  const C* g = Gw + (size_t)rr * bd.Kc + c;
  const C g00 = __ldg(g), g01 = __ldg(g + 1);
  const C g10 = __ldg(g + bd.Kc), g11 = __ldg(g + bd.Kc + 1);
  return clerp(clerp(g00, g01, fc), clerp(g10, g11, fc), fr);
}

__device__ __forceinline__ float2 sample_point(const float2* __restrict__ Gw, const Bounds& bd,
                                               const GatherT<float>& p, float u, float v,
                                               int* __restrict__ err) {
  if (!(isfinite(u) && isfinite(v))) return make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
  ff up = ff_add(ff_mul_f(u, p.cpa), ff_neg(ff_mul_f(v, p.spa)));
  ff vp = ff_add(ff_mul_f(u, p.spa), ff_mul_f(v, p.cpa));
  const bool neg = up.hi < 0.f;
  if (neg) {
    up = ff_neg(up);
    vp = ff_neg(vp);
  }
  const ff iu = ff_mul(up, p.S);
  const ff iv = ff_add_f(ff_mul(vp, p.S), p.half);
  int r, c;
  float fr, fc;
  cell_ff(iv.hi, iv.lo, p.N, r, fr);
  cell_ff(iu.hi, iu.lo, p.P, c, fc);
  float2 V = window_bilinear(Gw, bd, r, c, fr, fc, err);
  if (neg) V.y = -V.y;
  const ff ph = ff_add(ff_mul_f(u, p.phx), ff_mul_f(v, p.phy));
  const float n = rintf(ph.hi);
  const float fph = (ph.hi - n) + ph.lo;
  float sn, cs;
  sincospif(2.f * fph, &sn, &cs);
  return cmul(V, make_float2(cs, sn));
}

__device__ __forceinline__ double2 sample_point(const double2* __restrict__ Gw, const Bounds& bd,
                                                const GatherT<double>& p, double u, double v,
                                                int* __restrict__ err) {
  if (!(isfinite(u) && isfinite(v)))
    return make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
  double up = u * p.cpa - v * p.spa;
  double vp = u * p.spa + v * p.cpa;
  const bool neg = up < 0.0;
  if (neg) {
    up = -up;
    vp = -vp;
  }
  int r, c;
  double fr, fc;
  cell_d(p.half + vp * p.S, p.N, r, fr);
  cell_d(up * p.S, p.P, c, fc);
  double2 V = window_bilinear(Gw, bd, r, c, fr, fc, err);
  if (neg) V.y = -V.y;
  const double ph = u * p.phx + v * p.phy;
  const double fph = ph - rint(ph);
  double sn, cs;
  sincospi(2.0 * fph, &sn, &cs);
  return cmul(V, make_double2(cs, sn));
}

// per-thread compensated accumulators
struct AccF {  // float-float running sum
  ff s{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { s = ff_add_f(s, x); }
  __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};
struct AccD {  // Neumaier
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};
template <typename T> struct Acc;
template <> struct Acc<float> { using type = AccF; };
template <> struct Acc<double> { using type = AccD; };

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void load16(const T* __restrict__ p, int64_t q, T (&out)[Vec16<T>::W]) {
  using V = typename Vec16<T>::type;
  const V x = __ldcs(reinterpret_cast<const V*>(p) + q);
  if constexpr (Vec16<T>::W == 4) {
    out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
  } else {
    out[0] = x.x; out[1] = x.y;
  }
}

// block-wide sum of one double per thread, fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double x, double* ws) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[warp] = x;
  __syncthreads();
  x = 0.0;
  if (warp == 0) {
    x = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  }
  return x;
}

template <typename T, bool CHI2>
__global__ void __launch_bounds__(256)
gather_kernel(const cplx_t<T>* __restrict__ Gw, GatherT<T> p, const double* __restrict__ rho2,
              const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ re,
              const T* __restrict__ im, const T* __restrict__ w, int64_t M, int vec,
              cplx_t<T>* __restrict__ vis, double* __restrict__ partials,
              unsigned* __restrict__ counter, double* __restrict__ chi2_out, int* __restrict__ err) {
  using C = cplx_t<T>;
  constexpr int W = Vec16<T>::W;
  const Bounds bd = make_bounds(*rho2, p.Sd, p.N);
  typename Acc<T>::type acc;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nq = vec ? M / W : 0;
  for (int64_t q = gtid; q < nq; q += gstride) {
    T uu[W], vv[W];
    load16(u, q, uu);
    load16(v, q, vv);
    if constexpr (CHI2) {
      T rr[W], ii[W], ww[W];
      load16(re, q, rr);
      load16(im, q, ii);
      load16(w, q, ww);
#pragma unroll
      for (int e = 0; e < W; ++e) {
        const C V = sample_point(Gw, bd, p, uu[e], vv[e], err);
        const T dr = rr[e] - V.x, di = ii[e] - V.y;
        acc.add(ww[e] * (dr * dr + di * di));
      }
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) vis[q * W + e] = sample_point(Gw, bd, p, uu[e], vv[e], err);
    }
  }
  for (int64_t k = nq * W + gtid; k < M; k += gstride) {
    const C V = sample_point(Gw, bd, p, u[k], v[k], err);
    if constexpr (CHI2) {
      const T dr = re[k] - V.x, di = im[k] - V.y;
      acc.add(w[k] * (dr * dr + di * di));
    } else {
      vis[k] = V;
    }
  }
  if constexpr (CHI2) {
    __shared__ double ws[32];
    __shared__ bool last;
    const double bs = block_sum(acc.value(), ws);
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = bs;
      __threadfence();
      const unsigned prev = atomicAdd(counter, 1u);
      last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      AccD a;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a.add(__ldcg(partials + b));
      const double tot = block_sum(a.value(), ws);
      if (threadIdx.x == 0) {
        *chi2_out = tot;
        *counter = 0u;
      }
    }
  }
}

}  // namespace gal

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
namespace gal {

constexpr int kMaxDynSmem = 227 * 1024;

inline int row_threads_per_row(int N) { return N / 2 >= 8 ? N / 16 : 1; }
inline int col_threads_per_col(int N) { return N >= 8 ? N / 8 : 1; }

template <typename T> cudaError_t Launch<T>::init() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(row_pass_kernel<T, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(row_pass_kernel<T, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)))
    return e;
  return cudaFuncSetAttribute(col_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxDynSmem);
}

template <typename T> int Launch<T>::gather_blocks_per_sm(bool chi2) {
  int n = 0;
  if (chi2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, true>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, false>, 256, 0);
  return n < 1 ? 1 : n;
}

template <typename T> cudaError_t Launch<T>::twiddles(void* tw, int N, cudaStream_t st) {
  twiddle_kernel<T><<<(N + 255) / 256, 256, 0, st>>>(static_cast<cplx_t<T>*>(tw), N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::extent(const T* u, const T* v, int64_t M, double* rho2, int blocks,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(rho2, 0, sizeof(double), st);
  if (e) return e;
  if (M <= 0) return cudaSuccess;
  const int64_t need = (M + 255) / 256;
  const int grid = (int)(need < blocks ? need : blocks);
  extent_kernel<T><<<grid, 256, 0, st>>>(u, v, M, rho2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::sweep(const T* I, const SweepParams& sp, int N, T* img, int blocks,
                             cudaStream_t st) {
  const int64_t n = (int64_t)N * N;
  const int64_t need = (n + 255) / 256;
  const int grid = (int)(need < blocks ? need : blocks);
  sweep_kernel<T><<<grid, 256, 0, st>>>(I, sweep_cast<T>(sp), N, img);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::row_pass(const T* image, const T* I, const SweepParams& sp, int N,
                                const void* tw, void* F1, const double* rho2, double S,
                                cudaStream_t st) {
  using C = cplx_t<T>;
  const int M = N / 2;
  const int tg = row_threads_per_row(N);
  int rpb = 256 / tg;
  if (rpb < 1) rpb = 1;
  if (rpb > N) rpb = N;
  const int threads = tg * rpb;
  const size_t smem = (size_t)rpb * M * sizeof(C);
  const int grid = (N + rpb - 1) / rpb;
  const C* twc = static_cast<const C*>(tw);
  C* out = static_cast<C*>(F1);
  if (I)
    row_pass_kernel<T, true><<<grid, threads, smem, st>>>(nullptr, I, sweep_cast<T>(sp), N, twc,
                                                           out, rho2, S);
  else
    row_pass_kernel<T, false><<<grid, threads, smem, st>>>(image, nullptr, SweepT<T>{}, N, twc,
                                                            out, rho2, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::col_pass(const void* F1, void* Gw, int N, const void* tw,
                                const double* rho2, double S, cudaStream_t st) {
  using C = cplx_t<T>;
  const int tg = col_threads_per_col(N);
  int cpb = 256 / tg;
  if (cpb < 1) cpb = 1;
  const int P = N / 2 + 1;
  if (cpb > P) cpb = P;
  const int threads = tg * cpb;
  const size_t smem = (size_t)cpb * (N + 1) * sizeof(C);
  const int grid = (P + cpb - 1) / cpb;
  col_pass_kernel<T><<<grid, threads, smem, st>>>(static_cast<const C*>(F1), static_cast<C*>(Gw),
                                                  N, static_cast<const C*>(tw), rho2, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::gather(const void* Gw, const GatherParams& gp, const double* rho2,
                              const T* u, const T* v, const T* re, const T* im, const T* w,
                              int64_t M, void* vis, double* partials, unsigned* counter,
                              double* chi2, int* err, int blocks, cudaStream_t st) {
  using C = cplx_t<T>;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  int vec = al16(u) && al16(v);
  if (chi2) vec = vec && al16(re) && al16(im) && al16(w);
  const GatherT<T> p = GatherT<T>::make(gp);
  const C* g = static_cast<const C*>(Gw);
  if (chi2) {
    gather_kernel<T, true><<<blocks, 256, 0, st>>>(g, p, rho2, u, v, re, im, w, M, vec, nullptr,
                                                   partials, counter, chi2, err);
  } else {
    int64_t need = (M + 255) / 256;
    if (need < 1) need = 1;
    const int grid = (int)(need < blocks ? need : blocks);
    gather_kernel<T, false><<<grid, 256, 0, st>>>(g, p, rho2, u, v, nullptr, nullptr, nullptr, M,
                                                  vec, static_cast<C*>(vis), nullptr, nullptr,
                                                  nullptr, err);
  }
  return cudaGetLastError();
}

}  // namespace gal
