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
#include "gal_fft2.cuh"
#include "gal_fft3.cuh"
#include "gal_tma.cuh"

#include <atomic>
#include <limits>
#include <type_traits>
#include <utility>
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

// u_k = u_m,k nu_k / c and the same for v: baselines in metres at each
// visibility's own frequency, in wavelengths (Sect. 3, the frequency
// assumption lifted).  FP64 product then quotient, rounded to T once.
template <typename T>
__global__ void uv_from_frequency_kernel(const T* __restrict__ u_m, const T* __restrict__ v_m,
                                         const T* __restrict__ nu, int64_t M, T* __restrict__ u,
                                         T* __restrict__ v) {
  constexpr double kC = 299792458.0;  // m / s, exact by the definition of the metre
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double f = (double)nu[k];
    u[k] = (T)(__dmul_rn((double)u_m[k], f) / kC);  // (u_m nu) / c, each step rounded once
    v[k] = (T)(__dmul_rn((double)v_m[k], f) / kC);
  }
}

// min_k and max_k of u_k^2 + v_k^2 over the finite points (Sect. 3.3, criteria
// (i) and (iia)); range2[0] must start at +inf and range2[1] at 0.  Non-negative
// doubles order like their bit patterns, so the block results are combined
// with integer atomics.
template <typename T>
__global__ void uv_range_kernel(const T* __restrict__ u, const T* __restrict__ v, int64_t M,
                                double* __restrict__ range2) {
  double lo = __longlong_as_double(0x7ff0000000000000ll), hi = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)u[k], b = (double)v[k];
    const double r = a * a + b * b;
    if (r < lo) lo = r;  // NaN compares false both ways
    if (r > hi && r < __longlong_as_double(0x7ff0000000000000ll)) hi = r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_down_sync(0xffffffffu, lo, o);
    const double y = __shfl_down_sync(0xffffffffu, hi, o);
    if (x < lo) lo = x;
    if (y > hi) hi = y;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(reinterpret_cast<unsigned long long*>(range2), (unsigned long long)__double_as_longlong(lo));
    atomicMax(reinterpret_cast<unsigned long long*>(range2 + 1), (unsigned long long)__double_as_longlong(hi));
  }
}

// ---------------------------------------------------------------------------
// sweep: one pixel of the profile image (unshifted pixel (i, j)).
// ---------------------------------------------------------------------------
template <typename T> struct SweepT {
  T Rmin, inv_dR, xscale, yscale, area;
  int nr;
};

// Per-request kernel arguments.  Every pass takes a fixed-size array of K jobs
// as one __grid_constant__ parameter (read in place from the parameter bank,
// never copied): a single call launches K = 1, a batch launches up to
// kBatchJobs requests at once with job blockIdx.y in grid row y.
template <typename J, int K> struct Jobs {
  J j[K];
};

template <typename T> struct RowJob;
template <typename T> struct ColJob;
template <typename T> struct GatherJob;

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

// Primary-beam tables (Sect. 2.1: A is the antenna pattern normalised at the
// pointing centre, its central lobe a Gaussian of full width at half maximum
// K lambda / D): A(s) = exp(-c |s|^2), c = 4 ln 2 / fwhm^2, fixed on the
// phase centre.  After the PA rotation and the move o = (dRA, dDec) of
// Sect. 3.2, model pixel p = (x_j, y_i) lies on the sky at s = R^T p + o, and
// |R^T p + o| = |p + R o|, so A splits into a column term exp(-c (x_j + bx)^2)
// and a row term exp(-c (y_i + by)^2) with (bx, by) = R o.  Entry n < N is the
// column term of shifted column n (image column (n + N/2) mod N), entry N + n
// the row term of shifted row n; both in FP64, rounded once to T.
template <typename T>
__device__ __forceinline__ T beam_entry(int q, int N, double dxy, double c, double bx, double by) {
  const int n = q < N ? q : q - N;
  const int j = (n + N / 2) & (N - 1);
  const double s = (double)(N / 2 - j) * dxy + (q < N ? bx : by);
  return (T)exp(-c * s * s);
}

template <typename T>
__global__ void beam_table_kernel(T* __restrict__ tab, int N, double dxy, double c, double bx,
                                  double by) {
  grid_dep_launch();  // the row pass may start its image copies meanwhile
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 2 * N) tab[q] = beam_entry<T>(q, N, dxy, c, bx, by);
}

// the tables of up to K requests of a batch, grid row y = request y
template <typename T> struct BeamJob {
  T* tab;
  int N;
  double dxy, c, bx, by;
};
template <typename T, int K>
__global__ void beam_tables_kernel(const __grid_constant__ Jobs<BeamJob<T>, K> jobs) {
  const BeamJob<T>& jb = jobs.j[blockIdx.y];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * jb.N; q += gridDim.x * blockDim.x)
    jb.tab[q] = beam_entry<T>(q, jb.N, jb.dxy, jb.c, jb.bx, jb.by);
}

// Primary-beam factor (Sect. 2.1: the visibility is the transform of A I).
// The beam is a separable Gaussian on the image grid (see beam_table_kernel),
// tabulated in the fftshifted index order of the row pass: beam[n] for
// shifted column n, beam[N + i'] for shifted row i'.  A row-pass thread holds
// pixel pairs (2n, 2n + 1) of shifted row i' as one complex value.
template <typename T>
__device__ __forceinline__ cplx_t<T> beam_pair(cplx_t<T> z, const T* __restrict__ beam, int N,
                                               int row, int n) {
  const T ay = __ldg(beam + N + row);
  const cplx_t<T> ax = __ldg(reinterpret_cast<const cplx_t<T>*>(beam) + n);
  return mkc(z.x * (ay * ax.x), z.y * (ay * ax.y));
}

// ---------------------------------------------------------------------------
// Row pass.  F1 row i' (i' = 0..N-1) is the real-to-complex FFT of row i' of
// fftshift(image), i.e. of image row (i' + N/2) mod N with its two halves
// swapped; only the first Kc output bins are stored, column-major (column c
// holds bin c of the N rows).  The real row x is read as the complex
// sequence z_n = x_{2n} + i x_{2n+1} (M = N/2 points), transformed, and
// unpacked with
//   X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W_N^k (Z_k - conj Z_{M-k}).
// With SWEEP the row is generated from the profile instead of read.
// ---------------------------------------------------------------------------
template <typename T, bool SWEEP>
__global__ void __launch_bounds__(1024) row_pass_kernel(const T* __restrict__ image, const T* __restrict__ I,
                                SweepT<T> sp, int N, const cplx_t<T>* __restrict__ tw,
                                cplx_t<T>* __restrict__ F1, const double* __restrict__ rho2,
                                double S, const T* __restrict__ beam) {
  using C = cplx_t<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int M = N >> 1;
  const int Tg = M >= 8 ? M / 8 : 1;
  const int g = threadIdx.x / Tg, t = threadIdx.x % Tg;
  const int rpb = blockDim.x / Tg;
  const int row = blockIdx.x * rpb + g;
  const bool active = row < N;
  C* s = sm + (size_t)g * M;
  const Bounds bd = block_bounds(rho2, S, N);

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
      if (beam) z = beam_pair(z, beam, N, row, n);
      s[n] = z;
    }
  }
  __syncthreads();
  fft_inplace(s, M, t, Tg, tw, 2);
  if (active) {
    using R = T;
    for (int k = t; k < bd.Kc; k += Tg) {
      const C a = s[k & (M - 1)];
      const C b = cconj(s[(M - k) & (M - 1)]);
      const C e = mkc((R)0.5 * (a.x + b.x), (R)0.5 * (a.y + b.y));
      const C d = mkc((R)0.5 * (a.x - b.x), (R)0.5 * (a.y - b.y));
      const C o = cmul(cmul_mi(d), __ldg(tw + k));
      F1[(size_t)k * N + row] = cadd(e, o);  // column-major: column k holds N rows
    }
  }
}

// ---------------------------------------------------------------------------
// Column pass.  For each kept column c < Kc: complex FFT over the N rows of
// F1 (column-major, each column contiguous), then the v-axis fftshift: output
// row r holds frequency kv = (r + N/2) mod N.  Only rows r0 .. r0+nrw-1 are kept, written to the
// window Gp[rr Kc + c] (nrw x Kc).  Blocks loop over column groups (grid capped at a few blocks per SM), so a
// heavily pruned spectrum launches no idle blocks.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024)
col_pass_kernel(const cplx_t<T>* __restrict__ F1, cplx_t<T>* __restrict__ Gp, int N,
                const cplx_t<T>* __restrict__ tw, const double* __restrict__ rho2, double S) {
  using C = cplx_t<T>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const Bounds bd = block_bounds(rho2, S, N);
  const int Tg = N >= 8 ? N / 8 : 1;
  const int cpb = blockDim.x / Tg;
  const int g = threadIdx.x / Tg, t = threadIdx.x % Tg;
  const int ld = N + 1;  // padded column stride in shared memory
  for (int c0 = blockIdx.x * cpb; c0 < bd.Kc; c0 += gridDim.x * cpb) {
    for (int q = threadIdx.x; q < cpb * N; q += blockDim.x) {
      const int i = q % N, cl = q / N, c = c0 + cl;
      sm[(size_t)cl * ld + i] = c < bd.Kc ? F1[(size_t)c * N + i] : mkc((T)0, (T)0);
    }
    __syncthreads();
    fft_inplace(sm + (size_t)g * ld, N, t, Tg, tw, 1);
    for (int q = threadIdx.x; q < cpb * bd.nrw; q += blockDim.x) {
      const int cl = q % cpb, rr = q / cpb, c = c0 + cl;
      if (c < bd.Kc) {
        const int kv = (bd.r0 + rr + N / 2) & (N - 1);
        const C val = sm[(size_t)cl * ld + kv];
        Gp[(size_t)rr * bd.Kc + c] = val;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Compile-time-length row and column passes (gal_fft3.cuh), used whenever the
// transform length is at least V.
// ---------------------------------------------------------------------------
template <typename T> struct FftV;
template <> struct FftV<float> { static constexpr int V = 16; };
template <> struct FftV<double> { static constexpr int V = 8; };

// X_k = (A + B)/2 - (i/2) W (A - B), A = Z_k, B = conj Z_{M-k}, W = W_N^k
template <typename C> __device__ __forceinline__ C r2c_unpack(C zk, C zmk, C w) {
  using R = decltype(zk.x);
  const C b = cconj(zmk);
  const C e = mkc((R)0.5 * (zk.x + b.x), (R)0.5 * (zk.y + b.y));
  const C d = mkc((R)0.5 * (zk.x - b.x), (R)0.5 * (zk.y - b.y));
  return cadd(e, cmul(cmul_mi(d), w));
}

// Launch shape of the length-L passes: G sequences per block (at least 128
// threads), each with a shared-memory region of RS complex (padded, rounded
// to 16 bytes so that bulk copies into it stay aligned).
template <typename T, int L, int NSEQ, int MINT = 128, int VV = FftV<T>::V> struct Shape3 {
  using C = cplx_t<T>;
  static constexpr int V = VV;
  using P = P3<L, V>;
  static constexpr int G0 = P::T >= MINT ? 1 : MINT / P::T;
  static constexpr int G = G0 < NSEQ ? G0 : NSEQ;
  static constexpr int threads = G * P::T;
  static constexpr int RS = (P::padded * (int)sizeof(C) + 15) / 16 * 16 / (int)sizeof(C);
};

// Row pass: row i' of F1 (column-major) = first Kc bins of the real-to-complex FFT
// of row i' of fftshift(image), i.e. of image row (i' + N/2) mod N with its
// halves swapped, read as z_n = x_{2n} + i x_{2n+1} (M = N/2 points).
// TMA: persistent blocks own row groups blockIdx.x + k gridDim.x; thread 0
// keeps the next group in flight with bulk copies (the two half-row copies
// perform the fftshift) into a two-slot ring completed on one mbarrier per
// slot; each group is transformed in place (its slot and one work buffer).
// A wait that times out (never expected) sets bit 2 of *err, drains the
// copies still in flight (bounded) and ends the block.
// Otherwise (SWEEP, or an image that is not 16-byte aligned) each block loads
// or generates its rows directly.
// at most 128 registers per thread: four 128-thread blocks per SM
template <int THREADS> constexpr int min_blocks_128regs() {
  return THREADS >= 512 ? 1 : 512 / THREADS;
}

// BEAM: multiply the pixels by the primary-beam tables; the kernel is then
// launched as a programmatic dependent of beam_table_kernel and waits for it
// only before the first table read (its image copies are already in flight).
// MINT: least threads per block (rows per group G = MINT / threads per row,
// at least one): the row-group shape.  NSLOT: row groups in the bulk-copy
// ring (NSLOT - 1 stay in flight while one is transformed).  VR: values per
// thread, the radix of every stage but the last.
template <typename T, int LG, bool TMA, bool SWEEP, int K, bool BEAM = false, int MINT = 128,
          int NSLOT = 2, int VR = FftV<T>::V>
__global__ void __launch_bounds__(Shape3<T, (1 << LG), (2 << LG), MINT, VR>::threads,
                                  min_blocks_128regs<Shape3<T, (1 << LG), (2 << LG), MINT, VR>::threads>())
row_fft3_kernel(const __grid_constant__ Jobs<RowJob<T>, K> jobs, const cplx_t<T>* __restrict__ tw,
                int* __restrict__ err) {
  using C = cplx_t<T>;
  grid_dep_launch();  // the column pass may be scheduled as our blocks retire
  const RowJob<T>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  const T* __restrict__ image = jb.image;
  const T* __restrict__ I = jb.I;
  const SweepT<T>& sp = jb.sp;
  C* __restrict__ F1 = jb.F1;
  const double* __restrict__ rho2 = jb.rho2;
  const double S = jb.S;
  const T* __restrict__ beam = BEAM ? jb.beam : nullptr;
  constexpr int M = 1 << LG, N = 2 * M;
  using SH = Shape3<T, M, N, MINT, VR>;
  using P = typename SH::P;
  constexpr int V = SH::V, TT = P::T, G = SH::G, RS = SH::RS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  C* base = reinterpret_cast<C*>(smem_raw + 128);
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const Bounds bd = block_bounds(rho2, S, N);
  C tw1[V - 1];
  load_tw1<M, V, 2>(tw1, t, tw);
  const bool pruned = P::nstage >= 2 && bd.Kc <= P::Nsl;
  const bool one_j = bd.Kc <= TT;
  C twp[V];
  C wj = mkc((T)0, (T)0);
  if (pruned && one_j && t < bd.Kc) {
    load_twp<M, V, 2>(twp, t, tw);
    wj = __ldg(tw + t);
  }
  auto sync = [] { __syncthreads(); };
  // Transform the group held in registers v (stage-0 layout), A, B: buffers.
  auto transform = [&](C (&v)[V], C* A, C* B, int row) {
    Head3<M, V, 2, 0>::run(v, A, B, t, tw, tw1, sync);
    C* in = last_input<M, V>(A, B);
    C* out = F1 + row;  // column-major: bin j of this row at out[j N]
    if (pruned) {
      for (int j = t; j < bd.Kc; j += TT) {
        C zj, zmj;
        if (one_j) {
          pruned_pair3<M, V>(in, j, twp, zj, zmj);
          out[(size_t)j * N] = r2c_unpack(zj, zmj, wj);
        } else {
          C tj[V];
          load_twp<M, V, 2>(tj, j, tw);
          pruned_pair3<M, V>(in, j, tj, zj, zmj);
          out[(size_t)j * N] = r2c_unpack(zj, zmj, __ldg(tw + j));
        }
      }
    } else {
      last_full<M, V, 2>(v, in, t, tw);
      C* o = in == A ? B : A;
      store_full<M, V>(v, o, t);
      __syncthreads();
      // the G rows of the group are consecutive and all in shared memory
      // (row gg's buffer lies (gg - g) RS from ours): unpack bin by bin with
      // the G rows side by side, so each store fills G adjacent values of a
      // column instead of one value per sector
      const C* o0 = o - (size_t)g * RS;
      C* out0 = out - g;
      for (int q = threadIdx.x; q < bd.Kc * G; q += G * TT) {
        const int k = q / G, gg = q - k * G;
        const C* og = o0 + (size_t)gg * RS;
        out0[(size_t)k * N + gg] =
            r2c_unpack(og[pad3<V>(k & (M - 1))], og[pad3<V>((M - k) & (M - 1))], __ldg(tw + k));
      }
    }
  };
  if constexpr (TMA) {
    static_assert(NSLOT >= 2 && NSLOT <= 8, "ring of 2 to 8 slots");
    C* slot0 = base;
    C* work = base + NSLOT * G * RS;
    const int ngroups = N / G;
    const uint32_t half_bytes = (uint32_t)(M * sizeof(T));
    if (threadIdx.x == 0) {
      for (int k = 0; k < NSLOT; ++k) mbar_init(&bars[k], 1);
      mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int it) {  // thread 0 only
      const int grp = blockIdx.x + it * gridDim.x;
      if (grp >= ngroups) return;
      const int sl = it % NSLOT;
      mbar_arrive_expect_tx(&bars[sl], 2u * half_bytes * (uint32_t)G);
      for (int rl = 0; rl < G; ++rl) {
        const T* src = image + (size_t)(((grp * G + rl) + M) & (N - 1)) * N;
        T* dst = reinterpret_cast<T*>(slot0 + (size_t)(sl * G + rl) * RS);
        bulk_load(dst, src + M, half_bytes, &bars[sl]);
        bulk_load(dst + M, src, half_bytes, &bars[sl]);
      }
    };
    if (threadIdx.x == 0)
      for (int k = 0; k < NSLOT; ++k) issue(k);
    if constexpr (BEAM) grid_dep_wait();  // the beam tables
    for (int it = 0;; ++it) {
      const int grp = blockIdx.x + it * gridDim.x;
      if (grp >= ngroups) break;
      const int sl = it % NSLOT;
      const bool ok = mbar_wait(&bars[sl], (uint32_t)((it / NSLOT) & 1));
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicOr(err, 2);
          for (int k = it; k < it + NSLOT; ++k)
            if (blockIdx.x + k * gridDim.x < ngroups)
              mbar_wait(&bars[k % NSLOT], (uint32_t)((k / NSLOT) & 1));
        }
        return;
      }
      C* slot = slot0 + (size_t)(sl * G + g) * RS;
      C v[V];
#pragma unroll
      for (int r = 0; r < V; ++r) v[r] = slot[t + r * TT];
      if constexpr (BEAM) {
#pragma unroll
        for (int r = 0; r < V; ++r) v[r] = beam_pair(v[r], beam, N, grp * G + g, t + r * TT);
      }
      // stage 0 writes the work buffer; the slot is reused from stage 1 on,
      // after the barrier that ends stage 0
      transform(v, work + (size_t)g * RS, slot, grp * G + g);
      __syncthreads();  // every read of this slot is done
      if (threadIdx.x == 0) issue(it + NSLOT);
    }
  } else {
    C* A = base + (size_t)g * RS;
    C* B = base + (size_t)(G + g) * RS;
    const int row = blockIdx.x * G + g;
    const int irow = (row + M) & (N - 1);
    if constexpr (BEAM) grid_dep_wait();  // the beam tables
    C v[V];
#pragma unroll
    for (int r = 0; r < V; ++r) {
      const int n = t + r * TT;
      const int j = (2 * n + M) & (N - 1);
      if constexpr (SWEEP)
        v[r] = mkc(sweep_pixel(I, sp, N, irow, j), sweep_pixel(I, sp, N, irow, j + 1));
      else
        v[r] = *reinterpret_cast<const C*>(image + (size_t)irow * N + j);
      if constexpr (BEAM) v[r] = beam_pair(v[r], beam, N, row, n);
    }
    transform(v, A, B, row);
  }
}

// ---------------------------------------------------------------------------
// Row pass of the float 4096-wide image (M = 2048 complex points, stages
// 16 x 16 x 8), the shape of the large single-image evaluation.  Differences
// from row_fft3_kernel:
//  * rows are read with plain 8-byte loads straight into the stage-0
//    register layout, the next row in flight while this one is transformed
//    (the bulk-copy ring alone needs about as long as the whole pass);
//  * when the kept window has at most 64 columns, the pruned radix-8 last
//    stage runs in registers and warp shuffles: stage 1 gives thread
//    (k, blk) = (t >> 3, t & 7) the butterfly 16 blk + k, whose outputs are
//    Y[256 blk + k + 16 r']; the 8 lanes of one k hold every Y that the
//    outputs at in-block positions p = k (mod 16) need, and
//      X[p + 256 s] = sum_blk Y[p + 256 blk] W_2048^(blk p) W_8^(blk s)
//    is a sum over those 8 lanes (transpose-reduce: 7 complex shuffles per
//    lane).  Output slots: s = 0 for r' = 0..3 (X[j], j < 64) and s = 7 for
//    r' = 12..15 (X[2048 - j], j = 1..64).  The stage 0 -> 1 exchange goes
//    through an unpadded buffer with element 16 a + c at
//    16 a + ((c + 2a + (a >> 3)) & 15), free of bank conflicts for both the
//    stage-0 stores and the remapped stage-1 loads.
//  * otherwise (wider windows) each row takes row_fft3_kernel's transform.
// Every request of a launch (grid row y) takes the same branch for all its
// rows, and single calls and batches use this kernel alike, so their results
// stay bitwise equal.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int swz16(int a, int c) { return 16 * a + ((c + 2 * a + (a >> 3)) & 15); }

constexpr int kRowLdgLG = 11;      // the one transform length of row_fft3_ldg_kernel
constexpr int kRowLdgMaxKc = 64;   // widest window of its register last stage
constexpr int kRowLdgBlocks = 3;   // resident blocks per SM (168 registers each)

struct RowLdgShape {
  using P = P3<(1 << kRowLdgLG), 16>;
  static constexpr int M = 1 << kRowLdgLG, N = 2 * M, V = 16, TT = P::T;
  static constexpr int RS = (P::padded * 8 + 15) / 16 * 16 / 8;
  static constexpr int kZ = 2 * kRowLdgMaxKc + 1;  // Z[j] for j < 64, Z[M - j] for j = 1..64
  static constexpr size_t smem = (size_t)(2 * RS + kZ) * sizeof(float2);
};

template <int K, bool BEAM = false>
__global__ void __launch_bounds__(RowLdgShape::TT, kRowLdgBlocks)
row_fft3_ldg_kernel(const __grid_constant__ Jobs<RowJob<float>, K> jobs, const float2* __restrict__ tw) {
  using C = float2;
  using SH = RowLdgShape;
  using P = SH::P;
  constexpr int M = SH::M, N = SH::N, V = SH::V, TT = SH::TT, RS = SH::RS;
  static_assert(P::nstage == 3 && P::rlast == 8 && P::Nsl == 256 && TT == 128, "shape");
  grid_dep_launch();  // the column pass may be scheduled as our blocks retire
  const RowJob<float>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  const float* __restrict__ image = jb.image;
  const float* __restrict__ beam = BEAM ? jb.beam : nullptr;
  C* __restrict__ F1 = jb.F1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + RS;
  C* zlo = B + RS;                  // Z[j], j < 64
  C* zhi = zlo + kRowLdgMaxKc;      // Z[M - j] at index j, j = 1..64
  const int t = threadIdx.x;
  auto load_row = [&](C (&x)[V], int row) {
    // row `row` of fftshift(image): image row (row + N/2) mod N, halves
    // swapped: pixel pairs t + r TT of the shifted row are pairs M/2 + t + r TT
    // of the image row for r < V/2 and t + (r - V/2) TT after the wrap
    // (TT = M/8 pairs, so 2 (t + r TT) + M < N exactly when r < V/2)
    const C* src = reinterpret_cast<const C*>(image + (size_t)((row + M) & (N - 1)) * N) + t;
#pragma unroll
    for (int r = 0; r < V; ++r)
      x[r] = __ldcs(r < V / 2 ? src + M / 2 + r * TT : src + (r - V / 2) * TT);
  };
  // the first row is in flight while the bounds (one FP64 evaluation per
  // block) and the twiddles are read: this pass starts the evaluation, so
  // no earlier kernel hides its prologue
  int row = blockIdx.x;
  C v[V];
  if (row < N) load_row(v, row);
  // fast path: butterfly 16 blk + k of stage 1, twiddles of both stages
  // (read before the bounds are known; replaced below for wide windows)
  const int k = t >> 3, blk = t & 7;
  C tw1[V - 1];
  C twl[8];
#pragma unroll
  for (int r = 1; r < V; ++r) tw1[r - 1] = __ldg(tw + 16 * r * k);  // W_256^(r k)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int p = k + 16 * (i < 4 ? i : 8 + i);
    const int e = (blk * p + (i < 4 ? 0 : 256 * 7 * blk)) & (M - 1);
    twl[i] = __ldg(tw + 2 * e);  // W_2048^(blk p) W_8^(blk s)
  }
  const Bounds bd = block_bounds(jb.rho2, jb.S, N);
  const bool pruned = bd.Kc <= P::Nsl;
  const bool fast = bd.Kc <= kRowLdgMaxKc;  // uniform over the request
  C wj = mkc(0.f, 0.f);
  if (fast) {
    if (t < bd.Kc) wj = __ldg(tw + t);
  } else {
    load_tw1<M, V, 2>(tw1, t, tw);
  }
  C twp[V];
  if (!fast && pruned && t < bd.Kc) {
    load_twp<M, V, 2>(twp, t, tw);
    wj = __ldg(tw + t);
  }
  auto sync = [] { __syncthreads(); };
  if constexpr (BEAM) grid_dep_wait();  // the beam tables
  for (; row < N; row += gridDim.x) {
    const int nrow = row + gridDim.x;
    C nx[V];
    if (nrow < N) load_row(nx, nrow);
    if constexpr (BEAM) {
#pragma unroll
      for (int r = 0; r < V; ++r) v[r] = beam_pair(v[r], beam, N, row, t + r * TT);
    }
    C* out = F1 + row;  // column-major: bin j of this row at out[j N]
    if (fast) {
      // stage 0 (radix 16) into the swizzled buffer
      bflyR<V>(v);
#pragma unroll
      for (int r = 0; r < V; ++r) A[swz16(t, r)] = v[bfly_out<V>(r)];
      __syncthreads();
      // stage 1: butterfly b = 16 blk + k, inputs b + 128 r
#pragma unroll
      for (int r = 0; r < V; ++r) v[r] = A[swz16(blk + 8 * r, k)];
#pragma unroll
      for (int r = 1; r < V; ++r) v[r] = cmul(v[r], tw1[r - 1]);
      bflyR<V>(v);
      // last stage over the 8 lanes of this k
      C x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = cmul(v[bfly_out<V>(i < 4 ? i : 8 + i)], twl[i]);
      auto xs = [](C a, int m) {
        return mkc(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
      };
      const bool b2 = blk & 4, b1 = blk & 2, b0 = blk & 1;
      C y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] = cadd(b2 ? x[q + 4] : x[q], xs(b2 ? x[q] : x[q + 4], 4));
      C z2[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) z2[q] = cadd(b1 ? y[q + 2] : y[q], xs(b1 ? y[q] : y[q + 2], 2));
      const C zz = cadd(b0 ? z2[1] : z2[0], xs(b0 ? z2[0] : z2[1], 1));
      // lane blk now holds output slot blk
      if (blk < 4) zlo[k + 16 * blk] = zz;
      else zhi[256 - (k + 16 * (8 + blk))] = zz;
      __syncthreads();
      if (t < bd.Kc) {
        const C zj = zlo[t];
        out[(size_t)t * N] = r2c_unpack(zj, t == 0 ? zj : zhi[t], wj);
      }
    } else {
      Head3<M, V, 2, 0>::run(v, A, B, t, tw, tw1, sync);
      C* in = last_input<M, V>(A, B);
      if (pruned) {
        for (int j = t; j < bd.Kc; j += TT) {
          C zj, zmj;
          if (bd.Kc <= TT) {
            pruned_pair3<M, V>(in, j, twp, zj, zmj);
            out[(size_t)j * N] = r2c_unpack(zj, zmj, wj);
          } else {
            C tj[V];
            load_twp<M, V, 2>(tj, j, tw);
            pruned_pair3<M, V>(in, j, tj, zj, zmj);
            out[(size_t)j * N] = r2c_unpack(zj, zmj, __ldg(tw + j));
          }
        }
      } else {
        last_full<M, V, 2>(v, in, t, tw);
        C* o = in == A ? B : A;
        store_full<M, V>(v, o, t);
        __syncthreads();
        for (int q = t; q < bd.Kc; q += TT)
          out[(size_t)q * N] = r2c_unpack(o[pad3<V>(q & (M - 1))], o[pad3<V>((M - q) & (M - 1))], __ldg(tw + q));
      }
      __syncthreads();  // every read of A and B is done before the next row
    }
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = nx[r];
  }
}

// Column pass: for each kept column c < Kc (blocks loop over column groups),
// the complex FFT of length N down column c of F1 (contiguous); output row r
// of the v-shifted spectrum holds kv = (r + N/2) mod N, and rows r0 ..
// r0 + nrw - 1 are written to the window Gw (nrw x Kc).  When the window is
// pruned, only the kept frequencies +-j are evaluated.
// Blocks have at least 256 threads, so short columns come G >= 4 to a block:
// an unpruned window is then written a row at a time with the block's G
// adjacent columns side by side (whole 32-byte sectors, not one 8-byte value
// per sector).
template <typename T, int L, int VC = FftV<T>::V> using ColShape3 = Shape3<T, L, (1 << 30), 256, VC>;

// VC: values per thread, the radix of every stage but the last
template <typename T, int LG, int K, int VC = FftV<T>::V>
__global__ void __launch_bounds__(ColShape3<T, (1 << LG), VC>::threads)
col_fft3_kernel(const __grid_constant__ Jobs<ColJob<T>, K> jobs, const cplx_t<T>* __restrict__ tw) {
  const ColJob<T>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  const cplx_t<T>* __restrict__ F1 = jb.F1;
  cplx_t<T>* __restrict__ Gw = jb.Gw;
  const double* __restrict__ rho2 = jb.rho2;
  const double S = jb.S;
  grid_dep_launch();  // the gather may start its prologue on the SMs we leave idle
  using C = cplx_t<T>;
  constexpr int N = 1 << LG;
  using SH = ColShape3<T, N, VC>;
  using P = typename SH::P;
  constexpr int V = SH::V, TT = P::T, G = SH::G, RS = SH::RS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* base = reinterpret_cast<C*>(smem_raw);
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const Bounds bd = block_bounds(rho2, S, N);
  const int ncol = jb.full ? full_cols(bd, N).W : bd.Kc;  // window columns (and pitch)
  C tw1[V - 1];
  load_tw1<N, V, 1>(tw1, t, tw);
  const int kmax = N / 2 - bd.r0;
  const bool pruned = P::nstage >= 2 && bd.r0 > 0 && kmax < P::Nsl;
  const bool one_j = kmax < TT;
  C twp[V];
  if (pruned && one_j && t <= kmax) load_twp<N, V, 1>(twp, t, tw);
  C* A = base + (size_t)g * RS;
  C* B = base + (size_t)(G + g) * RS;
  auto sync = [] { __syncthreads(); };
  grid_dep_wait();  // F1 is the row pass's output
  for (int c0 = blockIdx.x * G; c0 < ncol; c0 += gridDim.x * G) {
    const int c = c0 + g;
    const bool act = c < ncol;
    C v[V];
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = act ? F1[(size_t)c * N + t + r * TT] : mkc((T)0, (T)0);
    Head3<N, V, 1, 0>::run(v, A, B, t, tw, tw1, sync);
    C* in = last_input<N, V>(A, B);
    if (pruned) {
      for (int j = t; j <= kmax; j += TT) {
        C xj, xmj;
        if (one_j) {
          pruned_pair3<N, V>(in, j, twp, xj, xmj);
        } else {
          C tj[V];
          load_twp<N, V, 1>(tj, j, tw);
          pruned_pair3<N, V>(in, j, tj, xj, xmj);
        }
        if (act) {
          Gw[(size_t)(kmax + j) * ncol + c] = xj;
          if (j > 0) Gw[(size_t)(kmax - j) * ncol + c] = xmj;
        }
      }
    } else {
      last_full<N, V, 1>(v, in, t, tw);
      C* o = in == A ? B : A;
      store_full<N, V>(v, o, t);
      __syncthreads();
      // every column of the group is in shared memory (group gg's output
      // buffer lies (gg - g) RS from ours): write row by row, G columns side by side
      const C* o0 = o - (size_t)g * RS;
      for (int q = threadIdx.x; q < bd.nrw * G; q += G * TT) {
        const int rr = q / G, gg = q - rr * G;
        if (c0 + gg < ncol)
          Gw[(size_t)rr * ncol + c0 + gg] = o0[(size_t)gg * RS + pad3<V>((bd.r0 + rr + N / 2) & (N - 1))];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Gather: per uv point, rotation (Sect. 3.2), grid index with Hermitian fold
// (App. D), bilinear interpolation clamped to the node range (Sect. 3.3),
// phase factor exp(+2 pi i (u dRA + v dDec)) (Sect. 3.2, App. D sign; the
// offset rotates with the uv points, and the dot product is rotation
// invariant, so the unrotated u, v are used).
//
// Clamping is done against the kept window.  When the window is pruned no
// point can reach its edge, and when it is not pruned it is the whole half
// spectrum, so window clamping is exactly the node-range clamping of App. D.
// ---------------------------------------------------------------------------
struct Window {
  int pitch;  // Kc nodes per row
  int cmax;   // last cell column, Kc - 2
  int rmax;   // last cell row, nrw - 2
  int rofs;   // N/2 - r0: window row of v = 0
  int cofs;   // window column of u = 0 (0 for the half spectrum)
  unsigned amax;  // node index of the last cell's first node, rmax * pitch + cmax
};
__device__ __forceinline__ Window make_window(const Bounds& b, int N) {
  Window w;
  w.pitch = b.Kc;
  w.cmax = b.Kc - 2;
  w.rmax = b.nrw - 2;
  w.rofs = N / 2 - b.r0;
  w.cofs = 0;
  w.amax = (unsigned)(w.rmax * w.pitch + w.cmax);
  return w;
}
// the full-plane window: both signs of u (full_cols), no fold
__device__ __forceinline__ Window make_window_full(const Bounds& b, int N) {
  const FullCols f = full_cols(b, N);
  Window w;
  w.pitch = f.W;
  w.cmax = f.W - 2;
  w.rmax = b.nrw - 2;
  w.rofs = N / 2 - b.r0;
  w.cofs = f.lo;
  w.amax = (unsigned)(w.rmax * w.pitch + w.cmax);
  return w;
}

template <typename T> struct GatherT;

// float path: A = cos(PA) N dxy and B = sin(PA) N dxy turn (u, v) into grid
// offsets x = u A - v B (along u') and y = u B + v A (along v'); PX, PY are
// dRA and dDec (turns per wavelength).  All four are float-float.
template <> struct GatherT<float> {
  ff A, B, PX, PY;
  // the same constants broadcast to both lanes of an f32x2 pair (read by the
  // two-point path straight from the kernel parameters)
  float2 Ah, Al, nAh, Bh, Bl, nBh, nBl, PXh, PXl, PYh, PYl, m1, twopi;
  double Sd;
  int N;
  __host__ static GatherT make(const GatherParams& g) {
    GatherT r;
    r.A = ff_split(g.cpa * g.S);
    r.B = ff_split(g.spa * g.S);
    r.PX = ff_split(g.phx);
    r.PY = ff_split(g.phy);
    auto b2 = [](float x) { return make_float2(x, x); };
    r.Ah = b2(r.A.hi);
    r.Al = b2(r.A.lo);
    r.nAh = b2(-r.A.hi);
    r.Bh = b2(r.B.hi);
    r.Bl = b2(r.B.lo);
    r.nBh = b2(-r.B.hi);
    r.nBl = b2(-r.B.lo);
    r.PXh = b2(r.PX.hi);
    r.PXl = b2(r.PX.lo);
    r.PYh = b2(r.PY.hi);
    r.PYl = b2(r.PY.lo);
    r.m1 = b2(-1.f);
    r.twopi = b2(6.28318530717958647692f);
    r.Sd = g.S;
    r.N = g.N;
    return r;
  }
};

template <typename T> struct RowJob {
  const T* image;       // nxy x nxy image (null when swept from I)
  const T* I;           // profile (SWEEP)
  SweepT<T> sp;
  cplx_t<T>* F1;        // row-pass output, column-major (Kc columns of N)
  const double* rho2;   // squared uv extent of the request's points
  double S;             // nxy * dxy
  const T* beam;        // primary-beam factors (beam_table_kernel), null: none
};
template <typename T> struct ColJob {
  const cplx_t<T>* F1;
  cplx_t<T>* Gw;        // window output, nrw x Kc (full plane: nrw x W)
  const double* rho2;
  double S;
  int full;             // 1: the full-plane window (full_cols(bd, N).W columns)
};

template <> struct GatherT<double> {
  double cpa, spa, S, phx, phy;
  double Sd;
  int N;
  __host__ static GatherT make(const GatherParams& g) {
    GatherT r;
    r.cpa = g.cpa;
    r.spa = g.spa;
    r.S = g.S;
    r.phx = g.phx;
    r.phy = g.phy;
    r.Sd = g.S;
    r.N = g.N;
    return r;
  }
};

template <typename T> struct GatherJob {
  const cplx_t<T>* Gw;
  GatherT<T> p;
  const double* rho2;
  const T *u, *v, *re, *im, *w;
  int64_t M;
  int vec;              // all point arrays 16-byte aligned
  cplx_t<T>* vis;       // sample mode output
  double* partials;     // chi2 mode: one slot per (virtual) block of the request
  unsigned* counter;    // chi2 mode: last-block-done counter (self-resetting)
  double* chi2_out;
  int vblocks = 0;      // batched launches: the request's virtual blocks (see gather_kernel)
};

// Offsets and amplitudes of the K copies of one model in a multi-source
// evaluation (end of Sect. 3.1): the sampled model visibility is multiplied by
// sum_k amp_k exp(+2 pi i (u dRA_k + v dDec_k)) instead of one phase factor.
constexpr int kMaxSources = 16;
template <typename T> struct MultiPhase;
template <> struct MultiPhase<float> {
  int K = 0;
  float2 PXh[kMaxSources], PXl[kMaxSources], PYh[kMaxSources], PYl[kMaxSources];  // broadcast
  float2 amp[kMaxSources];                                                      // broadcast
  float PXs[kMaxSources], PXsl[kMaxSources], PYs[kMaxSources], PYsl[kMaxSources];  // scalar
  float amps[kMaxSources];
  __host__ static MultiPhase make(int K, const double* dRA, const double* dDec, const double* a) {
    MultiPhase m;
    m.K = K;
    for (int k = 0; k < K; ++k) {
      const ff x = ff_split(dRA[k]), y = ff_split(dDec[k]);
      m.PXh[k] = make_float2(x.hi, x.hi);
      m.PXl[k] = make_float2(x.lo, x.lo);
      m.PYh[k] = make_float2(y.hi, y.hi);
      m.PYl[k] = make_float2(y.lo, y.lo);
      m.amp[k] = make_float2((float)a[k], (float)a[k]);
      m.PXs[k] = x.hi;
      m.PXsl[k] = x.lo;
      m.PYs[k] = y.hi;
      m.PYsl[k] = y.lo;
      m.amps[k] = (float)a[k];
    }
    return m;
  }
};
template <> struct MultiPhase<double> {
  int K = 0;
  double phx[kMaxSources], phy[kMaxSources], amp[kMaxSources];
  __host__ static MultiPhase make(int K, const double* dRA, const double* dDec, const double* a) {
    MultiPhase m;
    m.K = K;
    for (int k = 0; k < K; ++k) {
      m.phx[k] = dRA[k];
      m.phy[k] = dDec[k];
      m.amp[k] = a[k];
    }
    return m;
  }
};

// the gather's multi-source parameter: empty unless MULTI
template <typename T, bool MULTI> struct MultiArg {
  __device__ const MultiPhase<T>* get() const { return nullptr; }
};
template <typename T> struct MultiArg<T, true> {
  MultiPhase<T> m;
  __device__ const MultiPhase<T>* get() const { return &m; }
};

// a * b exactly as hi + lo (b float-float): hi = a b.hi rounded, lo = the rest
__device__ __forceinline__ float prod_hi_lo(float a, ff b, float& lo) {
  const float hi = a * b.hi;
  lo = fmaf(a, b.lo, fmaf(a, b.hi, -hi));
  return hi;
}

// a window node from global memory (read-only cache) or from shared memory
template <bool SMEM, typename C> __device__ __forceinline__ C ld_node(const C* p) {
  if constexpr (SMEM) return *p;
  else return __ldg(p);
}

// EDGE: clamp positions beyond the node range to the edge (App. D).  Needed
// only when the window is the whole half spectrum; for a pruned window no
// point can reach its edge, and the index clamps below only keep every read
// in bounds for non-finite input (whose result is NaN through the phase).
// phase of one offset (PX, PY float-float) in turns, reduced exactly to
// |f| <= 1/2: each product hi is reduced by its own nearest integer before the
// sum, then the low parts are added
__device__ __forceinline__ float phase_turns(float u, float v, ff PX, ff PY) {
  float pae, pbe;
  const float pa = prod_hi_lo(u, PX, pae), pb = prod_hi_lo(v, PY, pbe);
  float f = (pa - rintf(pa)) + (pb - rintf(pb));
  f += pae + pbe;
  return f - rintf(f);
}

template <bool SMEM, bool EDGE, bool MULTI = false, bool FULL = false>
__device__ __forceinline__ float2 sample_point(const cplx_t<float>* __restrict__ Gp, const Window& w,
                                               const GatherT<float>& p, float u, float v,
                                               const MultiPhase<float>* mp = nullptr) {
  float xae, xbe, yae, ybe;
  const float xa = prod_hi_lo(u, p.A, xae), xb = prod_hi_lo(v, p.B, xbe);
  const float ya = prod_hi_lo(u, p.B, yae), yb = prod_hi_lo(v, p.A, ybe);
  // x = (xa - xb) + errors, y = (ya + yb) + errors, each as hi + lo (TwoSum)
  float xh = xa - xb;
  float t = xh - xa;
  float xl = ((xa - (xh - t)) - (xb + t)) + (xae - xbe);
  float yh = ya + yb;
  t = yh - ya;
  float yl = ((ya - (yh - t)) + (yb - t)) + (yae + ybe);
  // Hermitian fold (half spectrum only): use (-u', -v') and conjugate.  The
  // sign is that of the whole position hi + lo (hi alone is 0 when the two
  // products cancel, with the position in lo).
  const bool neg = !FULL && xh + xl < 0.f;
  if (neg) {
    xh = -xh;
    xl = -xl;
    yh = -yh;
    yl = -yl;
  }
  // The cell of a position hi + lo is floor(hi + lo), taken from the sum
  // rounded down (exactly the floor of the exact sum; floor(hi) alone is one
  // cell off when lo carries the position across a node, and the bilinear
  // interpolant has a kink there).  The fraction (hi - cell) + lo is then
  // in [0, 1], with one rounding.  Every cell path computes both this way, so
  // the sampling and chi-square kernels agree bit for bit.
  const float cf = floorf(__fadd_rd(xh, xl)), rf = floorf(__fadd_rd(yh, yl));
  float fu = (xh - cf) + xl;
  float fv = (yh - rf) + yl;
  int c = FULL ? (int)fmaxf(fminf(cf, 32768.f), -32768.f) + w.cofs : (int)fminf(cf, 32768.f);
  int r = (int)fmaxf(fminf(rf, 32768.f), -32768.f) + w.rofs;
  if constexpr (EDGE) {
    if (FULL && c < 0) {
      c = 0;
      fu = 0.f;
    } else if (c > w.cmax) {
      c = w.cmax;
      fu = 1.f;
    }
    if (r < 0) {
      r = 0;
      fv = 0.f;
    } else if (r > w.rmax) {
      r = w.rmax;
      fv = 1.f;
    }
    c = max(c, 0);
  } else {
    c = min(max(c, 0), w.cmax);
    r = min(max(r, 0), w.rmax);
  }
  const float2* g = Gp + r * w.pitch + c;
  const float2 g00 = ld_node<SMEM>(g), g01 = ld_node<SMEM>(g + 1);
  const float2 g10 = ld_node<SMEM>(g + w.pitch), g11 = ld_node<SMEM>(g + w.pitch + 1);
  const float ar = fmaf(fu, g01.x - g00.x, g00.x), ai = fmaf(fu, g01.y - g00.y, g00.y);
  const float br = fmaf(fu, g11.x - g10.x, g10.x), bi = fmaf(fu, g11.y - g10.y, g10.y);
  const float Vr = fmaf(fv, br - ar, ar);
  float Vi = fmaf(fv, bi - ai, ai);
  if (neg) Vi = -Vi;
  float sn, cs;
  if constexpr (MULTI) {
    cs = 0.f;
    sn = 0.f;
    for (int k = 0; k < mp->K; ++k) {
      ff PX, PY;
      PX.hi = mp->PXs[k];
      PX.lo = mp->PXsl[k];
      PY.hi = mp->PYs[k];
      PY.lo = mp->PYsl[k];
      float sk, ck;
      __sincosf(6.28318530717958647692f * phase_turns(u, v, PX, PY), &sk, &ck);  // |arg| <= pi
      cs = fmaf(mp->amps[k], ck, cs);
      sn = fmaf(mp->amps[k], sk, sn);
    }
  } else {
    __sincosf(6.28318530717958647692f * phase_turns(u, v, p.PX, p.PY), &sn, &cs);  // |arg| <= pi
  }
  return make_float2(Vr * cs - Vi * sn, Vr * sn + Vi * cs);
}

// ---------------------------------------------------------------------------
// float path, two uv points per evaluation: every per-point FP32 operation
// runs as one packed f32x2 instruction (sm_100+: two FP32 results per issue
// slot), lane .x for the first point and .y for the second.  Subtractions
// are fma(a, -1, b), which is exact, so the error-free transformations keep
// their guarantees.  Same arithmetic as sample_point<float>.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a + b rounded towards minus infinity, both lanes
__device__ __forceinline__ float2 add2_rd(float2 a, float2 b) {
  auto pack = [](float2 f) {
    return ((unsigned long long)__float_as_uint(f.y) << 32) | __float_as_uint(f.x);
  };
  unsigned long long r;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack(a)), "l"(pack(b)));
  return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}

// Round to nearest integer on the FMA pipe: for |x| < 2^22, x + 1.5 2^23
// rounds x to an integer in the low mantissa bits.  rint_fma(x) is exact there;
// for larger |x| it returns a value within 1 of x that is exactly
// representable, so x - rint_fma(x) is still computed exactly (|.| <= 1).
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float rint_fma(float x) { return __fsub_rn(__fadd_rn(x, kMagic), kMagic); }
__device__ __forceinline__ float2 rint_fma2(float2 x) {
  return __fadd2_rn(__fadd2_rn(x, make_float2(kMagic, kMagic)), make_float2(-kMagic, -kMagic));
}
// floor(x) for |x| < 2^22, as float and int, without the XU pipe
__device__ __forceinline__ int floor_fma(float x, float& fl) {
  const float t = __fadd_rn(x, kMagic);
  int i = __float_as_int(t) - 0x4B400000;
  float r = __fsub_rn(t, kMagic);
  if (r > x) {
    r -= 1.f;
    i -= 1;
  }
  fl = r;
  return i;
}

using Pair2Const = GatherT<float>;  // the broadcast pairs live in the kernel parameters

// -a for both lanes, by flipping the sign bits (integer pipe): exactly the
// product by -1, which frees the FMA pipe the float-float steps load
__device__ __forceinline__ float2 neg2(float2 a) {
  return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                     __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
}

// x * c exactly as hi + lo for c = ch + cl: hi = x ch, lo = (x ch - hi) + x cl.
// (nch = -ch is no longer needed: -hi is hi with its sign flipped, which is
// x (-ch) exactly.)
__device__ __forceinline__ float2 prod2(float2 x, float2 ch, float2 nch, float2 cl, float2& lo) {
  (void)nch;
  const float2 hi = mul2(x, ch);
  lo = fma2(x, cl, fma2(x, ch, neg2(hi)));
  return hi;
}

// TwoSum of two pairs: a + b = s + e exactly
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2 m1, float2& e) {
  const float2 s = add2(a, b);
  const float2 bb = fma2(a, m1, s);   // s - a
  const float2 t = fma2(bb, m1, s);   // s - bb
  e = add2(fma2(t, m1, a), fma2(bb, m1, b));  // (a - t) + (b - bb)
  return s;
}

template <bool SMEM, bool EDGE, bool FULL = false>
__device__ __forceinline__ void cell_fetch(const float2* __restrict__ G, const Window& w, float xh,
                                           float xl, float yh, float yl, bool neg, float2& V) {
  // positions are grid offsets (|.| <= 8192), so the FMA-pipe floor applies;
  // non-finite input yields an arbitrary cell, clamped below, and NaN through
  // the phase
  // cell = floor(hi + lo) from the sum rounded down, fraction (hi - cell) +
  // lo, as in sample_point and cell_pair_pruned (same values, bit for bit)
  float cf, rf;
  int c = floor_fma(__fadd_rd(xh, xl), cf) + (FULL ? w.cofs : 0);
  int r = floor_fma(__fadd_rd(yh, yl), rf) + w.rofs;
  float fu = (xh - cf) + xl;
  float fv = (yh - rf) + yl;
  if constexpr (EDGE) {
    if (FULL && c < 0) {
      c = 0;
      fu = 0.f;
    } else if (c > w.cmax) {
      c = w.cmax;
      fu = 1.f;
    }
    if (r < 0) {
      r = 0;
      fv = 0.f;
    } else if (r > w.rmax) {
      r = w.rmax;
      fv = 1.f;
    }
    c = max(c, 0);
  } else {
    c = min(max(c, 0), w.cmax);
    r = min(max(r, 0), w.rmax);
  }
  const float2* g = G + r * w.pitch + c;
  const float2 g00 = ld_node<SMEM>(g), g01 = ld_node<SMEM>(g + 1);
  const float2 g10 = ld_node<SMEM>(g + w.pitch), g11 = ld_node<SMEM>(g + w.pitch + 1);
  const float2 m1 = pk(-1.f, -1.f);
  const float2 FU = pk(fu, fu), FV = pk(fv, fv);
  const float2 a = fma2(FU, fma2(g00, m1, g01), g00);
  const float2 b = fma2(FU, fma2(g10, m1, g11), g10);
  V = fma2(FV, fma2(a, m1, b), a);
  if (neg) V.y = -V.y;
}

// Both points' cells in a pruned window (no point can reach its edge), from
// the folded positions x = xh + xl, y = yh + yl (grid offsets, |.| < 2^22):
// the cell is floor(h + l), which is (h + l rounded down) + 1.5 2^23 rounded
// down (two adds per lane pair), whose low mantissa bits are the integer
// floor; the fraction (h - floor) is exact, plus the low part.  Non-finite input gives an arbitrary node
// index, clamped so every read stays in the window (its result is NaN
// through the phase).
template <bool SMEM, bool FULL = false>
__device__ __forceinline__ void cell_pair_pruned(const float2* __restrict__ G, const Window& w,
                                                 float2 xh, float2 xl, float2 yh, float2 yl,
                                                 float2 m1, float2& A0, float2& A1) {
  const float2 mg = make_float2(kMagic, kMagic), nmg = make_float2(-kMagic, -kMagic);
  // floor(hi + lo): the sum rounded down, then rounded down to an integer
  const float2 tx = add2_rd(add2_rd(xh, xl), mg), ty = add2_rd(add2_rd(yh, yl), mg);
  const float2 fu = add2(fma2(add2(tx, nmg), m1, xh), xl);
  const float2 fv = add2(fma2(add2(ty, nmg), m1, yh), yl);
  constexpr int kMagicBits = 0x4B400000;  // bit pattern of 1.5 2^23
  auto node = [&](float t_x, float t_y) {
    const int r = __float_as_int(t_y) - kMagicBits + w.rofs;
    const int c = __float_as_int(t_x) - kMagicBits + (FULL ? w.cofs : 0);
    return min((unsigned)(r * w.pitch + c), w.amax);
  };
  auto lerp = [&](unsigned a, float f_u, float f_v) {
    const float2* g = G + a;
    const float2 g00 = ld_node<SMEM>(g), g01 = ld_node<SMEM>(g + 1);
    const float2 g10 = ld_node<SMEM>(g + w.pitch), g11 = ld_node<SMEM>(g + w.pitch + 1);
    const float2 FU = pk(f_u, f_u), FV = pk(f_v, f_v);
    const float2 a0 = fma2(FU, fma2(g00, m1, g01), g00);
    const float2 b0 = fma2(FU, fma2(g10, m1, g11), g10);
    return fma2(FV, fma2(a0, m1, b0), a0);
  };
  A0 = lerp(node(tx.x, ty.x), fu.x, fv.x);
  A1 = lerp(node(tx.y, ty.y), fu.y, fv.y);
}

// phase of one offset for both lanes, in turns, reduced to |f| <= 1/2:
// (u dRA, v dDec) per lane, each reduced by its nearest integer, then summed
// with the low parts
__device__ __forceinline__ float2 phase_turns2(float2 U, float2 Vv, float2 PXh, float2 PXl,
                                               float2 PYh, float2 PYl, float2 m1) {
  const float2 pa = mul2(U, PXh), pb = mul2(Vv, PYh);
  const float2 pe1 = fma2(U, PXl, fma2(U, PXh, neg2(pa)));
  const float2 pe2 = fma2(Vv, PYl, fma2(Vv, PYh, neg2(pb)));
  const float2 ra = fma2(rint_fma2(pa), m1, pa);  // exact, |ra| <= 1
  const float2 rb = fma2(rint_fma2(pb), m1, pb);
  const float2 f = add2(add2(ra, rb), add2(pe1, pe2));
  return fma2(rint_fma2(f), m1, f);
}

template <bool SMEM, bool EDGE, bool MULTI = false, bool FULL = false>
__device__ __forceinline__ void sample_pair(const float2* __restrict__ G, const Window& w,
                                            const Pair2Const& k, float2 U, float2 Vv, float2& V0,
                                            float2& V1, const MultiPhase<float>* mp = nullptr) {
  // x = u A - v B, y = u B + v A, both lanes at once, as hi + lo
  float2 e1, e2, e3, e4, ex, ey;
  const float2 p1 = prod2(U, k.Ah, k.nAh, k.Al, e1);    //  u A
  const float2 p2 = prod2(Vv, k.nBh, k.Bh, k.nBl, e2);  // -v B
  const float2 xh2 = two_sum2(p1, p2, k.m1, ex);
  const float2 xl2 = add2(ex, add2(e1, e2));
  const float2 p3 = prod2(U, k.Bh, k.nBh, k.Bl, e3);    //  u B
  const float2 p4 = prod2(Vv, k.Ah, k.nAh, k.Al, e4);   //  v A
  const float2 yh2 = two_sum2(p3, p4, k.m1, ey);
  const float2 yl2 = add2(ey, add2(e3, e4));
  // phase factor c + i s per lane: one offset, or the amplitude-weighted sum
  // over the copies of a multi-source model
  float s0, c0, s1, c1;
  if constexpr (MULTI) {
    float2 C = pk(0.f, 0.f), S = pk(0.f, 0.f);
    for (int j = 0; j < mp->K; ++j) {
      const float2 ang = mul2(phase_turns2(U, Vv, mp->PXh[j], mp->PXl[j], mp->PYh[j],
                                           mp->PYl[j], k.m1),
                              k.twopi);  // |angle| <= pi
      float sa, ca, sb, cb;
      __sincosf(ang.x, &sa, &ca);
      __sincosf(ang.y, &sb, &cb);
      C = fma2(mp->amp[j], pk(ca, cb), C);
      S = fma2(mp->amp[j], pk(sa, sb), S);
    }
    c0 = C.x;
    c1 = C.y;
    s0 = S.x;
    s1 = S.y;
  } else {
    const float2 ang = mul2(phase_turns2(U, Vv, k.PXh, k.PXl, k.PYh, k.PYl, k.m1),
                            k.twopi);  // |angle| <= pi
    __sincosf(ang.x, &s0, &c0);
    __sincosf(ang.y, &s1, &c1);
  }
  float2 A0, A1;
  if constexpr (FULL) {  // full plane: both signs of u are in the window
    if constexpr (EDGE) {
      cell_fetch<SMEM, EDGE, true>(G, w, xh2.x, xl2.x, yh2.x, yl2.x, false, A0);
      cell_fetch<SMEM, EDGE, true>(G, w, xh2.y, xl2.y, yh2.y, yl2.y, false, A1);
    } else {
      cell_pair_pruned<SMEM, true>(G, w, xh2, xl2, yh2, yl2, k.m1, A0, A1);
    }
  } else {
    // Hermitian fold per lane, on the sign of the whole position hi + lo
    const float2 xs = add2(xh2, xl2);
    const bool n0 = xs.x < 0.f, n1 = xs.y < 0.f;
    // the fold negates by flipping sign bits (integer pipe), which is what a
    // product by -1 does to every value, NaN and zeros included
    const unsigned f0 = n0 ? 0x80000000u : 0u, f1 = n1 ? 0x80000000u : 0u;
    auto flip = [&](float2 a) {
      return make_float2(__uint_as_float(__float_as_uint(a.x) ^ f0),
                         __uint_as_float(__float_as_uint(a.y) ^ f1));
    };
    const float2 xh = flip(xh2), xl = flip(xl2), yh = flip(yh2), yl = flip(yl2);
    if constexpr (EDGE) {
      cell_fetch<SMEM, EDGE>(G, w, xh.x, xl.x, yh.x, yl.x, n0, A0);
      cell_fetch<SMEM, EDGE>(G, w, xh.y, xl.y, yh.y, yl.y, n1, A1);
    } else {
      cell_pair_pruned<SMEM>(G, w, xh, xl, yh, yl, k.m1, A0, A1);
      if (n0) A0.y = -A0.y;
      if (n1) A1.y = -A1.y;
    }
  }
  // rotate by the phase: V (c + i s) = c V + s (-Vi, Vr)
  V0 = fma2(pk(s0, s0), pk(-A0.y, A0.x), mul2(pk(c0, c0), A0));
  V1 = fma2(pk(s1, s1), pk(-A1.y, A1.x), mul2(pk(c1, c1), A1));
}

// cell of the position ofs + x (x relative to the window's origin row or
// column ofs), clamped to the window's node range [0, last + 1].  The floor
// is taken of x itself so the result does not depend on the window's size.
__device__ __forceinline__ void cell_d(double x, int ofs, int last, int& c, double& f) {
  double fl = floor(x);
  f = x - fl;
  fl = fmin(fmax(fl, -1.0e9), 1.0e9);
  c = (int)fl + ofs;
  if (c < 0) {
    c = 0;
    f = 0.0;
  } else if (c > last) {
    c = last;
    f = 1.0;
  }
}

template <bool SMEM, bool EDGE, bool MULTI = false, bool FULL = false>
__device__ __forceinline__ double2 sample_point(const cplx_t<double>* __restrict__ Gp, const Window& w,
                                                const GatherT<double>& p, double u, double v,
                                                const MultiPhase<double>* mp = nullptr) {
  if (!(isfinite(u) && isfinite(v)))
    return make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
  double up = u * p.cpa - v * p.spa;
  double vp = u * p.spa + v * p.cpa;
  const bool neg = !FULL && up < 0.0;  // Hermitian fold (half spectrum only)
  if (neg) {
    up = -up;
    vp = -vp;
  }
  int r, c;
  double fr, fc;
  cell_d(vp * p.S, w.rofs, w.rmax, r, fr);
  cell_d(up * p.S, FULL ? w.cofs : 0, w.cmax, c, fc);
  const double2* g = Gp + (size_t)r * w.pitch + c;
  const double2 g00 = ld_node<SMEM>(g), g01 = ld_node<SMEM>(g + 1);
  const double2 g10 = ld_node<SMEM>(g + w.pitch), g11 = ld_node<SMEM>(g + w.pitch + 1);
  double2 V = clerp(clerp(g00, g01, fc), clerp(g10, g11, fc), fr);
  if (neg) V.y = -V.y;
  double sn, cs;
  if constexpr (MULTI) {
    cs = 0.0;
    sn = 0.0;
    for (int k = 0; k < mp->K; ++k) {
      const double ph = u * mp->phx[k] + v * mp->phy[k];
      double sk, ck;
      sincospi(2.0 * (ph - rint(ph)), &sk, &ck);
      cs = fma(mp->amp[k], ck, cs);
      sn = fma(mp->amp[k], sk, sn);
    }
  } else {
    const double ph = u * p.phx + v * p.phy;
    const double fph = ph - rint(ph);
    sincospi(2.0 * fph, &sn, &cs);
  }
  return cmul(V, make_double2(cs, sn));
}

// per-thread compensated accumulators
// block-wide sum of one double per thread, fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double x, double* ws);

struct AccF {  // Kahan: s holds the sum, c the negated lost low-order part
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  // Block total (valid in thread 0): a float-float tree inside each warp and
  // across the warps, converted to FP64 once.  GB300 issues FP64 at a small
  // fraction of the FP32 rate, and a dependent FP64 tree across 16 warps
  // added about 1 us to the end of every block; the float-float sums carry
  // about 48 significant bits.  The sum over blocks stays FP64.
  __device__ __forceinline__ double block_total(double* ws) const {
    auto warp_tree = [](ff a) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ff b;
        b.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        a = ff_add(a, b);
      }
      return a;
    };
    ff a;
    a.hi = s;
    a.lo = -c;
    a = warp_tree(a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2* wf = reinterpret_cast<float2*>(ws);  // 32 doubles hold 32 float pairs
    __syncthreads();
    if (lane == 0) wf[warp] = make_float2(a.hi, a.lo);
    __syncthreads();
    double x = 0.0;
    if (warp == 0) {
      const float2 w = lane < (int)(blockDim.x >> 5) ? wf[lane] : make_float2(0.f, 0.f);
      a.hi = w.x;
      a.lo = w.y;
      a = warp_tree(a);
      x = (double)a.hi + (double)a.lo;
    }
    return x;
  }
};
struct AccD {  // Neumaier
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
  __device__ __forceinline__ double block_total(double* ws) const { return block_sum(value(), ws); }
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

// SMEM: the block first copies the kept window (nrw x Kc nodes) into shared
// memory and gathers from there; the random 4-node reads then cost shared
// memory bank cycles instead of one L1 tag lookup per distinct line.  The
// launch provides `smem_nodes` nodes of dynamic shared memory; a window that
// does not fit (never, when the host sized it from the same extent) is read
// from global memory instead.

// Loop over this thread's uv points, reading the window nodes through G
// (SMEM: G points into shared memory).
// The W points of one group: u, v and (chi-square mode) Re, Im, w.
template <typename T, bool CHI2> struct PointGroup {
  T uu[Vec16<T>::W], vv[Vec16<T>::W], rr[Vec16<T>::W], ii[Vec16<T>::W], ww[Vec16<T>::W];
  __device__ __forceinline__ void load(const T* __restrict__ u, const T* __restrict__ v,
                                       const T* __restrict__ re, const T* __restrict__ im,
                                       const T* __restrict__ w, int64_t q) {
    load16(u, q, uu);
    load16(v, q, vv);
    if constexpr (CHI2) {
      load16(re, q, rr);
      load16(im, q, ii);
      load16(w, q, ww);
    }
  }
};

// Grid-stride layout of the vector groups: whole rounds of gstride groups,
// then the remainder in equal contiguous slices, one per block (coalesced,
// and no few blocks run a round more than the rest).
// nblk blocks, this thread in block bid.
struct GroupSplit {
  int64_t nq, gstride, rounds, slice, rem_q, gtid;
  __device__ __forceinline__ GroupSplit(int64_t M, int W, int vec, int nblk, int bid) {
    nq = vec ? M / W : 0;
    gstride = (int64_t)nblk * blockDim.x;
    rounds = nq / gstride;
    const int64_t rem = nq - rounds * gstride;
    slice = (rem + nblk - 1) / nblk;  // <= blockDim.x
    rem_q = rounds * gstride + (int64_t)bid * slice + threadIdx.x;
    gtid = (int64_t)bid * blockDim.x + threadIdx.x;
  }
  __device__ __forceinline__ bool has_rem() const { return threadIdx.x < slice && rem_q < nq; }
};

// pre: this thread's first group (its grid index), already loaded by the
// caller when the grid has at least one whole round; null otherwise.
template <typename T, bool CHI2, bool SMEM, bool EDGE, bool MULTI, bool FULL, typename ACC>
__device__ __forceinline__ void gather_points(const cplx_t<T>* __restrict__ G, const Window& win,
                                              const GatherT<T>& p, const T* __restrict__ u,
                                              const T* __restrict__ v, const T* __restrict__ re,
                                              const T* __restrict__ im, const T* __restrict__ w,
                                              int64_t M, int vec, cplx_t<T>* __restrict__ vis,
                                              ACC& acc, const MultiPhase<T>* mp,
                                              const PointGroup<T, CHI2>* pre, const GroupSplit& sp) {
  using C = cplx_t<T>;
  constexpr int W = Vec16<T>::W;
  auto point = [&](T uu, T vv) {
    return sample_point<SMEM, EDGE, MULTI, FULL>(G, win, p, uu, vv, mp);
  };
  const int64_t gtid = sp.gtid;
  auto compute = [&](const PointGroup<T, CHI2>& g, int64_t q) {  // the W points of group q
    const T(&uu)[W] = g.uu;
    const T(&vv)[W] = g.vv;
    const T(&rr)[W] = g.rr;
    const T(&ii)[W] = g.ii;
    const T(&ww)[W] = g.ww;
    C Vs[W];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int e = 0; e < W; e += 2)
        sample_pair<SMEM, EDGE, MULTI, FULL>(G, win, p, pk(uu[e], uu[e + 1]), pk(vv[e], vv[e + 1]),
                                       Vs[e], Vs[e + 1], mp);
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) Vs[e] = point(uu[e], vv[e]);
    }
    if constexpr (CHI2) {
      T part = (T)0;
#pragma unroll
      for (int e = 0; e < W; ++e) {
        const T dr = rr[e] - Vs[e].x, di = ii[e] - Vs[e].y;
        part += ww[e] * (dr * dr + di * di);
      }
      acc.add(part);
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) vis[q * W + e] = Vs[e];
    }
  };
  auto group = [&](int64_t q) {
    PointGroup<T, CHI2> g;
    g.load(u, v, re, im, w, q);
    compute(g, q);
  };
  int64_t q = gtid;
  int64_t r = 0;
  if (pre) {
    compute(*pre, q);
    q += sp.gstride;
    r = 1;
  }
  for (; r < sp.rounds; ++r, q += sp.gstride) group(q);
  if (sp.has_rem()) group(sp.rem_q);
  for (int64_t k = sp.nq * W + gtid; k < M; k += sp.gstride) {
    const C V = point(u[k], v[k]);
    if constexpr (CHI2) {
      const T dr = re[k] - V.x, di = im[k] - V.y;
      acc.add(w[k] * (dr * dr + di * di));
    } else {
      vis[k] = V;
    }
  }
}

// block shape: 512-thread blocks, two per SM, when the window is staged in
// shared memory (each block its own copy, so one block's window copy and
// final reduction overlap the other's stream), 256-thread blocks otherwise.
// The full-plane window is about twice as large, so only one copy fits per
// SM: one 1024-thread block then keeps the same 32 warps resident.
template <bool SMEM, bool FULL = false> constexpr int gather_threads() {
  return SMEM ? (FULL ? 1024 : 512) : 256;
}
template <bool SMEM, bool FULL> constexpr int gather_min_blocks() { return SMEM ? (FULL ? 1 : 2) : 4; }

template <typename T, bool CHI2, bool SMEM, bool EDGE, int K, bool MULTI = false, bool FULL = false>
__global__ void __launch_bounds__(gather_threads<SMEM, FULL>(), gather_min_blocks<SMEM, FULL>())
gather_kernel(const __grid_constant__ Jobs<GatherJob<T>, K> jobs, int smem_nodes,
              const __grid_constant__ MultiArg<T, MULTI> multi) {
  using C = cplx_t<T>;
  const MultiPhase<T>* mp = multi.get();
  const GatherJob<T>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  const C* __restrict__ Gw = jb.Gw;
  const GatherT<T>& p = jb.p;
  const double* __restrict__ rho2 = jb.rho2;
  const T* __restrict__ u = jb.u;
  const T* __restrict__ v = jb.v;
  const T* __restrict__ re = jb.re;
  const T* __restrict__ im = jb.im;
  const T* __restrict__ w = jb.w;
  const int64_t M = jb.M;
  const int vec = jb.vec;
  C* __restrict__ vis = jb.vis;
  double* __restrict__ partials = jb.partials;
  unsigned* __restrict__ counter = jb.counter;
  double* __restrict__ chi2_out = jb.chi2_out;
  const Bounds bd = block_bounds(rho2, p.Sd, p.N);
  const Window win = FULL ? make_window_full(bd, p.N) : make_window(bd, p.N);
  // Virtual blocks: a batched launch may run fewer blocks than the request
  // has partial sums (nvb).  Block b then evaluates virtual blocks b,
  // b + gridDim.x, ... in turn, each exactly as block vb of a single call
  // (same points in the same order, same partial sum), so batched and single
  // results agree bit for bit while each block copies the window only once.
  const int nvb = K == 1 ? (int)gridDim.x : jb.vblocks;
  // The observation does not depend on the column pass: while that pass
  // finishes, load this thread's first group into registers (when the grid
  // has a whole round) and pull its remainder group, if any, towards L2.
  // (Single calls only: batched launches are not dependents.)
  constexpr int W = Vec16<T>::W;
  const GroupSplit gs(M, W, vec, nvb, blockIdx.x);
  PointGroup<T, CHI2> g0;
  const bool pre = K == 1 && gs.rounds > 0;  // uniform over the grid
  if constexpr (K == 1) {
    if (pre) g0.load(u, v, re, im, w, gs.gtid);
    if (gs.has_rem()) {
      const int64_t o = gs.rem_q * W;
      prefetch_l2(u + o);
      prefetch_l2(v + o);
      if constexpr (CHI2) {
        prefetch_l2(re + o);
        prefetch_l2(im + o);
        prefetch_l2(w + o);
      }
    }
  }
  grid_dep_wait();  // the window is the column pass's output
  C* sw = nullptr;
  bool win_ok = true;
  if constexpr (SMEM) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    sw = reinterpret_cast<C*>(smem_raw);
    const int nodes = bd.nrw * win.pitch;
    // the host sizes the shared window from the same extent, so this always
    // holds; otherwise the result is NaN rather than a read out of bounds
    win_ok = nodes <= smem_nodes;  // uniform over the grid
    if (win_ok) {
      // one bulk copy of the window (rounded up to 16 bytes; the window
      // buffer and the shared allocation both have the slack)
      __shared__ __align__(8) uint64_t wbar;
      const uint32_t bytes = ((uint32_t)(nodes * sizeof(C)) + 15u) & ~15u;
      if (threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        mbar_init_fence();
        mbar_arrive_expect_tx(&wbar, bytes);
        bulk_load(sw, Gw, bytes, &wbar);
      }
      __syncthreads();
      const bool ok = mbar_wait(&wbar, 0);
      if (__syncthreads_or(!ok)) {  // never expected: fall back to plain loads
        for (int i = threadIdx.x; i < nodes; i += blockDim.x) sw[i] = __ldg(Gw + i);
        __syncthreads();
      }
    }
  }
  __shared__ double ws[32];
  auto run = [&](int vb, const GroupSplit& sp, const PointGroup<T, CHI2>* g0p) {
    typename Acc<T>::type acc;
    if constexpr (SMEM) {
      if (win_ok) {
        gather_points<T, CHI2, true, EDGE, MULTI, FULL>(sw, win, p, u, v, re, im, w, M, vec, vis,
                                                        acc, mp, g0p, sp);
      } else {
        const T nan = std::numeric_limits<T>::quiet_NaN();
        if constexpr (CHI2) {
          acc.add(nan);
        } else {
          for (int64_t k = sp.gtid; k < M; k += sp.gstride) vis[k] = mkc(nan, nan);
        }
      }
    } else {
      gather_points<T, CHI2, false, EDGE, MULTI, FULL>(Gw, win, p, u, v, re, im, w, M, vec, vis,
                                                       acc, mp, g0p, sp);
    }
    if constexpr (CHI2) {
      const double bs = acc.block_total(ws);
      if (threadIdx.x == 0) partials[vb] = bs;
    }
  };
  if constexpr (K == 1) {
    run(blockIdx.x, gs, pre ? &g0 : nullptr);
  } else {
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) run(vb, GroupSplit(M, W, vec, nvb, vb), nullptr);
  }
  if constexpr (CHI2) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(counter, 1u);
      last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      // fixed order: thread i compensates partials i, i + blockDim.x, ...
      // (a single value is taken as it is, the same sum without FP64 work)
      double x;
      if (nvb <= (int)blockDim.x) {
        x = threadIdx.x < nvb ? __ldcg(partials + threadIdx.x) : 0.0;
      } else {
        AccD a;
        for (int b = threadIdx.x; b < nvb; b += blockDim.x) a.add(__ldcg(partials + b));
        x = a.value();
      }
      const double tot = block_sum(x, ws);
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

// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on
// the current device (the attribute is per device; set once per size).  The
// cache is atomic: the server's scheduler thread and callers' threads launch
// the same kernels on their own contexts.
template <auto Kern> cudaError_t ensure_smem_attr(size_t smem) {
  constexpr int kDev = 64;
  static std::atomic<size_t> done[kDev] = {};
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev >= 0 && dev < kDev && done[dev].load(std::memory_order_relaxed) >= smem)
    return cudaSuccess;
  e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < kDev) {
    size_t have = done[dev].load(std::memory_order_relaxed);
    while (have < smem && !done[dev].compare_exchange_weak(have, smem)) {
    }
  }
  return e;
}

// Launch `kern` as a programmatic dependent of the preceding kernel in `st`:
// it may be scheduled while that kernel finishes, and waits for it in
// grid_dep_wait() before reading what it wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
namespace gal {

constexpr int kMaxDynSmem = 224 * 1024;  // leaves room for the kernels' static shared memory
constexpr int kMaxWindowSmem = 200 * 1024;

inline int row_threads_per_row(int N) { return N / 2 >= 8 ? N / 16 : 1; }

// multiprocessor count of the current device (cached per device; atomic for
// the same reason as ensure_smem_attr)
inline int current_device_sms() {
  static std::atomic<int> cache[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 1;
  int c = cache[d].load(std::memory_order_relaxed);
  if (!c) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    c = n > 0 ? n : 1;
    cache[d].store(c, std::memory_order_relaxed);
  }
  return c;
}
inline int col_threads_per_col(int N) { return N >= 8 ? N / 8 : 1; }

template <typename T> cudaError_t Launch<T>::init() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(row_pass_kernel<T, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(row_pass_kernel<T, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)))
    return e;
  // the gather also holds a little static shared memory (reduction scratch),
  // so its dynamic budget stays below the per-block total
  if ((e = cudaFuncSetAttribute(gather_kernel<T, true, true, true, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxWindowSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(gather_kernel<T, true, true, false, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxWindowSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(gather_kernel<T, false, true, true, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxWindowSmem)))
    return e;
  if ((e = cudaFuncSetAttribute(gather_kernel<T, false, true, false, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxWindowSmem)))
    return e;
  return cudaFuncSetAttribute(col_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kMaxDynSmem);
}

template <typename T> int Launch<T>::gather_blocks_per_sm(bool chi2, size_t window_smem) {
  int n = 0;
  if (window_smem) {
    if (chi2)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, true, true, true, 1>,
                                                    gather_threads<true>(), window_smem);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, false, true, true, 1>,
                                                    gather_threads<true>(), window_smem);
  } else {
    if (chi2)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, true, false, true, 1>, 256, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather_kernel<T, false, false, true, 1>, 256, 0);
  }
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
cudaError_t Launch<T>::uv_from_frequency(const T* u_m, const T* v_m, const T* nu, int64_t M, T* u,
                                         T* v, int blocks, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const int64_t need = (M + 255) / 256;
  const int grid = (int)(need < blocks ? need : blocks);
  uv_from_frequency_kernel<T><<<grid, 256, 0, st>>>(u_m, v_m, nu, M, u, v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::uv_range(const T* u, const T* v, int64_t M, double* range2, int blocks,
                                cudaStream_t st) {
  const double init[2] = {std::numeric_limits<double>::infinity(), 0.0};
  cudaError_t e = cudaMemcpyAsync(range2, init, sizeof init, cudaMemcpyHostToDevice, st);
  if (e) return e;
  if (M <= 0) return cudaSuccess;
  const int64_t need = (M + 255) / 256;
  const int grid = (int)(need < blocks ? need : blocks);
  uv_range_kernel<T><<<grid, 256, 0, st>>>(u, v, M, range2);
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
                                const void* tw, void* F1, const double* rho2, double S, int* err,
                                const T* beam, cudaStream_t st, int radix) {
  using C = cplx_t<T>;
  const int M = N / 2;
  const bool al16 = I || (reinterpret_cast<uintptr_t>(image) & 15u) == 0;
  if (M >= FftV<T>::V && al16) {
    const cudaError_t e = row_fft3<T>(image, I, sp, N, tw, F1, rho2, S, err, beam, st, radix);
    if (e != cudaErrorNotSupported) return e;
  }
  const C* twc = static_cast<const C*>(tw);
  C* out = static_cast<C*>(F1);
  const int tg = row_threads_per_row(N);
  int rpb = 256 / tg;
  if (rpb < 1) rpb = 1;
  if (rpb > N) rpb = N;
  const int threads = tg * rpb;
  const size_t smem = (size_t)rpb * M * sizeof(C);
  const int grid = (N + rpb - 1) / rpb;
  if (I)
    row_pass_kernel<T, true><<<grid, threads, smem, st>>>(nullptr, I, sweep_cast<T>(sp), N, twc,
                                                           out, rho2, S, beam);
  else
    row_pass_kernel<T, false><<<grid, threads, smem, st>>>(image, nullptr, SweepT<T>{}, N, twc,
                                                            out, rho2, S, beam);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::beam_table(T* tab, int N, double dxy, double fwhm, double dRA, double dDec,
                                  double PA, cudaStream_t st) {
  const BeamParams b = beam_params(fwhm, dRA, dDec, PA);
  // small blocks spread the 2N FP64 exponentials over many SMs: the FP64
  // pipe of one SM, not the launch, bounds this kernel
  beam_table_kernel<T><<<(2 * N + 63) / 64, 64, 0, st>>>(tab, N, dxy, b.c, b.bx, b.by);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::col_pass(const void* F1, void* Gw, int N, const void* tw,
                                const double* rho2, double S, int kc_hint, bool full,
                                cudaStream_t st, int radix) {
  using C = cplx_t<T>;
  if (N >= FftV<T>::V) {
    const cudaError_t e = col_fft3<T>(F1, Gw, N, tw, rho2, S, kc_hint, full, st, radix);
    if (e != cudaErrorNotSupported) return e;
  }
  if (full) return cudaErrorNotSupported;  // the generic pass keeps the half plane only
  const int P = N / 2 + 1;
  const int tg = col_threads_per_col(N);
  int cpb = 256 / tg;
  if (cpb < 1) cpb = 1;
  if (cpb > P) cpb = P;
  const int threads = tg * cpb;
  const size_t smem = (size_t)cpb * (N + 1) * sizeof(C);
  int grid = (P + cpb - 1) / cpb;
  const int cap = 2 * current_device_sms();
  if (grid > cap) grid = cap;
  col_pass_kernel<T><<<grid, threads, smem, st>>>(static_cast<const C*>(F1), static_cast<C*>(Gw),
                                                  N, static_cast<const C*>(tw), rho2, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::gather(const void* Gw, const GatherParams& gp, const double* rho2,
                              const T* u, const T* v, const T* re, const T* im, const T* w,
                              int64_t M, void* vis, double* partials, unsigned* counter,
                              double* chi2, size_t window_smem, bool edge, int blocks,
                              const MultiSources* ms, cudaStream_t st) {
  using C = cplx_t<T>;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  int vec = al16(u) && al16(v);
  if (chi2) vec = vec && al16(re) && al16(im) && al16(w);
  const GatherT<T> p = GatherT<T>::make(gp);
  const C* g = static_cast<const C*>(Gw);
  const int nodes = (int)(window_smem / sizeof(C));
  const int threads = window_smem ? gather_threads<true>() : gather_threads<false>();
  int grid = blocks;
  if (!chi2) {
    int64_t need = (M + threads - 1) / threads;
    if (need < 1) need = 1;
    if (need < grid) grid = (int)need;
  }
  Jobs<GatherJob<T>, 1> jb;
  jb.j[0] = GatherJob<T>{g, p, rho2, u, v, re, im, w, M, vec, static_cast<C*>(vis), partials,
                         counter, chi2};
  cudaError_t le = cudaSuccess;
  auto pick = [&](auto chi2_c, auto smem_c, auto edge_c) {
    constexpr bool CH = decltype(chi2_c)::value, SM = decltype(smem_c)::value,
                   ED = decltype(edge_c)::value;
    const size_t smem = SM ? window_smem : 0;
    if (ms && ms->K > 0) {
      constexpr auto kern = gather_kernel<T, CH, SM, ED, 1, true>;
      le = ensure_smem_attr<kern>(smem);
      MultiArg<T, true> ma;
      ma.m = MultiPhase<T>::make(ms->K, ms->dRA, ms->dDec, ms->amp);
      if (le == cudaSuccess)
        le = launch_dependent(kern, dim3(grid), dim3(threads), smem, st, jb, nodes, ma);
    } else {
      constexpr auto kern = gather_kernel<T, CH, SM, ED, 1, false>;
      le = ensure_smem_attr<kern>(smem);
      if (le == cudaSuccess)
        le = launch_dependent(kern, dim3(grid), dim3(threads), smem, st, jb, nodes,
                              MultiArg<T, false>{});
    }
  };
  using TT = std::true_type;
  using FF = std::false_type;
  if (chi2) {
    if (window_smem) edge ? pick(TT{}, TT{}, TT{}) : pick(TT{}, TT{}, FF{});
    else edge ? pick(TT{}, FF{}, TT{}) : pick(TT{}, FF{}, FF{});
  } else {
    if (window_smem) edge ? pick(FF{}, TT{}, TT{}) : pick(FF{}, TT{}, FF{});
    else edge ? pick(FF{}, FF{}, TT{}) : pick(FF{}, FF{}, FF{});
  }
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

}  // namespace gal
