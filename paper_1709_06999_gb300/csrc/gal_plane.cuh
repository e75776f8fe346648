// Full-plane (complex-to-complex) spectrum path: the row pass transforms each
// real image row as a complex sequence of length N, keeps both signs of u,
// and the gather samples the window without the Hermitian fold.  The paper
// checks this transform against the real-to-complex one (Sect. 5); here it is
// an alternative spectrum path with its own kernels, and the primary-beam
// factor (Sect. 2.1) applies to it as to the half-plane path.
#pragma once

#include "gal_fft3_launch.cuh"

namespace gal {

// Longest full-plane transform: both ping-pong buffers of one row in shared
// memory, as for the column pass (8192 float2, 4096 double2).
template <typename T> constexpr int plane_max_lg() { return col3_max_lg<T>(); }

// Length-L complex transform of one row held in registers (v[r] at shifted
// index t + r T, stage-0 layout), and the store of its kept bins to row
// `row` of F1: bin k mod L at column k + fc.lo for k = -fc.lo .. fc.hi.
// Every thread of the block calls it (it synchronises); `act` masks the store.
template <typename T, int L> struct C2CRow {
  using C = cplx_t<T>;
  using P = P3<L, FftV<T>::V>;
  static constexpr int V = FftV<T>::V, TT = P::T;
  template <typename Sync>
  static __device__ __forceinline__ void run(C (&v)[V], C* A, C* B, int t,
                                             const C* __restrict__ tw, const C (&tw1)[V - 1],
                                             const C (&twp)[V], bool pruned, bool one_j,
                                             int kmax, const FullCols& fc, bool act, int row,
                                             C* __restrict__ F1, Sync&& sync) {
    Head3<L, V, 1, 0>::run(v, A, B, t, tw, tw1, sync);
    C* in = last_input<L, V>(A, B);
    if (pruned) {
      for (int j = t; j <= kmax; j += TT) {
        C xj, xmj;
        if (one_j) {
          pruned_pair3<L, V>(in, j, twp, xj, xmj);
        } else {
          C tj[V];
          load_twp<L, V, 1>(tj, j, tw);
          pruned_pair3<L, V>(in, j, tj, xj, xmj);
        }
        if (act) {
          if (j <= fc.hi) F1[(size_t)(fc.lo + j) * L + row] = xj;
          if (j > 0 && j <= fc.lo) F1[(size_t)(fc.lo - j) * L + row] = xmj;
        }
      }
    } else {
      last_full<L, V, 1>(v, in, t, tw);
      C* o = in == A ? B : A;
      store_full<L, V>(v, o, t);
      __syncthreads();
      if (act)
        for (int cc = t; cc < fc.W; cc += TT) F1[(size_t)cc * L + row] = o[pad3<V>((cc - fc.lo) & (L - 1))];
    }
    __syncthreads();
  }
};

// Row i' of F1 (column-major) holds, for u bins k = -lo .. hi of full_cols()
// (column k + lo), bin k mod N of the length-N complex FFT of row i' of
// fftshift(image) taken as x + 0i, i.e. of image row (i' + N/2) mod N with
// its halves swapped.  Pruned, X[j] and X[N - j] come from one evaluation of
// the last stage (pruned_pair3); otherwise the whole transform is kept.
// The beam tables, when given, multiply each pixel as in the half-plane pass.
template <typename T, int LG, bool SWEEP, int K = 1>
__global__ void __launch_bounds__(Shape3<T, (1 << LG), (1 << 30)>::threads,
                                  min_blocks_128regs<Shape3<T, (1 << LG), (1 << 30)>::threads>())
row_c2c_kernel(const __grid_constant__ Jobs<RowJob<T>, K> jobs, const cplx_t<T>* __restrict__ tw) {
  using C = cplx_t<T>;
  const RowJob<T>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  grid_dep_launch();  // the column pass may be scheduled as our blocks retire
  constexpr int N = 1 << LG;
  using SH = Shape3<T, N, (1 << 30)>;
  using P = typename SH::P;
  constexpr int V = SH::V, TT = P::T, G = SH::G, RS = SH::RS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* base = reinterpret_cast<C*>(smem_raw);
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const Bounds bd = block_bounds(jb.rho2, jb.S, N);
  const FullCols fc = full_cols(bd, N);
  const int kmax = fc.lo > fc.hi ? fc.lo : fc.hi;
  C tw1[V - 1];
  load_tw1<N, V, 1>(tw1, t, tw);
  const bool pruned = P::nstage >= 2 && kmax < P::Nsl;
  const bool one_j = kmax < TT;
  C twp[V];
  if (pruned && one_j && t <= kmax) load_twp<N, V, 1>(twp, t, tw);
  C* A = base + (size_t)g * RS;
  C* B = base + (size_t)(G + g) * RS;
  auto sync = [] { __syncthreads(); };
  const T* __restrict__ beam = jb.beam;
  C* __restrict__ F1 = jb.F1;
  if (beam) grid_dep_wait();  // launched as a dependent of beam_table_kernel
  for (int r0 = blockIdx.x * G; r0 < N; r0 += gridDim.x * G) {
    const int row = r0 + g;
    const bool act = row < N;
    const int irow = (row + N / 2) & (N - 1);
    C v[V];
#pragma unroll
    for (int r = 0; r < V; ++r) {
      const int n = t + r * TT;
      const int j = (n + N / 2) & (N - 1);
      T x = (T)0;
      if (act) {
        if constexpr (SWEEP)
          x = sweep_pixel(jb.I, jb.sp, N, irow, j);
        else
          x = jb.image[(size_t)irow * N + j];
        if (beam) x = x * (__ldg(beam + N + row) * __ldg(beam + n));
      }
      v[r] = mkc(x, (T)0);
    }
    C2CRow<T, N>::run(v, A, B, t, tw, tw1, twp, pruned, one_j, kmax, fc, act, row, F1, sync);
  }
}

// The same pass for a 16-byte aligned image, with the rows staged by bulk
// copies: persistent blocks own row groups blockIdx.x + k gridDim.x, thread 0
// keeps the next group in flight in a two-slot ring (the two half-row copies
// perform the fftshift), one mbarrier per slot.  Each slot is read into
// registers and released at once, so the transform's two buffers are
// separate.  A wait that times out (never expected) sets bit 2 of *err,
// drains the copies in flight (bounded) and ends the block.
template <typename T, int LG, int K = 1>
__global__ void __launch_bounds__(Shape3<T, (1 << LG), (1 << LG)>::threads,
                                  min_blocks_128regs<Shape3<T, (1 << LG), (1 << LG)>::threads>())
row_c2c_tma_kernel(const __grid_constant__ Jobs<RowJob<T>, K> jobs,
                   const cplx_t<T>* __restrict__ tw, int* __restrict__ err) {
  using C = cplx_t<T>;
  const RowJob<T>& jb = jobs.j[K == 1 ? 0 : blockIdx.y];
  grid_dep_launch();  // the column pass may be scheduled as our blocks retire
  constexpr int N = 1 << LG;
  using SH = Shape3<T, N, N>;
  using P = typename SH::P;
  constexpr int V = SH::V, TT = P::T, G = SH::G, RS = SH::RS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  T* slot0 = reinterpret_cast<T*>(smem_raw + 128);  // 2 G rows of N reals
  C* base = reinterpret_cast<C*>(smem_raw + 128 + (size_t)2 * G * N * sizeof(T));
  const int g = threadIdx.x / TT, t = threadIdx.x - g * TT;
  const Bounds bd = block_bounds(jb.rho2, jb.S, N);
  const FullCols fc = full_cols(bd, N);
  const int kmax = fc.lo > fc.hi ? fc.lo : fc.hi;
  C tw1[V - 1];
  load_tw1<N, V, 1>(tw1, t, tw);
  const bool pruned = P::nstage >= 2 && kmax < P::Nsl;
  const bool one_j = kmax < TT;
  C twp[V];
  if (pruned && one_j && t <= kmax) load_twp<N, V, 1>(twp, t, tw);
  C* A = base + (size_t)g * RS;
  C* B = base + (size_t)(G + g) * RS;
  auto sync = [] { __syncthreads(); };
  const T* __restrict__ image = jb.image;
  const T* __restrict__ beam = jb.beam;
  const int ngroups = N / G;
  const uint32_t half_bytes = (uint32_t)(N / 2 * sizeof(T));
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int it) {  // thread 0 only
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp >= ngroups) return;
    const int sl = it & 1;
    mbar_arrive_expect_tx(&bars[sl], 2u * half_bytes * (uint32_t)G);
    for (int rl = 0; rl < G; ++rl) {
      const T* src = image + (size_t)(((grp * G + rl) + N / 2) & (N - 1)) * N;
      T* dst = slot0 + (size_t)(sl * G + rl) * N;
      bulk_load(dst, src + N / 2, half_bytes, &bars[sl]);
      bulk_load(dst + N / 2, src, half_bytes, &bars[sl]);
    }
  };
  if (threadIdx.x == 0) {
    issue(0);
    issue(1);
  }
  if (beam) grid_dep_wait();  // launched as a dependent of beam_table_kernel
  for (int it = 0;; ++it) {
    const int grp = blockIdx.x + it * gridDim.x;
    if (grp >= ngroups) break;
    const int sl = it & 1;
    const bool ok = mbar_wait(&bars[sl], (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(err, 2);
        for (int k = it; k < it + 2; ++k)
          if (blockIdx.x + k * gridDim.x < ngroups) mbar_wait(&bars[k & 1], (uint32_t)((k >> 1) & 1));
      }
      return;
    }
    const int row = grp * G + g;
    const T* srow = slot0 + (size_t)(sl * G + g) * N;
    const T ay = beam ? __ldg(beam + N + row) : (T)1;
    C v[V];
#pragma unroll
    for (int r = 0; r < V; ++r) {
      const int n = t + r * TT;
      T x = srow[n];
      if (beam) x = x * (ay * __ldg(beam + n));
      v[r] = mkc(x, (T)0);
    }
    __syncthreads();  // every read of this slot is done
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      issue(it + 2);
    }
    C2CRow<T, N>::run(v, A, B, t, tw, tw1, twp, pruned, one_j, kmax, fc, true, row, jb.F1, sync);
  }
}

// Launchers of the full-plane row pass over n jobs (grid row y = job y).  Each
// job gets the GPU's resident blocks times `scale`, shared by the n jobs, as
// persistent blocks; `dep`: launch as a programmatic dependent (the jobs
// carry beam tables computed just before, single calls only).
template <typename T, int LG, bool SWEEP, int K>
cudaError_t launch_row_c2c(const Jobs<RowJob<T>, K>& jb, int n, int scale, bool dep,
                           const void* tw, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int N = 1 << LG;
  using SH = Shape3<T, N, (1 << 30)>;
  constexpr auto kern = row_c2c_kernel<T, LG, SWEEP, K>;
  const size_t smem = (size_t)2 * SH::G * SH::RS * sizeof(C);
  cudaError_t e = ensure_smem_attr<kern>(smem);
  if (e) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::threads, smem);
  if (e) return e;
  if (per_sm < 1) per_sm = 1;
  int x = (per_sm * current_device_sms() * (scale < 1 ? 1 : scale) + n - 1) / n;
  const int need = (N + SH::G - 1) / SH::G;
  if (x > need) x = need;
  if (x < 1) x = 1;
  if (dep)
    return launch_dependent(kern, dim3(x, n), dim3(SH::threads), smem, st, jb,
                            static_cast<const C*>(tw));
  kern<<<dim3(x, n), SH::threads, smem, st>>>(jb, static_cast<const C*>(tw));
  return cudaGetLastError();
}

template <typename T, int LG, int K>
cudaError_t launch_row_c2c_tma(const Jobs<RowJob<T>, K>& jb, int n, int scale, bool dep,
                               const void* tw, int* err, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int N = 1 << LG;
  using SH = Shape3<T, N, N>;
  constexpr auto kern = row_c2c_tma_kernel<T, LG, K>;
  const size_t smem = 128 + (size_t)2 * SH::G * N * sizeof(T) + (size_t)2 * SH::G * SH::RS * sizeof(C);
  cudaError_t e = ensure_smem_attr<kern>(smem);
  if (e) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::threads, smem);
  if (e) return e;
  if (per_sm < 1) per_sm = 1;
  int x = (per_sm * current_device_sms() * (scale < 1 ? 1 : scale) + n - 1) / n;
  if (x > N / SH::G) x = N / SH::G;
  if (x < 1) x = 1;
  if (dep)
    return launch_dependent(kern, dim3(x, n), dim3(SH::threads), smem, st, jb,
                            static_cast<const C*>(tw), err);
  kern<<<dim3(x, n), SH::threads, smem, st>>>(jb, static_cast<const C*>(tw), err);
  return cudaGetLastError();
}

// mode 0: staged image rows (16-byte aligned image), 1: plain loads, 2: sweep
template <typename T, int LG>
cudaError_t row_c2c_switch(int lg, const RowJob<T>& jb, int mode, const void* tw, int* err,
                           cudaStream_t st) {
  if constexpr (LG > plane_max_lg<T>()) {
    return cudaErrorNotSupported;
  } else {
    if (lg == LG) {
      Jobs<RowJob<T>, 1> j1;
      j1.j[0] = jb;
      const bool dep = jb.beam != nullptr;
      if (mode == 0) return launch_row_c2c_tma<T, LG, 1>(j1, 1, 1, dep, tw, err, st);
      if (mode == 2) return launch_row_c2c<T, LG, true, 1>(j1, 1, 1, dep, tw, st);
      return launch_row_c2c<T, LG, false, 1>(j1, 1, 1, dep, tw, st);
    }
    return row_c2c_switch<T, LG + 1>(lg, jb, mode, tw, err, st);
  }
}

template <typename T> bool Plane<T>::supported(int N) {
  return N >= FftV<T>::V && N <= (1 << plane_max_lg<T>()) && (N & (N - 1)) == 0;
}

template <typename T>
cudaError_t Plane<T>::rows(const T* image, const T* I, const SweepParams& sp, int N,
                           const void* tw, void* F1, const double* rho2, double S, const T* beam,
                           int* err, cudaStream_t st) {
  if (!supported(N)) return cudaErrorNotSupported;
  RowJob<T> jb{image, I, I ? sweep_cast<T>(sp) : SweepT<T>{}, static_cast<cplx_t<T>*>(F1), rho2, S,
               beam};
  const int mode = I ? 2 : (reinterpret_cast<uintptr_t>(image) & 15u) == 0 ? 0 : 1;
  constexpr int LG0 = ilog2c(FftV<T>::V);
  return row_c2c_switch<T, LG0>(ilog2i(N), jb, mode, tw, err, st);
}

template <typename T> int Plane<T>::gather_blocks_per_sm(bool chi2, size_t window_smem) {
  int n = 0;
  if (window_smem) {
    if (chi2) {
      constexpr auto kern = gather_kernel<T, true, true, true, 1, false, true>;
      if (ensure_smem_attr<kern>(window_smem) == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, gather_threads<true, true>(),
                                                      window_smem);
    } else {
      constexpr auto kern = gather_kernel<T, false, true, true, 1, false, true>;
      if (ensure_smem_attr<kern>(window_smem) == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, gather_threads<true, true>(),
                                                      window_smem);
    }
  } else {
    if (chi2)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, gather_kernel<T, true, false, true, 1, false, true>, gather_threads<false>(), 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, gather_kernel<T, false, false, true, 1, false, true>, gather_threads<false>(), 0);
  }
  (void)cudaGetLastError();
  return n < 1 ? 1 : n;
}

template <typename T>
cudaError_t Plane<T>::gather(const void* Gw, const GatherParams& gp, const double* rho2,
                             const T* u, const T* v, const T* re, const T* im, const T* w,
                             int64_t M, void* vis, double* partials, unsigned* counter,
                             double* chi2, size_t window_smem, bool edge, int blocks,
                             cudaStream_t st) {
  using C = cplx_t<T>;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  int vec = al16(u) && al16(v);
  if (chi2) vec = vec && al16(re) && al16(im) && al16(w);
  const int nodes = (int)(window_smem / sizeof(C));
  const int threads = window_smem ? gather_threads<true, true>() : gather_threads<false, true>();
  int grid = blocks;
  if (!chi2) {
    int64_t need = (M + threads - 1) / threads;
    if (need < 1) need = 1;
    if (need < grid) grid = (int)need;
  }
  Jobs<GatherJob<T>, 1> jb;
  jb.j[0] = GatherJob<T>{static_cast<const C*>(Gw), GatherT<T>::make(gp), rho2, u, v, re, im, w, M,
                         vec, static_cast<C*>(vis), partials, counter, chi2};
  cudaError_t le = cudaSuccess;
  auto pick = [&](auto chi2_c, auto smem_c, auto edge_c) {
    constexpr bool CH = decltype(chi2_c)::value, SM = decltype(smem_c)::value,
                   ED = decltype(edge_c)::value;
    constexpr auto kern = gather_kernel<T, CH, SM, ED, 1, false, true>;
    const size_t smem = SM ? window_smem : 0;
    le = ensure_smem_attr<kern>(smem);
    if (le == cudaSuccess)
      le = launch_dependent(kern, dim3(grid), dim3(threads), smem, st, jb, nodes,
                            MultiArg<T, false>{});
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
