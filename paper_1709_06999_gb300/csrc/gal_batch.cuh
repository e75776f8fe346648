// Batched passes: the row FFT, the column FFT and the gather/chi-square of
// many requests, one launch per pass, transform length and chunk of at most
// kBatchJobs requests.  Grid row y of a launch is request y of the chunk; its
// arguments come from the launch's __grid_constant__ job array.  Each request
// is computed by the same code and, for the gather, with the same block
// partition and reduction tree as a single call, so batched and single-call
// results are bitwise equal.
#pragma once

#include <type_traits>
#include <vector>

#include "gal_plane.cuh"

namespace gal {

template <typename T> bool BatchLaunch<T>::supported(int N) {
  const int lg = ilog2i(N);
  return (1 << lg) == N && N / 2 >= FftV<T>::V && lg - 1 <= 12 && lg <= col3_max_lg<T>();
}

namespace batch {

inline int chunk_of(const BatchShape& sh) {
  int k = sh.jobs_per_launch;
  return k < 1 ? 1 : (k > kBatchJobs ? kBatchJobs : k);
}

// rows: the chunk `idx[0..n)` of items, all of length 2^(LG+1), all swept
// (SWEEP) or all images, all with a beam (BEAM, its tables already computed
// earlier in the stream) or none
template <typename T, int LG, bool SWEEP, bool BEAM, int V = FftV<T>::V>
cudaError_t rows(const BatchItem* it, const int* idx, int n, const void* tw, int* err,
                 const BatchShape& sh, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int M = 1 << LG, N = 2 * M;
  using SH = Shape3<T, M, N, 128, V>;
  Jobs<RowJob<T>, kBatchJobs> jb{};
  for (int k = 0; k < n; ++k) {
    const BatchItem& b = it[idx[k]];
    jb.j[k] = RowJob<T>{static_cast<const T*>(b.image), static_cast<const T*>(b.I),
                        SWEEP ? sweep_cast<T>(b.sp) : SweepT<T>{}, static_cast<C*>(b.F1), b.rho2,
                        b.S, BEAM ? static_cast<const T*>(b.beam) : nullptr};
  }
  const C* twc = static_cast<const C*>(tw);
  if constexpr (row_ldg_shape<T, LG, SWEEP, V>()) {
    // the same kernel as single calls of this length (bitwise equal results)
    constexpr auto kern = row_fft3_ldg_kernel<kBatchJobs, BEAM>;
    const cudaError_t e = ensure_smem_attr<kern>(RowLdgShape::smem);
    if (e) return e;
    int x = row_ldg_grid<kern>(n) * (sh.row_blocks < 1 ? 1 : sh.row_blocks);
    if (x > RowLdgShape::N) x = RowLdgShape::N;
    if (x < 1) return cudaErrorInvalidConfiguration;
    kern<<<dim3(x, n), RowLdgShape::TT, RowLdgShape::smem, st>>>(jb, twc);
  } else if constexpr (!SWEEP) {
    constexpr auto kern = row_fft3_kernel<T, LG, true, false, kBatchJobs, BEAM, 128, 2, V>;
    const size_t smem = 128 + (size_t)3 * SH::G * SH::RS * sizeof(C);
    cudaError_t e = ensure_smem_attr<kern>(smem);
    if (e) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SH::threads, smem);
    if (e) return e;
    if (per_sm < 1) per_sm = 1;
    // persistent blocks per request: the GPU's resident blocks (times the
    // shape's factor) shared by the chunk's requests
    int x = (per_sm * current_device_sms() * (sh.row_blocks < 1 ? 1 : sh.row_blocks) + n - 1) / n;
    if (x > N / SH::G) x = N / SH::G;
    if (x < 1) x = 1;
    kern<<<dim3(x, n), SH::threads, smem, st>>>(jb, twc, err);
  } else {
    constexpr auto kern = row_fft3_kernel<T, LG, false, true, kBatchJobs, BEAM, 128, 2, V>;
    const size_t smem = 128 + (size_t)2 * SH::G * SH::RS * sizeof(C);
    const cudaError_t e = ensure_smem_attr<kern>(smem);
    if (e) return e;
    kern<<<dim3(N / SH::G, n), SH::threads, smem, st>>>(jb, twc, err);
  }
  return cudaGetLastError();
}

// full-plane rows: the chunk `idx[0..n)`, all of length 2^LG, all swept or
// all images (16-byte aligned, staged by bulk copies); beam tables, if any,
// were computed earlier in the stream
template <typename T, int LG, bool SWEEP>
cudaError_t rows_full(const BatchItem* it, const int* idx, int n, const void* tw, int* err,
                      const BatchShape& sh, cudaStream_t st) {
  using C = cplx_t<T>;
  Jobs<RowJob<T>, kBatchJobs> jb{};
  for (int k = 0; k < n; ++k) {
    const BatchItem& b = it[idx[k]];
    jb.j[k] = RowJob<T>{static_cast<const T*>(b.image), static_cast<const T*>(b.I),
                        SWEEP ? sweep_cast<T>(b.sp) : SweepT<T>{}, static_cast<C*>(b.F1), b.rho2,
                        b.S, static_cast<const T*>(b.beam)};
  }
  if constexpr (SWEEP) return launch_row_c2c<T, LG, true, kBatchJobs>(jb, n, sh.row_blocks, false, tw, st);
  else return launch_row_c2c_tma<T, LG, kBatchJobs>(jb, n, sh.row_blocks, false, tw, err, st);
}

template <typename T, int LG, int V = FftV<T>::V>
cudaError_t cols(const BatchItem* it, const int* idx, int n, const void* tw, cudaStream_t st) {
  using C = cplx_t<T>;
  constexpr int N = 1 << LG;
  using SH = ColShape3<T, N, V>;
  constexpr auto kern = col_fft3_kernel<T, LG, kBatchJobs, V>;
  const size_t smem = (size_t)2 * SH::G * SH::RS * sizeof(C);
  const cudaError_t e = ensure_smem_attr<kern>(smem);
  if (e) return e;
  Jobs<ColJob<T>, kBatchJobs> jb{};
  int kc = 1;
  for (int k = 0; k < n; ++k) {
    const BatchItem& b = it[idx[k]];
    jb.j[k] = ColJob<T>{static_cast<const C*>(b.F1), static_cast<C*>(b.Gw), b.rho2, b.S,
                        b.full ? 1 : 0};
    kc = b.ncol > kc ? b.ncol : kc;
  }
  int x = (kc + SH::G - 1) / SH::G;
  const int cap = 2 * current_device_sms();
  if (x > cap) x = cap;
  kern<<<dim3(x, n), SH::threads, smem, st>>>(jb, static_cast<const C*>(tw));
  return cudaGetLastError();
}

// Each request keeps the block partition of its single call (`grid` virtual
// blocks, one partial sum each); a launch of n requests runs min(n, fold) of
// them per block in turn (fold from the launch shape, kGatherFold by
// default), so a request's window is copied by that many times fewer blocks
// while the launch still fills the GPU (a launch of one request runs its
// single call's grid).
template <typename T, bool SMEM, bool EDGE, bool FULL>
cudaError_t gather(const BatchItem* it, const int* idx, int n, int grid, int fold_max,
                   cudaStream_t st) {
  using C = cplx_t<T>;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  Jobs<GatherJob<T>, kBatchJobs> jb{};
  size_t smem = 0;
  for (int k = 0; k < n; ++k) {
    const BatchItem& b = it[idx[k]];
    const int vec = al16(b.u) && al16(b.v) && al16(b.re) && al16(b.im) && al16(b.w);
    jb.j[k] = GatherJob<T>{static_cast<const C*>(b.Gw), GatherT<T>::make(b.gp), b.rho2,
                           static_cast<const T*>(b.u), static_cast<const T*>(b.v),
                           static_cast<const T*>(b.re), static_cast<const T*>(b.im),
                           static_cast<const T*>(b.w), b.M, vec, nullptr, b.partials,
                           b.counter, b.chi2_out, grid};
    smem = b.wbytes > smem ? b.wbytes : smem;
  }
  if (!SMEM) smem = 0;
  constexpr auto kern = gather_kernel<T, true, SMEM, EDGE, kBatchJobs, false, FULL>;
  const cudaError_t e = ensure_smem_attr<kern>(smem);
  if (e) return e;
  const int threads = gather_threads<SMEM, FULL>();
  if (fold_max < 1) fold_max = 1;
  if (fold_max > kMaxGatherFold) fold_max = kMaxGatherFold;
  const int fold = n < fold_max ? n : fold_max;
  const int blocks = (grid + fold - 1) / fold;
  kern<<<dim3(blocks, n), threads, smem, st>>>(jb, (int)(smem / sizeof(C)), MultiArg<T, false>{});
  return cudaGetLastError();
}

// length dispatch
template <typename T, int LG, typename F> cudaError_t by_lg(int lg, F&& f) {
  if constexpr (LG > 13) {
    return cudaErrorNotSupported;
  } else {
    if (lg == LG) return f(std::integral_constant<int, LG>{});
    return by_lg<T, LG + 1>(lg, f);
  }
}

// apply f(chunk indices, count) over the items selected by `pick`, grouped by
// key(item) and chunked
template <typename Key, typename Pick, typename F>
cudaError_t for_chunks(const BatchItem* it, int n, const BatchShape& sh, Pick&& pick, Key&& key,
                       F&& f) {
  const int cap = chunk_of(sh);
  std::vector<char> done(n, 0);
  std::vector<int> idx;
  idx.reserve(cap);
  for (int a = 0; a < n; ++a) {
    if (done[a] || !pick(it[a])) continue;
    const auto ka = key(it[a]);
    idx.clear();
    for (int b = a; b < n; ++b) {
      if (done[b] || !pick(it[b]) || !(key(it[b]) == ka)) continue;
      done[b] = 1;
      idx.push_back(b);
      if ((int)idx.size() == cap) {
        const cudaError_t e = f(idx.data(), (int)idx.size(), it[idx[0]]);
        if (e) return e;
        idx.clear();
      }
    }
    if (!idx.empty()) {
      const cudaError_t e = f(idx.data(), (int)idx.size(), it[idx[0]]);
      if (e) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace batch

template <typename T>
cudaError_t BatchLaunch<T>::beams(const BatchItem* it, int n, int* launches, cudaStream_t st) {
  const BatchShape sh{1, kBatchJobs, kGatherFold};
  auto pick = [](const BatchItem& b) { return b.beam != nullptr; };
  auto key = [](const BatchItem&) { return 0; };
  return batch::for_chunks(it, n, sh, pick, key, [&](const int* idx, int m, const BatchItem&) {
    Jobs<BeamJob<T>, kBatchJobs> jb{};
    int nmax = 1;
    for (int k = 0; k < m; ++k) {
      const BatchItem& b = it[idx[k]];
      jb.j[k] = BeamJob<T>{static_cast<T*>(b.beam), b.N, b.sp.dxy, b.bp.c, b.bp.bx, b.bp.by};
      nmax = b.N > nmax ? b.N : nmax;
    }
    beam_tables_kernel<T, kBatchJobs><<<dim3((2 * nmax + 63) / 64, m), 64, 0, st>>>(jb);
    const cudaError_t e = cudaGetLastError();
    if (!e) ++*launches;
    return e;
  });
}

template <typename T>
cudaError_t BatchLaunch<T>::rows(const BatchItem* it, int n, const void* const* tw, int* err,
                                 const BatchShape& sh, int* launches, cudaStream_t st) {
  auto pick = [](const BatchItem&) { return true; };
  auto key = [](const BatchItem& b) {
    return (b.N * 8 + (b.full ? 4 : 0) + (b.beam ? 2 : 0) + (b.I ? 1 : 0)) * 64 + b.radix_row;
  };
  return batch::for_chunks(it, n, sh, pick, key, [&](const int* idx, int m, const BatchItem& b0) {
    const int lg = ilog2i(b0.N);
    if (b0.full) {  // complex-to-complex rows of length N
      const cudaError_t e = batch::by_lg<T, ilog2c(FftV<T>::V)>(lg, [&](auto L) {
        constexpr int LG = decltype(L)::value;
        if constexpr (LG > plane_max_lg<T>()) {
          return cudaErrorNotSupported;
        } else {
          return b0.I ? batch::rows_full<T, LG, true>(it, idx, m, tw[lg], err, sh, st)
                      : batch::rows_full<T, LG, false>(it, idx, m, tw[lg], err, sh, st);
        }
      });
      if (!e) ++*launches;
      return e;
    }
    const cudaError_t e = batch::by_lg<T, ilog2c(FftV<T>::V)>(lg - 1, [&](auto L) {
      constexpr int LG = decltype(L)::value;
      if constexpr (LG > 12) {
        return cudaErrorNotSupported;
      } else {
        auto go = [&](auto v_c) {
          constexpr int VV = decltype(v_c)::value;
          if (b0.beam)
            return b0.I ? batch::rows<T, LG, true, true, VV>(it, idx, m, tw[lg], err, sh, st)
                        : batch::rows<T, LG, false, true, VV>(it, idx, m, tw[lg], err, sh, st);
          return b0.I ? batch::rows<T, LG, true, false, VV>(it, idx, m, tw[lg], err, sh, st)
                      : batch::rows<T, LG, false, false, VV>(it, idx, m, tw[lg], err, sh, st);
        };
        if constexpr (has_alt_radix<T, (2 << LG)>())
          if (b0.radix_row == kAltRadix) return go(std::integral_constant<int, kAltRadix>{});
        return go(std::integral_constant<int, FftV<T>::V>{});
      }
    });
    if (!e) ++*launches;
    return e;
  });
}

template <typename T>
cudaError_t BatchLaunch<T>::cols(const BatchItem* it, int n, const void* const* tw,
                                 const BatchShape& sh, int* launches, cudaStream_t st) {
  auto pick = [](const BatchItem&) { return true; };
  auto key = [](const BatchItem& b) { return b.N * 64 + b.radix_col; };
  return batch::for_chunks(it, n, sh, pick, key, [&](const int* idx, int m, const BatchItem& b0) {
    const int lg = ilog2i(b0.N);
    const cudaError_t e = batch::by_lg<T, ilog2c(FftV<T>::V)>(lg, [&](auto L) {
      constexpr int LG = decltype(L)::value;
      if constexpr (LG > col3_max_lg<T>()) {
        return cudaErrorNotSupported;
      } else {
        if constexpr (has_alt_radix<T, (1 << LG)>())
          if (b0.radix_col == kAltRadix) return batch::cols<T, LG, kAltRadix>(it, idx, m, tw[lg], st);
        return batch::cols<T, LG>(it, idx, m, tw[lg], st);
      }
    });
    if (!e) ++*launches;
    return e;
  });
}

template <typename T>
cudaError_t BatchLaunch<T>::gather(const BatchItem* it, int n, const BatchShape& sh,
                                   int* launches, cudaStream_t st) {
  auto pick = [](const BatchItem&) { return true; };
  // one launch shape per chunk: variant and blocks per request
  auto key = [](const BatchItem& b) {
    return (int64_t)b.grid * 8 + (b.full ? 4 : 0) + (b.wbytes ? 2 : 0) + (b.edge ? 1 : 0);
  };
  return batch::for_chunks(it, n, sh, pick, key, [&](const int* idx, int m, const BatchItem& b0) {
    cudaError_t e;
    auto go = [&](auto full_c) {
      constexpr bool F = decltype(full_c)::value;
      const int fold = sh.gather_fold;
      if (b0.wbytes)
        return b0.edge ? batch::gather<T, true, true, F>(it, idx, m, b0.grid, fold, st)
                       : batch::gather<T, true, false, F>(it, idx, m, b0.grid, fold, st);
      return b0.edge ? batch::gather<T, false, true, F>(it, idx, m, b0.grid, fold, st)
                     : batch::gather<T, false, false, F>(it, idx, m, b0.grid, fold, st);
    };
    e = b0.full ? go(std::true_type{}) : go(std::false_type{});
    if (!e) ++*launches;
    return e;
  });
}

}  // namespace gal
