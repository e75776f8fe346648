// Register-blocked Stockham FFT with conflict-free shared-memory exchanges.
//
// A group of T = L/V threads transforms one length-L sequence (L a power of
// two, L >= V).  Each thread holds V values (V = 16 for float2, 8 for
// double2).  The stages have radix V except possibly a smaller last one
// (L = V^k * R_last), so an FFT of length 2048 in float runs as 16 x 16 x 8:
// two exchanges through shared memory instead of four.
//
// Stage s (radix R, span Ns = product of the earlier radices): butterfly b
// takes the R values at b + r L/R, multiplies value r by W_{Ns R}^{r (b mod
// Ns)}, applies the radix-R DFT in registers and sends value r to
// (b - b mod Ns) R + (b mod Ns) + r Ns.  Thread t owns butterflies
// b = t + q T (q < V/R).  The first stage takes its inputs from registers
// (loaded by the caller straight from global memory), so shared memory is
// touched only between stages.
//
// Shared-memory addresses are XOR-swizzled, a' = a ^ ((a >> log2 V) & (V-1)):
// every store and load pattern of these plans then maps each half-warp
// (float2) or quarter-warp (double2) onto distinct banks.
//
// The last stage is left to the caller: fft_last() runs it fully, and
// pruned_pair() evaluates the two outputs X[j] and X[L-j] directly from the
// last stage's input, which is all the row and column passes need when only
// the low frequencies are kept.
#pragma once

#include <type_traits>

#include "gal_common.cuh"

namespace gal {

template <int V> struct VTraits;
template <> struct VTraits<16> { static constexpr int lg = 4; };
template <> struct VTraits<8> { static constexpr int lg = 3; };

template <int V> __device__ __forceinline__ int swz(int a) {
  return a ^ ((a >> VTraits<V>::lg) & (V - 1));
}

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

// Stage plan: radix V for every stage except the last, which takes the
// remainder (radix V when L is a power of V).
struct Plan2 {
  int nstage;
  int rlast;
  __host__ __device__ __forceinline__ int radix(int st) const { return st == nstage - 1 ? rlast : 0; }
};
template <int V> __host__ __device__ __forceinline__ Plan2 make_plan2(int L) {
  int lg = 0;
  while ((1 << lg) < L) ++lg;
  const int lv = VTraits<V>::lg;
  Plan2 p;
  p.nstage = (lg + lv - 1) / lv;
  const int rem = lg - (p.nstage - 1) * lv;  // bits of the last stage, in [1, lv]
  p.rlast = 1 << rem;
  return p;
}

// Twiddle the values of butterfly group q of a non-first stage.
template <int R, int V, typename C>
__device__ __forceinline__ void twiddle(C* v, int b, int Ns, int L, const C* __restrict__ tw,
                                        int tws) {
  const int k = b & (Ns - 1);
  const int step = (L / (Ns * R)) * tws * k;
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(tw + r * step));
}

// Apply radix-R butterflies (V/R per thread) to registers v (stage input
// layout v[q R + r] = x[b_q + r L/R]) and store the outputs to shared memory.
template <int R, int V, typename C>
__device__ __forceinline__ void stage_store(C* v, C* s, int L, int Ns, int t, int T,
                                            const C* __restrict__ tw, int tws) {
  constexpr int NB = V / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * T;
    if (Ns > 1) twiddle<R, V>(&v[q * R], b, Ns, L, tw, tws);
    bflyR<R>(&v[q * R]);
    const int k = b & (Ns - 1);
    const int base = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[swz<V>(base + r * Ns)] = v[q * R + bfly_out<R>(r)];
  }
}

template <int R, int V, typename C>
__device__ __forceinline__ void stage_load(C* v, const C* s, int L, int t, int T) {
  constexpr int NB = V / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int b = t + q * T;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = s[swz<V>(b + r * (L / R))];
  }
}

template <int V, typename C>
__device__ __forceinline__ void stage_store_any(int R, C* v, C* s, int L, int Ns, int t, int T,
                                                const C* __restrict__ tw, int tws) {
  if constexpr (V >= 16)
    if (R == 16) return stage_store<16, V>(v, s, L, Ns, t, T, tw, tws);
  if (R == 8) return stage_store<8, V>(v, s, L, Ns, t, T, tw, tws);
  if (R == 4) return stage_store<4, V>(v, s, L, Ns, t, T, tw, tws);
  stage_store<2, V>(v, s, L, Ns, t, T, tw, tws);
}

template <int V, typename C>
__device__ __forceinline__ void stage_load_any(int R, C* v, const C* s, int L, int t, int T) {
  if constexpr (V >= 16)
    if (R == 16) return stage_load<16, V>(v, s, L, t, T);
  if (R == 8) return stage_load<8, V>(v, s, L, t, T);
  if (R == 4) return stage_load<4, V>(v, s, L, t, T);
  stage_load<2, V>(v, s, L, t, T);
}

// All stages but the last.  On entry v holds the first stage's inputs
// (v[q R0 + r] = x[t + q T + r L/R0]); on exit shared memory s holds the
// last stage's input (swizzled) and the block has synchronised.  The caller
// must have synchronised s since its previous use.  Returns the last stage's
// span Ns = L / R_last.  Every thread of the block must call it.
template <int V, typename C>
__device__ __forceinline__ int fft_head(C (&v)[V], C* s, int L, int t, int T, const Plan2& p,
                                        const C* __restrict__ tw, int tws) {
  int Ns = 1;
  for (int st = 0; st < p.nstage - 1; ++st) {  // every stage but the last has radix V
    if (st > 0) {
      stage_load<V, V>(v, s, L, t, T);
      __syncthreads();
    }
    stage_store<V, V>(v, s, L, Ns, t, T, tw, tws);
    __syncthreads();
    Ns *= V;
  }
  return Ns;
}

// The full last stage: v receives outputs X[b + r L/R] of butterflies
// b = t + q T in v[q R + r].
template <int V, typename C>
__device__ __forceinline__ void fft_last(C (&v)[V], const C* s, int L, int Ns, int t, int T,
                                         const Plan2& p, const C* __restrict__ tw, int tws,
                                         bool from_registers) {
  const int R = p.rlast;
  if (!from_registers) stage_load_any<V>(R, v, s, L, t, T);
  auto run = [&](auto rc) {
    constexpr int RR = decltype(rc)::value;
#pragma unroll
    for (int q = 0; q < V / RR; ++q) {
      if (Ns > 1) twiddle<RR, V>(&v[q * RR], t + q * T, Ns, L, tw, tws);
      bflyR<RR>(&v[q * RR]);
      if constexpr (RR == 16) {
        C o[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) o[r] = v[q * RR + bfly_out<16>(r)];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[q * RR + r] = o[r];
      }
    }
  };
  if constexpr (V >= 16)
    if (R == 16) return run(std::integral_constant<int, 16>{});
  if (R == 8) return run(std::integral_constant<int, 8>{});
  if (R == 4) return run(std::integral_constant<int, 4>{});
  run(std::integral_constant<int, 2>{});
}

// Outputs X[j] and X[L - j] (X[L] = X[0]) of the transform whose last stage
// (radix R, span Ns = L/R, input in shared memory) has not been run, for
// 0 <= j <= Ns:
//   X[j]     = sum_r Y[j + r Ns]       W_L^( r j)     (needs j <  Ns)
//   X[L - j] = sum_r Y[(r+1) Ns - j]   W_L^(-r j)     (needs 1 <= j <= Ns)
template <int R, int V, typename C>
__device__ __forceinline__ void pruned_pair_r(const C* s, int L, int Ns, int j,
                                              const C* __restrict__ tw, int tws, C& xj, C& xmj) {
  C a = s[swz<V>(j)];
  C b = s[swz<V>((Ns - j) & (L - 1))];
#pragma unroll
  for (int r = 1; r < R; ++r) {
    const C w = __ldg(tw + ((r * j) & (L - 1)) * tws);
    const C ya = s[swz<V>(j + r * Ns)];
    const C yb = s[swz<V>(((r + 1) * Ns - j) & (L - 1))];
    a = cadd(a, cmul(ya, w));
    b = cadd(b, cmul(yb, cconj(w)));
  }
  xj = a;
  xmj = j == 0 ? a : b;
}

template <int V, typename C>
__device__ __forceinline__ void pruned_pair(const C* s, int L, int Ns, int j, const Plan2& p,
                                            const C* __restrict__ tw, int tws, C& xj, C& xmj) {
  const int R = p.rlast;
  if constexpr (V >= 16)
    if (R == 16) return pruned_pair_r<16, V>(s, L, Ns, j, tw, tws, xj, xmj);
  if (R == 8) return pruned_pair_r<8, V>(s, L, Ns, j, tw, tws, xj, xmj);
  if (R == 4) return pruned_pair_r<4, V>(s, L, Ns, j, tw, tws, xj, xmj);
  pruned_pair_r<2, V>(s, L, Ns, j, tw, tws, xj, xmj);
}

}  // namespace gal
