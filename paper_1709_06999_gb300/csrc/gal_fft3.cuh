// Compile-time-length, register-blocked Stockham FFT with padded shared-memory
// exchanges.
//
// A group of T = L/V threads transforms one length-L sequence (L a power of
// two, L >= V); each thread holds V values (V = 16 for float2, 8 for double2).
// Every stage has radix V except the last, which takes the remainder, so a
// length-2048 float transform runs as 16 x 16 x 8 with two exchanges.
//
// Stage s (radix R, span Ns = V^s): butterfly b takes the R values at
// b + r L/R, multiplies value r by W_{Ns R}^{r (b mod Ns)}, applies the
// radix-R DFT in registers and sends value r to (b - b mod Ns) R + (b mod Ns)
// + r Ns.  The first stage takes its inputs from registers.  Stages write to
// alternating buffers (ping-pong), so a stage needs one barrier, not two.
//
// Shared-memory element a lives at pad(a) = a + (a >> log2 V): every exchange
// pattern of these plans then hits distinct banks within each half-warp
// (float2) or quarter-warp (double2), and since L is a compile-time constant
// the padded addresses reduce to a per-thread base plus immediate offsets.
//
// The last stage is run by the caller: last_full() computes it completely,
// pruned_pair3() evaluates only X[j] and X[L-j] from its input.
#pragma once

#include "gal_common.cuh"
#include "gal_fft2.cuh"  // butterflies bfly2/4/8/16 and bfly_out

namespace gal {

constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
constexpr int ipowc(int b, int e) { return e == 0 ? 1 : b * ipowc(b, e - 1); }

template <int L, int V> struct P3 {
  static constexpr int lv = ilog2c(V);
  static constexpr int lg = ilog2c(L);
  static constexpr int nstage = (lg + lv - 1) / lv;
  static constexpr int rlast = 1 << (lg - (nstage - 1) * lv);
  static constexpr int T = L / V;        // threads per sequence
  static constexpr int Nsl = L / rlast;  // span of the last stage
  static constexpr int padded = L + (L >> lv);
};

template <int V> __device__ __forceinline__ int pad3(int a) { return a + (a >> ilog2c(V)); }

// address of element `base + r * step` when step is a multiple of V and base
// is any index: pad is then additive in r
template <int V> __device__ __forceinline__ constexpr int pad_step(int step) {
  return step + step / V;
}

template <int R, typename C> __device__ __forceinline__ void bfly_any(C* a) { bflyR<R>(a); }

// ---------------------------------------------------------------------------
// stages 0 .. nstage-2 (all radix V); ST is the stage index
// ---------------------------------------------------------------------------
template <int L, int V, int TWS, int ST> struct Head3 {
  using P = P3<L, V>;
  template <typename C, typename Sync>
  static __device__ __forceinline__ void run(C (&v)[V], C* A, C* B, int t, const C* __restrict__ tw,
                                             const C (&tw1)[V - 1], Sync&& sync) {
    if constexpr (ST < P::nstage - 1) {
      constexpr int T = P::T;
      constexpr int Ns = ipowc(V, ST);
      C* in = (ST % 2 == 1) ? A : B;   // output buffer of stage ST-1
      C* out = (ST % 2 == 0) ? A : B;
      if constexpr (ST > 0) {
        if constexpr (T % V == 0) {
          const int base = pad3<V>(t);
#pragma unroll
          for (int r = 0; r < V; ++r) v[r] = in[base + r * pad_step<V>(T)];
        } else {
#pragma unroll
          for (int r = 0; r < V; ++r) v[r] = in[pad3<V>(t + r * T)];
        }
        const int k = t & (Ns - 1);
        if constexpr (ST == 1) {
#pragma unroll
          for (int r = 1; r < V; ++r) v[r] = cmul(v[r], tw1[r - 1]);
        } else {
          constexpr int F = (L / (Ns * V)) * TWS;
#pragma unroll
          for (int r = 1; r < V; ++r) v[r] = cmul(v[r], __ldg(tw + r * F * k));
        }
      }
      bflyR<V>(v);
      if constexpr (ST == 0) {
        const int base = (V + 1) * t;  // pad(V t + r) for r < V
#pragma unroll
        for (int r = 0; r < V; ++r) out[base + r] = v[bfly_out<V>(r)];
      } else {
        const int k = t & (Ns - 1);
        const int base = pad3<V>((t - k) * V + k);
#pragma unroll
        for (int r = 0; r < V; ++r) out[base + r * pad_step<V>(Ns)] = v[bfly_out<V>(r)];
      }
      sync();
      Head3<L, V, TWS, ST + 1>::run(v, A, B, t, tw, tw1, sync);
    }
  }
};

// twiddles of stage 1 for thread t (loop-invariant across sequences)
template <int L, int V, int TWS, typename C>
__device__ __forceinline__ void load_tw1(C (&tw1)[V - 1], int t, const C* __restrict__ tw) {
  using P = P3<L, V>;
  if constexpr (P::nstage >= 3) {
    constexpr int Ns = V;
    constexpr int F = (L / (Ns * V)) * TWS;
    const int k = t & (Ns - 1);
#pragma unroll
    for (int r = 1; r < V; ++r) tw1[r - 1] = __ldg(tw + r * F * k);
  }
}

// buffer that holds the last stage's input after the head
template <int L, int V, typename C> __device__ __forceinline__ C* last_input(C* A, C* B) {
  return ((P3<L, V>::nstage - 2) % 2 == 0) ? A : B;
}

// Full last stage (radix R = rlast, span Nsl): v[q R + r] <- X[t + q T + r L/R].
// Reads `in`; for nstage == 1 the inputs are taken from registers instead.
template <int L, int V, int TWS, typename C>
__device__ __forceinline__ void last_full(C (&v)[V], const C* in, int t, const C* __restrict__ tw) {
  using P = P3<L, V>;
  constexpr int R = P::rlast, T = P::T;
  if constexpr (P::nstage == 1) {
    bflyR<V>(v);
    C o[V];
#pragma unroll
    for (int r = 0; r < V; ++r) o[r] = v[bfly_out<V>(r)];
#pragma unroll
    for (int r = 0; r < V; ++r) v[r] = o[r];
  } else {
#pragma unroll
    for (int q = 0; q < V / R; ++q) {
      const int b = t + q * T;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = in[pad3<V>(b + r * (L / R))];
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], __ldg(tw + r * b * TWS));
      bflyR<R>(&v[q * R]);
      C o[R];
#pragma unroll
      for (int r = 0; r < R; ++r) o[r] = v[q * R + bfly_out<R>(r)];
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = o[r];
    }
  }
}

// store the outputs of last_full in natural order to `out` (padded)
template <int L, int V, typename C>
__device__ __forceinline__ void store_full(const C (&v)[V], C* out, int t) {
  using P = P3<L, V>;
  constexpr int R = P::rlast, T = P::T;
#pragma unroll
  for (int q = 0; q < V / R; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) out[pad3<V>(t + q * T + r * (L / R))] = v[q * R + r];
}

// twiddles for pruned_pair at index j (loop-invariant when j is fixed)
template <int L, int V, int TWS, typename C>
__device__ __forceinline__ void load_twp(C (&twp)[V], int j, const C* __restrict__ tw) {
  constexpr int R = P3<L, V>::rlast;
#pragma unroll
  for (int r = 1; r < R; ++r) twp[r - 1] = __ldg(tw + r * j * TWS);
}

// X[j] and X[L-j] (X[L] = X[0]) from the last stage's input, 0 <= j < Nsl:
//   X[j]   = sum_r Y[j + r Ns] W_L^(r j),   X[L-j] = sum_r Y[(r+1) Ns - j] W_L^(-r j)
// twp[r-1] = W_L^(r j).  Requires nstage >= 2.
template <int L, int V, typename C>
__device__ __forceinline__ void pruned_pair3(const C* in, int j, const C (&twp)[V], C& xj, C& xmj) {
  using P = P3<L, V>;
  constexpr int R = P::rlast, Ns = P::Nsl;
  const int jb = j == 0 ? Ns : j;  // j = 0 reads valid addresses; its X[L] is X[0]
  const int ba = pad3<V>(j);
  const int bb = -jb + ((-jb) >> P::lv);  // pad of (-jb), with floor shift
  C a = in[ba];
  C b = in[bb + pad_step<V>(Ns)];
#pragma unroll
  for (int r = 1; r < R; ++r) {
    const C w = twp[r - 1];
    a = cadd(a, cmul(in[ba + r * pad_step<V>(Ns)], w));
    b = cadd(b, cmul(in[bb + (r + 1) * pad_step<V>(Ns)], cconj(w)));
  }
  xj = a;
  xmj = j == 0 ? a : b;
}

}  // namespace gal
