// C ABI of the library (declared in include/galario_gb300.h): context and
// observation handles, argument checks, workspace management and the
// sequencing of the kernels for each operation of Fig. 3 of the paper.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <initializer_list>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/galario_gb300.h"
#include "gal_common.cuh"
#include "gal_internal.h"
#include "gal_reorder.h"

namespace {

constexpr int kMaxLog2 = 13;  // nxy <= 8192
constexpr int kStages = 4;    // 0 extent, 1 row pass, 2 column pass, 3 gather
// largest spectrum window staged in shared memory by the chi2 gather (two
// blocks per SM while two copies fit, one above; larger windows are read
// through L2)
constexpr size_t kWindowSmem = 200 * 1024;

struct TimedStage {
  int stage;
  cudaEvent_t a, b;
};

}  // namespace

struct gal_ctx {
  int device = 0;
  int num_sms = 0;
  void* F1 = nullptr;  // row-pass output: Kc columns of nxy complex values (column-major)
  size_t F1_bytes = 0;
  void* Gw = nullptr;  // pruned spectrum window as node pairs (nrw x (Kc-1) x 2 complex)
  size_t Gw_bytes = 0;
  double* partials = nullptr;  // per-block chi2 partial sums
  int partials_len = 0;
  unsigned* counter = nullptr;  // last-block-done counter (self-resetting)
  double* rho2 = nullptr;       // uv extent scratch for raw-pointer calls
  double* uvrange = nullptr;    // min / max of u^2 + v^2 (image sizing)
  int* err = nullptr;           // index-check flag
  double* chi2_dev = nullptr;   // result slot for the host-buffer entry points
  void* stage_img = nullptr;    // image staging for the host-buffer entry points
  size_t stage_img_bytes = 0;
  void* beam = nullptr;         // primary-beam tables of the last call with a beam
  size_t beam_bytes = 0;
  // pipelined host-buffer calls: two staging images used in turn, a copy
  // stream, and per-buffer events (copy done, compute done)
  void* pipe_img[2] = {};
  size_t pipe_img_bytes[2] = {};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t pipe_copied[2] = {}, pipe_done[2] = {};
  double* pipe_chi2 = nullptr;  // device result slots, one per staging image
  uint64_t pipe_k = 0;          // pipelined calls so far
  void* tw[2][kMaxLog2 + 1] = {};
  int gather_blocks[2][2] = {};  // [f64?][chi2?], global-memory window
  size_t smem_blocks_key[2] = {};  // window bytes the cached count below is for
  int smem_blocks[2] = {};         // chi2 gather blocks with a shared-memory window
  int aux_blocks = 0;
  uint64_t launches = 0;
  int timing = 0;  // bit s: time stage s
  std::vector<TimedStage> timed;
  std::vector<cudaEvent_t> event_pool;
  double stage_ms[kStages] = {};
  int64_t stage_n[kStages] = {};
  char last_err[256] = {0};
  // batches
  void* batch_ws = nullptr;  // per-request spectra, windows and partial sums
  size_t batch_ws_bytes = 0;
  unsigned* batch_ctr = nullptr;  // per-request last-block counters, zero at rest
  size_t batch_ctr_n = 0;
  uint64_t ws_generation = 0;  // bumped whenever a workspace is reallocated
  bool batch_tuning = true;
  std::map<std::tuple<int, int, int>, gal::BatchShape> batch_shapes;
  size_t hbm_budget = 0;  // workspace limit in bytes (0: none)
};

struct gal_data {
  gal_ctx* ctx = nullptr;  // the context it was registered on
  int device = 0;          // usable by every context on this device
  int real_bytes = 0;
  int64_t M = 0;
  const void *u = nullptr, *v = nullptr, *re = nullptr, *im = nullptr, *w = nullptr;
  double* rho2 = nullptr;  // device scalar: max(u^2 + v^2)
  double rho2_host = 0.0;  // the same value, read back once at registration
  void* uv_own = nullptr;  // arrays the handle owns: u, v in wavelengths when registered
                           // from metres, or all five when registered in Z-order
};

namespace {

int cuda_fail(gal_ctx* ctx, cudaError_t e) {
  if (ctx) snprintf(ctx->last_err, sizeof ctx->last_err, "%s", cudaGetErrorString(e));
  (void)cudaGetLastError();  // a failed call must not poison the next launch check
  return e == cudaErrorMemoryAllocation ? GAL_E_NOMEM : GAL_E_CUDA;
}

#define GAL_CUDA(ctx, call)                      \
  do {                                           \
    cudaError_t _e = (call);                     \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e); \
  } while (0)

bool pow2_size(int n) { return n >= 4 && n <= (1 << kMaxLog2) && (n & (n - 1)) == 0; }
int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// every reallocation of any context's workspace (contexts may live on
// different host threads, e.g. the server's workers)
std::atomic<uint64_t> g_ws_generation{0};

// Grow one workspace buffer to `need` bytes (contents are not kept).  Growth
// that would take the context's workspace past its HBM budget fails as an
// allocation failure would (GAL_E_NOMEM), leaving the buffer as it was.
cudaError_t grow(gal_ctx* ctx, void** p, size_t* have, size_t need) {
  if (*have >= need) return cudaSuccess;
  if (ctx->hbm_budget && gal_workspace_bytes(ctx) - *have + need > ctx->hbm_budget)
    return cudaErrorMemoryAllocation;
  ++g_ws_generation;
  if (*p) {
    cudaError_t e = cudaFree(*p);
    if (e) return e;
    *p = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(p, need);
  if (e == cudaSuccess) *have = need;
  return e;
}

template <typename T> constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }

// Workspace and twiddles for images of side nxy in precision T (full: the
// full-plane path, whose row pass keeps up to nxy columns).
template <typename T> int ensure(gal_ctx* ctx, int nxy, bool full = false) {
  using C = gal::cplx_t<T>;
  const size_t spec = (size_t)nxy * (nxy / 2 + 1) * sizeof(C);
  GAL_CUDA(ctx, grow(ctx, &ctx->F1, &ctx->F1_bytes, full ? (size_t)nxy * nxy * sizeof(C) : spec));
  GAL_CUDA(ctx, grow(ctx, &ctx->Gw, &ctx->Gw_bytes, 2 * spec));  // horizontal node pairs
  const int l = log2i(nxy);
  void*& tw = ctx->tw[prec_index<T>()][l];
  if (!tw) {
    GAL_CUDA(ctx, cudaMalloc(&tw, (size_t)nxy * sizeof(C)));
    GAL_CUDA(ctx, gal::Launch<T>::twiddles(tw, nxy, 0));
    GAL_CUDA(ctx, cudaStreamSynchronize(0));
    ctx->launches++;
  }
  return GAL_OK;
}

cudaEvent_t pool_event(gal_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void harvest(gal_ctx* ctx, size_t keep) {
  // fold the oldest timed stages (all but `keep`) into the per-stage sums
  if (ctx->timed.size() <= keep) return;
  const size_t n = ctx->timed.size() - keep;
  for (size_t i = 0; i < n; ++i) {
    TimedStage& t = ctx->timed[i];
    float ms = 0.f;
    cudaEventSynchronize(t.b);
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      ctx->stage_ms[t.stage] += ms;
      ctx->stage_n[t.stage] += 1;
    }
    ctx->event_pool.push_back(t.a);
    ctx->event_pool.push_back(t.b);
  }
  ctx->timed.erase(ctx->timed.begin(), ctx->timed.begin() + n);
}

// Launch wrapper: counts the launch and, when timing, brackets it with events.
template <typename F> int stage(gal_ctx* ctx, int id, cudaStream_t st, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  // drop a launch error left behind by an earlier, unrelated runtime call so
  // that the check after our launch reports our launch only
  (void)cudaGetLastError();
  const bool timed = (ctx->timing >> id) & 1;
  if (timed) {
    if (ctx->timed.size() > 8192) harvest(ctx, 4096);
    a = pool_event(ctx);
    b = pool_event(ctx);
    cudaEventRecord(a, st);
  }
  cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  ctx->launches++;
  if (timed) {
    cudaEventRecord(b, st);
    ctx->timed.push_back({id, a, b});
  }
  return GAL_OK;
}

#define GAL_TRY(expr)            \
  do {                           \
    int _s = (expr);             \
    if (_s != GAL_OK) return _s; \
  } while (0)

int check_geometry(int nxy, double dxy) {
  if (!pow2_size(nxy)) return GAL_E_INVAL;
  if (!(dxy > 0.0) || !std::isfinite(dxy)) return GAL_E_INVAL;
  return GAL_OK;
}

int check_profile(const void* I, int nr, double Rmin, double dR, double inc) {
  if (!I || nr < 2) return GAL_E_INVAL;
  if (!(dR > 0.0) || !std::isfinite(dR) || !std::isfinite(Rmin)) return GAL_E_INVAL;
  if (!(std::fabs(inc) < M_PI / 2)) return GAL_E_INVAL;
  return GAL_OK;
}

gal::GatherParams gather_params(int nxy, double dxy, double dRA, double dDec, double PA) {
  gal::GatherParams g;
  g.cpa = std::cos(PA);
  g.spa = std::sin(PA);
  g.S = (double)nxy * dxy;
  g.phx = dRA;
  g.phy = dDec;
  g.N = nxy;
  return g;
}

// Options of the extended calls (gal_opts): primary-beam FWHM (0: none) and
// the full-plane spectrum.
struct CallOpts {
  double pb_fwhm = 0.0;
  bool full = false;
};

int read_opts(const gal_opts* o, CallOpts* out) {
  CallOpts c;
  if (o) {
    if (!(o->pb_fwhm >= 0.0) || !std::isfinite(o->pb_fwhm)) return GAL_E_INVAL;
    if (o->full_plane != 0 && o->full_plane != 1) return GAL_E_INVAL;
    c.pb_fwhm = o->pb_fwhm;
    c.full = o->full_plane == 1;
  }
  *out = c;
  return GAL_OK;
}

// Primary-beam tables of a call into ctx->beam (*out = null without a beam).
template <typename T>
int beam_tables(gal_ctx* ctx, const CallOpts& o, int nxy, double dxy, double dRA, double dDec,
                double PA, cudaStream_t st, const T** out) {
  *out = nullptr;
  if (!(o.pb_fwhm > 0.0)) return GAL_OK;
  GAL_CUDA(ctx, grow(ctx, &ctx->beam, &ctx->beam_bytes, 2 * (size_t)nxy * sizeof(T)));
  T* tab = static_cast<T*>(ctx->beam);
  GAL_TRY(stage(ctx, 1, st, [&] {
    return gal::Launch<T>::beam_table(tab, nxy, dxy, o.pb_fwhm, dRA, dDec, PA, st);
  }));
  *out = tab;
  return GAL_OK;
}

// Everything a call of side nxy may grow, grown before it enqueues anything,
// so that a failed allocation (or the HBM budget) leaves nothing enqueued.
template <typename T> int reserve_call(gal_ctx* ctx, int nxy, const CallOpts& o) {
  GAL_TRY(ensure<T>(ctx, nxy, o.full));
  if (o.pb_fwhm > 0.0)
    GAL_CUDA(ctx, grow(ctx, &ctx->beam, &ctx->beam_bytes, 2 * (size_t)nxy * sizeof(T)));
  return GAL_OK;
}

// ---------------------------------------------------------------------------
// FFT plans.  For float images of side 32 .. kAltRadixMaxSide the row and
// column passes exist at radix 16 and at radix 8; the plan of a side says
// which one runs.  There is one plan per device, side and precision for the
// whole process, so single calls, batches, served requests and the
// allocation-free entry point compute a request with the same arithmetic
// (bitwise equal results).  A side's plan is fixed at its first use on a
// context: timed on that context's workspace and stream when its tuning is on
// and the stream is not being captured (each radix, each pass, best of three,
// the smaller radix kept only when at least 5 % faster), otherwise the
// default; gal_set_fft_radix overrides it.
// ---------------------------------------------------------------------------
namespace plans {
constexpr int kDevices = 64;
std::mutex mu;
int table[kDevices][2][kMaxLog2 + 1][2] = {};  // [device][f64?][log2 side]{row, col}; 0: unset
}  // namespace plans

template <typename T> bool plan_tunable(int nxy) {
  return sizeof(T) == 4 && nxy >= 32 && nxy <= gal::kAltRadixMaxSide;
}

// the plan of side nxy on `device` if chosen (returns false and the defaults otherwise)
template <typename T> bool plan_lookup(int device, int nxy, int* rv, int* cv) {
  *rv = *cv = gal::fft_radix_default<T>();
  if (device < 0 || device >= plans::kDevices || !plan_tunable<T>(nxy)) return true;
  std::lock_guard<std::mutex> lk(plans::mu);
  const int* e = plans::table[device][prec_index<T>()][log2i(nxy)];
  if (!e[0]) return false;
  *rv = e[0];
  *cv = e[1];
  return true;
}

template <typename T> void plan_store(int device, int nxy, int rv, int cv, bool overwrite) {
  if (device < 0 || device >= plans::kDevices || !plan_tunable<T>(nxy)) return;
  std::lock_guard<std::mutex> lk(plans::mu);
  int* e = plans::table[device][prec_index<T>()][log2i(nxy)];
  if (e[0] && !overwrite) return;  // the first choice stands
  e[0] = rv;
  e[1] = cv;
}

// Time both radices of the row and column passes of side nxy on the
// context's own workspace (its contents serve as input: only the time
// matters) with the uv extent of the whole half spectrum.
template <typename T> int tune_fft(gal_ctx* ctx, int nxy, cudaStream_t st, int* rv, int* cv) {
  GAL_TRY(ensure<T>(ctx, nxy));
  const void* tw = ctx->tw[prec_index<T>()][log2i(nxy)];
  const double big = 1e300;  // beyond any grid: nothing is pruned
  GAL_CUDA(ctx, cudaMemcpyAsync(ctx->rho2, &big, sizeof(double), cudaMemcpyHostToDevice, st));
  const T* img = static_cast<const T*>(ctx->Gw);
  const double S = 1.0;
  cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
  auto best_of = [&](auto&& launch, float* ms) -> int {
    *ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      GAL_CUDA(ctx, cudaEventRecord(a, st));
      GAL_CUDA(ctx, launch());
      ctx->launches++;
      GAL_CUDA(ctx, cudaEventRecord(b, st));
      GAL_CUDA(ctx, cudaEventSynchronize(b));
      float t = 0.f;
      GAL_CUDA(ctx, cudaEventElapsedTime(&t, a, b));
      if (rep > 0 && t < *ms) *ms = t;  // the first run warms up
    }
    return GAL_OK;
  };
  const int r0 = gal::fft_radix_default<T>(), r1 = gal::kAltRadix;
  float row[2], col[2];
  for (int k = 0; k < 2; ++k) {
    const int r = k ? r1 : r0;
    GAL_TRY(best_of([&] {
      return gal::Launch<T>::row_pass(img, nullptr, gal::SweepParams{}, nxy, tw, ctx->F1, ctx->rho2,
                                      S, ctx->err, nullptr, st, r);
    }, &row[k]));
    GAL_TRY(best_of([&] {
      return gal::Launch<T>::col_pass(ctx->F1, ctx->Gw, nxy, tw, ctx->rho2, S, 0, false, st, r);
    }, &col[k]));
  }
  ctx->event_pool.push_back(a);
  ctx->event_pool.push_back(b);
  *rv = row[1] < 0.95f * row[0] ? r1 : r0;
  *cv = col[1] < 0.95f * col[0] ? r1 : r0;
  return GAL_OK;
}

// Fix (or look up) the plan of side nxy before a call enqueues anything.
template <typename T> int fft_plan(gal_ctx* ctx, int nxy, cudaStream_t st) {
  int rv, cv;
  if (plan_lookup<T>(ctx->device, nxy, &rv, &cv)) return GAL_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GAL_CUDA(ctx, cudaStreamIsCapturing(st, &cap));
  rv = cv = gal::fft_radix_default<T>();
  if (ctx->batch_tuning && cap == cudaStreamCaptureStatusNone)
    GAL_TRY(tune_fft<T>(ctx, nxy, st, &rv, &cv));
  plan_store<T>(ctx->device, nxy, rv, cv, false);
  return GAL_OK;
}

// FFT of the image (or of the swept profile) into the pruned window ctx->Gw;
// `beam` multiplies the pixels (null: none), `full` keeps both signs of u.
template <typename T>
int spectrum(gal_ctx* ctx, const T* image, const T* I, const gal::SweepParams& sp, int nxy,
             double dxy, const double* rho2, int kc_hint, cudaStream_t st,
             const T* beam = nullptr, bool full = false) {
  GAL_TRY(ensure<T>(ctx, nxy, full));
  const void* tw = ctx->tw[prec_index<T>()][log2i(nxy)];
  const double S = (double)nxy * dxy;
  int rv, cv;
  plan_lookup<T>(ctx->device, nxy, &rv, &cv);
  GAL_TRY(stage(ctx, 1, st, [&] {
    if (full) return gal::Plane<T>::rows(image, I, sp, nxy, tw, ctx->F1, rho2, S, beam, ctx->err, st);
    return gal::Launch<T>::row_pass(image, I, sp, nxy, tw, ctx->F1, rho2, S, ctx->err, beam, st, rv);
  }));
  GAL_TRY(stage(ctx, 2, st, [&] {
    return gal::Launch<T>::col_pass(ctx->F1, ctx->Gw, nxy, tw, rho2, S, kc_hint, full, st, cv);
  }));
  return GAL_OK;
}

template <typename T>
int sample_impl(gal_ctx* ctx, const T* image, const T* I, const gal::SweepParams& sp, int nxy,
                double dxy, double dRA, double dDec, double PA, int64_t M, const T* u,
                const T* v, T* vis, cudaStream_t st,
                const gal::MultiSources* ms = nullptr, const CallOpts& o = CallOpts{}) {
  if (!ctx) return GAL_E_INVAL;
  GAL_TRY(check_geometry(nxy, dxy));
  if (o.full && (ms || !gal::Plane<T>::supported(nxy))) return GAL_E_INVAL;
  if (M < 0) return GAL_E_INVAL;
  if (M == 0) return GAL_OK;
  if (!u || !v || !vis) return GAL_E_INVAL;
  if (!aligned(u, sizeof(T)) || !aligned(v, sizeof(T)) || !aligned(vis, 2 * sizeof(T)))
    return GAL_E_INVAL;
  GAL_TRY(reserve_call<T>(ctx, nxy, o));
  GAL_TRY(fft_plan<T>(ctx, nxy, st));
  GAL_TRY(stage(ctx, 0, st, [&] {
    return gal::Launch<T>::extent(u, v, M, ctx->rho2, ctx->aux_blocks, st);
  }));
  const T* beam;
  GAL_TRY(beam_tables<T>(ctx, o, nxy, dxy, dRA, dDec, PA, st, &beam));
  GAL_TRY(spectrum<T>(ctx, image, I, sp, nxy, dxy, ctx->rho2, 0, st, beam, o.full));
  const gal::GatherParams gp = gather_params(nxy, dxy, dRA, dDec, PA);
  if (o.full) {
    const int blocks = ctx->num_sms * gal::Plane<T>::gather_blocks_per_sm(false, 0);
    return stage(ctx, 3, st, [&] {
      return gal::Plane<T>::gather(ctx->Gw, gp, ctx->rho2, u, v, nullptr, nullptr, nullptr, M,
                                   vis, nullptr, nullptr, nullptr, 0, true, blocks, st);
    });
  }
  const int blocks = ctx->gather_blocks[prec_index<T>()][0];
  return stage(ctx, 3, st, [&] {
    return gal::Launch<T>::gather(ctx->Gw, gp, ctx->rho2, u, v, nullptr, nullptr, nullptr, M,
                                  vis, nullptr, nullptr, nullptr, 0, true, blocks, ms, st);
  });
}

// Shape of the chi2 gather for a request with window `bd`: the window bytes to
// stage in shared memory (0: read from L2) and the number of blocks.  Single
// calls and batches use the same shape, so they reduce in the same order.
template <typename T> int chi2_gather_shape(gal_ctx* ctx, const gal::Bounds& bd, size_t* wbytes_out) {
  using C = gal::cplx_t<T>;
  // Stage the kept spectrum window in shared memory when it is small enough
  // (the pruned windows of long-baseline-free data usually are).
  size_t wbytes = ((size_t)bd.nrw * bd.Kc * sizeof(C) + 15) & ~size_t(15);  // bulk-copy size
  if (wbytes > kWindowSmem) wbytes = 0;
  int blocks = ctx->gather_blocks[prec_index<T>()][1];
  if (wbytes) {
    if (wbytes != ctx->smem_blocks_key[prec_index<T>()]) {
      ctx->smem_blocks_key[prec_index<T>()] = wbytes;
      ctx->smem_blocks[prec_index<T>()] =
          ctx->num_sms * gal::Launch<T>::gather_blocks_per_sm(true, wbytes);
    }
    blocks = ctx->smem_blocks[prec_index<T>()];
  }
  if (blocks > ctx->partials_len) blocks = ctx->partials_len;
  *wbytes_out = wbytes;
  return blocks;
}

template <typename T>
int chi2_impl(gal_ctx* ctx, const T* image, const T* I, const gal::SweepParams& sp, int nxy,
              double dxy, double dRA, double dDec, double PA, const gal_data* d, double* chi2,
              cudaStream_t st, const gal::MultiSources* ms = nullptr,
              const CallOpts& o = CallOpts{}) {
  if (!ctx || !d || !chi2) return GAL_E_INVAL;
  if (d->device != ctx->device || d->real_bytes != (int)sizeof(T)) return GAL_E_INVAL;
  GAL_TRY(check_geometry(nxy, dxy));
  if (o.full && (ms || !gal::Plane<T>::supported(nxy))) return GAL_E_INVAL;
  if (!aligned(chi2, sizeof(double))) return GAL_E_INVAL;
  if (d->M == 0) {
    GAL_CUDA(ctx, cudaMemsetAsync(chi2, 0, sizeof(double), st));
    return GAL_OK;
  }
  using C = gal::cplx_t<T>;
  GAL_TRY(reserve_call<T>(ctx, nxy, o));
  GAL_TRY(fft_plan<T>(ctx, nxy, st));
  const gal::Bounds bd = gal::make_bounds(d->rho2_host, (double)nxy * dxy, nxy);
  const T* beam;
  GAL_TRY(beam_tables<T>(ctx, o, nxy, dxy, dRA, dDec, PA, st, &beam));
  const gal::GatherParams gp = gather_params(nxy, dxy, dRA, dDec, PA);
  if (o.full) {
    const int W = gal::full_cols(bd, nxy).W;
    GAL_TRY(spectrum<T>(ctx, image, I, sp, nxy, dxy, d->rho2, W, st, beam, true));
    size_t wbytes = ((size_t)bd.nrw * W * sizeof(C) + 15) & ~size_t(15);  // bulk-copy size
    if (wbytes > kWindowSmem) wbytes = 0;
    int blocks = ctx->num_sms * gal::Plane<T>::gather_blocks_per_sm(true, wbytes);
    if (blocks > ctx->partials_len) blocks = ctx->partials_len;
    return stage(ctx, 3, st, [&] {
      return gal::Plane<T>::gather(ctx->Gw, gp, d->rho2, static_cast<const T*>(d->u),
                                   static_cast<const T*>(d->v), static_cast<const T*>(d->re),
                                   static_cast<const T*>(d->im), static_cast<const T*>(d->w),
                                   d->M, nullptr, ctx->partials, ctx->counter, chi2, wbytes,
                                   /*edge=*/bd.r0 == 0, blocks, st);
    });
  }
  GAL_TRY(spectrum<T>(ctx, image, I, sp, nxy, dxy, d->rho2, bd.Kc, st, beam));
  size_t wbytes;
  const int blocks = chi2_gather_shape<T>(ctx, bd, &wbytes);
  return stage(ctx, 3, st, [&] {
    return gal::Launch<T>::gather(ctx->Gw, gp, d->rho2, static_cast<const T*>(d->u),
                                  static_cast<const T*>(d->v), static_cast<const T*>(d->re),
                                  static_cast<const T*>(d->im), static_cast<const T*>(d->w), d->M,
                                  nullptr, ctx->partials, ctx->counter, chi2, wbytes,
                                  /*edge=*/bd.r0 == 0, blocks, ms, st);
  });
}

template <typename T>
int sample_image_t(gal_ctx* ctx, const T* image, int nxy, double dxy, double dRA, double dDec,
                   double PA, int64_t M, const T* u, const T* v, T* vis, void* stream,
                   const gal_opts* opts = nullptr) {
  CallOpts o;
  GAL_TRY(read_opts(opts, &o));
  if (!image || !aligned(image, 2 * sizeof(T))) return GAL_E_INVAL;
  gal::SweepParams sp{};
  return sample_impl<T>(ctx, image, nullptr, sp, nxy, dxy, dRA, dDec, PA, M, u, v, vis,
                        static_cast<cudaStream_t>(stream), nullptr, o);
}

template <typename T>
int sample_profile_t(gal_ctx* ctx, const T* I, int nr, double Rmin, double dR, int nxy, double dxy,
                     double inc, double dRA, double dDec, double PA, int64_t M, const T* u,
                     const T* v, T* vis, void* stream, const gal_opts* opts = nullptr) {
  CallOpts o;
  GAL_TRY(read_opts(opts, &o));
  GAL_TRY(check_profile(I, nr, Rmin, dR, inc));
  if (!aligned(I, sizeof(T))) return GAL_E_INVAL;
  gal::SweepParams sp{Rmin, dR, dxy, inc, nr};
  return sample_impl<T>(ctx, nullptr, I, sp, nxy, dxy, dRA, dDec, PA, M, u, v, vis,
                        static_cast<cudaStream_t>(stream), nullptr, o);
}

template <typename T>
int chi2_image_t(gal_ctx* ctx, const T* image, int nxy, double dxy, double dRA, double dDec,
                 double PA, const gal_data* d, double* chi2, void* stream,
                 const gal_opts* opts = nullptr) {
  CallOpts o;
  GAL_TRY(read_opts(opts, &o));
  if (!image || !aligned(image, 2 * sizeof(T))) return GAL_E_INVAL;
  gal::SweepParams sp{};
  return chi2_impl<T>(ctx, image, nullptr, sp, nxy, dxy, dRA, dDec, PA, d, chi2,
                      static_cast<cudaStream_t>(stream), nullptr, o);
}

template <typename T>
int chi2_profile_t(gal_ctx* ctx, const T* I, int nr, double Rmin, double dR, int nxy, double dxy,
                   double inc, double dRA, double dDec, double PA, const gal_data* d, double* chi2,
                   void* stream, const gal_opts* opts = nullptr) {
  CallOpts o;
  GAL_TRY(read_opts(opts, &o));
  GAL_TRY(check_profile(I, nr, Rmin, dR, inc));
  if (!aligned(I, sizeof(T))) return GAL_E_INVAL;
  gal::SweepParams sp{Rmin, dR, dxy, inc, nr};
  return chi2_impl<T>(ctx, nullptr, I, sp, nxy, dxy, dRA, dDec, PA, d, chi2,
                      static_cast<cudaStream_t>(stream), nullptr, o);
}

// Multi-source arguments: K in [1, 16] finite offsets and amplitudes (host).
int check_multi(int K, const double* dRA, const double* dDec, const double* amp) {
  if (K < 1 || K > 16 || !dRA || !dDec || !amp) return GAL_E_INVAL;
  for (int k = 0; k < K; ++k)
    if (!std::isfinite(dRA[k]) || !std::isfinite(dDec[k]) || !std::isfinite(amp[k]))
      return GAL_E_INVAL;
  return GAL_OK;
}

template <typename T>
int sample_image_multi_t(gal_ctx* ctx, const T* image, int nxy, double dxy, double PA, int K,
                         const double* dRA, const double* dDec, const double* amp, int64_t M,
                         const T* u, const T* v, T* vis, void* stream) {
  if (!image || !aligned(image, 2 * sizeof(T))) return GAL_E_INVAL;
  GAL_TRY(check_multi(K, dRA, dDec, amp));
  const gal::MultiSources ms{K, dRA, dDec, amp};
  gal::SweepParams sp{};
  return sample_impl<T>(ctx, image, nullptr, sp, nxy, dxy, 0.0, 0.0, PA, M, u, v, vis,
                        static_cast<cudaStream_t>(stream), &ms);
}

template <typename T>
int chi2_multi_t(gal_ctx* ctx, const T* image, const T* I, const gal::SweepParams& sp, int nxy,
                 double dxy, double PA, int K, const double* dRA, const double* dDec,
                 const double* amp, const gal_data* d, double* chi2, void* stream) {
  GAL_TRY(check_multi(K, dRA, dDec, amp));
  const gal::MultiSources ms{K, dRA, dDec, amp};
  return chi2_impl<T>(ctx, image, I, sp, nxy, dxy, 0.0, 0.0, PA, d, chi2,
                      static_cast<cudaStream_t>(stream), &ms);
}

template <typename T>
int sweep_t(gal_ctx* ctx, const T* I, int nr, double Rmin, double dR, int nxy, double dxy,
            double inc, T* img, void* stream) {
  if (!ctx || !img) return GAL_E_INVAL;
  GAL_TRY(check_geometry(nxy, dxy));
  GAL_TRY(check_profile(I, nr, Rmin, dR, inc));
  if (!aligned(I, sizeof(T)) || !aligned(img, sizeof(T))) return GAL_E_INVAL;
  gal::SweepParams sp{Rmin, dR, dxy, inc, nr};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return stage(ctx, 1, st, [&] {
    return gal::Launch<T>::sweep(I, sp, nxy, img, ctx->aux_blocks, st);
  });
}

template <typename T>
int data_create_t(gal_ctx* ctx, const T* u, const T* v, const T* re, const T* im, const T* w,
                  int64_t M, void* stream, gal_data** out) {
  if (!ctx || !out || M < 0) return GAL_E_INVAL;
  if (M > 0 && (!u || !v || !re || !im || !w)) return GAL_E_INVAL;
  for (const void* p : {(const void*)u, (const void*)v, (const void*)re, (const void*)im,
                        (const void*)w})
    if (!aligned(p, sizeof(T))) return GAL_E_INVAL;
  gal_data* d = new (std::nothrow) gal_data;
  if (!d) return GAL_E_NOMEM;
  d->ctx = ctx;
  d->device = ctx->device;
  d->real_bytes = sizeof(T);
  d->M = M;
  d->u = u;
  d->v = v;
  d->re = re;
  d->im = im;
  d->w = w;
  cudaError_t e = cudaMalloc(&d->rho2, sizeof(double));
  if (e != cudaSuccess) {
    delete d;
    return cuda_fail(ctx, e);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int s = stage(ctx, 0, st, [&] {
    return gal::Launch<T>::extent(u, v, M, d->rho2, ctx->aux_blocks, st);
  });
  if (s == GAL_OK) {
    // one read-back at registration: the host sizes the gather's shared
    // window from it (the kernels read the device copy)
    cudaError_t e2 = cudaMemcpyAsync(&d->rho2_host, d->rho2, sizeof(double),
                                     cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (e2 != cudaSuccess) s = cuda_fail(ctx, e2);
  }
  if (s != GAL_OK) {
    cudaFree(d->rho2);
    delete d;
    return s;
  }
  *out = d;
  return GAL_OK;
}

// Registration from baselines in metres and one frequency per visibility:
// u, v in wavelengths (u_m nu / c) are computed once into arrays the handle
// owns, then the observation is registered as usual.
template <typename T>
int data_create_freq_t(gal_ctx* ctx, const T* u_m, const T* v_m, const T* nu, const T* re,
                       const T* im, const T* w, int64_t M, void* stream, gal_data** out) {
  if (!ctx || !out || M < 0) return GAL_E_INVAL;
  if (M > 0 && (!u_m || !v_m || !nu)) return GAL_E_INVAL;
  for (const void* p : {(const void*)u_m, (const void*)v_m, (const void*)nu})
    if (!aligned(p, sizeof(T))) return GAL_E_INVAL;
  void* own = nullptr;
  if (M > 0) GAL_CUDA(ctx, cudaMalloc(&own, 2 * sizeof(T) * (size_t)M + 16));
  T* u = static_cast<T*>(own);
  // v starts 16-byte aligned so the gather can read both as vectors
  T* v = u ? reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(u + M) + 15) & ~uintptr_t(15))
           : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int s = GAL_OK;
  if (M > 0)
    s = stage(ctx, 0, st, [&] {
      return gal::Launch<T>::uv_from_frequency(u_m, v_m, nu, M, u, v, ctx->aux_blocks, st);
    });
  if (s == GAL_OK) s = data_create_t<T>(ctx, u, v, re, im, w, M, stream, out);
  if (s != GAL_OK) {
    if (own) cudaFree(own);
    return s;
  }
  (*out)->uv_own = own;
  return GAL_OK;
}


// Registration from copies in Z-order (gal_reorder.h): the order is computed
// on the host from u and v, the five arrays are gathered into one buffer the
// handle owns, then the copies are registered as usual.
template <typename T>
int data_create_sorted_t(gal_ctx* ctx, const T* u, const T* v, const T* re, const T* im,
                         const T* w, int64_t M, void* stream, gal_data** out) {
  if (!ctx || !out || M < 0) return GAL_E_INVAL;
  if (M > 0 && (!u || !v || !re || !im || !w)) return GAL_E_INVAL;
  for (const void* p : {(const void*)u, (const void*)v, (const void*)re, (const void*)im,
                        (const void*)w})
    if (!aligned(p, sizeof(T))) return GAL_E_INVAL;
  if (M == 0) return data_create_t<T>(ctx, u, v, re, im, w, M, stream, out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int64_t> perm;
  try {
    std::vector<T> hu((size_t)M), hv((size_t)M);
    GAL_CUDA(ctx, cudaMemcpyAsync(hu.data(), u, sizeof(T) * (size_t)M, cudaMemcpyDeviceToHost, st));
    GAL_CUDA(ctx, cudaMemcpyAsync(hv.data(), v, sizeof(T) * (size_t)M, cudaMemcpyDeviceToHost, st));
    GAL_CUDA(ctx, cudaStreamSynchronize(st));
    gal::z_order<T>(hu.data(), hv.data(), M, perm);
  } catch (const std::bad_alloc&) {
    return GAL_E_NOMEM;
  }
  // five arrays, each starting on a 256-byte boundary (16-byte vector loads)
  const size_t stride = (sizeof(T) * (size_t)M + 255) & ~size_t(255);
  void* own = nullptr;
  int64_t* dperm = nullptr;
  GAL_CUDA(ctx, cudaMalloc(&own, 5 * stride));
  cudaError_t e = cudaMalloc(&dperm, sizeof(int64_t) * (size_t)M);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dperm, perm.data(), sizeof(int64_t) * (size_t)M, cudaMemcpyHostToDevice,
                        st);
  T* o[5];
  for (int k = 0; k < 5; ++k) o[k] = reinterpret_cast<T*>(static_cast<char*>(own) + k * stride);
  const T* in[5] = {u, v, re, im, w};
  int s = e == cudaSuccess ? GAL_OK : cuda_fail(ctx, e);
  if (s == GAL_OK)
    s = stage(ctx, 0, st, [&] { return gal::permute5<T>(dperm, M, in, o, ctx->aux_blocks, st); });
  if (s == GAL_OK) {
    e = cudaStreamSynchronize(st);  // the permutation is freed below
    if (e != cudaSuccess) s = cuda_fail(ctx, e);
  }
  if (dperm) cudaFree(dperm);
  if (s == GAL_OK) s = data_create_t<T>(ctx, o[0], o[1], o[2], o[3], o[4], M, stream, out);
  if (s != GAL_OK) {
    cudaFree(own);
    return s;
  }
  (*out)->uv_own = own;
  return GAL_OK;
}

// The Z-order of host arrays u, v into perm_out (gal_z_order_*).
template <typename T> int z_order_t(const T* u, const T* v, int64_t M, int64_t* perm_out) {
  if (M < 0 || (M > 0 && (!u || !v || !perm_out))) return GAL_E_INVAL;
  try {
    std::vector<int64_t> perm;
    gal::z_order<T>(u, v, M, perm);
    if (M > 0) std::memcpy(perm_out, perm.data(), sizeof(int64_t) * (size_t)M);
  } catch (const std::bad_alloc&) {
    return GAL_E_NOMEM;
  }
  return GAL_OK;
}

template <typename T>
int chi2_image_host_t(gal_ctx* ctx, const T* image_host, int nxy, double dxy, double dRA,
                      double dDec, double PA, const gal_data* d, double* chi2_host, void* stream) {
  if (!ctx || !image_host || !chi2_host) return GAL_E_INVAL;
  GAL_TRY(check_geometry(nxy, dxy));
  const size_t bytes = (size_t)nxy * nxy * sizeof(T);
  GAL_CUDA(ctx, grow(ctx, &ctx->stage_img, &ctx->stage_img_bytes, bytes));
  GAL_TRY(reserve_call<T>(ctx, nxy, CallOpts{}));  // before the copy is enqueued
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GAL_CUDA(ctx, cudaMemcpyAsync(ctx->stage_img, image_host, bytes, cudaMemcpyHostToDevice, st));
  GAL_TRY(chi2_image_t<T>(ctx, static_cast<const T*>(ctx->stage_img), nxy, dxy, dRA, dDec, PA, d,
                          ctx->chi2_dev, stream));
  GAL_CUDA(ctx, cudaMemcpyAsync(chi2_host, ctx->chi2_dev, sizeof(double), cudaMemcpyDeviceToHost,
                                st));
  GAL_CUDA(ctx, cudaStreamSynchronize(st));
  return GAL_OK;
}

// Pipelined host-buffer chi2Image: the image goes into one of two staging
// buffers on the context's copy stream, so it overlaps the compute of the
// previous call; the compute waits for its copy, and the next copy into the
// same buffer waits for that compute.  The result is copied to *chi2_host on
// `stream`; nothing here synchronises.
template <typename T>
int chi2_image_host_async_t(gal_ctx* ctx, const T* image_host, int nxy, double dxy, double dRA,
                            double dDec, double PA, const gal_data* d, double* chi2_host,
                            void* stream) {
  if (!ctx || !image_host || !chi2_host || !d) return GAL_E_INVAL;
  GAL_TRY(check_geometry(nxy, dxy));
  if (d->device != ctx->device || d->real_bytes != (int)sizeof(T)) return GAL_E_INVAL;
  if (!aligned(chi2_host, sizeof(double))) return GAL_E_INVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ctx->copy_stream) {
    // the events and result slots first: copy_stream marks a complete set-up
    for (int s = 0; s < 2; ++s) {
      if (!ctx->pipe_copied[s])
        GAL_CUDA(ctx, cudaEventCreateWithFlags(&ctx->pipe_copied[s], cudaEventDisableTiming));
      if (!ctx->pipe_done[s])
        GAL_CUDA(ctx, cudaEventCreateWithFlags(&ctx->pipe_done[s], cudaEventDisableTiming));
    }
    if (!ctx->pipe_chi2) GAL_CUDA(ctx, cudaMalloc(&ctx->pipe_chi2, 2 * sizeof(double)));
    GAL_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  }
  const int s = (int)(ctx->pipe_k & 1);
  const size_t bytes = (size_t)nxy * nxy * sizeof(T);
  if (ctx->pipe_img_bytes[s] < bytes) {  // regrow only once the buffer's last use is done
    GAL_CUDA(ctx, cudaEventSynchronize(ctx->pipe_done[s]));
    GAL_CUDA(ctx, grow(ctx, &ctx->pipe_img[s], &ctx->pipe_img_bytes[s], bytes));
  }
  GAL_TRY(reserve_call<T>(ctx, nxy, CallOpts{}));  // before the copy is enqueued
  GAL_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->pipe_done[s], 0));
  GAL_CUDA(ctx, cudaMemcpyAsync(ctx->pipe_img[s], image_host, bytes, cudaMemcpyHostToDevice,
                                ctx->copy_stream));
  GAL_CUDA(ctx, cudaEventRecord(ctx->pipe_copied[s], ctx->copy_stream));
  GAL_CUDA(ctx, cudaStreamWaitEvent(st, ctx->pipe_copied[s], 0));
  GAL_TRY(chi2_image_t<T>(ctx, static_cast<const T*>(ctx->pipe_img[s]), nxy, dxy, dRA, dDec, PA, d,
                          ctx->pipe_chi2 + s, stream));
  GAL_CUDA(ctx, cudaMemcpyAsync(chi2_host, ctx->pipe_chi2 + s, sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  GAL_CUDA(ctx, cudaEventRecord(ctx->pipe_done[s], st));
  ctx->pipe_k++;
  return GAL_OK;
}

// Kernel attributes (dynamic shared-memory limits) are per device: set them
// once on each device a context is created on, with that device current.
constexpr int kInitDevices = 64;
std::mutex g_init_mutex;
bool g_init_done[kInitDevices] = {};

int init_current_device(int device) {
  if (device < 0 || device >= kInitDevices) return GAL_E_DEVICE;
  std::lock_guard<std::mutex> lk(g_init_mutex);
  if (g_init_done[device]) return GAL_OK;
  cudaError_t e = gal::Launch<float>::init();
  if (e == cudaSuccess) e = gal::Launch<double>::init();
  if (e != cudaSuccess) return GAL_E_DEVICE;  // e.g. no sm_103a image for this GPU
  g_init_done[device] = true;
  return GAL_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
template <typename T>
int image_size_t(gal_ctx* ctx, const T* u, const T* v, int64_t M, double PB, double f_min,
                 double f_max, int64_t* nxy_out, double* dxy_out, void* stream) {
  if (!ctx || !u || !v || !nxy_out || !dxy_out || M < 1) return GAL_E_INVAL;
  if (!aligned(u, sizeof(T)) || !aligned(v, sizeof(T))) return GAL_E_INVAL;
  if (!(f_min > 1.0) || !(f_max > 2.0) || !std::isfinite(f_min) || !std::isfinite(f_max))
    return GAL_E_INVAL;
  if (!(PB >= 0.0) || !std::isfinite(PB)) return GAL_E_INVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GAL_TRY(stage(ctx, 0, st, [&] {
    return gal::Launch<T>::uv_range(u, v, M, ctx->uvrange, ctx->aux_blocks, st);
  }));
  double r2[2];
  GAL_CUDA(ctx, cudaMemcpyAsync(r2, ctx->uvrange, sizeof r2, cudaMemcpyDeviceToHost, st));
  GAL_CUDA(ctx, cudaStreamSynchronize(st));
  if (!(r2[0] > 0.0) || !(r2[1] >= r2[0]) || !std::isfinite(r2[1])) return GAL_E_INVAL;
  const double rho_min = std::sqrt(r2[0]), rho_max = std::sqrt(r2[1]);
  constexpr double kGamma = 0.6;  // ALMA's value of the MRS constant (Sect. 3.3)
  double duv = rho_min / (kGamma * f_min);  // criterion (iia)
  if (PB > 0.0 && 1.0 / PB < duv) duv = 1.0 / PB;  // criterion (iib)
  const double need = 2.0 * f_max * rho_max / duv;  // criterion (i)
  if (!(need <= 4.611686018427388e18)) return GAL_E_RANGE;  // 2^62
  int64_t n = 1;
  while ((double)n < need) n <<= 1;
  *nxy_out = n;
  *dxy_out = 1.0 / ((double)n * duv);
  return GAL_OK;
}


namespace {

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct BatchPlan {
  std::vector<gal::BatchItem> items[2];  // per precision (0 float, 1 double)
  std::vector<int> single;               // requests run as single calls
  std::vector<int> empty;                // requests with M == 0
  int max_nxy[2] = {0, 0};
};

int check_request(gal_ctx* ctx, const gal_request& r) {
  const gal_data* d = r.data;
  if (!d || d->device != ctx->device) return GAL_E_INVAL;
  GAL_TRY(check_geometry(r.nxy, r.dxy));
  if (!std::isfinite(r.dRA) || !std::isfinite(r.dDec) || !std::isfinite(r.PA)) return GAL_E_INVAL;
  if (!(r.pb_fwhm >= 0.0) || !std::isfinite(r.pb_fwhm)) return GAL_E_INVAL;
  if (r.full_plane != 0 && r.full_plane != 1) return GAL_E_INVAL;
  const size_t rb = (size_t)d->real_bytes;
  if (r.full_plane && !(rb == 8 ? gal::Plane<double>::supported(r.nxy)
                                : gal::Plane<float>::supported(r.nxy)))
    return GAL_E_INVAL;
  if ((r.image != nullptr) == (r.intensity != nullptr)) return GAL_E_INVAL;
  if (r.image) {
    if (!aligned(r.image, 2 * rb)) return GAL_E_INVAL;
  } else {
    GAL_TRY(check_profile(r.intensity, r.nr, r.Rmin, r.dR, r.inc));
    if (!aligned(r.intensity, rb)) return GAL_E_INVAL;
  }
  return GAL_OK;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename T>
bool batchable(const gal_request& r) {
  return gal::BatchLaunch<T>::supported(r.nxy) && (!r.image || aligned(r.image, 16));
}

// Validate every request, sort them into batched / single / empty, and lay
// out (growing if needed) the batch workspace.
int plan_batch(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out, BatchPlan& pl) {
  for (int i = 0; i < n; ++i) GAL_TRY(check_request(ctx, reqs[i]));
  size_t bytes = 0;
  size_t nctr = 0;
  struct Off {
    size_t f1, gw, part, bm;
  };
  std::vector<Off> offs[2];
  for (int i = 0; i < n; ++i) {
    const gal_request& r = reqs[i];
    const gal_data* d = r.data;
    const int p = d->real_bytes == 8 ? 1 : 0;
    if (d->M == 0) {
      pl.empty.push_back(i);
      continue;
    }
    const bool ok = p ? batchable<double>(r) : batchable<float>(r);
    if (!ok) {
      pl.single.push_back(i);
      continue;
    }
    gal::BatchItem b{};
    b.image = r.image;
    b.I = r.intensity;
    b.sp = gal::SweepParams{r.Rmin, r.dR, r.dxy, r.inc, r.nr};
    b.N = r.nxy;
    b.S = (double)r.nxy * r.dxy;
    b.rho2 = d->rho2;
    const gal::Bounds bd = gal::make_bounds(d->rho2_host, b.S, r.nxy);
    b.Kc = bd.Kc;
    b.nrw = bd.nrw;
    b.gp = gather_params(r.nxy, r.dxy, r.dRA, r.dDec, r.PA);
    b.u = d->u;
    b.v = d->v;
    b.re = d->re;
    b.im = d->im;
    b.w = d->w;
    b.M = d->M;
    b.chi2_out = chi2_out + i;
    b.edge = bd.r0 == 0;
    const size_t cb = 2 * (size_t)d->real_bytes;  // complex value
    b.full = r.full_plane == 1;
    if (b.full) {  // the single full-plane call's window and gather shape
      b.ncol = gal::full_cols(bd, r.nxy).W;
      b.wbytes = round_up((size_t)bd.nrw * b.ncol * cb, 16);
      if (b.wbytes > kWindowSmem) b.wbytes = 0;
      b.grid = ctx->num_sms * (p ? gal::Plane<double>::gather_blocks_per_sm(true, b.wbytes)
                                 : gal::Plane<float>::gather_blocks_per_sm(true, b.wbytes));
      if (b.grid > ctx->partials_len) b.grid = ctx->partials_len;
    } else {
      b.ncol = bd.Kc;
      b.grid = p ? chi2_gather_shape<double>(ctx, bd, &b.wbytes)
                 : chi2_gather_shape<float>(ctx, bd, &b.wbytes);
    }
    Off o;
    o.f1 = bytes;
    bytes = round_up(bytes + (size_t)r.nxy * b.ncol * cb, 256);
    o.gw = bytes;
    bytes = round_up(bytes + round_up((size_t)bd.nrw * b.ncol * cb, 16) + 16, 256);
    o.part = bytes;
    bytes = round_up(bytes + sizeof(double) * (size_t)b.grid, 256);
    o.bm = 0;
    if (r.pb_fwhm > 0.0) {  // the request's beam tables: 2N values
      o.bm = bytes;
      bytes = round_up(bytes + 2 * (size_t)r.nxy * (size_t)d->real_bytes, 256);
      b.bp = gal::beam_params(r.pb_fwhm, r.dRA, r.dDec, r.PA);
    }
    b.counter = reinterpret_cast<unsigned*>(nctr);  // index, resolved below
    ++nctr;
    pl.items[p].push_back(b);
    offs[p].push_back(o);
    pl.max_nxy[p] = std::max(pl.max_nxy[p], r.nxy);
  }
  GAL_CUDA(ctx, grow(ctx, &ctx->batch_ws, &ctx->batch_ws_bytes, bytes));
  if (nctr > ctx->batch_ctr_n) {
    size_t have = ctx->batch_ctr_n * sizeof(unsigned);
    GAL_CUDA(ctx, grow(ctx, reinterpret_cast<void**>(&ctx->batch_ctr), &have, nctr * sizeof(unsigned)));
    GAL_CUDA(ctx, cudaMemset(ctx->batch_ctr, 0, nctr * sizeof(unsigned)));
    // the memset runs on the legacy stream, which a non-blocking stream does
    // not wait for: finish it before any launch reads the counters
    GAL_CUDA(ctx, cudaStreamSynchronize(0));
    ctx->batch_ctr_n = nctr;
  }
  char* base = static_cast<char*>(ctx->batch_ws);
  for (int p = 0; p < 2; ++p)
    for (size_t k = 0; k < pl.items[p].size(); ++k) {
      gal::BatchItem& b = pl.items[p][k];
      b.F1 = base + offs[p][k].f1;
      b.Gw = base + offs[p][k].gw;
      b.partials = reinterpret_cast<double*>(base + offs[p][k].part);
      b.beam = offs[p][k].bm ? base + offs[p][k].bm : nullptr;
      b.counter = ctx->batch_ctr + reinterpret_cast<size_t>(b.counter);
    }
  return GAL_OK;
}

template <typename T> int ensure_twiddles(gal_ctx* ctx, int nxy) {
  using C = gal::cplx_t<T>;
  void*& tw = ctx->tw[prec_index<T>()][log2i(nxy)];
  if (!tw) {
    GAL_CUDA(ctx, cudaMalloc(&tw, (size_t)nxy * sizeof(C)));
    ++g_ws_generation;
    GAL_CUDA(ctx, gal::Launch<T>::twiddles(tw, nxy, 0));
    GAL_CUDA(ctx, cudaStreamSynchronize(0));
    ctx->launches++;
  }
  return GAL_OK;
}

// Enqueue the batched passes of one precision with launch shape `sh`.
template <typename T>
int enqueue_items(gal_ctx* ctx, const std::vector<gal::BatchItem>& items,
                  const gal::BatchShape& sh, cudaStream_t st) {
  if (items.empty()) return GAL_OK;
  const void* const* tw = ctx->tw[prec_index<T>()];
  const int n = (int)items.size();
  int nl = 0;
  if (std::any_of(items.begin(), items.end(), [](const gal::BatchItem& b) { return b.beam; })) {
    GAL_TRY(stage(ctx, 1, st, [&] {
      return gal::BatchLaunch<T>::beams(items.data(), n, &nl, st);
    }));
    ctx->launches += nl - 1;
    nl = 0;
  }
  GAL_TRY(stage(ctx, 1, st, [&] {
    return gal::BatchLaunch<T>::rows(items.data(), n, tw, ctx->err, sh, &nl, st);
  }));
  ctx->launches += nl - 1;
  nl = 0;
  GAL_TRY(stage(ctx, 2, st, [&] {
    return gal::BatchLaunch<T>::cols(items.data(), n, tw, sh, &nl, st);
  }));
  ctx->launches += nl - 1;
  nl = 0;
  GAL_TRY(stage(ctx, 3, st, [&] {
    return gal::BatchLaunch<T>::gather(items.data(), n, sh, &nl, st);
  }));
  ctx->launches += nl - 1;
  return GAL_OK;
}

constexpr gal::BatchShape kDefaultShape{1, gal::kBatchJobs, gal::kGatherFold};

// Everything of a planned batch except the batched passes' shapes.
int enqueue_rest(gal_ctx* ctx, const gal_request* reqs, const BatchPlan& pl, double* chi2_out,
                 cudaStream_t st) {
  for (int i : pl.empty) GAL_CUDA(ctx, cudaMemsetAsync(chi2_out + i, 0, sizeof(double), st));
  for (int i : pl.single) {
    const gal_request& r = reqs[i];
    const gal::SweepParams sp{r.Rmin, r.dR, r.dxy, r.inc, r.nr};
    CallOpts o;
    o.pb_fwhm = r.pb_fwhm;
    o.full = r.full_plane == 1;
    if (r.data->real_bytes == 8)
      GAL_TRY(chi2_impl<double>(ctx, static_cast<const double*>(r.image),
                                static_cast<const double*>(r.intensity), sp, r.nxy, r.dxy, r.dRA,
                                r.dDec, r.PA, r.data, chi2_out + i, st, nullptr, o));
    else
      GAL_TRY(chi2_impl<float>(ctx, static_cast<const float*>(r.image),
                               static_cast<const float*>(r.intensity), sp, r.nxy, r.dxy, r.dRA,
                               r.dDec, r.PA, r.data, chi2_out + i, st, nullptr, o));
  }
  return GAL_OK;
}

// Launch shape for precision p of this plan: cached (tuned earlier or set by
// gal_set_batch_shape), or tuned now by timing candidates on the stream
// (results are identical for all of them).  Two stages: the row-pass blocks
// and requests per launch at the default gather fold, then the gather fold
// with the pair that won.
int batch_shape(gal_ctx* ctx, const BatchPlan& pl, int p, cudaStream_t st, gal::BatchShape* out) {
  *out = kDefaultShape;
  const int n = (int)pl.items[p].size();
  if (n == 0) return GAL_OK;
  const auto key = std::make_tuple(p, n, pl.max_nxy[p]);
  auto it = ctx->batch_shapes.find(key);
  if (it != ctx->batch_shapes.end()) {
    *out = it->second;
    return GAL_OK;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GAL_CUDA(ctx, cudaStreamIsCapturing(st, &cap));
  if (!ctx->batch_tuning || cap != cudaStreamCaptureStatusNone) return GAL_OK;
  constexpr int F = gal::kGatherFold;
  const gal::BatchShape stage1[] = {{1, 32, F}, {2, 32, F}, {4, 32, F},
                                    {1, 8, F},  {2, 8, F},  {4, 16, F}};
  cudaEvent_t a, b;
  GAL_CUDA(ctx, cudaEventCreate(&a));
  GAL_CUDA(ctx, cudaEventCreate(&b));
  float best = 1e30f;
  gal::BatchShape pick = kDefaultShape;
  const int saved_timing = ctx->timing;
  ctx->timing = 0;
  int status = GAL_OK;
  auto time_one = [&](const gal::BatchShape& c) {
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && status == GAL_OK; ++rep) {  // first run warms up
      cudaEventRecord(a, st);
      status = p ? enqueue_items<double>(ctx, pl.items[1], c, st)
                 : enqueue_items<float>(ctx, pl.items[0], c, st);
      cudaEventRecord(b, st);
      if (status == GAL_OK && cudaEventSynchronize(b) == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        ms = std::min(ms, t);
      }
    }
    if (status == GAL_OK && ms < best) {
      best = ms;
      pick = c;
    }
  };
  for (const auto& c : stage1) {
    if (status != GAL_OK) break;
    time_one(c);
  }
  // the gather fold matters only when a launch holds more than one request
  const int per_launch = std::min(n, pick.jobs_per_launch);
  if (per_launch > 1) {
    const gal::BatchShape pair = pick;
    for (int fold : {1, 2, 8}) {
      if (status != GAL_OK) break;
      if (fold > per_launch && fold != 1) continue;  // same launch as min(n, fold)
      time_one(gal::BatchShape{pair.row_blocks, pair.jobs_per_launch, fold});
    }
  }
  ctx->timing = saved_timing;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (status != GAL_OK) return status;
  ctx->batch_shapes[key] = pick;
  *out = pick;
  return GAL_OK;
}

int run_batch(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out, cudaStream_t st,
              bool allow_setup) {
  BatchPlan pl;
  GAL_TRY(plan_batch(ctx, reqs, n, chi2_out, pl));
  if (allow_setup) {
    for (const auto& b : pl.items[0]) GAL_TRY(ensure_twiddles<float>(ctx, b.N));
    for (const auto& b : pl.items[1]) GAL_TRY(ensure_twiddles<double>(ctx, b.N));
    for (const auto& b : pl.items[0]) GAL_TRY(fft_plan<float>(ctx, b.N, st));
  }
  // every request runs with the FFT plan of its side (the same as a single call's)
  for (auto& b : pl.items[0]) plan_lookup<float>(ctx->device, b.N, &b.radix_row, &b.radix_col);
  for (auto& b : pl.items[1]) plan_lookup<double>(ctx->device, b.N, &b.radix_row, &b.radix_col);
  gal::BatchShape sh[2];
  for (int p = 0; p < 2; ++p) GAL_TRY(batch_shape(ctx, pl, p, st, &sh[p]));
  GAL_TRY(enqueue_items<float>(ctx, pl.items[0], sh[0], st));
  GAL_TRY(enqueue_items<double>(ctx, pl.items[1], sh[1], st));
  return enqueue_rest(ctx, reqs, pl, chi2_out, st);
}

}  // namespace

struct gal_graph {
  gal_ctx* ctx = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<gal_request> reqs;
  double* chi2_out = nullptr;
  uint64_t generation = 0;  // workspace generation the graph was recorded against
  uint64_t launches = 0;    // kernels per replay
};

namespace {

// Record the batch into a new graph (nothing runs).  The workspace and
// twiddles must already exist (a preceding run_batch on the same requests).
int record_batch(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out, cudaGraph_t* g,
                 uint64_t* launches) {
  cudaStream_t cs;
  GAL_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const int saved_timing = ctx->timing;
  ctx->timing = 0;
  const uint64_t l0 = ctx->launches;
  const uint64_t gen0 = g_ws_generation;
  int s = GAL_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s = run_batch(ctx, reqs, n, chi2_out, cs, false);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (s == GAL_OK && e == cudaSuccess && g_ws_generation != gen0) s = GAL_E_INVAL;
    if (s == GAL_OK && e == cudaSuccess) {
      *g = graph;
    } else if (graph) {
      cudaGraphDestroy(graph);
    }
  }
  *launches = ctx->launches - l0;
  ctx->launches = l0;
  ctx->timing = saved_timing;
  cudaStreamDestroy(cs);
  if (s != GAL_OK) return s;
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  return GAL_OK;
}

bool same_structure(const std::vector<gal_request>& a, const gal_request* b, int n) {
  if ((int)a.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (a[i].data != b[i].data || a[i].nxy != b[i].nxy ||
        (a[i].image == nullptr) != (b[i].image == nullptr) ||
        (a[i].pb_fwhm > 0.0) != (b[i].pb_fwhm > 0.0) || a[i].full_plane != b[i].full_plane)
      return false;
  return true;
}

int graph_record_into(gal_graph* gr, const gal_request* reqs, int n, double* chi2_out) {
  gal_ctx* ctx = gr->ctx;
  cudaGraph_t g = nullptr;
  uint64_t nl = 0;
  GAL_TRY(record_batch(ctx, reqs, n, chi2_out, &g, &nl));
  cudaError_t e = cudaSuccess;
  if (gr->exec) {
    cudaGraphExecUpdateResultInfo info;
    e = cudaGraphExecUpdate(gr->exec, g, &info);
    if (e != cudaSuccess) {  // topology changed: instantiate afresh
      (void)cudaGetLastError();
      cudaGraphExecDestroy(gr->exec);
      gr->exec = nullptr;
    }
  }
  if (!gr->exec) e = cudaGraphInstantiate(&gr->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  gr->reqs.assign(reqs, reqs + n);
  gr->chi2_out = chi2_out;
  gr->generation = g_ws_generation;
  gr->launches = nl;
  return GAL_OK;
}

}  // namespace

extern "C" {

const char* gal_strerror(int s) {
  switch (s) {
    case GAL_OK: return "ok";
    case GAL_E_INVAL: return "invalid argument";
    case GAL_E_NOMEM: return "device allocation failed";
    case GAL_E_CUDA: return "CUDA error";
    case GAL_E_RANGE: return "internal index check tripped";
    case GAL_E_DEVICE: return "no usable CUDA device";
    case GAL_E_BUSY: return "queue full or request not finished";
    case GAL_E_TIMEOUT: return "wait timed out";
    default: return "unknown status";
  }
}

int gal_create(gal_ctx** out, int device) {
  if (!out) return GAL_E_INVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GAL_E_DEVICE;
  if (cudaSetDevice(device) != cudaSuccess) return GAL_E_DEVICE;
  if (const int st = init_current_device(device); st != GAL_OK) return st;
  gal_ctx* ctx = new (std::nothrow) gal_ctx;
  if (!ctx) return GAL_E_NOMEM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  ctx->gather_blocks[0][0] = ctx->num_sms * gal::Launch<float>::gather_blocks_per_sm(false, 0);
  ctx->gather_blocks[0][1] = ctx->num_sms * gal::Launch<float>::gather_blocks_per_sm(true, 0);
  ctx->gather_blocks[1][0] = ctx->num_sms * gal::Launch<double>::gather_blocks_per_sm(false, 0);
  ctx->gather_blocks[1][1] = ctx->num_sms * gal::Launch<double>::gather_blocks_per_sm(true, 0);
  ctx->aux_blocks = ctx->num_sms * 8;
  int maxb = 0;
  for (auto& a : ctx->gather_blocks)
    for (int b : a) maxb = b > maxb ? b : maxb;
  ctx->partials_len = maxb;
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMalloc(&ctx->partials, sizeof(double) * (size_t)maxb);
  if (!e) e = cudaMalloc(&ctx->counter, sizeof(unsigned));
  if (!e) e = cudaMalloc(&ctx->rho2, sizeof(double));
  if (!e) e = cudaMalloc(&ctx->uvrange, 2 * sizeof(double));
  if (!e) e = cudaMalloc(&ctx->err, sizeof(int));
  if (!e) e = cudaMalloc(&ctx->chi2_dev, sizeof(double));
  if (!e) e = cudaMemset(ctx->counter, 0, sizeof(unsigned));
  if (!e) e = cudaMemset(ctx->err, 0, sizeof(int));
  if (!e) e = cudaDeviceSynchronize();
  if (e) {
    int s = cuda_fail(ctx, e);
    gal_destroy(ctx);
    return s;
  }
  *out = ctx;
  return GAL_OK;
}

void gal_destroy(gal_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (void* p : {ctx->F1, ctx->Gw, (void*)ctx->partials, (void*)ctx->counter, (void*)ctx->rho2,
                  (void*)ctx->uvrange, ctx->batch_ws, (void*)ctx->batch_ctr,
                  (void*)ctx->err, (void*)ctx->chi2_dev, ctx->stage_img, ctx->beam,
                  ctx->pipe_img[0], ctx->pipe_img[1], (void*)ctx->pipe_chi2})
    if (p) cudaFree(p);
  for (cudaEvent_t e : {ctx->pipe_copied[0], ctx->pipe_copied[1], ctx->pipe_done[0],
                        ctx->pipe_done[1]})
    if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (auto& a : ctx->tw)
    for (void* p : a)
      if (p) cudaFree(p);
  for (auto& t : ctx->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
}

int gal_reserve(gal_ctx* ctx, int nxy, int real_bytes) {
  if (!ctx || !pow2_size(nxy)) return GAL_E_INVAL;
  if (real_bytes == 4) return ensure<float>(ctx, nxy);
  if (real_bytes == 8) return ensure<double>(ctx, nxy);
  return GAL_E_INVAL;
}

const char* gal_last_cuda_error(const gal_ctx* ctx) { return ctx ? ctx->last_err : ""; }

int gal_check(gal_ctx* ctx) {
  if (!ctx) return GAL_E_INVAL;
  GAL_CUDA(ctx, cudaDeviceSynchronize());
  int flag = 0;
  GAL_CUDA(ctx, cudaMemcpy(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost));
  GAL_CUDA(ctx, cudaMemset(ctx->err, 0, sizeof(int)));
  GAL_CUDA(ctx, cudaStreamSynchronize(0));  // cleared before any later launch
  return flag ? GAL_E_RANGE : GAL_OK;
}

uint64_t gal_launch_count(const gal_ctx* ctx) { return ctx ? ctx->launches : 0; }

int gal_set_stage_timing(gal_ctx* ctx, int stage_mask) {
  if (!ctx || stage_mask < 0 || stage_mask > GAL_STAGE_ALL) return GAL_E_INVAL;
  harvest(ctx, 0);
  ctx->timing = stage_mask;
  for (int s = 0; s < kStages; ++s) {
    ctx->stage_ms[s] = 0.0;
    ctx->stage_n[s] = 0;
  }
  return GAL_OK;
}

int gal_stage_times(gal_ctx* ctx, double* ms_out4, int64_t* count_out4) {
  if (!ctx) return GAL_E_INVAL;
  harvest(ctx, 0);
  for (int s = 0; s < kStages; ++s) {
    if (ms_out4) ms_out4[s] = ctx->stage_ms[s];
    if (count_out4) count_out4[s] = ctx->stage_n[s];
  }
  return GAL_OK;
}

size_t gal_workspace_bytes(const gal_ctx* ctx) {
  if (!ctx) return 0;
  size_t b = ctx->F1_bytes + ctx->Gw_bytes + ctx->batch_ws_bytes + ctx->stage_img_bytes +
             ctx->batch_ctr_n * sizeof(unsigned) + sizeof(double) * (size_t)ctx->partials_len +
             ctx->beam_bytes + ctx->pipe_img_bytes[0] + ctx->pipe_img_bytes[1] +
             (ctx->pipe_chi2 ? 2 * sizeof(double) : 0);
  for (int p = 0; p < 2; ++p)
    for (int l = 0; l <= kMaxLog2; ++l)
      if (ctx->tw[p][l]) b += ((size_t)1 << l) * (p ? 16 : 8);
  return b;
}

int gal_device(const gal_ctx* ctx) { return ctx ? ctx->device : -1; }

int gal_set_hbm_budget(gal_ctx* ctx, size_t bytes) {
  if (!ctx) return GAL_E_INVAL;
  ctx->hbm_budget = bytes;
  return GAL_OK;
}

int gal_chi2_batch(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out, void* stream) {
  if (!ctx || n < 0 || (n > 0 && (!reqs || !chi2_out))) return GAL_E_INVAL;
  if (n == 0) return GAL_OK;
  if (!aligned(chi2_out, sizeof(double))) return GAL_E_INVAL;
  return run_batch(ctx, reqs, n, chi2_out, static_cast<cudaStream_t>(stream), true);
}

int gal_set_batch_tuning(gal_ctx* ctx, int enable) {
  if (!ctx) return GAL_E_INVAL;
  ctx->batch_tuning = enable != 0;
  return GAL_OK;
}

int gal_set_batch_shape(gal_ctx* ctx, int real_bytes, int n, int max_nxy, int row_blocks,
                        int jobs_per_launch, int gather_fold) {
  if (!ctx || (real_bytes != 4 && real_bytes != 8) || n < 1 || !pow2_size(max_nxy))
    return GAL_E_INVAL;
  if (row_blocks < 1 || row_blocks > 8 || jobs_per_launch < 1 ||
      jobs_per_launch > gal::kBatchJobs || gather_fold < 1 || gather_fold > gal::kMaxGatherFold)
    return GAL_E_INVAL;
  ctx->batch_shapes[std::make_tuple(real_bytes == 8 ? 1 : 0, n, max_nxy)] =
      gal::BatchShape{row_blocks, jobs_per_launch, gather_fold};
  return GAL_OK;
}

int gal_get_batch_shape(const gal_ctx* ctx, int real_bytes, int n, int max_nxy, int* shape_out3,
                        int* cached) {
  if (!ctx || !shape_out3 || (real_bytes != 4 && real_bytes != 8) || n < 1 || max_nxy < 1)
    return GAL_E_INVAL;
  gal::BatchShape sh = kDefaultShape;
  auto it = ctx->batch_shapes.find(std::make_tuple(real_bytes == 8 ? 1 : 0, n, max_nxy));
  const bool have = it != ctx->batch_shapes.end();
  if (have) sh = it->second;
  shape_out3[0] = sh.row_blocks;
  shape_out3[1] = sh.jobs_per_launch;
  shape_out3[2] = sh.gather_fold;
  if (cached) *cached = have ? 1 : 0;
  return GAL_OK;
}

int gal_set_fft_radix(int device, int real_bytes, int nxy, int row_radix, int col_radix) {
  if (device < 0 || device >= plans::kDevices || !pow2_size(nxy)) return GAL_E_INVAL;
  auto ok = [](int r, int dflt, bool alt) { return r == dflt || (alt && r == gal::kAltRadix); };
  if (real_bytes == 4) {
    const bool alt = plan_tunable<float>(nxy);
    if (!ok(row_radix, 16, alt) || !ok(col_radix, 16, alt)) return GAL_E_INVAL;
    plan_store<float>(device, nxy, row_radix, col_radix, true);
    return GAL_OK;
  }
  if (real_bytes == 8) return row_radix == 8 && col_radix == 8 ? GAL_OK : GAL_E_INVAL;
  return GAL_E_INVAL;
}

int gal_get_fft_radix(int device, int real_bytes, int nxy, int* row_radix, int* col_radix) {
  if (!row_radix || !col_radix || device < 0 || device >= plans::kDevices || !pow2_size(nxy))
    return GAL_E_INVAL;
  bool set;
  if (real_bytes == 4) set = plan_lookup<float>(device, nxy, row_radix, col_radix);
  else if (real_bytes == 8) set = plan_lookup<double>(device, nxy, row_radix, col_radix);
  else return GAL_E_INVAL;
  if (!set) *row_radix = *col_radix = 0;
  return GAL_OK;
}

int gal_chi2_batch_capture(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out,
                           void* stream, gal_graph** out) {
  if (!out) return GAL_E_INVAL;
  *out = nullptr;
  if (!ctx || n < 1 || !reqs || !chi2_out || !aligned(chi2_out, sizeof(double)))
    return GAL_E_INVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one ordinary run: workspace, twiddles and launch shapes are set up here
  GAL_TRY(run_batch(ctx, reqs, n, chi2_out, st, true));
  GAL_CUDA(ctx, cudaStreamSynchronize(st));
  gal_graph* g = new (std::nothrow) gal_graph;
  if (!g) return GAL_E_NOMEM;
  g->ctx = ctx;
  const int s = graph_record_into(g, reqs, n, chi2_out);
  if (s != GAL_OK) {
    gal_graph_destroy(g);
    return s;
  }
  *out = g;
  return GAL_OK;
}

int gal_graph_update(gal_graph* g, const gal_request* reqs, int n, double* chi2_out) {
  if (!g || !reqs || !chi2_out || !aligned(chi2_out, sizeof(double))) return GAL_E_INVAL;
  if (!same_structure(g->reqs, reqs, n)) return GAL_E_INVAL;
  for (int i = 0; i < n; ++i) GAL_TRY(check_request(g->ctx, reqs[i]));
  return graph_record_into(g, reqs, n, chi2_out);
}

int gal_graph_launch(gal_graph* g, void* stream) {
  if (!g || !g->exec) return GAL_E_INVAL;
  gal_ctx* ctx = g->ctx;
  if (g->generation != g_ws_generation) {
    // a workspace the graph points into was reallocated since it was recorded:
    // set the batch up again (allocations happen here, outside any capture)
    // and re-record it
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchPlan pl;
    GAL_TRY(plan_batch(ctx, g->reqs.data(), (int)g->reqs.size(), g->chi2_out, pl));
    for (const auto& b : pl.items[0]) GAL_TRY(ensure_twiddles<float>(ctx, b.N));
    for (const auto& b : pl.items[1]) GAL_TRY(ensure_twiddles<double>(ctx, b.N));
    for (int i : pl.single) {
      const gal_request& r = g->reqs[i];
      GAL_TRY(r.data->real_bytes == 8 ? ensure<double>(ctx, r.nxy) : ensure<float>(ctx, r.nxy));
    }
    GAL_CUDA(ctx, cudaStreamSynchronize(st));
    const std::vector<gal_request> reqs = g->reqs;
    GAL_TRY(graph_record_into(g, reqs.data(), (int)reqs.size(), g->chi2_out));
  }
  GAL_CUDA(ctx, cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  ctx->launches += g->launches;
  return GAL_OK;
}

void gal_graph_destroy(gal_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

int gal_get_image_size_f32(gal_ctx* ctx, const float* u, const float* v, int64_t M, double PB,
                           double f_min, double f_max, int64_t* nxy_out, double* dxy_out,
                           void* stream) {
  return image_size_t<float>(ctx, u, v, M, PB, f_min, f_max, nxy_out, dxy_out, stream);
}
int gal_get_image_size_f64(gal_ctx* ctx, const double* u, const double* v, int64_t M, double PB,
                           double f_min, double f_max, int64_t* nxy_out, double* dxy_out,
                           void* stream) {
  return image_size_t<double>(ctx, u, v, M, PB, f_min, f_max, nxy_out, dxy_out, stream);
}

int gal_data_create_f32(gal_ctx* ctx, const float* u, const float* v, const float* re,
                        const float* im, const float* w, int64_t M, void* stream, gal_data** out) {
  return data_create_t<float>(ctx, u, v, re, im, w, M, stream, out);
}
int gal_data_create_f64(gal_ctx* ctx, const double* u, const double* v, const double* re,
                        const double* im, const double* w, int64_t M, void* stream,
                        gal_data** out) {
  return data_create_t<double>(ctx, u, v, re, im, w, M, stream, out);
}
int gal_data_create_sorted_f32(gal_ctx* ctx, const float* u, const float* v, const float* re,
                               const float* im, const float* w, int64_t M, void* stream,
                               gal_data** out) {
  return data_create_sorted_t<float>(ctx, u, v, re, im, w, M, stream, out);
}
int gal_data_create_sorted_f64(gal_ctx* ctx, const double* u, const double* v, const double* re,
                               const double* im, const double* w, int64_t M, void* stream,
                               gal_data** out) {
  return data_create_sorted_t<double>(ctx, u, v, re, im, w, M, stream, out);
}
int gal_z_order_f32(const float* u, const float* v, int64_t M, int64_t* perm_out) {
  return z_order_t<float>(u, v, M, perm_out);
}
int gal_z_order_f64(const double* u, const double* v, int64_t M, int64_t* perm_out) {
  return z_order_t<double>(u, v, M, perm_out);
}
int gal_data_create_freq_f32(gal_ctx* ctx, const float* u_m, const float* v_m, const float* nu,
                             const float* re, const float* im, const float* w, int64_t M,
                             void* stream, gal_data** out) {
  return data_create_freq_t<float>(ctx, u_m, v_m, nu, re, im, w, M, stream, out);
}
int gal_data_create_freq_f64(gal_ctx* ctx, const double* u_m, const double* v_m,
                             const double* nu, const double* re, const double* im,
                             const double* w, int64_t M, void* stream, gal_data** out) {
  return data_create_freq_t<double>(ctx, u_m, v_m, nu, re, im, w, M, stream, out);
}

int gal_sample_image_multi_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double PA,
                               int K, const double* dRA, const double* dDec, const double* amp,
                               int64_t M, const float* u, const float* v, float* vis_out,
                               void* stream) {
  return sample_image_multi_t<float>(ctx, image, nxy, dxy, PA, K, dRA, dDec, amp, M, u, v,
                                     vis_out, stream);
}
int gal_sample_image_multi_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double PA,
                               int K, const double* dRA, const double* dDec, const double* amp,
                               int64_t M, const double* u, const double* v, double* vis_out,
                               void* stream) {
  return sample_image_multi_t<double>(ctx, image, nxy, dxy, PA, K, dRA, dDec, amp, M, u, v,
                                      vis_out, stream);
}
int gal_chi2_image_multi_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double PA,
                             int K, const double* dRA, const double* dDec, const double* amp,
                             const gal_data* data, double* chi2_out, void* stream) {
  if (!image || !aligned(image, 8)) return GAL_E_INVAL;
  return chi2_multi_t<float>(ctx, image, nullptr, gal::SweepParams{}, nxy, dxy, PA, K, dRA, dDec,
                             amp, data, chi2_out, stream);
}
int gal_chi2_image_multi_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double PA,
                             int K, const double* dRA, const double* dDec, const double* amp,
                             const gal_data* data, double* chi2_out, void* stream) {
  if (!image || !aligned(image, 16)) return GAL_E_INVAL;
  return chi2_multi_t<double>(ctx, image, nullptr, gal::SweepParams{}, nxy, dxy, PA, K, dRA,
                              dDec, amp, data, chi2_out, stream);
}
int gal_chi2_profile_multi_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR,
                               int nxy, double dxy, double inc, double PA, int K,
                               const double* dRA, const double* dDec, const double* amp,
                               const gal_data* data, double* chi2_out, void* stream) {
  GAL_TRY(check_profile(I, nr, Rmin, dR, inc));
  if (!aligned(I, sizeof(float))) return GAL_E_INVAL;
  return chi2_multi_t<float>(ctx, nullptr, I, gal::SweepParams{Rmin, dR, dxy, inc, nr}, nxy, dxy,
                             PA, K, dRA, dDec, amp, data, chi2_out, stream);
}
int gal_chi2_profile_multi_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR,
                               int nxy, double dxy, double inc, double PA, int K,
                               const double* dRA, const double* dDec, const double* amp,
                               const gal_data* data, double* chi2_out, void* stream) {
  GAL_TRY(check_profile(I, nr, Rmin, dR, inc));
  if (!aligned(I, sizeof(double))) return GAL_E_INVAL;
  return chi2_multi_t<double>(ctx, nullptr, I, gal::SweepParams{Rmin, dR, dxy, inc, nr}, nxy,
                              dxy, PA, K, dRA, dDec, amp, data, chi2_out, stream);
}

int gal_data_info(const gal_data* d, int64_t* M_out, int* real_bytes_out) {
  if (!d) return GAL_E_INVAL;
  if (M_out) *M_out = d->M;
  if (real_bytes_out) *real_bytes_out = d->real_bytes;
  return GAL_OK;
}

void gal_data_destroy(gal_data* d) {
  if (!d) return;
  cudaDeviceSynchronize();
  if (d->rho2) cudaFree(d->rho2);
  if (d->uv_own) cudaFree(d->uv_own);
  delete d;
}

int gal_sweep_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                  double dxy, double inc, float* image_out, void* stream) {
  return sweep_t<float>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, image_out, stream);
}
int gal_sweep_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                  double dxy, double inc, double* image_out, void* stream) {
  return sweep_t<double>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, image_out, stream);
}

int gal_sample_image_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                         double dDec, double PA, int64_t M, const float* u, const float* v,
                         float* vis_out, void* stream) {
  return sample_image_t<float>(ctx, image, nxy, dxy, dRA, dDec, PA, M, u, v, vis_out, stream);
}
int gal_sample_image_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                         double dDec, double PA, int64_t M, const double* u, const double* v,
                         double* vis_out, void* stream) {
  return sample_image_t<double>(ctx, image, nxy, dxy, dRA, dDec, PA, M, u, v, vis_out, stream);
}

int gal_sample_profile_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                           double dxy, double inc, double dRA, double dDec, double PA, int64_t M,
                           const float* u, const float* v, float* vis_out, void* stream) {
  return sample_profile_t<float>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, M, u, v,
                                 vis_out, stream);
}
int gal_sample_profile_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                           double dxy, double inc, double dRA, double dDec, double PA, int64_t M,
                           const double* u, const double* v, double* vis_out, void* stream) {
  return sample_profile_t<double>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, M, u, v,
                                  vis_out, stream);
}

int gal_chi2_image_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                       double dDec, double PA, const gal_data* data, double* chi2_out,
                       void* stream) {
  return chi2_image_t<float>(ctx, image, nxy, dxy, dRA, dDec, PA, data, chi2_out, stream);
}
int gal_chi2_image_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                       double dDec, double PA, const gal_data* data, double* chi2_out,
                       void* stream) {
  return chi2_image_t<double>(ctx, image, nxy, dxy, dRA, dDec, PA, data, chi2_out, stream);
}

int gal_chi2_profile_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                         double dxy, double inc, double dRA, double dDec, double PA,
                         const gal_data* data, double* chi2_out, void* stream) {
  return chi2_profile_t<float>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, data,
                               chi2_out, stream);
}
int gal_chi2_profile_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                         double dxy, double inc, double dRA, double dDec, double PA,
                         const gal_data* data, double* chi2_out, void* stream) {
  return chi2_profile_t<double>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, data,
                                chi2_out, stream);
}

int gal_sample_image_ex_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                            double dDec, double PA, const gal_opts* opts, int64_t M,
                            const float* u, const float* v, float* vis_out, void* stream) {
  return sample_image_t<float>(ctx, image, nxy, dxy, dRA, dDec, PA, M, u, v, vis_out, stream,
                               opts);
}
int gal_sample_image_ex_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                            double dDec, double PA, const gal_opts* opts, int64_t M,
                            const double* u, const double* v, double* vis_out, void* stream) {
  return sample_image_t<double>(ctx, image, nxy, dxy, dRA, dDec, PA, M, u, v, vis_out, stream,
                                opts);
}
int gal_sample_profile_ex_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR,
                              int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                              const gal_opts* opts, int64_t M, const float* u, const float* v,
                              float* vis_out, void* stream) {
  return sample_profile_t<float>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, M, u, v,
                                 vis_out, stream, opts);
}
int gal_sample_profile_ex_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR,
                              int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                              const gal_opts* opts, int64_t M, const double* u, const double* v,
                              double* vis_out, void* stream) {
  return sample_profile_t<double>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, M, u, v,
                                  vis_out, stream, opts);
}
int gal_chi2_image_ex_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                          double dDec, double PA, const gal_opts* opts, const gal_data* data,
                          double* chi2_out, void* stream) {
  return chi2_image_t<float>(ctx, image, nxy, dxy, dRA, dDec, PA, data, chi2_out, stream, opts);
}
int gal_chi2_image_ex_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                          double dDec, double PA, const gal_opts* opts, const gal_data* data,
                          double* chi2_out, void* stream) {
  return chi2_image_t<double>(ctx, image, nxy, dxy, dRA, dDec, PA, data, chi2_out, stream, opts);
}
int gal_chi2_profile_ex_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                            double dxy, double inc, double dRA, double dDec, double PA,
                            const gal_opts* opts, const gal_data* data, double* chi2_out,
                            void* stream) {
  return chi2_profile_t<float>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, data,
                               chi2_out, stream, opts);
}
int gal_chi2_profile_ex_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                            double dxy, double inc, double dRA, double dDec, double PA,
                            const gal_opts* opts, const gal_data* data, double* chi2_out,
                            void* stream) {
  return chi2_profile_t<double>(ctx, I, nr, Rmin, dR, nxy, dxy, inc, dRA, dDec, PA, data,
                                chi2_out, stream, opts);
}

int gal_chi2_image_host_async_f32(gal_ctx* ctx, const float* image_host, int nxy, double dxy,
                                  double dRA, double dDec, double PA, const gal_data* data,
                                  double* chi2_host, void* stream) {
  return chi2_image_host_async_t<float>(ctx, image_host, nxy, dxy, dRA, dDec, PA, data, chi2_host,
                                        stream);
}
int gal_chi2_image_host_async_f64(gal_ctx* ctx, const double* image_host, int nxy, double dxy,
                                  double dRA, double dDec, double PA, const gal_data* data,
                                  double* chi2_host, void* stream) {
  return chi2_image_host_async_t<double>(ctx, image_host, nxy, dxy, dRA, dDec, PA, data, chi2_host,
                                         stream);
}

int gal_chi2_image_host_f32(gal_ctx* ctx, const float* image_host, int nxy, double dxy,
                            double dRA, double dDec, double PA, const gal_data* data,
                            double* chi2_host, void* stream) {
  return chi2_image_host_t<float>(ctx, image_host, nxy, dxy, dRA, dDec, PA, data, chi2_host,
                                  stream);
}
int gal_chi2_image_host_f64(gal_ctx* ctx, const double* image_host, int nxy, double dxy,
                            double dRA, double dDec, double PA, const gal_data* data,
                            double* chi2_host, void* stream) {
  return chi2_image_host_t<double>(ctx, image_host, nxy, dxy, dRA, dDec, PA, data, chi2_host,
                                   stream);
}

}  // extern "C"

namespace gal {
void fft_plan_lookup_f32(int device, int nxy, int* rv, int* cv) {
  plan_lookup<float>(device, nxy, rv, cv);
}
}  // namespace gal
