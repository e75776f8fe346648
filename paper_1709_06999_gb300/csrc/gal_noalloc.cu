// Allocation-free chi-square of a model image (float32), for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host application whose own memory
// manager has already reserved the GPU's memory, a plug-in that is not allowed
// to grow the process's device footprint, or a latency-critical loop in which
// an allocation's implicit device synchronisation is unacceptable.  This entry
// point serves them: it runs the same kernels as gal_chi2_image_f32, but its
// scratch (twiddle table, spectrum buffers, reduction partials and counters)
// lives in one file-scope device array of fixed size.  The array exists on
// every GPU that loads the library, for as long as the library stays loaded.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/galario_gb300.h"
#include "gal_common.cuh"
#include "gal_internal.h"

namespace {

constexpr int kMaxN = GAL_NOALLOC_MAX_NXY;                         // largest image side
constexpr size_t kSpecElems = (size_t)kMaxN * (kMaxN / 2 + 1);     // half spectrum, complex
constexpr int kMaxBlocks = 8192;                                  // reduction partials
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffTw = 0;
constexpr size_t kOffF1 = kOffTw + align256(sizeof(float2) * kMaxN);
constexpr size_t kOffGw = kOffF1 + align256(sizeof(float2) * kSpecElems);
constexpr size_t kOffPartials = kOffGw + align256(2 * sizeof(float2) * kSpecElems);
constexpr size_t kOffRho2 = kOffPartials + align256(sizeof(double) * kMaxBlocks);
constexpr size_t kOffCounter = kOffRho2 + 256;
constexpr size_t kOffErr = kOffCounter + 256;
constexpr size_t kScratchBytes = kOffErr + 256;

// The scratch.  In host code this name is only a stand-in for the device
// array, never a usable address: the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  int gather_blocks = 0;
  int aux_blocks = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: resolve the array's device
// address and the launch shapes.  No allocation happens here.
int setup_current_device(DeviceSetup** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GAL_E_DEVICE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GAL_E_DEVICE;
    if (gal::Launch<float>::init() != cudaSuccess) return GAL_E_DEVICE;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return GAL_E_DEVICE;
    int blocks = sms * gal::Launch<float>::gather_blocks_per_sm(true, 0);
    s.gather_blocks = blocks < kMaxBlocks ? blocks : kMaxBlocks;
    s.aux_blocks = sms * 8;
    s.base = static_cast<unsigned char*>(p);
  }
  *out = &s;
  return GAL_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }


// After the gather: a bounded wait of the row pass that gave up (the error
// word is non-zero) left the spectrum incomplete, so the result is replaced by
// NaN.  With no context there is no gal_check to report it; the NaN does.
__global__ void noalloc_status_kernel(const int* __restrict__ err, double* __restrict__ chi2_out) {
  if (*err != 0) *chi2_out = __longlong_as_double(0x7ff8000000000000ll);
}

}  // namespace

extern "C" int gal_chi2_image_noalloc_f32(const float* image, int nxy, double dxy, double dRA,
                                          double dDec, double PA, const float* u, const float* v,
                                          const float* re, const float* im, const float* w,
                                          int64_t M, double* chi2_out, void* stream) {
  if (!image || !chi2_out || M < 0) return GAL_E_INVAL;
  if (nxy < 4 || nxy > kMaxN || (nxy & (nxy - 1))) return GAL_E_INVAL;  // beyond the scratch
  if (!(dxy > 0.0) || !std::isfinite(dxy)) return GAL_E_INVAL;
  if (M > 0 && (!u || !v || !re || !im || !w)) return GAL_E_INVAL;
  if (!aligned(image, 8) || !aligned(chi2_out, 8)) return GAL_E_INVAL;
  for (const void* p : {(const void*)u, (const void*)v, (const void*)re, (const void*)im,
                        (const void*)w})
    if (!aligned(p, 4)) return GAL_E_INVAL;

  DeviceSetup* s = nullptr;
  int st = setup_current_device(&s);
  if (st != GAL_OK) return st;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (M == 0) return cudaMemsetAsync(chi2_out, 0, sizeof(double), cs) ? GAL_E_CUDA : GAL_OK;

  void* tw = s->base + kOffTw;
  void* F1 = s->base + kOffF1;
  void* Gw = s->base + kOffGw;
  double* partials = reinterpret_cast<double*>(s->base + kOffPartials);
  double* rho2 = reinterpret_cast<double*>(s->base + kOffRho2);
  unsigned* counter = reinterpret_cast<unsigned*>(s->base + kOffCounter);
  int* err = reinterpret_cast<int*>(s->base + kOffErr);

  // The array keeps whatever the previous call left: reset what must start at
  // zero (the extent launcher clears rho2 itself), rebuild the twiddles for
  // this nxy.
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), cs) != cudaSuccess) return GAL_E_CUDA;
  if (cudaMemsetAsync(err, 0, sizeof(int), cs) != cudaSuccess) return GAL_E_CUDA;
  if (gal::Launch<float>::twiddles(tw, nxy, cs) != cudaSuccess) return GAL_E_CUDA;
  if (gal::Launch<float>::extent(u, v, M, rho2, s->aux_blocks, cs) != cudaSuccess)
    return GAL_E_CUDA;
  const double S = (double)nxy * dxy;
  gal::SweepParams none{};
  int dev = 0, rv = 0, cv = 0;
  cudaGetDevice(&dev);
  gal::fft_plan_lookup_f32(dev, nxy, &rv, &cv);
  if (gal::Launch<float>::row_pass(image, nullptr, none, nxy, tw, F1, rho2, S, err, nullptr, cs,
                                   rv) != cudaSuccess)
    return GAL_E_CUDA;
  if (gal::Launch<float>::col_pass(F1, Gw, nxy, tw, rho2, S, 0, false, cs, cv) != cudaSuccess)
    return GAL_E_CUDA;
  gal::GatherParams gp;
  gp.cpa = std::cos(PA);
  gp.spa = std::sin(PA);
  gp.S = S;
  gp.phx = dRA;
  gp.phy = dDec;
  gp.N = nxy;
  if (gal::Launch<float>::gather(Gw, gp, rho2, u, v, re, im, w, M, nullptr, partials, counter,
                                 chi2_out, 0, true, s->gather_blocks, nullptr, cs) != cudaSuccess)
    return GAL_E_CUDA;
  noalloc_status_kernel<<<1, 1, 0, cs>>>(err, chi2_out);
  return cudaGetLastError() == cudaSuccess ? GAL_OK : GAL_E_CUDA;
}
