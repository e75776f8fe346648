// Internal interface between the C-ABI layer (gal_api.cu) and the kernel
// translation units (gal_kernels_f32.cu, gal_kernels_f64.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace gal {

// Parameters of the primary-beam tables (Sect. 2.1): c = 4 ln 2 / fwhm^2 and
// the beam centre (bx, by) = R (dRA, dDec) on the image grid, R the matrix of
// the Sect. 3.2 rotation (see beam_table_kernel).  One host function serves
// single calls and batches, so their tables are identical.
struct BeamParams {
  double c, bx, by;
};
inline BeamParams beam_params(double fwhm, double dRA, double dDec, double PA) {
  const double cp = std::cos(PA), sp = std::sin(PA);
  return BeamParams{4.0 * std::log(2.0) / (fwhm * fwhm), dRA * cp - dDec * sp, dRA * sp + dDec * cp};
}

// profile -> image parameters (all radians; Sect. 2 sampleProfile)
struct SweepParams {
  double Rmin, dR, dxy, inc;
  int nr;
};

// per-call sampling parameters: cos/sin PA, S = nxy * dxy (grid cells per
// wavelength^-1), and the phase offsets (dRA, dDec) so that the phase in turns
// is u * phx + v * phy.
struct GatherParams {
  double cpa, spa, S, phx, phy;
  int N;
};

// K offset copies of one model (multi-source composition): host arrays of
// K offsets (radians) and amplitudes, K in [1, 16].
struct MultiSources {
  int K;
  const double* dRA;
  const double* dDec;
  const double* amp;
};

// Host launchers, one explicit instantiation per precision.
template <typename T> struct Launch {
  static cudaError_t init();  // kernel attributes; once per process
  // resident gather blocks per SM; window_smem > 0 selects the variant that
  // stages the spectrum window (that many bytes) in shared memory.  The gather
  // takes `edge` = false only when the window is known to be pruned (no uv
  // point can reach the edge of the half spectrum).
  static int gather_blocks_per_sm(bool chi2, size_t window_smem);
  static cudaError_t twiddles(void* tw, int N, cudaStream_t st);
  static cudaError_t extent(const T* u, const T* v, int64_t M, double* rho2, int blocks,
                            cudaStream_t st);
  // u = u_m nu / c, v = v_m nu / c (metres and Hz to wavelengths), in FP64,
  // rounded once to T
  static cudaError_t uv_from_frequency(const T* u_m, const T* v_m, const T* nu, int64_t M, T* u,
                                       T* v, int blocks, cudaStream_t st);
  // range2[0] = min_k, range2[1] = max_k of u_k^2 + v_k^2 (finite points)
  static cudaError_t uv_range(const T* u, const T* v, int64_t M, double* range2, int blocks,
                              cudaStream_t st);
  static cudaError_t sweep(const T* I, const SweepParams& sp, int N, T* img, int blocks,
                           cudaStream_t st);
  // err: bit 2 is set if a staged copy's wait timed out (never expected);
  // beam: primary-beam tables of beam_table (null: no beam); radix: values per
  // thread of the compile-time FFT stages (0: the default, fft_radix_default)
  static cudaError_t row_pass(const T* image, const T* I, const SweepParams& sp, int N,
                              const void* tw, void* F1, const double* rho2, double S, int* err,
                              const T* beam, cudaStream_t st, int radix = 0);
  // primary-beam tables (2 N values) for a beam of FWHM fwhm > 0 on the
  // pointing centre, seen from a model moved by (dRA, dDec) at position angle PA
  static cudaError_t beam_table(T* tab, int N, double dxy, double fwhm, double dRA, double dDec,
                                double PA, cudaStream_t st);
  // kc_hint: window columns if the host knows them (0: unknown); full: the
  // full-plane window of full_cols (lengths of the compile-time passes only)
  static cudaError_t col_pass(const void* F1, void* Gw, int N, const void* tw,
                              const double* rho2, double S, int kc_hint, bool full,
                              cudaStream_t st, int radix = 0);
  // ms: multi-source offsets (null: the single offset of gp)
  static cudaError_t gather(const void* Gw, const GatherParams& gp, const double* rho2,
                            const T* u, const T* v, const T* re, const T* im, const T* w,
                            int64_t M, void* vis, double* partials, unsigned* counter,
                            double* chi2, size_t window_smem, bool edge, int blocks,
                            const MultiSources* ms, cudaStream_t st);
};

// Full-plane (complex-to-complex) spectrum path (gal_plane.cuh), instantiated
// per precision in gal_plane_f32.cu / gal_plane_f64.cu.  F1 then holds W =
// full_cols(bounds, N).W columns and the window nrw x W nodes; the column
// pass runs with full = true.
template <typename T> struct Plane {
  static bool supported(int N);  // transform lengths of the full-plane row pass
  // err: bit 2 is set if a staged copy's wait timed out (never expected)
  static cudaError_t rows(const T* image, const T* I, const SweepParams& sp, int N,
                          const void* tw, void* F1, const double* rho2, double S, const T* beam,
                          int* err, cudaStream_t st);
  static int gather_blocks_per_sm(bool chi2, size_t window_smem);
  static cudaError_t gather(const void* Gw, const GatherParams& gp, const double* rho2,
                            const T* u, const T* v, const T* re, const T* im, const T* w,
                            int64_t M, void* vis, double* partials, unsigned* counter,
                            double* chi2, size_t window_smem, bool edge, int blocks,
                            cudaStream_t st);
};

// Requests per launch of the batched passes (their job arrays are kernel
// parameters: 32 gather jobs take about 8 KB of the 32 KB parameter space).
constexpr int kBatchJobs = 32;

// FFT radix (values per thread of every stage but the last) of the
// compile-time row and column passes.  Float transforms run at radix 16; for
// image sides up to kAltRadixMaxSide the radix-8 passes exist too, and the
// FFT plan (a per-device choice per side, see gal_set_fft_radix) says which
// of the two a call uses.  Double transforms always run at radix 8.
template <typename T> constexpr int fft_radix_default() { return sizeof(T) == 4 ? 16 : 8; }
constexpr int kAltRadix = 8;
constexpr int kAltRadixMaxSide = 512;
// the FFT plan of a float32 side on `device` if one is fixed, the defaults
// otherwise (fixes nothing; for callers without a context)
void fft_plan_lookup_f32(int device, int nxy, int* rv, int* cv);

// One request of a batch, planned by the C-ABI layer (host values and device
// pointers).  Exactly one of image / I is set.
struct BatchItem {
  const void* image;   // nxy x nxy image, 16-byte aligned
  const void* I;       // radial profile (the sweep runs inside the row pass)
  SweepParams sp;
  int N;
  double S;            // N * dxy
  const double* rho2;  // device: squared uv extent of the observation
  int Kc, nrw;         // kept window (same rule as the kernels' bounds)
  void* F1;            // workspace: Kc columns of N complex values
  void* Gw;            // workspace: the window, nrw x Kc complex (+16 B)
  GatherParams gp;
  const void *u, *v, *re, *im, *w;
  int64_t M;
  double* partials;    // workspace: one slot per gather block
  unsigned* counter;   // workspace: zero at rest
  double* chi2_out;    // device result slot
  size_t wbytes;       // window bytes staged in shared memory (0: read from L2)
  bool edge;           // window reaches the edge of the half spectrum
  int grid;            // gather blocks (those of a single call of this request)
  void* beam;          // workspace: the request's 2N beam factors (null: no beam)
  BeamParams bp;       // their parameters
  bool full;           // full-plane spectrum (complex-to-complex rows, no fold)
  int ncol;            // window columns: Kc, or full_cols(...).W for the full plane
  int radix_row;       // FFT plan of side N: row and column pass radix (0: default)
  int radix_col;
};

// Launch shape of the batched passes.  Results do not depend on it (every
// request keeps the block partition and reduction tree of a single call), so
// it is free for the autotuner to choose.
struct BatchShape {
  int row_blocks;       // persistent row-pass blocks per SM and request group (1, 2, 4)
  int jobs_per_launch;  // requests per launch (<= kBatchJobs)
  int gather_fold;      // a request's single-call gather blocks run per launched block (1..8)
};
constexpr int kGatherFold = 4;     // default gather fold
constexpr int kMaxGatherFold = 8;  // largest fold a shape may ask for

// Batched passes: each launch covers up to jobs_per_launch requests of one
// transform length (grid row y = request).  `tw[lg]` is the twiddle table of
// length 2^lg.  `launches` is incremented per kernel launched.
template <typename T> struct BatchLaunch {
  static bool supported(int N);  // lengths the batched passes cover
  // the beam tables of the items that have a beam (launches only if some do)
  static cudaError_t beams(const BatchItem* items, int n, int* launches, cudaStream_t st);
  static cudaError_t rows(const BatchItem* items, int n, const void* const* tw, int* err,
                          const BatchShape& shape, int* launches, cudaStream_t st);
  static cudaError_t cols(const BatchItem* items, int n, const void* const* tw,
                          const BatchShape& shape, int* launches, cudaStream_t st);
  static cudaError_t gather(const BatchItem* items, int n, const BatchShape& shape,
                            int* launches, cudaStream_t st);
};

// Compile-time-length FFT passes (gal_fft3.cuh), instantiated per precision in
// gal_fft3_f32.cu / gal_fft3_f64.cu.  They return cudaErrorNotSupported when
// the length is outside their range (the caller then uses the generic passes).
template <typename T>
cudaError_t row_fft3(const T* image, const T* I, const SweepParams& sp, int N, const void* tw,
                     void* F1, const double* rho2, double S, int* err, const T* beam,
                     cudaStream_t st, int radix);
template <typename T>
cudaError_t col_fft3(const void* F1, void* Gw, int N, const void* tw, const double* rho2, double S,
                     int kc_hint, bool full, cudaStream_t st, int radix);

}  // namespace gal
