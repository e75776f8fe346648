/*
 * galario_gb300.h -- C ABI of the GB300 (sm_103a) visibility / chi-square library.
 *
 * The library computes synthetic interferometric visibilities of a model image,
 * or of an axisymmetric radial profile swept into an image, at a set of uv
 * points, and their weighted chi-square against observed visibilities: the hot
 * path of GALARIO (Tazzari, Beaujean & Testi, arXiv 1709.06999).  Every step
 * runs in hand-written CUDA kernels; this header is the whole public surface.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Units (Sect. 2 "Basic usage"): images are in Jy/pixel, profiles in Jy/sr,
 *   u and v in wavelengths; dxy, Rmin, dR, dRA, dDec, PA and inc in radians.
 *   Geometry scalars are `double` in both precisions.
 * Image layout (Sect. 2, Sect. 3.3): nxy x nxy, row-major, row 0 at the top
 *   (North), column 0 at the left (East); the origin is the centre pixel
 *   (nxy/2, nxy/2).  nxy must be a power of two with 4 <= nxy <= 8192.
 * Visibility output: interleaved (Re, Im) pairs, 2*M values of the entry
 *   point's precision.
 * Pointers: unless a name ends in `_host`, every array argument is DEVICE
 *   memory on the context's device, owned by the caller, borrowed for the
 *   duration of the stream-ordered work; inputs are never modified.  Arrays of
 *   the _f32 entry points must be 4-byte aligned, of the _f64 ones 8-byte
 *   aligned (16-byte alignment enables vector loads).
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Entry points only enqueue work; they do not synchronise unless
 *   documented (the `_host` variants do).  A context must be used by one host
 *   thread and one stream at a time: its workspace is shared by its calls.
 * Device: work is enqueued on the calling thread's current CUDA device, which
 *   must be the context's (gal_create makes it current); a stream of another
 *   device makes the launch fail with GAL_E_CUDA.
 * Errors: every int-returning call returns GAL_OK (0) or a negative GAL_E_*
 *   code; gal_strerror() names it.  On error nothing has been enqueued, except
 *   for GAL_E_CUDA, which reports a failed CUDA call (the message of the last
 *   CUDA error is kept in the context, see gal_last_cuda_error()).
 * Off-grid uv points: a point whose grid index lies beyond the half spectrum
 *   is evaluated at the nearest edge node, as the App. D reference does.
 * First use of a size: the first call with a new nxy (per precision) allocates
 *   workspace and twiddle tables.  gal_reserve() performs that allocation up
 *   front; after it, calls allocate nothing and may be captured in a CUDA graph.
 */
#ifndef GALARIO_GB300_H
#define GALARIO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GAL_OK          0
#define GAL_E_INVAL    -1   /* bad argument: null pointer, nxy not a power of two in [4, 8192],
                               nr < 2, dR <= 0, dxy <= 0, |inc| >= pi/2, M < 0, misaligned array */
#define GAL_E_NOMEM    -2   /* device allocation failed, or the context's HBM budget is reached */
#define GAL_E_CUDA     -3   /* a CUDA runtime call failed */
#define GAL_E_RANGE    -4   /* internal index check tripped (see gal_check) */
#define GAL_E_DEVICE   -5   /* no usable CUDA device / wrong architecture */
#define GAL_E_BUSY     -6   /* server: queue full (submit) */
#define GAL_E_TIMEOUT  -7   /* server: the result was not ready within the wait's limit */

typedef struct gal_ctx gal_ctx;     /* workspace, twiddle tables, launch shapes, counters */
typedef struct gal_data gal_data;   /* a registered observation: u, v, Re, Im, w + uv extent */

/* ---- context ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device` (made current for the call).  Owns all
 * library workspace.  Returns GAL_E_DEVICE if the device is absent. */
int gal_create(gal_ctx** out, int device);
/* Free the context and all workspace.  Waits for the device.  NULL is ignored. */
void gal_destroy(gal_ctx* ctx);
/* Pre-allocate workspace and twiddles for images up to `nxy` in precision
 * `real_bytes` (4 or 8), so that later calls allocate nothing. */
int gal_reserve(gal_ctx* ctx, int nxy, int real_bytes);
/* Name of a status code. */
const char* gal_strerror(int status);
/* Text of the last CUDA error seen by this context ("" if none). */
const char* gal_last_cuda_error(const gal_ctx* ctx);
/* Synchronise the device and report whether any kernel's internal index check
 * tripped since the last gal_check (GAL_E_RANGE) -- it never should. */
int gal_check(gal_ctx* ctx);
/* Number of kernels this context has launched since creation. */
uint64_t gal_launch_count(const gal_ctx* ctx);
/* Per-stage device timing.  Bit s of stage_mask enables stage s: each launch
 * of an enabled stage is bracketed with CUDA events (two event records on the
 * call's stream, so enable only the stages you need inside a timed loop).
 * gal_stage_times synchronises and returns, per stage, the summed milliseconds
 * and the number of timed launches since the mask was last set.
 * Stages: 0 uv extent, 1 row FFT (with sweep), 2 column FFT, 3 sample/chi2.
 * 0 disables timing; a mask outside [0, GAL_STAGE_ALL] is GAL_E_INVAL. */
#define GAL_STAGE_ALL 0xF
int gal_set_stage_timing(gal_ctx* ctx, int stage_mask);
int gal_stage_times(gal_ctx* ctx, double* ms_out4, int64_t* count_out4);

/* ---- observations ------------------------------------------------------------------- */

/* Device workspace the context holds now (spectra, windows, partial sums,
 * twiddles, beam tables, staging images), in bytes; and the device it was
 * created on. */
size_t gal_workspace_bytes(const gal_ctx* ctx);
int gal_device(const gal_ctx* ctx);
/* Limit the context's workspace (as gal_workspace_bytes counts it) to `bytes`;
 * 0, the default, sets no limit.  A call that would grow the workspace past
 * the limit returns GAL_E_NOMEM without evaluating anything (no output is
 * written), and the workspace already held is kept (lowering the limit frees
 * nothing; gal_destroy does).  GAL_E_INVAL for a NULL context. */
int gal_set_hbm_budget(gal_ctx* ctx, size_t bytes);

/* Register an observation of M visibilities: u, v (wavelengths), Re_obs, Im_obs (Jy)
 * and weights w = 1/sigma^2 (Sect. 3.1, Eq. chap6.eq:def.chi.square).  The arrays
 * are borrowed (device memory, must outlive the handle).  Enqueues on `stream` one
 * reduction for the largest baseline sqrt(u^2+v^2) (Sect. 3.3, criterion (i)),
 * which later calls use to restrict the FFT to the part of the spectrum the uv
 * points can reach (an exact pruning), and reads that one value back
 * (synchronising `stream` once).  The handle may be used by every context on
 * the same device. */
int gal_data_create_f32(gal_ctx* ctx, const float* u, const float* v, const float* re,
                        const float* im, const float* w, int64_t M, void* stream, gal_data** out);
int gal_data_create_f64(gal_ctx* ctx, const double* u, const double* v, const double* re,
                        const double* im, const double* w, int64_t M, void* stream, gal_data** out);
/* Register an observation as gal_data_create_* does, from copies the handle
 * owns, stored in Z-order (Morton order) of the uv plane: both axes quantised
 * to 16 bits over [-rho, rho] (rho the largest finite baseline), the two cells
 * bit-interleaved, points sorted stably by that key (non-finite points last).
 * The chi-square (Sect. 3.1, Eq. chap6.eq:def.chi.square) is a sum over the
 * points, so it is unchanged up to the rounding of the new order, and results
 * are the same on every run.  Points close in the uv plane then sample
 * neighbouring cells of the spectrum next to each other in memory, which
 * matters when a model's kept spectrum is too large for shared memory and is
 * read through L2.  u, v, re, im, w are read during the
 * call only: u and v are copied to the host and ordered there (a radix sort),
 * the five arrays gathered on `stream` into one device buffer of 5 M values
 * (freed by gal_data_destroy); the call synchronises `stream`.  Same errors as
 * gal_data_create_*, plus GAL_E_NOMEM when the host or device buffers cannot
 * be allocated. */
int gal_data_create_sorted_f32(gal_ctx* ctx, const float* u, const float* v, const float* re,
                               const float* im, const float* w, int64_t M, void* stream,
                               gal_data** out);
int gal_data_create_sorted_f64(gal_ctx* ctx, const double* u, const double* v, const double* re,
                               const double* im, const double* w, int64_t M, void* stream,
                               gal_data** out);
/* The order gal_data_create_sorted_* stores an observation in, computed on the
 * host from host arrays u, v: perm_out[i] (M values, caller-owned) is the input
 * index of the i-th stored point.  No device work.  GAL_E_INVAL for M < 0 or a
 * null pointer with M > 0; GAL_E_NOMEM if the host buffers cannot be had. */
int gal_z_order_f32(const float* u, const float* v, int64_t M, int64_t* perm_out);
int gal_z_order_f64(const double* u, const double* v, int64_t M, int64_t* perm_out);
/* Register an observation whose baselines u_m, v_m are in metres, with the
 * frequency nu (Hz) of every visibility (lifts the single-frequency assumption
 * of Sect. 3: each visibility samples the model at its own u_m nu / c).  The
 * wavelengths u = u_m nu / c, v = v_m nu / c are computed once, in FP64 and
 * rounded to the precision, into device arrays the handle owns (2 M values,
 * freed by gal_data_destroy); u_m, v_m, nu are not used after the call returns.
 * re, im, w are borrowed as in gal_data_create_*.  Same errors, plus
 * GAL_E_NOMEM if the owned arrays cannot be allocated. */
int gal_data_create_freq_f32(gal_ctx* ctx, const float* u_m, const float* v_m, const float* nu,
                             const float* re, const float* im, const float* w, int64_t M,
                             void* stream, gal_data** out);
int gal_data_create_freq_f64(gal_ctx* ctx, const double* u_m, const double* v_m,
                             const double* nu, const double* re, const double* im,
                             const double* w, int64_t M, void* stream, gal_data** out);
/* Release a handle (not the borrowed arrays).  Waits for the device. */
void gal_data_destroy(gal_data* data);
/* Number of visibilities and bytes per real value (4 or 8) of a handle. */
int gal_data_info(const gal_data* data, int64_t* M_out, int* real_bytes_out);

/* ---- the operations of Fig. 3 --------------------------------------------------------- */

/* sweep: image_out[nxy*nxy] (Jy/pixel) of the profile I[nr] (Jy/sr) sampled at radii
 * Rmin + k*dR, swept over 2*pi and inclined by `inc` about the North-South axis
 * (Sect. 2 sampleProfile, Sect. 4 "sweep", App. D): linear interpolation in r,
 * zero outside [Rmin, Rmin + (nr-1) dR], centre pixel linearly extrapolated to
 * r = 0, multiplied by dxy^2. */
int gal_sweep_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                  double dxy, double inc, float* image_out, void* stream);
int gal_sweep_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                  double dxy, double inc, double* image_out, void* stream);

/* sampleImage (Sect. 2, Fig. 3): visibilities of `image` at the M points (u, v),
 * with the model rotated by PA and shifted by (dRA, dDec) (Sect. 3.2).  Steps:
 * fftshift -> real-to-complex 2D FFT -> fftshift along v (Sect. 4), uv rotation,
 * bilinear interpolation (Sect. 3.3), phase factor exp(+2 pi i (u dRA + v dDec))
 * (App. D sign).  vis_out: 2*M values.  Computes the uv extent first (one extra
 * read of u and v). */
int gal_sample_image_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                         double dDec, double PA, int64_t M, const float* u, const float* v,
                         float* vis_out, void* stream);
int gal_sample_image_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                         double dDec, double PA, int64_t M, const double* u, const double* v,
                         double* vis_out, void* stream);

/* sampleProfile (Sect. 2, Fig. 3): as sample_image for the image that gal_sweep
 * would produce; the sweep runs inside the row FFT, so no image is written. */
int gal_sample_profile_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR,
                           int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                           int64_t M, const float* u, const float* v, float* vis_out,
                           void* stream);
int gal_sample_profile_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR,
                           int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                           int64_t M, const double* u, const double* v, double* vis_out,
                           void* stream);

/* chi2Image (Sect. 2, Eq. chap6.eq:def.chi.square): writes to *chi2_out (one
 * double in device memory) sum_k w_k [(Re_k - Re_mod)^2 + (Im_k - Im_mod)^2] of
 * the registered observation against the model image.  The reduction order is
 * fixed, so repeated calls give bitwise identical results on one device.  The
 * observation's precision must match the entry point's. */
int gal_chi2_image_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                       double dDec, double PA, const gal_data* data, double* chi2_out,
                       void* stream);
int gal_chi2_image_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                       double dDec, double PA, const gal_data* data, double* chi2_out,
                       void* stream);

/* chi2Profile (Sect. 2): chi2_image of the swept profile (sweep fused into the FFT). */
int gal_chi2_profile_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                         double dxy, double inc, double dRA, double dDec, double PA,
                         const gal_data* data, double* chi2_out, void* stream);
int gal_chi2_profile_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                         double dxy, double inc, double dRA, double dDec, double PA,
                         const gal_data* data, double* chi2_out, void* stream);

/* Host-buffer chi2Image (the paper's calling pattern, Sect. 4 "memory
 * operations"): `image_host` (nxy*nxy values in host memory, ideally pinned) is
 * copied to context workspace, chi2_image runs on `stream`, and the result is
 * copied back to *chi2_host.  Synchronises `stream` before returning. */
int gal_chi2_image_host_f32(gal_ctx* ctx, const float* image_host, int nxy, double dxy,
                            double dRA, double dDec, double PA, const gal_data* data,
                            double* chi2_host, void* stream);
int gal_chi2_image_host_f64(gal_ctx* ctx, const double* image_host, int nxy, double dxy,
                            double dRA, double dDec, double PA, const gal_data* data,
                            double* chi2_host, void* stream);

/* ---- primary beam and full-plane spectrum ---------------------------------------------- */

/* Options of the extended calls below; a NULL pointer means all defaults, and
 * the call is then identical to its plain counterpart.
 *
 * pb_fwhm: full width at half maximum (radians) of a primary beam applied to
 *   the model before the transform (Sect. 2.1: the visibility is the transform
 *   of A I, A being the antenna pattern normalised at the pointing centre,
 *   whose central lobe is close to a Gaussian of FWHM K lambda / D; the first
 *   release left A to the caller and never applied it to profiles).  A is the
 *   circular Gaussian exp(-4 ln 2 |s|^2 / pb_fwhm^2), fixed on the phase centre
 *   and evaluated at each model pixel's sky position after the PA rotation and
 *   the (dRA, dDec) move, so a model moved away from the centre is attenuated
 *   as the sky would attenuate it.  The image (or the swept profile) is then
 *   the bare brightness I.  0 = no beam; negative or non-finite values are
 *   GAL_E_INVAL.  The factor is applied inside the row FFT (no extra pass).
 * full_plane: 1 = compute the full complex-to-complex spectrum (both signs of
 *   u, no Hermitian fold) instead of the real-to-complex half spectrum; the
 *   paper checks one against the other (Sect. 5).  Off-grid points are
 *   clamped to the node range -nxy/2 .. nxy/2-1 of both axes.  Supported for
 *   16 <= nxy <= 8192 (_f32) and 8 <= nxy <= 4096 (_f64); other sizes, and
 *   values other than 0 and 1, are GAL_E_INVAL. */
typedef struct gal_opts {
  double pb_fwhm;
  int full_plane;
} gal_opts;

int gal_sample_image_ex_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                            double dDec, double PA, const gal_opts* opts, int64_t M,
                            const float* u, const float* v, float* vis_out, void* stream);
int gal_sample_image_ex_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                            double dDec, double PA, const gal_opts* opts, int64_t M,
                            const double* u, const double* v, double* vis_out, void* stream);
int gal_sample_profile_ex_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR,
                              int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                              const gal_opts* opts, int64_t M, const float* u, const float* v,
                              float* vis_out, void* stream);
int gal_sample_profile_ex_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR,
                              int nxy, double dxy, double inc, double dRA, double dDec, double PA,
                              const gal_opts* opts, int64_t M, const double* u, const double* v,
                              double* vis_out, void* stream);
int gal_chi2_image_ex_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double dRA,
                          double dDec, double PA, const gal_opts* opts, const gal_data* data,
                          double* chi2_out, void* stream);
int gal_chi2_image_ex_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double dRA,
                          double dDec, double PA, const gal_opts* opts, const gal_data* data,
                          double* chi2_out, void* stream);
int gal_chi2_profile_ex_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR, int nxy,
                            double dxy, double inc, double dRA, double dDec, double PA,
                            const gal_opts* opts, const gal_data* data, double* chi2_out,
                            void* stream);
int gal_chi2_profile_ex_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR, int nxy,
                            double dxy, double inc, double dRA, double dDec, double PA,
                            const gal_opts* opts, const gal_data* data, double* chi2_out,
                            void* stream);

/* Pipelined host-buffer chi2Image, for a caller that streams model images from
 * the host (Sect. 4: host-device transfers dominate the paper's GPU timings).
 * The image is copied into one of two context staging buffers on a context-
 * owned copy stream, so the copy overlaps the compute of the previous call;
 * the compute runs on `stream` once its copy is done, and the result is
 * copied to *chi2_host (ideally pinned) on `stream`.  Nothing is synchronised:
 * *chi2_host is written, and `image_host` (ideally pinned) may be modified or
 * freed, only once `stream` has passed this call's work (e.g. after
 * cudaStreamSynchronize).  Results equal gal_chi2_image_host's bitwise. */
int gal_chi2_image_host_async_f32(gal_ctx* ctx, const float* image_host, int nxy, double dxy,
                                  double dRA, double dDec, double PA, const gal_data* data,
                                  double* chi2_host, void* stream);
int gal_chi2_image_host_async_f64(gal_ctx* ctx, const double* image_host, int nxy, double dxy,
                                  double dRA, double dDec, double PA, const gal_data* data,
                                  double* chi2_host, void* stream);

/* ---- multi-source composition --------------------------------------------------------- */

/* Largest number of copies in one multi-source call. */
#define GAL_MAX_SOURCES 16

/* Visibilities (and chi-square) of K copies of one model: copy k scaled by
 * amp[k] and displaced by (dRA[k], dDec[k]) radians, all rotated by PA (end of
 * Sect. 3.1: by the linearity of the Fourier transform, identical sources at
 * different places need one transform; each is displaced by its own phase,
 * Sect. 3.2).  The sampled model visibility is multiplied by
 *   sum_k amp[k] exp(+2 pi i (u dRA[k] + v dDec[k]))
 * instead of one phase factor: one FFT and one interpolation per uv point
 * serve all K copies.  dRA, dDec, amp: K host doubles, K in [1, GAL_MAX_SOURCES]
 * (GAL_E_INVAL otherwise or for non-finite values); with K = 1 and amp = 1
 * the result is bitwise that of the single-offset call.  Other arguments as in
 * the single-source calls. */
int gal_sample_image_multi_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double PA,
                               int K, const double* dRA, const double* dDec, const double* amp,
                               int64_t M, const float* u, const float* v, float* vis_out,
                               void* stream);
int gal_sample_image_multi_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double PA,
                               int K, const double* dRA, const double* dDec, const double* amp,
                               int64_t M, const double* u, const double* v, double* vis_out,
                               void* stream);
int gal_chi2_image_multi_f32(gal_ctx* ctx, const float* image, int nxy, double dxy, double PA,
                             int K, const double* dRA, const double* dDec, const double* amp,
                             const gal_data* data, double* chi2_out, void* stream);
int gal_chi2_image_multi_f64(gal_ctx* ctx, const double* image, int nxy, double dxy, double PA,
                             int K, const double* dRA, const double* dDec, const double* amp,
                             const gal_data* data, double* chi2_out, void* stream);
int gal_chi2_profile_multi_f32(gal_ctx* ctx, const float* I, int nr, double Rmin, double dR,
                               int nxy, double dxy, double inc, double PA, int K,
                               const double* dRA, const double* dDec, const double* amp,
                               const gal_data* data, double* chi2_out, void* stream);
int gal_chi2_profile_multi_f64(gal_ctx* ctx, const double* I, int nr, double Rmin, double dR,
                               int nxy, double dxy, double inc, double PA, int K,
                               const double* dRA, const double* dDec, const double* amp,
                               const gal_data* data, double* chi2_out, void* stream);

/* ---- batches ------------------------------------------------------------------------- */

/* One chi-square request of a batch: chi2Image when `image` is set, chi2Profile
 * when `intensity` is set (exactly one of the two), with the arguments of
 * gal_chi2_image_* / gal_chi2_profile_* (Sect. 2).  The arrays' precision is the
 * observation's (`data`); nr, Rmin, dR and inc are read for profiles only. */
typedef struct gal_request {
  const void* image;      /* nxy*nxy values (device) or NULL */
  const void* intensity;  /* nr values (device) or NULL */
  int nr;
  double Rmin, dR, inc;
  int nxy;
  double dxy, dRA, dDec, PA;
  const gal_data* data;
  double pb_fwhm;         /* primary-beam FWHM (radians), 0 = none: as gal_opts.pb_fwhm, e.g.
                             one beam per spectral channel of a cube */
  int full_plane;         /* 1 = full-plane spectrum, as gal_opts.full_plane (0 or 1) */
} gal_request;

/* chi2_out[i] (device, n doubles) = the chi-square of request i: the many
 * spectral channels or MCMC walkers of one fit in a few launches.  Requests of
 * one precision and image side share each launch of the row FFT, of the column
 * FFT and of the gather (up to 32 requests per launch; grid row = request), so
 * the whole batch costs about three launches per distinct image side instead
 * of three per request.  Every result is bitwise equal to the corresponding
 * single call on the same context (same kernels, block partitions and
 * reduction trees: a batched gather runs each request's single-call blocks as
 * virtual blocks, several to a launched block, so the request's spectrum
 * window is copied into shared memory fewer times).  Requests the batched
 * kernels do not cover (nxy < 32 in
 * float32 / < 16 in float64, nxy above 8192 / 4096, images not 16-byte
 * aligned) run as single calls inside the batch.
 * Launch shapes: the first batch of each (precision, request count, largest
 * side) is run once per candidate shape, timed with events on `stream`
 * (synchronising it) and the fastest shape is kept for the context; results do
 * not depend on the shape (gal_set_batch_shape below lists the candidates).
 * gal_set_batch_tuning(ctx, 0) turns this off (default shape).  The batch workspace (about nxy*Kc*2 complex values per
 * request) grows on first use; like every call on a context, batches on
 * different streams must not overlap.
 * Errors: GAL_E_INVAL if any request is invalid (nothing is launched then). */
int gal_chi2_batch(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out, void* stream);
/* enable = 0 turns off the context's tuning: launch shapes of batches and the
 * FFT plans of sides it is first to use (which then take the default). */
int gal_set_batch_tuning(gal_ctx* ctx, int enable);

/* Launch shapes of batches (an implementation choice: the paper evaluates one
 * model per call, Sect. 4).  A shape is three integers:
 *   row_blocks       persistent row-pass blocks per SM for each group of
 *                    requests (1 .. 8);
 *   jobs_per_launch  requests per launch of each pass (1 .. 32);
 *   gather_fold      how many of a request's single-call gather blocks one
 *                    launched block runs in turn (1 .. 8; a launch of m
 *                    requests uses min(m, gather_fold)), so that its window
 *                    is copied into shared memory that many times fewer.
 * The context keeps one shape per key (real_bytes 4 or 8; n, the number of
 * the batch's requests of that precision that run in the batched kernels;
 * max_nxy, the largest side among them).  The first batch of a key tunes it
 * when tuning is on: the six pairs (row_blocks, jobs_per_launch) of (1, 32),
 * (2, 32), (4, 32), (1, 8), (2, 8), (4, 16) at fold 4, then folds 1, 2 and 8
 * with the fastest pair, each run twice on the batch's stream (the first run
 * warms up); the fastest is kept.  Without tuning (off, or the stream being
 * captured) a key takes the default (1, 32, 4).  Results are bitwise the same
 * for every shape.
 *   gal_set_batch_shape  fixes the shape of a key (before or after tuning);
 *                        GAL_E_INVAL for a NULL context, real_bytes other
 *                        than 4 or 8, n < 1, a value outside the ranges
 *                        above or max_nxy not a power of two in 4 .. 8192.
 *   gal_get_batch_shape  writes the shape the next batch of that key will use
 *                        to shape_out3 = {row_blocks, jobs_per_launch,
 *                        gather_fold}: the kept one, or the default when none
 *                        is kept yet; *cached (may be NULL) = 1 if one is kept. */
int gal_set_batch_shape(gal_ctx* ctx, int real_bytes, int n, int max_nxy, int row_blocks,
                        int jobs_per_launch, int gather_fold);
int gal_get_batch_shape(const gal_ctx* ctx, int real_bytes, int n, int max_nxy, int* shape_out3,
                        int* cached);

/* FFT plans (an implementation choice; the paper's transform is any FFT,
 * Sect. 4).  The row and column passes of a float32 image of side 32 .. 512
 * exist at two radices (values per thread in the register-blocked stages):
 * 16 and 8.  Which one runs is the plan of that side, one per device and
 * precision for the whole process, so that single calls, batches, graphs,
 * served requests and gal_chi2_image_noalloc_f32 compute a request with the
 * same arithmetic (their results stay bitwise equal).  A side's plan is fixed
 * at its first use by a context: the context times both radices of both
 * passes on its workspace and stream (synchronising the stream once) and keeps
 * radix 8 for a pass only if it is at least 5 % faster -- unless its tuning is
 * off or the stream is being captured, when the side takes the default (16).
 * Sides above 512 run at radix 16, float64 transforms at radix 8.  The two
 * radices round differently, so results may differ in the last bits between
 * processes whose plans differ; set the plan explicitly to fix them.
 *   gal_set_fft_radix   sets the plan of (device, real_bytes 4 or 8, nxy):
 *                       row_radix, col_radix 16 or 8 for float32 sides 32..512,
 *                       16 for other float32 sides, 8 for float64.  It applies
 *                       to calls enqueued afterwards.  GAL_E_INVAL otherwise.
 *   gal_get_fft_radix   the plan of that side, or 0, 0 when it is not fixed yet. */
int gal_set_fft_radix(int device, int real_bytes, int nxy, int row_radix, int col_radix);
int gal_get_fft_radix(int device, int real_bytes, int nxy, int* row_radix, int* col_radix);

/* A batch captured into a CUDA graph.  gal_chi2_batch_capture runs the batch
 * once on `stream` (workspace, twiddles and launch-shape tuning happen there)
 * and then records its launches into a graph, which gal_graph_launch replays
 * on any stream.  The replay reads the requests' arrays (images, profiles,
 * observations) as they are at replay time, so a fit that rewrites its model
 * images in place relaunches the same graph; scalar arguments are those of the
 * capture.  gal_graph_update re-records the batch with new requests of the
 * same structure (same count, sides, kinds and observations) and updates the
 * executable graph in place (GAL_E_INVAL if the structure changed).  A graph
 * uses its context's batch workspace: keep the context alive, and do not run
 * other batches on it while a replay may be in flight. */
typedef struct gal_graph gal_graph;
int gal_chi2_batch_capture(gal_ctx* ctx, const gal_request* reqs, int n, double* chi2_out,
                           void* stream, gal_graph** out);
int gal_graph_update(gal_graph* g, const gal_request* reqs, int n, double* chi2_out);
int gal_graph_launch(gal_graph* g, void* stream);
void gal_graph_destroy(gal_graph* g);

/* ---- serving ------------------------------------------------------------------------- */

/* A request loop for chi-square requests of mixed kinds and sizes on one GPU
 * (the paper has no counterpart; it serves many independent evaluations the
 * way an MCMC or a fitting service issues them).
 *
 * A scheduler thread owns `slots` worker contexts, each with its own CUDA
 * stream.  Submitted requests wait in a FIFO queue.  Whenever a slot is free
 * the scheduler admits the head of the queue -- together with up to
 * max_batch - 1 more queued requests of the same precision, run as one
 * gal_chi2_batch -- if the HBM budget allows, so requests that arrive while
 * others are on the GPU join as slots and memory free up and their work
 * overlaps on the device.  Budget: the bytes of the observations added with
 * gal_server_add_data plus the workspace every slot holds, where a slot about
 * to take a launch is charged the workspace that launch may grow it to
 * (3 half spectra of each request's side and precision).  The head request
 * waits while that sum would exceed hbm_budget_bytes; one that can never fit
 * fails with GAL_E_NOMEM.  Each result is bitwise equal to a single call of
 * the request (batching does not change it).
 *
 * Observations must be added with gal_server_add_data_* (the budget counts
 * them); a request's arrays (image or profile) must stay valid until its
 * result has been waited for.  Latency is measured on the host from submit to
 * the scheduler's observation that the result is in host memory. */
typedef struct gal_server gal_server;
int gal_server_create(int device, size_t hbm_budget_bytes, int slots, int max_batch,
                      gal_server** out);
/* As gal_data_create_*, on the server's device, charged to its budget
 * (5 M real values; GAL_E_NOMEM if over).  Destroyed with the server. */
int gal_server_add_data_f32(gal_server* s, const float* u, const float* v, const float* re,
                            const float* im, const float* w, int64_t M, gal_data** out);
int gal_server_add_data_f64(gal_server* s, const double* u, const double* v, const double* re,
                            const double* im, const double* w, int64_t M, gal_data** out);
/* As gal_server_add_data_*, registered in Z-order as gal_data_create_sorted_*
 * does (the server keeps its own copies; the arrays may be freed after the
 * call, which synchronises the device).  Same budget charge and errors. */
int gal_server_add_data_sorted_f32(gal_server* s, const float* u, const float* v, const float* re,
                                   const float* im, const float* w, int64_t M, gal_data** out);
int gal_server_add_data_sorted_f64(gal_server* s, const double* u, const double* v,
                                   const double* re, const double* im, const double* w, int64_t M,
                                   gal_data** out);
/* Queue one request (copied); *ticket identifies it.  GAL_E_INVAL for an invalid
 * request, GAL_E_BUSY when 65536 requests are already waiting. */
int gal_server_submit(gal_server* s, const gal_request* req, uint64_t* ticket);
/* Queue n requests at once (tickets[n]): all or none (GAL_E_INVAL / GAL_E_BUSY). */
int gal_server_submit_many(gal_server* s, const gal_request* reqs, int n, uint64_t* tickets);
/* Wait up to timeout_ms (< 0: forever) for a ticket: its chi-square and its
 * latency in seconds.  Returns the request's own status (GAL_OK, or the error
 * its evaluation met), GAL_E_TIMEOUT if not finished in time, GAL_E_INVAL for
 * an unknown or already collected ticket.  A collected ticket is forgotten. */
int gal_server_wait(gal_server* s, uint64_t ticket, int timeout_ms, double* chi2,
                    double* latency_s);
typedef struct gal_server_stats {
  uint64_t submitted, completed, launches;  /* launches: single calls + batches */
  uint64_t max_inflight;                    /* most requests on the GPU at once */
  size_t data_bytes, workspace_bytes;       /* charged to the budget now */
  size_t peak_bytes;                        /* largest charge seen */
} gal_server_stats;
int gal_server_get_stats(gal_server* s, gal_server_stats* out);
/* Finish every queued request, stop the scheduler, free everything. */
void gal_server_destroy(gal_server* s);

/* ---- image sizing --------------------------------------------------------------------- */

/* get_image_size (Sect. 3.3, criteria (i), (iia), (iib)): the image side *nxy_out
 * (a power of two, possibly above the 8192 the transforms accept) and pixel
 * size *dxy_out (radians) for the M points (u, v) (wavelengths, device memory).
 * With rho_min / rho_max the shortest / longest baseline (finite points only):
 *   (iia), PB == 0:  duv = rho_min / (Gamma f_min), Gamma = 0.6
 *   (iib), PB > 0:   duv = min(1 / PB, rho_min / (Gamma f_min))   (PB: primary
 *                    beam FWHM in radians; the field covers both the beam and
 *                    f_min times the largest recoverable scale)
 *   nxy = smallest power of two >= 2 f_max rho_max / duv   (criterion (i))
 *   dxy = 1 / (nxy duv)
 * f_min > 1 and f_max > 2 as the criteria require (the paper uses 5 and 2.5).
 * Reads two doubles back: synchronises `stream`.  GAL_E_INVAL for M < 1, bad
 * factors, PB < 0, or rho_min == 0 (a zero-length baseline) or no finite point;
 * GAL_E_RANGE if nxy would exceed 2^62. */
int gal_get_image_size_f32(gal_ctx* ctx, const float* u, const float* v, int64_t M, double PB,
                           double f_min, double f_max, int64_t* nxy_out, double* dxy_out,
                           void* stream);
int gal_get_image_size_f64(gal_ctx* ctx, const double* u, const double* v, int64_t M, double PB,
                           double f_min, double f_max, int64_t* nxy_out, double* dxy_out,
                           void* stream);

/* ---- allocation-free variant ---------------------------------------------------------- */

/* Largest image side accepted by gal_chi2_image_noalloc_f32. */
#define GAL_NOALLOC_MAX_NXY 1024

/* chi2Image in float32 without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * -- for example a host application whose own allocator has already reserved
 * the GPU's memory, a plug-in that may not grow the process's device
 * footprint, or a latency-critical loop that cannot afford the device
 * synchronisation an allocation implies.
 *
 * It computes what gal_data_create_f32 + gal_chi2_image_f32 compute (same
 * kernels, same result) but takes the observation as plain arrays and needs no
 * context.  Its scratch is one fixed device array of about 12.7 MB inside the
 * library, present on every GPU that loads the library until the process
 * exits; no call allocates or frees anything.
 *   image     nxy*nxy floats (device), 8-byte aligned; nxy a power of two in
 *             [4, GAL_NOALLOC_MAX_NXY] -- larger images return GAL_E_INVAL
 *   u, v, re, im, w   M floats each (device), as for gal_data_create_f32
 *   chi2_out  one double (device)
 * The first call on a device (with that device current) looks up the array's
 * device address; make that first call before any stream capture.  Every call
 * uses the same array and leaves its contents behind (each call re-initialises
 * what it needs), so calls that may overlap on the GPU -- other streams, other
 * host threads -- race with each other and must be serialised by the caller.
 * Errors: argument errors return GAL_E_INVAL and enqueue nothing.  A bounded
 * device wait that gives up (never expected) cannot be reported through a
 * context here, so the call then writes NaN to *chi2_out.
 * The transforms use the FFT plan of the side if one is fixed on the device
 * (gal_set_fft_radix), the default radix otherwise.  The window of the
 * spectrum is always read through L2 and clamped as at the grid's edge, with
 * four 256-thread gather blocks per SM: the result is bitwise
 * gal_chi2_image_f32's when that call takes the same shape (a window larger
 * than its 200 KB shared-memory budget that spans every row) under the same
 * plan, and equal to rounding otherwise. */
int gal_chi2_image_noalloc_f32(const float* image, int nxy, double dxy, double dRA, double dDec,
                               double PA, const float* u, const float* v, const float* re,
                               const float* im, const float* w, int64_t M, double* chi2_out,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GALARIO_GB300_H */
