/*
 * fbf.h -- C ABI of the GB300 (sm_103a) shiftable Fourier-kernel bilateral filter.
 *
 * Method: Ghosh & Chaudhury, "On Fast Bilateral Filtering using Fourier
 * Kernels" (arXiv 1603.08081).  The bilateral filter of eq. (1),
 *
 *     f_BF(i) = sum_j w(j) phi(f(i-j) - f(i)) f(i-j) / sum_j w(j) phi(f(i-j) - f(i)),
 *
 * is approximated by replacing the range kernel phi with the cosine series of
 * eq. (6), phi_N(t) = d_0 + sum_{n=1}^{K-1} d_n cos(n omega t), omega = pi / T,
 * whose coefficients minimise the squared error on the grid {0, ..., T}
 * (eqs. (7)-(8), Algorithm 2).  The approximation (eq. (9)) is then computed as
 * K rounds of modulate / convolve with w / demodulate / accumulate, followed
 * by one division (Algorithm 1, eqs. (4)-(5)).
 *
 * Conventions.
 *   - K counts the coefficients d_0 .. d_{K-1}.  (The paper's Tables 3-4 call
 *     this number N; Algorithm 2's column counter is the same K.)
 *   - Images are single channel, row-major, with a row pitch in BYTES.
 *   - Device pointers are plain CUDA device pointers; every device call is
 *     asynchronous on the given stream, never synchronises, and (unless stated)
 *     allocates nothing.  The caller owns every buffer.  Calls that need
 *     scratch take it stream-ordered from a memory pool the library creates
 *     per device on first use; the pool keeps the memory it has reserved, so
 *     the next call re-uses it (the memory stays reserved while the process
 *     runs).
 *   - Errors are returned as fbf_status; nothing is thrown across the ABI.
 *     A fault inside a kernel surfaces at the caller's next synchronisation.
 */
#ifndef FBF_H
#define FBF_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FBF_OK = 0,
  FBF_ERR_INVALID_ARGUMENT = 1, /* null pointer, bad size/pitch, sigma <= 0, ... */
  FBF_ERR_NOT_CONVERGED = 2,    /* fit: eps not reached within the column limit */
  FBF_ERR_RANGE = 3,            /* window or order beyond the compiled limits     */
  FBF_ERR_UNSUPPORTED = 4,      /* valid request this build does not implement   */
  FBF_ERR_CUDA = 5,             /* a CUDA runtime call or launch failed            */
  FBF_ERR_TIMEOUT = 6           /* a bounded device-side wait gave up              */
} fbf_status;

/* Range kernel phi.  Gaussian: eq. (3), phi(t) = exp(-t^2 / (2 sigma_r^2)).
 * Exponential: phi(t) = exp(-|t| / sigma_r) (the kernel of the works cited in
 * Sec. I; the paper names it without printing the formula). */
typedef enum { FBF_RANGE_GAUSSIAN = 0, FBF_RANGE_EXPONENTIAL = 1 } fbf_range_kernel;

/* Spatial kernel w on Omega = [-W, W]^2 (Sec. I).  Gaussian: eq. (2),
 * separable; box: uniform.  Weights are normalised to sum 1 (Sec. IV). */
typedef enum {
  FBF_SPATIAL_GAUSSIAN = 0,
  FBF_SPATIAL_BOX = 1,
  /* The recursive Gaussian (the constant-time Gaussian filtering that Sec. II
   * cites after eq. (5): Deriche's fourth-order approximation, two damped
   * sinusoids per direction realised as causal + anticausal recursions, unit
   * gain).  Its cost per pixel does not depend on sigma_s: there is no window
   * (W is not used).  TRUNCATE: zero outside the image; REFLECT: each line
   * extended by ceil(8 sigma_s) mirrored samples.  0.5 <= sigma_s <= 256; the
   * FP32 form (AUTO selects it) on uint8 images; fbf_filter then takes 40
   * bytes per pixel and harmonic of scratch (at most 4 GiB, harmonics in
   * chunks beyond that) stream-ordered from the library's pool. */
  FBF_SPATIAL_GAUSSIAN_RECURSIVE = 2
} fbf_spatial_kernel;

/* Border rule (the paper leaves it open).  REFLECT: half-sample symmetric
 * extension (index -1 -> 0, -2 -> 1, ...; repeated for windows wider than the
 * image).  TRUNCATE: the window sums of eq. (1) run only over pixels inside the
 * image (equivalently, both modulated channels are zero outside). */
typedef enum { FBF_BORDER_REFLECT = 0, FBF_BORDER_TRUNCATE = 1 } fbf_border;

/* Element type of the input image. */
typedef enum { FBF_U8 = 0, FBF_F32 = 1 } fbf_dtype;

/* Arithmetic form of the device filter.  FP32: every step in FP32 on the FMA
 * pipe.  TC_FP16 / TC_BF16: both 1-D passes as banded-Toeplitz products on the
 * tensor cores (tcgen05) with FP32 accumulation; data split into hi + lo
 * 16-bit parts (BF16 splits the weights too); uint8 input only.
 * TC_FP16_SINGLE: the same with data and weights rounded to FP16 once (half the
 * tensor-core products); on 8-bit images its error against the exact
 * Algorithm 1 stays near 0.02-0.05 gray level for sigma_r >= 20 and grows as
 * sigma_r shrinks (about 0.1 at sigma_r = 5), where the split forms stay below
 * 2e-3.  TC_BF16_SINGLE: data and weights rounded to BF16 once (one product,
 * the speed of TC_FP16_SINGLE; BF16 keeps 8 significand bits to FP16's 11):
 * with the REFLECT border its error stays within 0.35 gray level for
 * sigma_r >= 15 and sigma_s >= 1 (an FP64 emulation of its rounding steps gives
 * 0.08-0.31 over Gaussian and box windows W = 3..48) and reaches 0.5 near
 * sigma_r = 10 or with a window of one dominant tap (sigma_s < 1); with
 * TRUNCATE the same holds away from the image border, while near a corner,
 * where a quarter of the window remains, the error grows up to about four
 * times (0.48 measured at W = 16).  Callers opt in.
 * AUTO: the faster of FP32 and TC_FP16 for the window, as measured on GB300
 * (TC_FP16 from W = 4 up, for the Gaussian and the box kernel alike; FP32,
 * which runs the box kernel as running window sums, below); AUTO never picks
 * TC_FP16_SINGLE or TC_BF16_SINGLE. */
typedef enum {
  FBF_FORM_AUTO = 0,
  FBF_FORM_FP32 = 1,
  FBF_FORM_TC_FP16 = 2,
  FBF_FORM_TC_BF16 = 3,
  FBF_FORM_TC_FP16_SINGLE = 4,
  FBF_FORM_TC_BF16_SINGLE = 5
} fbf_form;

#define FBF_KMAX 256 /* maximum number of coefficients K                 */
#define FBF_WMAX 48  /* maximum half window W (taps 2W+1 <= 97)           */

/* Fitted range-kernel approximation, eq. (6): phi_N(t) = sum_k d[k] cos(k omega t). */
typedef struct {
  int K;             /* number of coefficients d[0..K-1]                      */
  int levels;        /* grid size used by the fit (T+1 for the integer grid)  */
  double T;          /* half period; omega = pi / T                           */
  double omega;      /* pi / T                                                */
  double resid_l2;   /* ||b - A d||_2 on the grid (the E of Algorithm 2)      */
  double resid_linf; /* max_t |phi(t) - phi_N(t)| on the grid (eq. (10))     */
  double d[FBF_KMAX];
} fbf_coeffs;

/* Filter parameters. */
typedef struct {
  fbf_spatial_kernel spatial;
  double sigma_s;           /* Gaussian spatial scale (ignored for the box)      */
  int W;                    /* half window; <= 0 selects ceil(3 sigma_s)         */
  fbf_border border;
  fbf_form form;
  const fbf_coeffs *coeffs; /* host pointer, read during the call only           */
} fbf_params;

/*
 * fbf_fit_coeffs -- Algorithm 2 (Progressive Fourier Approximation), host, FP64.
 *
 * Samples b = [phi(t)] on the grid, then grows the basis {1, cos(wt),
 * cos(2wt), ...} one column at a time, updating a QR factorisation by one
 * modified Gram-Schmidt step per column, solving R d = Q^T b by
 * back-substitution, and stopping at the first K with ||b - A d||_2 <= eps
 * (Sec. III; the residual is evaluated as b - A d).
 *
 *   kernel, sigma_r  range kernel phi and its scale (> 0)
 *   T                half period (> 0); omega = pi / T
 *   eps              tolerance (> 0) when K_fixed == 0
 *   K_fixed          > 0: fit exactly this many coefficients, ignore eps
 *   levels           0: grid {0, 1, ..., T} (T must be an integer);
 *                    >= 2: that many equispaced points on [0, T]
 *   out              filled on FBF_OK and on FBF_ERR_NOT_CONVERGED (then with
 *                    the largest order tried: min(grid size, FBF_KMAX))
 * Returns FBF_ERR_INVALID_ARGUMENT for bad inputs, FBF_ERR_RANGE if K_fixed
 * exceeds FBF_KMAX or the grid size.
 */
fbf_status fbf_fit_coeffs(fbf_range_kernel kernel, double sigma_r, double T, double eps,
                          int K_fixed, int levels, fbf_coeffs *out);

/*
 * fbf_fit_coeffs_samples -- Algorithm 2 for a range kernel given by its
 * samples, host, FP64.  Sec. III states that the progressive fit applies to
 * any kernel whose Fourier series converges pointwise (the Gaussian and the
 * exponential are two of them); this entry point takes such a kernel as
 * samples instead of an enum.
 *
 *   phi      host array of L values phi(t_l) at t_l = l * T / (L - 1),
 *            l = 0 .. L-1 (for integer T and L = T + 1: the grid {0, ..., T});
 *            phi is even, so only [0, T] is sampled; read during the call only
 *   L        number of samples (>= 2)
 *   T        half period (> 0); omega = pi / T
 *   eps      tolerance on ||b - A d||_2 (> 0) when K_fixed == 0
 *   K_fixed  > 0: fit exactly this many coefficients, ignore eps
 *   out      as fbf_fit_coeffs (out->levels = L)
 * Returns FBF_ERR_INVALID_ARGUMENT for a null pointer, L < 2, a non-finite
 * sample or bad T / eps; FBF_ERR_RANGE if K_fixed exceeds FBF_KMAX or L;
 * FBF_ERR_NOT_CONVERGED (out filled) when eps is not reached by
 * min(L, FBF_KMAX) coefficients.
 */
fbf_status fbf_fit_coeffs_samples(const double *phi, int L, double T, double eps, int K_fixed,
                                  fbf_coeffs *out);

/*
 * fbf_filter -- Algorithm 1 (Shiftable Bilateral Filtering) on the GPU.
 *
 * Computes, for every pixel, fhat(i) = P(i) / Q(i) with
 *   P = sum_n d_n Re[e^{-i n w f} (w * (f e^{i n w f}))],
 *   Q = sum_n d_n Re[e^{-i n w f} (w * e^{i n w f})],
 * i.e. eq. (9) with phi_N, by one fused kernel that stages each image tile and
 * its W halo in shared memory, generates the modulated channels on the fly,
 * runs the separable row and column passes and accumulates all K terms in
 * registers: the image is read once and only the output is written.
 *
 *   p          parameters; p->coeffs from fbf_fit_coeffs (K <= FBF_KMAX)
 *   d_in       device image, H rows of Wd elements of type dtype, row pitch
 *              in_pitch bytes (>= Wd * element size)
 *   dtype      FBF_U8: values 0..255, coeffs->T must be an integer >= 1
 *              (the phase n*omega*f is reduced exactly in integers);
 *              FBF_F32: any finite values, any T > 0; FP32 form only, W <= 32
 *   d_out      device FP32 output, H x Wd, row pitch out_pitch bytes; must not
 *              overlap d_in
 *   stream     CUDA stream (0 = legacy default stream)
 * The approximation guarantee of eq. (12) needs 0 <= f <= T and
 * T >= every window difference.  H == 0 or Wd == 0 is a no-op.
 * Returns FBF_ERR_RANGE when W > FBF_WMAX, FBF_ERR_UNSUPPORTED for a form or
 * dtype this build does not implement, FBF_ERR_CUDA when the launch fails.
 */
fbf_status fbf_filter(const fbf_params *p, const void *d_in, fbf_dtype dtype, int H, int Wd,
                      size_t in_pitch, float *d_out, size_t out_pitch, cudaStream_t stream);

/* ---- Batched filtering ---------------------------------------------------
 * Many uint8 images of uneven sizes, each with its own spatial window, range
 * kernel, sigma_r, T and tolerance (hence its own K), filtered by one
 * CUDA graph whose schedule (persistent launches over all the images, or one
 * launch per image) the plan picks by timing the candidates on the batch
 * itself. */

typedef struct fbf_plan fbf_plan; /* owns its device tables and the graph */

typedef struct {
  const void *d_in;           /* device uint8 image, row pitch in_pitch bytes            */
  float *d_out;               /* device FP32 output, row pitch out_pitch bytes           */
  int H, Wd;                  /* rows, columns                                           */
  size_t in_pitch, out_pitch; /* bytes                                                   */
  fbf_spatial_kernel spatial;
  double sigma_s;
  int W;                      /* half window; <= 0 selects ceil(3 sigma_s); <= FBF_WMAX  */
  fbf_range_kernel range;
  double sigma_r, T, eps;     /* as fbf_fit_coeffs (T an integer for uint8 images)       */
  int K_fixed, levels;        /* as fbf_fit_coeffs                                       */
} fbf_image_desc;

/* Schedules a plan can replay (see fbf_plan_create). */
typedef enum {
  FBF_SCHEDULE_PERSISTENT = 0,      /* one persistent FP32 launch, 32 x 192 tiles     */
  FBF_SCHEDULE_PERSISTENT_WIDE = 1, /* one persistent FP32 launch, 64 x 96 tiles      */
  FBF_SCHEDULE_PER_IMAGE_FP32 = 2,  /* one single-image FP32 launch per image         */
  FBF_SCHEDULE_PER_IMAGE_FORM = 3,  /* one launch per image in the plan's form        */
  FBF_SCHEDULE_PER_IMAGE_FP32_STREAMS = 4, /* PER_IMAGE_FP32 on 4 concurrent branches */
  FBF_SCHEDULE_PER_IMAGE_FORM_STREAMS = 5, /* PER_IMAGE_FORM on 4 concurrent branches */
  FBF_SCHEDULE_PERSISTENT_TC = 6           /* persistent tensor-core launches, one per window band */
} fbf_schedule;

/*
 * fbf_plan_create -- fit every image's coefficients (Algorithm 2, host FP64)
 * and capture the plan's schedule in a CUDA graph on the current device.
 * Candidate schedules: PERSISTENT (one CTA per SM pulling cost-sorted (image,
 * tile) items from a counter; FP32 tile body with run-time taps), its 64 x 96
 * tile variant PERSISTENT_WIDE (when every W <= 16), PER_IMAGE_FP32 (the
 * single-image FP32 kernels, one launch each), PER_IMAGE_FORM (one launch
 * per image in `form`) and the two per-image schedules with their launches
 * spread over four concurrent graph branches (largest images first, each to
 * the least loaded branch), so that small images and the last wave of one
 * image's tiles share the GPU with other images (PERSISTENT needs every
 * W <= 32), and PERSISTENT_TC: one persistent launch of the tensor-core
 * kernel per window band present (W <= 16, 17..32, 33..48), each with one CTA
 * per SM taking the (image, tile) items of the band's images -- sorted by
 * estimated cost, most expensive first, CTA b taking items b, b + #SMs, ...
 * -- and rebuilding the image's Toeplitz matrices whenever its next item
 * belongs to another image (tiles 32 x (128 - 2W), every W <= FBF_WMAX,
 * T <= 255).
 * form FP32: PERSISTENT, PERSISTENT_WIDE and both PER_IMAGE_FP32 schedules;
 * AUTO: those and both PER_IMAGE_FORM schedules (per image as fbf_filter's
 * AUTO); TC_FP16_SINGLE: PERSISTENT_TC and both PER_IMAGE_FORM schedules; the
 * split tensor-core forms: both PER_IMAGE_FORM schedules.
 * The concurrent schedules need images whose outputs overlap no other
 * image's output or input.
 * With more than one candidate the plan autotunes: it replays every
 * candidate on the given images -- writing their outputs -- times each with
 * CUDA events (three rounds over the candidates, three replays a round, each
 * candidate's best round) and keeps the fastest (fbf_plan_schedule reports
 * which, with that time); this
 * synchronises the device.  The pointers in `descs` are baked into the plan:
 * the images must stay allocated while the plan is used.  Allocates device
 * memory (synchronously) for the persistent tables.  A fit that misses its
 * tolerance returns FBF_ERR_NOT_CONVERGED.
 */
fbf_status fbf_plan_create(const fbf_image_desc *descs, int n, fbf_form form, fbf_border border,
                           fbf_plan **out);
/* As fbf_plan_create, but captures the one given schedule without autotuning
 * (no replay at creation).  FBF_ERR_INVALID_ARGUMENT when `schedule` is not a
 * candidate of `form` (or out of range). */
fbf_status fbf_plan_create_schedule(const fbf_image_desc *descs, int n, fbf_form form, fbf_border border,
                                    fbf_schedule schedule, fbf_plan **out);
/* Filter every image of the plan: one cudaGraphLaunch on `stream`. */
fbf_status fbf_filter_batched(fbf_plan *plan, cudaStream_t stream);
/* Release the plan (the caller synchronises first if a launch is in flight). */
fbf_status fbf_plan_destroy(fbf_plan *plan);
/* Number of images and (image, tile) work items of a plan. */
fbf_status fbf_plan_size(const fbf_plan *plan, int *n_images, int *n_items);
/* The schedule the plan replays and the time autotuning measured for it (ms
 * per replay; 0 when the plan had a single candidate). */
fbf_status fbf_plan_schedule(const fbf_plan *plan, fbf_schedule *schedule, double *ms);

/*
 * fbf_filter_backward -- gradient of L = sum_i g(i) fhat(i) with respect to the
 * input image f, where fhat is eq. (9) computed by fbf_filter (FP32 form,
 * FBF_F32 input).  T, omega and the coefficients are constants.
 *
 * With a = g / Q and b = g fhat / Q, f(m) enters eq. (9) both as a neighbour
 * and as the centre; per harmonic n the derivative takes the forward channels
 * Fbar_n, Gbar_n (recomputed per tile, not stored) and the transposed
 * convolutions of a e^{-i n w f} and b e^{-i n w f}: eight real channels.
 * Under REFLECT the transposed border is exact (mirrored contributions are
 * folded back onto their source pixels).
 *
 *   d_in       FP32 image (H x Wd), row pitch `pitch` bytes (multiple of 4)
 *   d_gout     FP32 upstream gradient g, same shape and pitch
 *   d_out_fwd  ignored (may be NULL): Q is needed, so the forward is recomputed
 *   d_gin      FP32 output dL/df, same shape and pitch
 * Allocates its scratch (8 bytes per pixel, plus (H+2W)(Wd+2W) floats under
 * REFLECT) stream-ordered from the library's pool on `stream`.
 * W <= 32.  Returns FBF_ERR_UNSUPPORTED for the tensor-core forms.
 */
fbf_status fbf_filter_backward(const fbf_params *p, const float *d_in, const float *d_gout,
                               const float *d_out_fwd, float *d_gin, int H, int Wd, size_t pitch,
                               cudaStream_t stream);

/*
 * fbf_filter_backward_noalloc -- the same gradient as fbf_filter_backward, for
 * callers that must not allocate device memory (the paper has no counterpart:
 * this is a deployment variant).  Typical such callers: an application whose
 * framework has already reserved the device memory for its own allocator, or a
 * real-time loop where an allocation call (which may block, synchronise, or
 * fail under memory pressure) is not allowed.
 *
 * Arguments, results and limits are those of fbf_filter_backward.  Scratch comes
 * from one array of FBF_NOALLOC_SCRATCH_BYTES bytes that the library keeps in
 * device memory on every GPU that loads it, until the process exits; nothing is
 * allocated or freed.  A request needing more than that (8 bytes per pixel,
 * plus (H+2W)(Wd+2W) floats under REFLECT, rounded up to 256 bytes) returns
 * FBF_ERR_RANGE.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress, which allocates nothing); the first
 * lookup on a device may load the library's device code, so make the first
 * call on a device before any stream capture.  All calls share the array:
 * calls whose GPU work overlaps (e.g. on two streams) race and give wrong
 * results; serialise them.
 */
#define FBF_NOALLOC_SCRATCH_BYTES (16u << 20)
fbf_status fbf_filter_backward_noalloc(const fbf_params *p, const float *d_in, const float *d_gout,
                                       const float *d_out_fwd, float *d_gin, int H, int Wd, size_t pitch,
                                       cudaStream_t stream);

/*
 * fbf_filter_stack / fbf_filter_backward_stack -- N images of one size under
 * one set of parameters (a stack, e.g. a batch of a training step): image i
 * starts at d_in + i * in_image_stride bytes (its output, gradient and
 * gradient-input likewise with their own stride), and each image is filtered
 * (or differentiated) exactly as fbf_filter (fbf_filter_backward) would, one
 * launch after the other on `stream`.  Image strides must be at least H times
 * the row pitch (images do not overlap); N = 0 does nothing.  The backward
 * allocates its scratch once for the stack (one image's worth, reused
 * stream-ordered).  Errors as for the single-image calls, plus
 * FBF_ERR_INVALID_ARGUMENT for N < 0 or a short image stride.
 */
fbf_status fbf_filter_stack(const fbf_params *p, const void *d_in, fbf_dtype dtype, int N, int H, int Wd,
                            size_t in_pitch, size_t in_image_stride, float *d_out, size_t out_pitch,
                            size_t out_image_stride, cudaStream_t stream);
fbf_status fbf_filter_backward_stack(const fbf_params *p, const float *d_in, const float *d_gout, float *d_gin,
                                     int N, int H, int Wd, size_t pitch, size_t image_stride,
                                     cudaStream_t stream);

/* Dynamic range T of an 8-bit image over the window Omega = [-W, W]^2: the
 * quantity defined at the start of Sec. III, T = max over pixels i and offsets
 * j in Omega of |f(i - j) - f(i)|, neighbours outside the image excluded (the
 * mirrored neighbours of REFLECT are image pixels inside the same clipped
 * window, so both borders give the same T).  Passing this T (instead of the
 * full 255) to fbf_fit_coeffs gives omega = pi / T and, for the same sigma_r
 * and eps, no more -- often fewer -- terms (Sec. III).
 *
 * d_in: H x Wd bytes (dtype FBF_U8), row pitch `pitch` bytes >= Wd.  d_T: one
 * device uint32 that receives T in 0..255; it is zeroed on `stream` first,
 * then written by the kernel (asynchronous: read it after the stream).  W in
 * 0..FBF_WMAX.  Empty images give T = 0.  Errors: FBF_ERR_INVALID_ARGUMENT
 * (null pointers, negative sizes, pitch < Wd), FBF_ERR_UNSUPPORTED (float
 * input), FBF_ERR_RANGE (W > FBF_WMAX).  Allocates nothing. */
fbf_status fbf_local_range(const void *d_in, fbf_dtype dtype, int H, int Wd, size_t pitch, int W,
                           unsigned int *d_T, cudaStream_t stream);

/* Half window actually used for the parameters (W, or ceil(3 sigma_s) when
 * W <= 0), or -1 when invalid.  Host only. */
int fbf_resolve_window(const fbf_params *p);

/* Reads and clears the library's device-side error word on the current device
 * (non-zero when a bounded wait inside a kernel gave up: that kernel then
 * abandoned its remaining tiles, so its output is incomplete).  Synchronises
 * the device.  *code receives the word; returns FBF_ERR_TIMEOUT when it is
 * non-zero, FBF_OK when it is zero, FBF_ERR_CUDA when the device cannot be
 * read. */
fbf_status fbf_device_error(unsigned int *code);

/* Poll limit of the tensor-core kernels' bounded waits (mbarrier waits on
 * their MMAs and TMA copies), for the calls launched after it: polls >= 0 sets
 * it (0: every wait gives up at once -- a way to exercise the failure path,
 * which then leaves the outputs incomplete and sets the device error word),
 * polls < 0 restores the default (about a second of polling).  A process-wide
 * setting; not part of the filter.  FBF_ERR_RANGE above 2^32 - 1. */
fbf_status fbf_set_wait_limit(long long polls);

/* FP32-pipe throughput probe (the roofline denominator of the FP32 form).
 * Runs independent FMA chains on every SM of `device` -- scalar FFMA when
 * packed == 0, the two-lane fma.rn.f32x2 otherwise -- and writes the measured
 * throughput in TFLOP/s (2 flops per FMA) to *tflops.  Not part of the filter:
 * it allocates and frees a small result buffer and synchronises the device. */
fbf_status fbf_measure_fp32_peak(int device, int packed, double *tflops);

/* Static description of a status code. */
const char *fbf_status_string(fbf_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int fbf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FBF_H */
