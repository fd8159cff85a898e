/*
 * lensed.h -- C ABI of the GB300 (sm_103a) ray-tracing likelihood library.
 *
 * The library computes, for parametric lens and source models, the expected
 * image of a strong-lensing system and its Gaussian log-likelihood, as
 * defined in Tessore, Bellagamba & Metcalf, "Lensed: a code for the forward
 * reconstruction of lenses and sources from strong lensing observations":
 *
 *   Sec. 2.1, Eq. 1   lens equation            y = x - alpha(x)
 *   Sec. 2.1, Eq. 2   image-plane brightness   I(x) = I_L(x) + I_S(y(x))
 *   Sec. 2.1, Eq. 3   pixel luminosity         L_i = integral of I over pixel i
 *   Sec. 3.1, Eq. 14  quadrature               L_i ~ sum_k w_k I(x_k)
 *   Sec. 3.1, Eq. 15  PSF                      L*_ij = sum_kl F_{-k,-l} L_{i+k,j+l}
 *                     (PSF normalised to unit sum, border padded by
 *                      repeating the nearest pixel)
 *   Sec. 3.2, Eq. 17  loglike = -1/2 sum_i w_i (d_i - L*_i)^2, w_i = 1/s_i^2,
 *                     a masked pixel has w_i = 0
 *   Sec. 3.3, Eq. 21  s_i^2 = (d_i + b_i) / g_i when no variance is given,
 *                     times an optional multiplicative extra weight
 *   Sec. 4.1, Eqs. 22-23  elliptical Sersic profile, geometric-mean radius
 *
 * Conventions (the paper leaves them open):
 *   - images are row-major [ny][nx]; row i runs along +y, column j along +x;
 *     pixel (i, j) is the square of side h centred on
 *     ((j - (nx-1)/2) h, (i - (ny-1)/2) h) arcsec;
 *   - a PSF array is row-major [psf_ny][psf_nx] = [2p+1][2q+1], centred on
 *     its middle element F_{0,0}; both sizes odd;
 *   - position angles in degrees, counter-clockwise from +x to the major axis;
 *   - component parameters, in this order:
 *       LENSED_SIE        x, y, b, q, pa, s      (Einstein radius b in the
 *                          geometric-mean convention, core radius s)
 *       LENSED_SHEAR      x, y, gamma, phi       (about the centre x, y)
 *       LENSED_POINTMASS  x, y, theta_E
 *       LENSED_SERSIC     x, y, r_e, mag, n, q, pa
 *       LENSED_DEVAUC     x, y, r_e, mag, q, pa  (Sersic with n = 4)
 *       LENSED_GAUSS      x, y, sigma, mag, q, pa
 *       LENSED_SKY        S                      (flat sky, Sec. 5: constant
 *                          surface brightness S per arcsec^2 in the data's
 *                          flux units, either sign)
 *     Total flux of a light profile is 10^(-0.4 (mag - zeropoint)).
 *     A source on LENSED_PLANE_SOURCE_IMAGE (image-plane prior, Sec. 5)
 *     takes x, y as an image-plane position theta and is centred on
 *     theta - alpha(theta), the same point's lens deflection (Eq. 1).
 *
 * Memory and streams: every input array of lensed_create_model is copied
 * into library-owned device memory, so the caller may free it on return.
 * Parameter and output arrays of the evaluation calls are caller-owned
 * device pointers (unless the call name ends in _host); the library never
 * frees caller memory.  Work is enqueued on the caller's CUDA stream
 * (NULL = legacy default stream) and the calls return without synchronising,
 * except lensed_create_model, lensed_autotune and the _host calls.  A model
 * must not be used from two host threads at once.  Scratch memory is owned
 * by the model, grown on demand and released by lensed_destroy.
 *
 * Errors: every call returns a lensed_status; nothing aborts the process or
 * traps the GPU.  lensed_last_error() returns a thread-local message for the
 * last failing call of the calling thread.  A parameter point outside the
 * model's domain (an axis ratio outside (0, 1], a non-positive radius or
 * Sersic index, a negative Einstein radius or core) is not an error: its
 * log-likelihood is -inf.
 */
#ifndef LENSED_GB300_H
#define LENSED_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LENSED_OK = 0,
    LENSED_E_ARG = -1,         /* invalid argument or descriptor */
    LENSED_E_NOMEM = -2,       /* device or host allocation failed */
    LENSED_E_CUDA = -3,        /* a CUDA runtime call failed */
    LENSED_E_NONFINITE = -4,   /* non-finite data, variance, weight or PSF */
    LENSED_E_TIMEOUT = -5,     /* a bounded device-side wait expired */
    LENSED_E_UNSUPPORTED = -6  /* valid request this build cannot serve */
} lensed_status;

enum {
    LENSED_SIE = 1,
    LENSED_SHEAR = 2,
    LENSED_POINTMASS = 3,
    LENSED_SERSIC = 4,
    LENSED_DEVAUC = 5,
    LENSED_GAUSS = 6,
    LENSED_SKY = 7
};

enum {
    LENSED_PLANE_LENS = 0,        /* mass: contributes to alpha */
    LENSED_PLANE_FOREGROUND = 1,  /* light evaluated at the image position x */
    LENSED_PLANE_SOURCE = 2,      /* light evaluated at the traced position y */
    LENSED_PLANE_SOURCE_IMAGE = 3 /* as SOURCE, position given on the image
                                     plane (image-plane prior); not for SKY */
};

/* Integration rules (Sec. 3.1, Eq. 14; rule list of Sec. 4.5), each the
 * Cartesian square of a 1-D rule on the pixel:
 *   LENSED_RULE_POINT  one ray at the pixel centre (rule_order ignored)
 *   LENSED_RULE_SUB    rule_order x rule_order uniform sub-sampling
 *   LENSED_RULE_GL     rule_order x rule_order Gauss-Legendre
 *   LENSED_RULE_GK     Gauss-Kronrod: the (2N+1) x (2N+1) Kronrod extension
 *                      of the N x N Gauss rule, N = rule_order in 1..7
 *                      (g3k7 is N = 3, the paper's default; g5k11 N = 5;
 *                      g7k15 N = 7); lensed_render_error gives its
 *                      embedded-Gauss error estimate per pixel            */
enum { LENSED_RULE_POINT = 0, LENSED_RULE_SUB = 1, LENSED_RULE_GL = 2, LENSED_RULE_GK = 3 };
#define LENSED_MAX_KRONROD_ORDER 7

/* Arithmetic of the evaluation, and its accuracy against an FP64 evaluation
 * of the same discretised model (the target being |dlogL| <= 1e-3 where
 * chi^2 / N <= 10, and <= 1e-6 |logL| elsewhere):
 *   LENSED_PREC_FP32   rays, brightness and PSF in FP32; chi^2 summed in FP64.
 *                      Misses the target: the float grid of traced positions
 *                      leaves up to ~1e-2 absolute (a few 1e-6 relative) on
 *                      steep, compact sources.
 *   LENSED_PREC_MIXED  as FP32, but the SIE deflection is evaluated in FP64
 *                      for axis ratios close to 1 (e = sqrt(1-q^2) < 0.05)
 *                      and for rays within 2 s / q of the SIE centre.  Misses
 *                      the target like FP32.
 *   LENSED_PREC_FP64   everything in FP64 (validation mode).  Meets it.
 *   LENSED_PREC_MIXED_FF  as MIXED, and every ray whose FP32 source-plane
 *                      position falls within half an effective radius of a
 *                      Sersic-type source (R < r/2) is re-traced with the lens
 *                      equation in float-float arithmetic (~44 bits).  Meets
 *                      the target on the 64x64 and 200x200 workloads and near
 *                      the posterior of large images; far from the posterior
 *                      on large, high signal-to-noise images (chi^2 / N of a
 *                      few, |logL| >= 1e4) FP32 storage of the images leaves
 *                      a few 1e-6 relative.  1.4-3x the cost of MIXED.
 *                      Its batched calls also keep a queue for the second
 *                      pass of the re-traces (a 24-byte header per trace
 *                      block and point, and 4 bytes per re-traced ray, at
 *                      most 256 MiB) beside the image scratch. */
enum { LENSED_PREC_FP32 = 0, LENSED_PREC_MIXED = 1, LENSED_PREC_FP64 = 2,
       LENSED_PREC_MIXED_FF = 3 };

enum { LENSED_RENDER_UNCONVOLVED = 0, LENSED_RENDER_CONVOLVED = 1 };

#define LENSED_MAX_COMPONENT_PARAMS 8
#define LENSED_MAX_COMPONENTS 16
#define LENSED_MAX_RULE_ORDER 16
#define LENSED_MAX_PSF_HALF 15     /* PSF sizes up to 31 x 31 */
#define LENSED_MAX_IMAGE_SIDE 4096

/* One model component.  Parameter k is free when free_index[k] >= 0 (then
 * it is read from the parameter vector at that index; several components
 * may share an index, which ties parameters) and fixed to value[k]
 * otherwise. */
typedef struct {
    int type;   /* LENSED_SIE ... LENSED_SKY */
    int plane;  /* LENSED_PLANE_* (mass types must be LENSED_PLANE_LENS) */
    int free_index[LENSED_MAX_COMPONENT_PARAMS];
    double value[LENSED_MAX_COMPONENT_PARAMS];
} lensed_component;

/* One imaging system (Sec. 3, steps (i)-(ii) of the high-level algorithm):
 * data, variance or gain/offset, mask, PSF, rule and model.  All pointers
 * are HOST pointers, read during lensed_create_model only. */
typedef struct {
    int nx, ny;                    /* image size, 1 .. LENSED_MAX_IMAGE_SIDE */
    double pixel_scale;            /* h, arcsec per pixel, > 0 */
    const double *data;            /* [ny*nx] observed d_i; required */
    const double *variance;        /* [ny*nx] s_i^2, or NULL: use gain/offset */
    double gain, offset;           /* Eq. 21: s_i^2 = (d_i + offset) / gain */
    const double *extra_weight;    /* [ny*nx] factor on w_i, or NULL */
    const unsigned char *mask;     /* [ny*nx], nonzero = excluded, or NULL */
    const double *psf;             /* [psf_ny*psf_nx] or NULL (no PSF) */
    int psf_nx, psf_ny;            /* odd, <= 2*LENSED_MAX_PSF_HALF+1 */
    int rule, rule_order;          /* LENSED_RULE_*, order 1..LENSED_MAX_RULE_ORDER */
    double zeropoint;              /* magnitude zero point */
    int n_components;              /* 1 .. LENSED_MAX_COMPONENTS */
    const lensed_component *components;
    int n_params;                  /* length of this system's parameter vector */
} lensed_system_desc;

typedef struct lensed_model lensed_model; /* opaque, library-owned */

typedef struct {
    int n_systems;
    int n_params_max;        /* row stride of the parameter arrays */
    int precision;
    long long total_pixels;  /* sum over systems of nx*ny */
    long long rays_per_eval_all;     /* sum over systems of nx*ny*rays/pixel */
    long long rays_per_eval_traced;  /* rays lensed_loglike_* traces per point
                                        and system (pixels the masked chi^2
                                        needs, through the PSF footprint) */
    long long psf_taps_per_eval;     /* multiply-adds of the PSF per point */
    double flops_per_ray;    /* algorithmic FP32 operations per traced ray,
                                counted from the formulas (add, mul, div,
                                sqrt, transcendental = 1, fused pair = 2),
                                averaged over the traced rays */
    double transcendentals_per_ray;  /* of which atan/atanh/exp2/log2/sqrt */
} lensed_model_info;

/* Build a model of n_systems imaging systems (Sec. 3, steps (i)-(ii)).
 * Validates every descriptor, computes the weights w_i (Sec. 3.2-3.3),
 * normalises the PSF (Sec. 3.1), builds the quadrature table (Eq. 14) and
 * copies everything to the current CUDA device.  Synchronous.
 * Returns LENSED_E_ARG for a malformed descriptor (sizes, even PSF, unknown
 * type or plane, free index >= n_params), LENSED_E_NONFINITE for non-finite
 * data/variance/weights/PSF or a non-positive variance on an unmasked pixel,
 * LENSED_E_NOMEM/LENSED_E_CUDA on device failures.  *out is set only on
 * success. */
int lensed_create_model(const lensed_system_desc *systems, int n_systems, int precision,
                        lensed_model **out);

/* The 1-D integration rule on the unit pixel that a system with this rule
 * and order uses (Sec. 3.1, Eq. 14; the 2-D rule is its Cartesian square):
 * writes the offsets t (in (-1/2, 1/2), ascending) and weights w (summing
 * to one) into HOST arrays of at least LENSED_MAX_RULE_ORDER doubles, and
 * for LENSED_RULE_GK the embedded Gauss weights into w_gauss (zero on the
 * Kronrod-only nodes; may be NULL).  Returns the number of nodes, or
 * LENSED_E_ARG for an unknown rule or an order out of range.  Host only:
 * needs no device. */
int lensed_rule_nodes(int rule, int order, double *t, double *w, double *w_gauss);

/* Free everything the model owns.  NULL-safe.  Synchronises the device
 * work the model has in flight before freeing. */
void lensed_destroy(lensed_model *m);

/* Describe the model (sizes and work per evaluation). */
int lensed_model_info_get(const lensed_model *m, lensed_model_info *info);

/* Expected image of one system at one parameter point (Eqs. 1-3, 14, and
 * Eq. 15 when flags == LENSED_RENDER_CONVOLVED): writes L or L* for every
 * pixel into out_image, a DEVICE array of ny*nx floats.  params is a
 * DEVICE array of the system's n_params doubles.  If the point is outside
 * the domain the image is filled with NaN.  Asynchronous on stream. */
int lensed_render(lensed_model *m, int system, const double *params, int flags,
                  float *out_image, void *stream);

/* Per-pixel integration error estimate of one Gauss-Kronrod system (Sec.
 * 3.1: the Gauss rule embedded in the Kronrod rule estimates each pixel's
 * quadrature error, kept as a diagnostic beside the image).  Writes
 * |L_K - L_G| for every pixel into out_error, a DEVICE array of ny*nx floats
 * (row-major), where L_K is the unconvolved pixel luminosity by the
 * (2N+1)^2-point Kronrod rule (what lensed_render writes with
 * LENSED_RENDER_UNCONVOLVED) and L_G the one by the N^2-point Gauss rule on
 * the shared nodes, both in the model's precision.  params is a DEVICE
 * array of the system's n_params doubles.  Returns LENSED_E_ARG if the
 * system's rule is not LENSED_RULE_GK.  Outside the domain the map is NaN.
 * Asynchronous on stream; it shares the model's render scratch with
 * lensed_render, so render calls on one model must not overlap. */
int lensed_render_error(lensed_model *m, int system, const double *params, float *out_error,
                        void *stream);

/* Log-likelihood (Eq. 17) of P parameter points for every system, batched:
 * params is a DEVICE array [n_systems][P][n_params_max] of doubles (entries
 * beyond a system's n_params are ignored), out_loglike a DEVICE array
 * [n_systems][P] of doubles.  All points of all systems go through one
 * CUDA-graph launch whose tile configuration comes from the autotuner (or
 * a default).  Asynchronous on stream.  P must be >= 1. */
int lensed_loglike_batch(lensed_model *m, const double *params, int P, double *out_loglike,
                         void *stream);

/* Same result as lensed_loglike_batch, computed the way the paper's code
 * schedules it: one parameter point of one system at a time, each with its
 * own kernel launches and no graph.  Kept as the baseline the batched path
 * is measured against.  Results are bit-identical to lensed_loglike_batch. */
int lensed_loglike_plain(lensed_model *m, const double *params, int P, double *out_loglike,
                         void *stream);

/* lensed_loglike_batch with HOST arrays: copies params to the device,
 * evaluates, copies the results back and synchronises the stream before
 * returning.  Pinned host memory gives the fastest copies. */
int lensed_loglike_batch_host(lensed_model *m, const double *params_host, int P,
                              double *out_host, void *stream);

/* lensed_loglike_batch for callers that cannot allocate device memory
 * during evaluation: for example a sampler embedded in a framework that has
 * reserved nearly all device memory for its own pool (so cudaMalloc fails),
 * or a service whose device-memory budget is fixed at start-up.  This call
 * allocates nothing: its scratch (per-point constants, validity flags,
 * pixel luminosities, chi^2 partials) lives in one fixed 32 MiB device array
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.  The paper has no counterpart; it is a property
 * of this library's interface.
 *   - Same arguments and results as lensed_loglike_batch (params and
 *     out_loglike are caller-owned DEVICE arrays), bit for bit, launched
 *     directly on stream without a graph.
 *   - It uses the model's launch configuration except that, in
 *     LENSED_PREC_MIXED_FF, the float-float re-traces always run inside
 *     the trace blocks (the second-pass queue would need memory of its own);
 *     both forms give the same bits, so only the speed can differ from the
 *     configuration lensed_tuned_config reports.
 *   - P is limited by the array: the per-point scratch of all P points plus
 *     the pixel luminosities of at least one point must fit in 32 MiB;
 *     larger requests return LENSED_E_ARG with the limit in the message.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the one array and overwrites it; calls whose work
 *     overlaps on the GPU (two streams, or two host threads) race and give
 *     wrong results: serialise them.
 *   - Nothing in the array needs clearing: every value is written before
 *     it is read within the call. */
int lensed_loglike_batch_noalloc(lensed_model *m, const double *params, int P,
                                 double *out_loglike, void *stream);

/* Time the candidate launch configurations (trace block size; PSF applied
 * directly or, where the PSF has numerical rank <= 3, as separable passes;
 * the trace as one CTA per (trace block, point) or as a persistent,
 * work-queued launch whose resident CTAs take those items from a counter;
 * for LENSED_PREC_MIXED_FF also whether the float-float re-traces run inside
 * the trace blocks or in a second kernel) on a batch of P points drawn
 * inside the given DEVICE parameter array (same layout as
 * lensed_loglike_batch) and keep the fastest for later calls; then, with
 * that configuration, time whole scratch chunks against chunks sized to half
 * and a quarter of L2 (lensed_set_chunk_points) and keep the faster.  The
 * trace block size, the launch form, the place of the re-traces and the
 * chunk size never change a result; the PSF mode changes the FP32 summation
 * order of Eq. 15 (differences at the float rounding level).  Synchronous. */
int lensed_autotune(lensed_model *m, const double *params, int P, void *stream);

/* Index of the configuration in use (-1: default) and its description (with
 * the chunk limit, if one is set), for reports. */
int lensed_tuned_config(const lensed_model *m, char *buf, int buflen);

/* Measured FP32 throughput of this GPU for the roofline (the paper has no
 * counterpart): *fma_tflops = FP32 fused multiply-adds (2 flops each) per
 * second, *mufu_tops = special-function (ex2) operations per second, both in
 * units of 1e12, from probes of independent dependency chains over every SM.
 * Synchronous; allocates a small scratch buffer. */
int lensed_measure_alu_peaks(double *fma_tflops, double *mufu_tops, void *stream);

/* Accuracy probe of the FP32 SIE's inverse tangents (Sec. 2.1, Eqs. 2-3:
 * the deflection's atan(e x' / (psi + s)) and atanh(e y' / (psi + q^2 s))).
 * For i < count, with DEVICE arrays n[count], d[count] (d >= 0; |n| < d for
 * atanh) it writes to the DEVICE array out[4 * count]: out[i] = the kernel's
 * atan(n/d), out[count + i] = its atanh(n/d), out[2 count + i] = CUDA's
 * atanf of the rounded FP32 quotient, out[3 count + i] = atanhf of it.
 * Asynchronous on `stream`; LENSED_E_ARG for a negative count or a NULL
 * pointer with count > 0. */
int lensed_eval_sie_trig(const float *n, const float *d, long long count, float *out,
                         void *stream);

/* Use configuration `index` (0 .. n-1 as lensed_tuned_config numbers them,
 * -1 = default) instead of the autotuner's choice; returns the number of
 * configurations n, or LENSED_E_ARG for an index out of range.  n = 12:
 * 0-5 = trace blocks of 128, 256, 64 pixels with the direct PSF, then the
 * same three with separable passes; 6-11 = 0-5 with the trace as a
 * persistent, work-queued launch.  LENSED_PREC_MIXED_FF: n = 24, and
 * 12 + k runs configuration k with the float-float re-traces in a second
 * kernel. */
int lensed_set_config(lensed_model *m, int index);

/* Points per scratch chunk of the batched schedule (a8; the paper has no
 * counterpart).  lensed_loglike_batch runs the trace and PSF passes over
 * chunks of points whose pixel luminosities fit the model's scratch; with
 * points > 0 a chunk holds at most that many points, so that a chunk's
 * luminosities can stay in L2 between the trace pass that writes them and
 * the PSF pass that reads them; points = 0 lifts the limit.  Chunks are
 * independent ranges of points, so the limit never changes a result, only
 * the number of launches and the DRAM traffic.  lensed_autotune sets it too
 * (no limit, or half or a quarter of L2 over one point's luminosities);
 * lensed_set_config leaves it as it is.  LENSED_E_ARG for points < 0. */
int lensed_set_chunk_points(lensed_model *m, int points);

/* Launch plan of one lensed_loglike_batch call with P points: number of
 * kernels it launches (*launches) and the number of points per scratch
 * chunk (*chunk_points).  Nothing is launched. */
int lensed_batch_plan(lensed_model *m, int P, int *launches, int *chunk_points);

/* Run the batched schedule of lensed_loglike_batch once without the graph,
 * with CUDA events around every launch on stream, and report the device
 * milliseconds spent per stage in stage_ms[4]: prologue, trace (rays,
 * Eqs. 1-3, 14), PSF + chi^2 (Eqs. 15, 17), finalize; and in
 * *trace_launches the number of trace launches.  Same results as
 * lensed_loglike_batch.  Synchronous. */
int lensed_profile_batch(lensed_model *m, const double *params, int P, double *out_loglike,
                         void *stream, double *stage_ms, int *trace_launches);

/* ------------------------------------------------------------------------
 * Log-likelihood surrogate network (the paper has no counterpart; the
 * sampling driver uses it to pre-screen proposals, and the exact likelihood
 * decides every point it accepts):
 *     h1 = silu(x W1^T + b1), h2 = silu(h1 W2^T + b2), h3 = silu(h2 W3^T + b3),
 *     y  = h3 . w4 + b4,   loss = mean over the batch of (y - t)^2 / 2.
 * BF16 weights and activations on the tensor cores, FP32 accumulation, FP32
 * master weights with Adam (beta 0.9 / 0.999, eps 1e-8).  Flat parameter
 * order: W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], w4 [H],
 * b4 [1], each W stored [out][in].  Inputs X are row-major [B][n_in] FP32
 * DEVICE arrays (the caller normalises them); targets t and outputs y are
 * [B] FP32 DEVICE arrays.  The products run on the tensor cores
 * (tcgen05.mma, accumulators in tensor memory); their waits are bounded, and
 * an expired wait is reported as LENSED_E_TIMEOUT by the next
 * lensed_mlp_get_params.  Errors: status codes, message from
 * lensed_mlp_last_error(). */
typedef struct lensed_mlp lensed_mlp;


/* n_in 1..64, hidden a multiple of 64, max_batch >= 1 (largest B of a
 * gradient or training call; forward calls of any B run in slices of it).
 * Parameters start at zero: set them with lensed_mlp_set_params. */
int lensed_mlp_create(int n_in, int hidden, int max_batch, lensed_mlp **out);
void lensed_mlp_destroy(lensed_mlp *m);                       /* NULL-safe */
long long lensed_mlp_param_count(const lensed_mlp *m);
/* HOST arrays of lensed_mlp_param_count floats; setting resets Adam and
 * clears a recorded expired wait (see lensed_mlp_get_params). */
int lensed_mlp_set_params(lensed_mlp *m, const float *host_params);
int lensed_mlp_get_params(const lensed_mlp *m, float *host_params);
/* y[0..B) = network(X[0..B)); asynchronous on stream. */
int lensed_mlp_forward(lensed_mlp *m, const float *X, int B, float *y, void *stream);
/* Loss (DEVICE scalar) and its gradient (DEVICE [param_count]) on one batch,
 * B <= max_batch; asynchronous. */
int lensed_mlp_gradient(lensed_mlp *m, const float *X, const float *t, int B, float *grad,
                        float *loss, void *stream);
/* One Adam step on one batch (B <= max_batch); writes the batch loss before
 * the step to the DEVICE scalar loss; asynchronous. */
int lensed_mlp_train_step(lensed_mlp *m, const float *X, const float *t, int B, float lr,
                          float *loss, void *stream);
const char *lensed_mlp_last_error(void);

/* Proposals for the nested-sampling driver (Sec. 3.2 samples the prior
 * inside the current likelihood contour; the network's pre-screen is this
 * library's own addition): n candidates, numbered first .. first+n-1 of the
 * counter-based stream `seed` (Philox4x32-10), each a uniform draw inside
 * the ellipsoid v = center + chol z, |z| <= 1.  v lives in the sampler's
 * unit-cube coordinates with each periodic axis shifted by shift[j] (0 on
 * the other axes); the candidate's point is u = v + shift wrapped into
 * [0, 1), which keeps the draws uniform and lets a likelihood contour that
 * straddles the ends of a periodic parameter's range be bounded by one
 * ellipsoid.  A candidate survives when v lies inside the open unit cube
 * and, if m is not NULL, the network's output at x = x_whiten (u - x_center)
 * is below y_cut (the caller's threshold in the network's output units).
 *   d = the dimension (1..32; m's n_in when m is given);
 *   center [d], chol [d][d] (row-major, lower triangle read), shift [d] (or
 *   NULL: no shift), x_center [d], x_whiten [d][d] (row-major): DEVICE
 *   float arrays, caller-owned (the candidates are drawn in FP32 and
 *   returned as doubles);
 *   u_out [n][d] DEVICE doubles, idx_out [n] DEVICE ints, n_out DEVICE int:
 *   the survivors' points and candidate numbers (relative to `first`) in the
 *   first *n_out rows, in no particular order (sort by idx_out for a
 *   reproducible order; each candidate's point is a function of its number
 *   alone).  Asynchronous on stream; grows the network's screening scratch
 *   (synchronising the stream) when n exceeds every earlier n. */
int lensed_mlp_screen_ellipsoid(lensed_mlp *m, int d, int n, unsigned long long seed,
                                unsigned long long first, const float *center,
                                const float *chol, const float *shift,
                                const float *x_center, const float *x_whiten, float y_cut,
                                double *u_out, int *idx_out, int *n_out, void *stream);

/* Fault-injection hooks for tests of the error paths (the paper has no
 * counterpart).  They cause no GPU fault: the failures are made on the host
 * or by a wait that is allowed to give up early.
 *   lensed_debug_fail_alloc(after): process-wide; after >= 0 lets `after`
 *     more device allocations of the library (models and networks) succeed
 *     and refuses every later one with LENSED_E_NOMEM, before cudaMalloc
 *     is called; after < 0 switches the injection off.  Returns the number
 *     of device buffers the library holds at that moment (for leak checks).
 *     A refused lensed_create_model / lensed_mlp_create frees what it had
 *     allocated; a refused per-batch allocation leaves the model usable.
 *   lensed_mlp_debug_spin_limit(m, polls): the pipeline waits of the
 *     network's later tensor-core products give up after `polls` polls of
 *     their mbarrier (0: at once) instead of ~16M.  A product whose wait
 *     gives up waits with the full limit for the tensor-core work it has
 *     already issued, frees its tensor memory, writes no output and records
 *     the expiry, which the next lensed_mlp_get_params reports as
 *     LENSED_E_TIMEOUT; lensed_mlp_set_params clears it.  Values above the
 *     default are clamped to it.
 *   lensed_debug_ff_queue_cap(m, cap): MIXED_FF launches whose float-float
 *     re-traces go to a second kernel see a queue of at most `cap` entries
 *     (cap < 0: the allocated size).  A warp whose rays do not fit marks its
 *     slots empty and re-traces them itself, so the results are unchanged;
 *     the hook exercises that path.  Synchronises the device. */
long long lensed_debug_fail_alloc(long long after);
int lensed_debug_ff_queue_cap(lensed_model *m, long long cap);
int lensed_mlp_debug_spin_limit(lensed_mlp *m, int polls);

/* Thread-local message of the last failing call ("" if none). */
const char *lensed_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LENSED_GB300_H */
