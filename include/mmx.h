/*
 * mmx.h -- C ABI of libmmx, a single-GPU (GB300, sm_103a) integrator of the
 * Landau-Lifshitz-Gilbert equation with FFT demagnetising field and the demag
 * polynomial extrapolation of Lepadatu, arXiv 2107.06729 (Sec. II).
 *
 * Conventions shared by every call:
 *   - Return value: 0 on success, negative on error (MMX_ERR_*), positive for
 *     a warning (MMX_WARN_*).  No C++ exception crosses this boundary.  The
 *     text of the last error of a context is available from mmx_last_error.
 *   - Magnetisation arrays hold unit vectors m = M/Ms in SoA layout
 *     [3][nz][ny][nx] (x fastest), element type double for MMX_FP64 and float
 *     for MMX_FP32_MIXED.  A cell whose m is exactly (0, 0, 0) holds no
 *     material (vacuum, e.g. between the particles of an array, Sec. III):
 *     it adds nothing to the demag field, feels no torque and stays 0.
 *     Fields are in A/m, lengths in m, times in s.
 *   - Every pointer passed in stays owned by the caller.  The library owns the
 *     device buffers it allocates in mmx_create (spectra, stage buffers,
 *     history of exact demag fields) and frees them in mmx_destroy.
 *   - All device work is enqueued on the CUDA stream given to mmx_create
 *     (NULL = legacy default stream).  Calls that return host-visible results
 *     (mmx_run, mmx_step, mmx_get_stats, mmx_save_state) synchronise it.
 *   - Mesh sizes: nx, ny, nz must be powers of two; nx >= 2; ny and nz may be
 *     1 (no padding along that axis); ny = 1 together with nz > 8 (FP32) or
 *     nz > 4 (FP64) is not supported.  Other sizes return MMX_ERR_ARG.
 */
#ifndef MMX_H
#define MMX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMX_OK 0
#define MMX_WARN_HMIN 1       /* an error above e_max was accepted at h_min */
#define MMX_ERR_ARG (-1)      /* invalid argument; nothing was enqueued      */
#define MMX_ERR_OOM (-2)      /* a device or host allocation failed          */
#define MMX_ERR_CUDA (-3)     /* a CUDA runtime call failed                  */
#define MMX_ERR_NONFINITE (-4)/* the error estimate became NaN/Inf           */
#define MMX_ERR_TIMEOUT (-5)  /* attempt or wall-time limit of a run reached */
#define MMX_ERR_STATE (-6)    /* call not valid in the current state         */

/* Cell-centred finite-difference mesh (Sec. II, Eq. 2): nx*ny*nz cells of
 * dx*dy*dz metres. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
} mmx_mesh;

/* Material (Sec. II, Eq. 1 and the effective-field terms): saturation
 * magnetisation Ms [A/m], exchange stiffness A [J/m], uniaxial anisotropy
 * constant K [J/m^3] along the unit axis ku, Gilbert damping alpha, and
 * gyromagnetic ratio gamma [m/(A s)]. */
typedef struct {
    double Ms, A, K, ku[3], alpha, gamma;
} mmx_material;

/* Applied field [A/m]: H(t) = H0 + pulse_H for t_on <= t < t_off, else H0. */
typedef struct {
    double H0[3];
    double pulse_H[3];
    double t_on, t_off;
} mmx_field;

/* Explicit evaluation methods of Sec. II (Eq. 3-4 with their tableaux). */
typedef enum {
    MMX_RK4 = 0,     /* classical RK4, fixed step                        */
    MMX_HEUN12 = 1,  /* adaptive Heun (2) with Euler (1) estimate        */
    MMX_RK23_BS = 2, /* Bogacki-Shampine 3(2), FSAL                      */
    MMX_RKF45 = 3,   /* Runge-Kutta-Fehlberg, propagates order 4         */
    MMX_RKCK45 = 4,  /* Cash-Karp, propagates order 4                    */
    MMX_RKDP54 = 5,  /* Dormand-Prince 5(4), FSAL                        */
    MMX_RKF56 = 6,   /* Runge-Kutta-Fehlberg, propagates order 5         */
    MMX_ABM2 = 7     /* Adams-Bashforth-Moulton 2, predictor-corrector:
                      * variable-step AB2 predictor, trapezoidal corrector,
                      * error = corrector - predictor, two evaluations per
                      * step (at t and, extrapolated when p >= 0, t + h);
                      * the first step after a (re)start predicts by Euler */
} mmx_method;

/* Integrator settings.  extrap_order = p >= 0 evaluates Eq. 2 once per step
 * (stage 1) and approximates it at the other stages by the order-p
 * polynomial extrapolation of Eq. 6 (the first p steps prime the history
 * with full evaluations); extrap_order = -1 evaluates Eq. 2 at every stage.
 * adaptive = 0 keeps h fixed; adaptive = 1 uses the controller of Eq. 5 with
 * tol = e_max, step bounds hmin/hmax and factor bounds cmin/cmax (the paper's
 * values are 1e-5, 1 fs, 3 ps, 0.01, 2).  safety is the factor 0.8 of Eq. 5. */
typedef struct {
    int method;
    int extrap_order;
    int adaptive;
    double h, tol, hmin, hmax, cmin, cmax, safety;
} mmx_integrator;

typedef enum {
    MMX_FP64 = 0,       /* all fields, FFTs and stages in double            */
    MMX_FP32_MIXED = 1  /* fields, FFTs and stages in float; extrapolation
                           weights, error norm, controller and time in double */
} mmx_precision;

typedef struct {
    double t;             /* simulated time [s]                               */
    double h;             /* step proposed by the controller for the next step */
    double last_err;      /* error estimate e of the last attempt (Sec. II)   */
    long long accepted, rejected;
    long long exact_evals;  /* evaluations of Eq. 2 (FFT convolutions)        */
    long long extrap_evals; /* stage fields from Eq. 6                        */
    long long forced_accepts;
    long long attempts;
    long long kernel_launches; /* kernels of this library launched so far     */
} mmx_stats;

typedef struct mmx_ctx mmx_ctx;

/* Creates a context: validates the description, computes the Newell tensor
 * of the mesh (Sec. II, ref. [24]) on the host in binary128, its padded
 * spectrum, and allocates all device buffers.  precision is an
 * mmx_precision.  cuda_stream is a cudaStream_t (NULL = default stream).
 * Errors: MMX_ERR_ARG for invalid sizes or parameters (no CUDA call made),
 * MMX_ERR_OOM, MMX_ERR_CUDA.  On error *out is NULL. */
int mmx_create(const mmx_mesh *mesh, const mmx_material *mat, const mmx_field *field,
               const mmx_integrator *integ, int precision, void *cuda_stream, mmx_ctx **out);

/* Copies the magnetisation in from m (host or device pointer, 3*nx*ny*nz
 * elements of the context's precision) and resets the extrapolation history
 * (the next p steps prime it again, Sec. II after Eq. 6). */
int mmx_set_m(mmx_ctx *ctx, const void *m);

/* Copies the current magnetisation out to m (host or device pointer). */
int mmx_get_m(mmx_ctx *ctx, void *m);

/* Sets the simulated time (and resets the extrapolation history). */
int mmx_set_time(mmx_ctx *ctx, double t);

/* One exact evaluation of Eq. 2, H(r0) = -sum_r N(r - r0) Ms m(r), self term
 * included, by the zero-padded FFT convolution.  m_dev and H_dev are device
 * pointers of the context's precision, layout [3][nz][ny][nx]; H in A/m.
 * Does not touch the integrator state. */
int mmx_demag(mmx_ctx *ctx, const void *m_dev, void *H_dev);

/* Integrates Eq. 1 from the current time to t_end with the configured method
 * (Eq. 3-5, and Eq. 6 when extrap_order >= 0); the last step is clipped to
 * land on t_end.  Returns MMX_WARN_HMIN if an error above e_max had to be
 * accepted at h_min, MMX_ERR_NONFINITE if the error estimate became
 * non-finite (the state is left at the last accepted step). */
int mmx_run(mmx_ctx *ctx, double t_end);

/* Integrates until n_accepted more steps have been accepted. */
int mmx_step(mmx_ctx *ctx, int n_accepted);

/* Copies the counters out (synchronises the stream). */
int mmx_get_stats(mmx_ctx *ctx, mmx_stats *out);

/* Checkpoint: writes (t, h, m, history of exact fields, counters) to buf.
 * With buf == NULL only *len is set to the size needed.  The blob is only
 * valid for a context created with the same mesh, method and precision. */
int mmx_save_state(mmx_ctx *ctx, void *buf, size_t *len);
int mmx_load_state(mmx_ctx *ctx, const void *buf, size_t len);

/* Per-kernel-class device timing with CUDA events on the context stream.
 * While enabled, mmx_run runs each attempted step as a CUDA graph with an
 * event-record node before and after every kernel (the host reads the loop
 * flag between attempts, so runs are slower than without profiling, but
 * the kernels themselves run back to back as in the step loop), and
 * mmx_demag records and synchronises an event pair around each pass.
 * mmx_get_profile returns, per class (0: x-forward FFT, 1: yz FFT + tensor
 * multiply, 2: x-inverse FFT, 3: LLG stage, 4: last stage (error norm, and
 * the Eq. 3 solution unless stage S-2 of an FSAL tableau formed it), 5:
 * controller (Eq. 5 and the next attempt's coefficients)), the summed
 * milliseconds and the number of launches.  ms
 * and launches point to arrays of MMX_NPROF.  enable: 0 off, 1 an event
 * pair around every launch, 2 the same except that the stage kernels of an
 * extrapolated attempt (every stage but the last; no demag pass runs between
 * them) share one pair, so that class 3 then times them back to back without
 * event-record nodes between them and counts every launch of the run; any
 * other value is MMX_ERR_ARG.  Switching the mode clears the sums. */
#define MMX_NPROF 6
int mmx_set_profiling(mmx_ctx *ctx, int enable);
int mmx_get_profile(mmx_ctx *ctx, double *ms, long long *launches);

/* Configuration of the exact demag evaluation chosen for this context.  At
 * mmx_create the library times the candidate configurations of its FFT
 * passes on the context's own buffers and keeps the fastest (unless the
 * environment forces one: MMX_AUTOTUNE=0, MMX_FORCE_SPLIT, MMX_NO_TMA,
 * MMX_TROWS); results are cached per mesh and precision for the life of the
 * process.  The candidates:
 *   x_rows   rows of the x transforms per CTA in the plain x passes (2-16);
 *   xi_tma   inverse x pass fed by tensor-memory-access tile copies (FP32);
 * and, set by the mesh:
 *   yz_pass  0: one CTA transforms a whole y-z column (meshes where it
 *            fits); 1: split y / z passes through an HBM y spectrum.
 * demag_us is the timed evaluation of the chosen configuration (0 when not
 * tuned); kernels_per_demag the launches of one evaluation. */
typedef struct {
    int yz_pass;
    int x_rows;
    int xi_tma;
    int tuned;
    int kernels_per_demag;
    double demag_us;
} mmx_plan;
int mmx_get_plan(const mmx_ctx *ctx, mmx_plan *out);

/* Allocation-free exact demag evaluation.  No counterpart in the paper: it
 * serves callers that cannot allocate device memory, e.g. code running while
 * its stream is being captured into a CUDA graph (cudaMalloc is not allowed
 * there) or code in a process whose device memory belongs to another
 * allocator, and who therefore cannot create a context with mmx_create.
 * It computes the same field as mmx_demag (Eq. 2, self term included) for a
 * mesh with saturation magnetisation Ms, with the same FFT kernels, but the
 * tensor spectrum, the twiddle tables and the FFT scratch live in one
 * file-scope device array of MMX_STATIC_SCRATCH_BYTES inside this library,
 * which every GPU that loads the library holds until the process exits.
 * m_dev and H_dev are device pointers of the given precision's element
 * type, layout [3][nz][ny][nx]; H in A/m; the work is enqueued on
 * cuda_stream (NULL = default stream).
 *   - No device memory is allocated or freed, and no CUDA library or torch
 *     routine that allocates is called.  The first call on a device looks up
 *     the array's device address (cudaGetSymbolAddress), and the first call
 *     for a new mesh, Ms or precision computes the Newell tensor on the host
 *     (host memory only) and copies its spectrum into the array; make that
 *     first call before any stream capture (such a first call made while
 *     cuda_stream is capturing returns MMX_ERR_ARG and enqueues nothing).
 *     Later calls with the same description (mesh sizes, cell sizes, Ms and
 *     precision compared field by field) reuse the spectrum the array still
 *     holds.
 *   - Every call shares the array: calls that overlap on the GPU (other
 *     streams, other host threads) race; serialise them.
 *   - Meshes whose spectrum, tables and scratch exceed the array, or whose
 *     y-z column does not fit one CTA (the split passes need a second
 *     spectrum buffer; this includes nz > 8 in FP32, nz > 4 in FP64), return
 *     MMX_ERR_ARG (text from mmx_last_error(NULL)); the other errors are
 *     those of mmx_create and mmx_demag. */
#define MMX_STATIC_SCRATCH_BYTES (16u << 20)
int mmx_demag_static(const mmx_mesh *mesh, double Ms, int precision, const void *m_dev, void *H_dev,
                     void *cuda_stream);

/* Batched ensemble of independent simulations (no counterpart in the paper:
 * the method of Sec. II applied to many unrelated samples at once).  A batch
 * groups n existing contexts of any mesh size, material, method, order and
 * precision; mmx_batch_run integrates every member to its own end time with
 * ONE CUDA-graph launch on cuda_stream (NULL = default stream).  The graph
 * holds, per member, the preparation kernel and the member's own device-side
 * loops (the priming loop, then the extrapolated loop, each a conditional
 * while node stepped by the member's controller), with no dependency between
 * members, so the GPU runs the members side by side.  Every member keeps its
 * own step size, accept/reject decisions and history (Eq. 5, Eq. 6): the
 * result of each member is the one mmx_run(member, t_end[i]) gives.
 *   - members: n distinct contexts (1 <= n <= 4096), owned by the caller, that
 *     must outlive the batch; the batch only reads their buffers.  While the
 *     batch exists, the members may still be used on their own (mmx_set_m,
 *     mmx_run, ...), but not concurrently with mmx_batch_run.
 *   - The graph is built at the first mmx_batch_run, kept, and reused.
 *   - MMX_ERR_ARG for a NULL or duplicate member or n out of range (text from
 *     mmx_last_error(NULL)). */
typedef struct mmx_batch mmx_batch;
int mmx_batch_create(int n, mmx_ctx *const *members, void *cuda_stream, mmx_batch **out);

/* Integrates member i from its current time to t_end[i] (host array of n);
 * members with t_end[i] <= their time are left as they are.  status, if not
 * NULL, receives per member what mmx_run would have returned (MMX_OK,
 * MMX_WARN_HMIN, MMX_ERR_NONFINITE, MMX_ERR_TIMEOUT, ...; the member's own
 * mmx_last_error holds the text).  Returns the most severe member status
 * (the first negative one, else MMX_WARN_HMIN if any, else MMX_OK), or a
 * batch error (MMX_ERR_CUDA, text from mmx_batch_last_error).  Synchronises
 * cuda_stream.  Per-member counters: mmx_get_stats on each member. */
int mmx_batch_run(mmx_batch *b, const double *t_end, int *status);

/* Text of the batch's own error from its last mmx_batch_run ("" when the
 * run had none, e.g. when only members failed); with b == NULL the text of
 * the last failed mmx_batch_create of this thread. */
const char *mmx_batch_last_error(const mmx_batch *b);

/* Frees the batch's graph (not its members). */
void mmx_batch_destroy(mmx_batch *b);

/* Text of the last error (never NULL; "" if none).  ctx may be NULL, then
 * the text of the last failed mmx_create of this thread is returned. */
const char *mmx_last_error(const mmx_ctx *ctx);

/* Frees every resource of the context (synchronises its stream). */
void mmx_destroy(mmx_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* MMX_H */
