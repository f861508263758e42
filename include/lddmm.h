/*
 * lddmm.h -- C ABI of the GB300 PDE-EPDiff LDDMM library (liblddmm.so).
 *
 * The method (Hernandez, arXiv 1807.04638, Sec. 3) minimises, over the initial
 * velocity v0 of an EPDiff geodesic,
 *
 *     E(v0) = w <L v0, v0> + || m(1) - I1 ||^2,     L = (Id - alpha Lap)^s,
 *
 * where v_t solves EPDiff  dv/dt = -K ad*_v L v  (K = L^-1, Sec. 2.2) and
 * m(1) = I0 o phi_1^-1 solves the transport state equation dm/dt + grad m . v = 0.
 * The reduced gradient is carried from t = 1 back to t = 0 by the adjoint
 * Jacobi equations, and the Gauss-Newton Hessian-vector product by the same
 * backward sweep after a forward incremental EPDiff / Jacobi-field sweep
 * (Sec. 3); PCG with preconditioner K solves H dv0 = -grad E inside an inexact
 * Gauss-Newton-Krylov loop (Sec. 2.3, Sec. 3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grid n = (n0, n1, n2), axis 2 fastest, periodic box [0, len_a), spacing
 *    h_a = len_a / n_a.  Each n_a must factor into 2, 3 and 5 only and lie in
 *    [2, 512].
 *  - A scalar field is n0*n1*n2 contiguous values [n0][n1][n2]; a vector field
 *    is three such planes [3][n0][n1][n2]; component c points along axis c.
 *  - Inner products are <f, g> = h0 h1 h2 sum_x sum_c f_c g_c, always
 *    accumulated in double precision on the device.
 *  - Array arguments are DEVICE pointers owned by the caller, in the handle's
 *    compute type (double for LDDMM_F64, float for LDDMM_F32), unless stated
 *    otherwise.  They must not alias each other.  Calls are enqueued on the
 *    handle's stream and return before the work completes, except where a
 *    host output (energy, kinetic, report) forces a synchronisation.
 *  - The handle owns its workspace (stored time states, FFT scratch, PCG
 *    vectors).  A handle must not be used from two host threads at once.
 *  - No exception or abort crosses the ABI.  The first failure is sticky:
 *    later calls on the same handle return the same status until
 *    lddmm_destroy.  Every call that takes device arrays first scans them
 *    on the device (one extra launch over the inputs); a NaN or Inf there is
 *    reported as LDDMM_ERR_NONFINITE by that call, which still enqueues its
 *    work (its outputs are then undefined) and waits only for the scan's
 *    verdict, not for the rest of its work.  A NaN or Inf in an energy or a
 *    report gives the same status.  lddmm_apply_metric_noalloc does not scan.
 */
#ifndef LDDMM_H
#define LDDMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDDMM_OK = 0,
    LDDMM_ERR_ARG = 1,            /* a null handle, null pointer or bad enum    */
    LDDMM_ERR_SHAPE = 2,          /* a grid size the FFTs do not support       */
    LDDMM_ERR_OOM = 3,            /* device allocation failed                  */
    LDDMM_ERR_CUDA = 4,           /* a CUDA runtime call failed                */
    LDDMM_ERR_NOT_LINEARIZED = 5, /* hessvec / jacobi call before gradient     */
    LDDMM_ERR_NONFINITE = 6,      /* NaN or Inf in an input, energy or result  */
    LDDMM_ERR_DEVICE_CHECK = 7,   /* a device-side check recorded an error     */
    LDDMM_ERR_TIMEOUT = 8,        /* a host-side wait exceeded its limit       */
    LDDMM_WARN_LINESEARCH = 9,    /* Armijo search failed; registration stopped */
    LDDMM_ERR_TOO_LARGE = 10      /* grid exceeds lddmm_apply_metric_noalloc's scratch */
} lddmm_status;

enum { LDDMM_F64 = 0, LDDMM_F32 = 1, LDDMM_BF16 = 2 };          /* number types   */
enum { LDDMM_INTERP_CUBIC = 0, LDDMM_INTERP_LINEAR = 1 };       /* SL interpolant */
enum { LDDMM_SPACE_V = 0, LDDMM_SPACE_L2 = 1 };                 /* metric of g, Hv */
enum { LDDMM_OPT_GN = 0, LDDMM_OPT_GD = 1 };                     /* lddmm_register  */
enum { LDDMM_GRAD_JACOBI = 0, LDDMM_GRAD_DISCRETE = 1 };         /* gradient_mode   */

typedef struct {
    int n[3];        /* grid points per axis                                  */
    double len[3];   /* box lengths; 0 means 2*pi                             */
} lddmm_grid;

typedef struct {
    double alpha;        /* L = (Id - alpha Lap)^s, Sec. 2.1; alpha > 0        */
    int s;               /* integer power s >= 1                               */
    double weight;       /* w in E = w <L v0, v0> + ||m1 - I1||^2 (w = sigma^2) */
    int nt;              /* Heun time steps on [0, 1]                          */
    int interp;          /* LDDMM_INTERP_*: Catmull-Rom (default) or trilinear */
    int space;           /* LDDMM_SPACE_*: gradient / Hv metric (Sec. 3, last paragraph) */
    int compute_dtype;   /* LDDMM_F64 or LDDMM_F32                             */
    int state_dtype;     /* stored time states: compute_dtype, or LDDMM_BF16 with
                            LDDMM_F32 compute (the stage fields are evaluated in
                            FP32 and stored rounded to bfloat16)              */
    int checkpoint_every;/* 1: keep the fields of every Heun stage; c > 1: keep
                            the spectral velocity every c steps and re-shoot
                            one segment of c steps inside each sweep (memory of
                            c steps' states instead of nt, one more shoot per
                            sweep; the answer is unchanged)                   */
    int gn_maxit;        /* Gauss-Newton iterations of lddmm_register          */
    int pcg_maxit;       /* PCG iterations per Gauss-Newton step (cap)         */
    double pcg_rtol;     /* PCG relative residual tolerance                    */
    double armijo_c1;    /* Armijo sufficient-decrease constant                */
    int ls_maxit;        /* Armijo halvings before giving up                   */
    int dealias;         /* 1 (default): 2/3-rule projector P on the products of
                            the EPDiff and Jacobi equations, modes |k_a| <=
                            (n_a - 1)/3 kept; 0: unfiltered products           */
    int optimizer;       /* LDDMM_OPT_GN (default): Gauss-Newton-Krylov;
                            LDDMM_OPT_GD: gradient descent in V (Sec. 2.2) */
    int gradient_mode;   /* LDDMM_GRAD_JACOBI (default): the reduced gradient of
                            Sec. 3 (adjoint Jacobi sweep from the final-time
                            source, delta m1 = -grad m1 . xi1);
                            LDDMM_GRAD_DISCRETE: the exact gradient of the
                            discrete energy, through the transposes of the
                            semi-Lagrangian map steps and of the warp (needs
                            state_dtype = compute_dtype and checkpoint_every
                            <= 1; keeps every map u_k, 6 (nt + 1) more real
                            fields).  The Gauss-Newton Hv is the same in both. */
} lddmm_params;

#define LDDMM_TRACE_MAX 64
typedef struct {
    int gn_iters;                          /* Gauss-Newton iterations taken    */
    int pcg_iters_total;                   /* sum over iterations (Table 1)    */
    double mse_rel;                        /* ||m1-I1||^2/||I0-I1||^2 (Sec. 4) */
    double gnorm_rel;                      /* ||g_n||_inf / ||g_0||_inf        */
    double jac_min, jac_max;               /* extrema of det(I + D u1)         */
    double energy[LDDMM_TRACE_MAX + 1];    /* E before each step and at the end */
    int pcg_iters[LDDMM_TRACE_MAX];        /* per Gauss-Newton step            */
    double step[LDDMM_TRACE_MAX];          /* accepted Armijo step (0: failed) */
} lddmm_report;

typedef struct lddmm_handle lddmm_handle;

/* Fill *p with the defaults: alpha 0.01, s 2, weight 1e-3, nt 10, cubic, V,
 * F64 compute and states, checkpoint 1, 5 GN x 10 PCG, rtol 0.1, c1 1e-4,
 * 10 halvings, dealiasing on, Gauss-Newton. */
void lddmm_default_params(lddmm_params *p);

/* Device bytes that lddmm_create would allocate for (g, p); 0 if invalid.
 * Used by callers to admit work against a memory budget. */
size_t lddmm_workspace_bytes(const lddmm_grid *g, const lddmm_params *p);

/* Create a handle bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Allocates the whole
 * workspace with cudaMalloc.  On failure *h is NULL. */
lddmm_status lddmm_create(lddmm_handle **h, const lddmm_grid *g, const lddmm_params *p,
                          void *cuda_stream);
lddmm_status lddmm_destroy(lddmm_handle *h);
const char *lddmm_status_string(lddmm_status s);
/* Status of the handle (sticky first error), without synchronising. */
lddmm_status lddmm_last_status(const lddmm_handle *h);
/* Block until the handle's stream is idle; returns the handle's status. */
lddmm_status lddmm_synchronize(lddmm_handle *h);

/* Geodesic shooting (Sec. 2.2 EPDiff + Sec. 3 state equation): Heun steps of
 * dv/dt = -K P ad*_v L v from P v0, semi-Lagrangian transport of the inverse
 * map psi = x + u, m1 = I0(x + u1).  With I0 != NULL the shoot also stores
 * grad m1 and becomes the linearisation point of lddmm_shoot_vjp,
 * lddmm_hessvec and lddmm_jacobi_*.
 *   v0      [3][N]  initial velocity
 *   I0      [N]     source image (may be NULL when m1 is NULL)
 *   m1      [N]     out, warped source (nullable)
 *   u1      [3][N]  out, inverse-map displacement at t = 1 (nullable)
 *   kinetic host [nt+1] out, <L v_k, v_k> (nullable; synchronises) */
lddmm_status lddmm_shoot(lddmm_handle *h, const void *v0, const void *I0, void *m1, void *u1,
                         double *kinetic);

/* Reduced gradient of E(v0) = w <L v0, v0> + ||m1(P v0) - I1||^2 (Sec. 3:
 * grad_{v1}E = lambda(1) grad m(1), lambda(1) = -2 (m(1) - I1), carried back
 * by the adjoint Jacobi equations).
 *   grad   [3][N] out, g_V = K g_L2 (LDDMM_SPACE_V) or g_L2 (LDDMM_SPACE_L2)
 *   energy host [3] out (nullable; synchronises): E, data term, regulariser.
 * Stores the linearisation point (time states, grad m1) in the handle for
 * lddmm_hessvec / lddmm_jacobi_*. */
lddmm_status lddmm_gradient(lddmm_handle *h, const void *v0, const void *I0, const void *I1,
                            void *grad, double *energy);

/* Gauss-Newton Hessian-vector product at the last gradient's v0 (Sec. 3,
 * incremental EPDiff + reduced incremental adjoint Jacobi equations with the
 * Gauss-Newton drops):  H dv0 = 2 w L dv0 + T^T [2 (grad m1 . xi1) grad m1],
 * returned in the metric of `space` (V: K H_L2).  dv0, Hdv [3][N]. */
lddmm_status lddmm_hessvec(lddmm_handle *h, const void *dv0, void *Hdv);

/* Vector-Jacobian product of the shooting map v0 -> m1 = I0 o phi_1^-1
 * (reverse-mode derivative; Sec. 3: the gradient is computed at t = 1 and
 * carried back by the adjoint Jacobi equations).  With the Jacobi-field
 * linearisation delta m1 = -grad m1 . xi1,
 *     out = P T^T (-G grad m1),
 * the derivative of sum_x G(x) m1(x) with respect to v0 (sum pairing, no cell
 * volume).  Valid at the last lddmm_gradient or lddmm_shoot with I0 != NULL;
 * otherwise LDDMM_ERR_NOT_LINEARIZED.  G [N], out [3][N]. */
lddmm_status lddmm_shoot_vjp(lddmm_handle *h, const void *G, void *out);

/* Forward Jacobi (tangent) sweep T at the last gradient's v0: from
 * (eta0, xi0) = (dv0, 0) integrate eta' = R'(v) eta, xi' = eta + ad_v xi;
 * writes eta1 and xi1 ([3][N] each, both nullable). */
lddmm_status lddmm_jacobi_forward(lddmm_handle *h, const void *dv0, void *eta1, void *xi1);

/* Backward (adjoint Jacobi) sweep T^T, the exact transpose of
 * lddmm_jacobi_forward: cotangents b_eta (nullable = 0) and b_xi on
 * (eta1, xi1) -> cotangent on dv0, written to out [3][N] (L2 pairing). */
lddmm_status lddmm_jacobi_adjoint(lddmm_handle *h, const void *b_eta, const void *b_xi, void *out);

/* Spectral metric operator: out = L^power in  (power -1 is K, Sec. 2.1),
 * for `ncomp` scalar fields stored back to back.  power in [-4, 4]. */
lddmm_status lddmm_apply_metric(lddmm_handle *h, const void *in, void *out, int ncomp, int power);

/* J = det(I + D u) of psi = x + u (Sec. 4 reports its extrema).
 *   u [3][N] in;  J [N] out (nullable);  minmax host [2] out (nullable; synchronises). */
lddmm_status lddmm_jacobian_det(lddmm_handle *h, const void *u, void *J, double *minmax);

/* Inexact Gauss-Newton-Krylov registration (Sec. 3): gn_maxit iterations of
 * gradient -> PCG (preconditioner K, Hv per iteration, FP64 scalars) ->
 * Armijo backtracking -> v0 <- v0 + eps dv0.  With optimizer LDDMM_OPT_GD the
 * same loop takes the gradient-descent step in V of Sec. 2.2 instead,
 * v0 <- v0 - eps K g_L2 (no PCG): Armijo backtracking starts at the step that
 * moves max |K g_L2| by one voxel (min_a h_a) in the first iteration and at
 * twice the last accepted step afterwards.  v0_inout [3][N] is the start
 * and receives the result.  report (host, nullable) receives the Sec. 4
 * metrics and the per-iteration trace.  Synchronises.  Returns
 * LDDMM_WARN_LINESEARCH (not sticky) when a line search failed. */
lddmm_status lddmm_register(lddmm_handle *h, const void *I0, const void *I1, void *v0_inout,
                            lddmm_report *report);

/* Optional kernel profiler (tracing; no counterpart in the paper).  When
 * enabled, CUDA events bracket every kernel launch of the handle on its
 * stream.  lddmm_profile_read returns, for one kernel class, the summed
 * device time in ms, the algorithmic bytes (the compulsory reads + writes of
 * each launch, counted from its arguments) and the number of launches since
 * the last enable.  Enabling resets the counters; reading synchronises. */
int lddmm_profile_num_classes(void);
const char *lddmm_profile_class_name(int cls);
lddmm_status lddmm_profile(lddmm_handle *h, int enable);
lddmm_status lddmm_profile_read(lddmm_handle *h, int cls, double *ms, double *bytes, long long *launches);

/* Metric operator without device allocation (no counterpart in the paper).
 * For callers that cannot call cudaMalloc -- code running while a CUDA graph
 * is captured, real-time loops that must stay out of the allocator, plug-ins
 * whose host application owns every device allocation -- and so cannot
 * create a handle.  Computes out = L^power in (power -1 is K; L = (Id -
 * alpha Lap)^s, no dealiasing) for `ncomp` scalar fields stored back to back
 * on the grid g, in LDDMM_F64 or LDDMM_F32 (`dtype`), on `cuda_stream`.
 * in / out are caller-owned device pointers; out may equal in.
 * Scratch: a fixed static device array of lddmm_apply_metric_noalloc_capacity()
 * bytes (24 MiB) compiled into the library; each GPU that loads the library
 * holds it until the process exits.  A grid whose scratch need
 * (lddmm_apply_metric_noalloc_scratch_bytes) exceeds it is rejected with
 * LDDMM_ERR_TOO_LARGE before any device work (e.g. 128^3 fits in F32, not in
 * F64).  The first call on each device looks up the array's device address
 * (with that device current); make it before any stream capture.  Every call
 * rewrites the scratch it reads; calls that overlap on the GPU share the one
 * array and race.  Allocates nothing, host or device. */
lddmm_status lddmm_apply_metric_noalloc(const lddmm_grid *g, double alpha, int s, int power, int dtype,
                                        const void *in, void *out, int ncomp, void *cuda_stream);
size_t lddmm_apply_metric_noalloc_scratch_bytes(const lddmm_grid *g, int dtype);
size_t lddmm_apply_metric_noalloc_capacity(void);

/* FP64 fused multiply-add rate probe (measurement; no counterpart in the
 * paper).  Launches `blocks` blocks of lddmm_probe_fp64_fma_threads() threads
 * on `cuda_stream`; every thread runs `iters` rounds of independent FP64 FMA
 * chains and writes one double to out[thread] (caller-owned device buffer of
 * blocks * threads doubles).  lddmm_probe_fp64_fma_flops gives the launch's
 * flop count (2 per FMA); time the launch with CUDA events to get the FP64
 * rate that bounds the plain FP64 method's FFT passes.  Returns
 * LDDMM_ERR_ARG for a null buffer or non-positive sizes. */
lddmm_status lddmm_probe_fp64_fma(double *out, int blocks, int iters, void *cuda_stream);
double lddmm_probe_fp64_fma_flops(int blocks, int iters);
int lddmm_probe_fp64_fma_threads(void);

#ifdef __cplusplus
}
#endif
#endif /* LDDMM_H */
