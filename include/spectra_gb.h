/*
 * spectra_gb -- GB300 (sm_103a) boundary oracle and random walks for
 * spectrahedra S = { x in R^n : F(x) = A_0 + sum_i x_i A_i >= 0 }
 * (arXiv 2010.03817, "Efficient Sampling from Feasible Sets of SDPs and
 * Volume Approximation", Eq. 1).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Return value: SP_OK (0) or one of the SP_E* codes below.  A non-zero
 *   code means nothing was launched (argument errors) or a CUDA call failed
 *   (SP_ECUDA); sp_last_error() gives a one-line message (thread-local).
 * - "device" pointers are caller-owned global-memory pointers (for example
 *   torch tensors' data_ptr()), contiguous, float64 unless stated.  The
 *   library never frees or retains them past the call, and writes nothing
 *   but the documented outputs.
 * - "host" pointers are ordinary CPU memory.  Entry points that accept
 *   "host or device" detect the kind with cudaPointerGetAttributes and copy
 *   host data through their own staging buffers.
 * - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *   enqueued asynchronously on it; outputs are ready when the stream is.
 * - Per-item results carry a status word (SP_ST_*) in a caller buffer.
 * - mode selects the arithmetic: SP_MODE_FP64 (plain FP64 path) or
 *   SP_MODE_MIXED (see below).
 *
 * Handles own their device memory (allocated in the create/init calls,
 * released by the matching destroy call).
 */
#ifndef SPECTRA_GB_H
#define SPECTRA_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SP_OK 0
#define SP_EINVAL 1      /* bad argument (null handle, size, mode, ...) */
#define SP_ENOTPD 2      /* a start point is not interior: F(x) is not positive definite */
#define SP_EUNBOUNDED 3  /* a ray never meets the boundary (S must be bounded) */
#define SP_ENOCONV 4     /* an eigen-solve hit its iteration cap */
#define SP_ECUDA 5       /* a CUDA runtime call failed */
#define SP_ENOMEM 6      /* device allocation failed */

/* per-item / per-chain status words */
#define SP_ST_OK 0
#define SP_ST_NOT_PD 1      /* point not interior (Cholesky of F failed) */
#define SP_ST_UNBOUNDED 2   /* no positive root: t+ = +inf */
#define SP_ST_NOCONV 3      /* Lanczos hit its cap; the result is the last Ritz value */
#define SP_ST_RHO 4         /* Billiard: more than rho reflections, point kept (Alg. 5) */
#define SP_ST_DEGENERATE 5  /* normal undefined: rank F(p+) <= m-2 (Lemma "Gradient of det F") */
#define SP_ST_INVALID 6     /* a non-finite entry in the point or the direction (nothing computed) */

/* arithmetic modes */
#define SP_MODE_FP64 0   /* every step in FP64 */
#define SP_MODE_MIXED 1  /* tensor-core V formation and normals (exact digit splitting,
                            FP64 quality), FP32 estimate, double-float factorisation next to
                            the boundary and refinement of t+ and u (FP64 as the fallback);
                            needs n <= 224 (normals on the tensor cores: m <= 224) */
#define SP_MODE_LEARNED 2  /* the mixed path with the network's warm start (sp_attach_mlp):
                              the Billiard walk and sp_reflect start stage 1 from the
                              network's prediction; sp_intersect (which also needs t-, not
                              predicted) and the chord walks run as SP_MODE_MIXED; without
                              an attached network SP_EINVAL */

/* walk kinds (sp_chain_stats slots are SP_STAT_*) */
#define SP_STAT_SEGMENTS 0     /* boundary-oracle calls */
#define SP_STAT_REFLECTIONS 1  /* Billiard reflections */
#define SP_STAT_BAD_STEPS 2    /* steps that ended with a non-OK status (point kept) */
#define SP_STAT_LANCZOS 3      /* Lanczos iterations */
#define SP_STAT_SHIFT_RETRY 4  /* shifted factorisations redone unshifted */
#define SP_STAT_NOCONV 5       /* eigen-solves that hit the iteration cap */
#define SP_STAT_FALLBACK 6     /* mixed path: segments whose stage 2 fell back to FP64 */
#define SP_STAT_POWER 7        /* mixed path: power iterations next to the boundary */
#define SP_STAT_LEARNED_OK 8   /* learned path: warm starts accepted by the certificate */
#define SP_STAT_LEARNED_MISS 9 /* learned path: warm starts rejected (plain stage 1 instead) */
#define SP_NUM_STATS 12

typedef struct sp_spec sp_spec;
typedef struct sp_chains sp_chains;

/* Message of the last failed call on this thread ("" if none). */
const char* sp_last_error(void);

/* Library version string. */
const char* sp_version(void);

/*
 * Create a spectrahedron handle from the LMI F(x) = A_0 + sum x_i A_i (Eq. 1).
 *   n, m  : dimension and matrix size, 1 <= n <= 4096, 1 <= m <= 4096.
 *   A     : host pointer, (n+1) x m x m float64 row-major, A[0] = A_0.  Each
 *           A_i must be symmetric (checked to 1e-12 relative; SP_EINVAL
 *           otherwise).  The library copies and packs it (lower triangles) to
 *           device memory; the caller keeps ownership of A.
 *   flags : bit 0 (SP_FLAG_FP64_ONLY): skip the mixed path's precomputed
 *           operands (digit stacks, FP32 pairs); other bits reserved, 0.
 *   out   : receives the handle; free with sp_destroy_spectrahedron.
 */
#define SP_FLAG_FP64_ONLY 1u
int sp_create_spectrahedron(int n, int m, const double* A, uint32_t flags, sp_spec** out);
int sp_destroy_spectrahedron(sp_spec* s);
int sp_spec_dims(const sp_spec* s, int* n, int* m);

/*
 * MEMBERSHIP (Sec. 2.2, Alg. 1) in the strict sense: inside[c] = 1 iff
 * F(x_c) is positive definite (its Cholesky factorisation succeeds).
 *   x: device, count x n.  inside: device int32, count.
 */
int sp_membership(sp_spec* s, int count, const double* x, int* inside, void* stream);

/*
 * INTERSECTION (Sec. 2.3, Alg. 2; Lemma "PEP and S cap C") for the lines
 * x_c + t v_c: t_minus[c] < 0 < t_plus[c] are the roots of det(F(x_c) + t V_c)
 * (V = sum v_i A_i) closest to 0 on either side.
 *   x, v    : device, count x n (v need not be unit).
 *   t_minus : device, count (-inf if none).   t_plus: device, count (+inf if none).
 *   u       : device, count x m, or NULL: unit null vector of F(x + t+ v),
 *             largest-magnitude entry positive.
 *   status  : device int32, count (SP_ST_*).
 *   mode    : SP_MODE_FP64, SP_MODE_MIXED (t+ and t- to 1e-9 relative of the FP64
 *             result) or SP_MODE_LEARNED (runs as SP_MODE_MIXED).
 */
int sp_intersect(sp_spec* s, int count, const double* x, const double* v, double* t_minus,
                 double* t_plus, double* u, int* status, int mode, void* stream);

/*
 * REFLECTION (Sec. 2.4, Alg. 3; Eq. "reflection"; Lemma "Gradient of det F"):
 * t_plus[c] as in sp_intersect, the unit normal w_hat = w/|w| with
 * w_j = u^T A_j u (j = 1..n, u the null vector at the hit point; it points
 * into S), and the reflected direction s = v - 2 <v, w_hat> w_hat.
 *   x, v: device, count x n.  t_plus: device, count.  w_hat, s: device, count x n.
 *   status: device int32, count.
 *   mode: SP_MODE_FP64, SP_MODE_MIXED or SP_MODE_LEARNED (the attached
 *   network's warm start for stage 1; a prediction the factorisation or the
 *   Lanczos test rejects falls back to the plain stage 1, so the results
 *   meet the mixed path's accuracy either way; sp_learned_counts reports
 *   the accepted and rejected warm starts of the last call).
 */
int sp_reflect(sp_spec* s, int count, const double* x, const double* v, double* t_plus,
               double* w_hat, double* s_out, int* status, int mode, void* stream);

/*
 * The pencil of the lines x_c + t v_c (Lemma "PEP and S cap C"):
 * F_out[c] = F(x_c) = A_0 + sum_i x_ci A_i and V_out[c] = sum_i v_ci A_i, as
 * packed lower triangles (count x m(m+1)/2, device).  x / F_out or v / V_out
 * may both be NULL.  SP_MODE_FP64: FP64 arithmetic.  SP_MODE_MIXED: BF16
 * tensor cores with exact digit splitting of both operands (eight 7-bit
 * digits, FP64 result; error below n 2^-51 max_j |c_j| max_{j>=1} |A_j[p]|
 * plus one FP64 rounding).
 */
int sp_form_pencil(sp_spec* s, int count, const double* x, const double* v, double* F_out,
                   double* V_out, int mode, void* stream);

/*
 * Chains: C independent walkers with state (x, step counter) on the device.
 *   x0    : host or device, C x n start points, or NULL for the origin.
 *           Every start point must be interior (checked: SP_ENOTPD).
 *   seed  : Philox4x32-10 key.  Chain c draws from counter (chain0 + c, step, stream, i).
 *   chain0: offset of this handle's chains in the Philox counter space
 *           (lets several handles / GPUs share one seed without overlap).
 */
int sp_init_chains(sp_spec* s, int C, const double* x0, uint64_t seed, uint32_t chain0,
                   sp_chains** out, void* stream);
int sp_destroy_chains(sp_chains* ch);

/*
 * Billiard walk (Sec. 3.2, Alg. 5): `steps` steps on every chain.
 *   tau   : length scale, l = -tau ln eta (the paper takes tau ~ diam(S)).
 *   rho   : reflection bound; a step with more than rho reflections keeps its
 *           start point (status SP_ST_RHO, counted in SP_STAT_BAD_STEPS).
 *   kappa : after a hit at t+ the walker moves to (1 - kappa) t+ (0 <= kappa < 1),
 *           keeping F positive definite; the remaining length drops by t+.
 */
int sp_step_billiard(sp_chains* ch, int steps, double tau, int rho, double kappa, int mode,
                     void* stream);

/* Hit-and-Run (Sec. 3.1, Alg. 4), uniform point on the chord [t-, t+]. */
int sp_step_hnr(sp_chains* ch, int steps, int mode, void* stream);

/* Coordinate-direction Hit-and-Run (Sec. 3.1, CDHR): direction e_j, j uniform. */
int sp_step_cdhr(sp_chains* ch, int steps, int mode, void* stream);

/*
 * REFLECTION on the trajectories of HMC for the Boltzmann density
 * pi(x) ~ exp(-c.x / T) (Sec. 3.3, Alg. 6; FP64; m <= 64).  For f(x) = c.x / T
 * the Hamiltonian ODE has the exact solution Phi(t) = x + v t - (c / (2T)) t^2,
 * so F(Phi(t)) = F(x) + t V + t^2 C (V = sum v_j A_j, C = -(1/(2T)) sum c_j A_j),
 * a quadratic eigenvalue problem (Sec. 2.1) solved through its companion
 * linearisation of size 2m: t_plus[k] is its first positive root (+inf and
 * SP_ST_UNBOUNDED when there is none), w_hat the unit normal w / |w|,
 * w_j = u^T A_j u at Phi(t_plus) (pointing into S), s the velocity
 * Phi'(t_plus) = v - (c / T) t_plus reflected on it:
 * s = Phi' - 2 <Phi', w_hat> w_hat (Sec. 2.4).
 *   x, v: device, count x n (start points, interior; initial velocities).
 *   c: host or device, n.  T > 0.
 *   t_plus: device, count.  w_hat, s: device, count x n (zero unless status
 *   is SP_ST_OK).  status: device int32, count (SP_ST_NOTPD for a start
 *   outside S, SP_ST_NOCONV when the eigenvalue iteration hits its cap).
 * Errors: SP_EINVAL for m > 64, count < 0, T <= 0 or a NULL argument.
 */
int sp_curve_reflect(sp_spec* s, int count, const double* x, const double* v, const double* c,
                     double T, double* t_plus, double* w_hat, double* s_out, int* status,
                     void* stream);

/*
 * HMC with reflections (Sec. 3.3, Alg. 6) for pi(x) ~ exp(-c.x / T): `steps`
 * steps on every chain (FP64; m <= 64).  Each step draws the momentum
 * v ~ N(0, I_n) (Philox stream 0, not normalised) and the length
 * l = tau eta (eta uniform, stream 1), then follows Phi from the chain's
 * point, reflecting (as sp_curve_reflect) until l is used up; after a hit
 * at t+ the walker moves to Phi((1 - kappa) t+) and the remaining length
 * drops by t+.  A step with more than rho reflections, or whose boundary
 * oracle fails, keeps its start point (status as sp_step_billiard).
 *   c: host or device, n.  T, tau > 0, rho >= 0, 0 <= kappa < 1.
 */
int sp_step_hmc(sp_chains* ch, int steps, const double* c, double T, double tau, int rho,
                double kappa, void* stream);

/*
 * Volume of S by multiphase Monte Carlo over a sequence of balls (Sec. 4.1,
 * the multiphase scheme with the Billiard walk): radii r_0 = r_inner < r_1 <
 * ... < r_q = r_outer, geometric, q = ceil(n ln(r_outer / r_inner) / ln(1 /
 * ratio)) so that each ratio vol(S cap B(r_{i-1})) / vol(S cap B(r_i)) is
 * about `ratio` for a body that fills its balls; then
 *   vol(S) = vol(B(r_0)) prod_i 1 / f_i,
 * f_i the fraction of samples of S cap B(r_i) in B(r_{i-1}).  Each phase
 * creates the spectrahedron S cap B(r_i) (the ball block [[r_i, x^T],
 * [x, r_i I_n]] appended to the LMI), starts `chains` chains at the origin
 * (seed + i), runs `burn_in` steps and then `steps` steps, counting every
 * chain's point after every step.  walk: 0 Billiard (tau = 2 r_i, rho =
 * 1000, kappa = 1e-6), 1 Hit-and-Run; mode: SP_MODE_FP64 or SP_MODE_MIXED.
 * Requires the origin interior to S, B(r_inner) inside S and S inside
 * B(r_outer) (otherwise the result is the volume of S cap B(r_outer) times
 * vol(B(r_inner)) / vol(S cap B(r_inner))).  vol (host): the estimate; info
 * (host, 4 doubles, may be NULL): phases q, samples per phase, relative
 * standard error from the per-phase binomial errors (the chains'
 * autocorrelation is ignored, so it is optimistic), wall seconds.
 * Synchronises `stream`.  SP_EINVAL for bad arguments or a phase with no
 * sample in the smaller ball.
 */
int sp_volume_estimate(sp_spec* s, double r_inner, double r_outer, double ratio, int chains,
                       int burn_in, int steps, int walk, int mode, uint64_t seed, double* vol,
                       double* info, void* stream);

/*
 * The Monte Carlo estimate of the expected value of f(x) = 1(c.x <= b1 or
 * c.x >= b2) -- the indicator of S cap H for the union H of two half-spaces
 * (Sec. 4.2) -- over the chains' current points, in `groups` consecutive
 * groups of C / groups chains: frac_out[g] (host) = the fraction of group g's
 * points in H.  c: host or device, n doubles.  SP_EINVAL unless groups
 * divides C and b1 < b2.  Synchronises `stream`.
 */
int sp_halfspace_fraction(sp_chains* ch, const double* c, double b1, double b2, int groups,
                          double* frac_out, void* stream);

/*
 * A batch of spectrahedra of uneven sizes (n, m) walked together: the
 * Billiard walk (Sec. 3.2, Alg. 5) of every chain of every body in ONE
 * persistent launch on the FP64 path.  Work items are (body, chain) pairs
 * handed out by a device-side queue in decreasing order of the estimated
 * cost of a segment (formation, Cholesky, Lanczos, normal), so that the
 * longest items start first; a block carves its shared memory for each
 * item's body (factor in shared memory when it fits, else in global
 * memory) and runs all its steps with the body's Cholesky panel width.
 *   sp_create_batch : bodies handles (not owned; they must outlive the
 *                     batch), chains[i] chains each, all starting at their
 *                     body's origin (checked interior: SP_ENOTPD); body i's
 *                     chain c draws from Philox chain chain0_i + c with
 *                     chain0_i = chains[0] + ... + chains[i-1], key `seed`.
 *   sp_batch_billiard: `steps` steps of every chain; tau (host, one per
 *                     body), rho, kappa as in sp_step_billiard.
 *   sp_batch_dims   : n, m, chains and chain0 of body i (host outputs, may be NULL).
 *   sp_batch_state  : x_out (host or device, chains[i] x n) <- body i's points.
 *   sp_batch_stats  : stats (host, bodies x SP_NUM_STATS) summed per body.
 *   sp_batch_panels : read (panel_out) and / or set (panel_in) the Cholesky
 *                     panel widths (host, one per body: 4, 8 or 16; default 8).
 *   sp_batch_tune   : the autotuner: for every body, the panel width whose
 *                     calibration (REFLECTION of two lines per SM from the
 *                     origin, one untimed and one timed launch per width) is
 *                     fastest; results are cached per (device name, n, m) in
 *                     the text file cache_path (read if present, rewritten
 *                     with new entries; NULL: no cache).  times_out (host,
 *                     bodies x 3, may be NULL): the calibration ms of widths
 *                     4, 8, 16 (from the cache when found there).
 */
typedef struct sp_batch sp_batch;
int sp_create_batch(int bodies, sp_spec* const* specs, const int* chains, uint64_t seed,
                    sp_batch** out, void* stream);
int sp_destroy_batch(sp_batch* b);
int sp_batch_billiard(sp_batch* b, int steps, const double* tau, int rho, double kappa,
                      void* stream);
int sp_batch_dims(const sp_batch* b, int body, int* n, int* m, int* chains, int* chain0);
int sp_batch_state(sp_batch* b, int body, double* x_out, uint32_t* step_out, void* stream);
int sp_batch_stats(sp_batch* b, long long* stats, void* stream);
int sp_batch_panels(sp_batch* b, int* panel_out, const int* panel_in);
int sp_batch_tune(sp_batch* b, const char* cache_path, double* times_out, void* stream);

/*
 * Chain state.
 *   sp_get_state: x_out (host or device, C x n) <- current points; *step_out <-
 *                 the next step number.  Synchronises `stream` when x_out is host.
 *   sp_set_state: replace the points (host or device, C x n; interior is not
 *                 re-checked) and the step number (resume from a checkpoint).
 *   sp_chain_status: status (device int32, C) of each chain's last failed step
 *                 (SP_ST_OK if none), and stats (host int64, SP_NUM_STATS) summed
 *                 over chains since init (synchronises `stream`).
 */
int sp_get_state(sp_chains* ch, double* x_out, uint32_t* step_out, void* stream);
int sp_set_state(sp_chains* ch, const double* x, uint32_t step, void* stream);
int sp_chain_status(sp_chains* ch, int* status, long long* stats, void* stream);

/*
 * INTERSECTION without any allocation (no counterpart in the paper; an
 * interface for callers that cannot allocate device memory).
 *
 * Callers that live inside another runtime's memory pool, run under an
 * allocator policy that forbids cudaMalloc, or sit in a loop where a driver
 * allocation would stall, cannot create a spectrahedron handle (which owns
 * device memory).  This entry point takes everything from the caller instead
 * and allocates nothing: its working memory is one 8 MiB array of device
 * memory declared statically in the library, present on every GPU that loads
 * the library until the process exits.
 *   n, m     : dimension and matrix size.  m is limited to what one thread
 *              block's shared memory holds (about m <= 210), and the work
 *              space of at least one block must fit in the 8 MiB array;
 *              larger problems return SP_EINVAL.  One block's work space is
 *              m^2 + m(m+1)/2 + 96 m doubles, so the array holds
 *              floor((2^20 - ceil(m(m+1)/4)) / that) blocks: 13 at m = 200,
 *              52 at m = 100 (at most one per SM).  The call therefore runs
 *              on that many SMs, well below the one block per SM of
 *              sp_intersect for m above about 90.
 *   A_packed : device, (n+1) x m(m+1)/2 float64, caller-owned: row j is the
 *              lower triangle of A_j packed row by row (element (i, k), i >= k,
 *              at i(i+1)/2 + k).
 *   count, x, v, t_minus, t_plus, status: as in sp_intersect (device).
 * Results equal those of sp_intersect (SP_MODE_FP64, default solver).  The
 * first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the one array, which keeps whatever the previous call left in
 * it: calls that overlap on the GPU (different streams or host threads) race
 * and must be serialised by the caller.
 */
int sp_intersect_noalloc(int n, int m, const double* A_packed, int count, const double* x,
                         const double* v, double* t_minus, double* t_plus, int* status,
                         void* stream);

/*
 * The learned warm start (not in the paper): a three-layer perceptron
 * din -> dh -> dh -> dout (ReLU) that maps a line (x, v) to (log t+, u) so
 * that the boundary oracle can shift the pencil next to the boundary and
 * start its eigen-iteration from u.  BF16 weights and activations, FP32
 * accumulation on the tensor cores; FP32 master weights, Adam.
 * Parameter layout (floats): W1 [dh x ceil8(din)] (columns >= din zero),
 * b1 [dh], W2 [dh x dh], b2 [dh], W3 [ceil16(dout) x dh] (rows >= dout
 * zero), b3 [ceil16(dout)].
 * Training loss per sample, batch mean:
 *   (Y_0 - T_0)^2 + 1 - (a.b)^2 / (|a|^2 |b|^2),  a = Y_1.., b = T_1..
 *   sp_mlp_create : dh a multiple of 8; He initialisation from `seed`.
 *   sp_mlp_params : copy the parameters to host_out and / or from host_in (host).
 *   sp_mlp_forward: X (device f32, count x din) -> Y (device f32, count x dout).
 *   sp_mlp_gradients: one forward + backward on (X, T) (device, T count x dout,
 *                   count a multiple of 8); gradients (host, parameter layout)
 *                   and the loss (host).  Synchronises `stream`.
 *   sp_mlp_train  : `epochs` passes of Adam over count / batch mini-batches in
 *                   order; losses_host[e] = last mini-batch loss of epoch e.
 */
typedef struct sp_mlp sp_mlp;
int sp_mlp_create(int din, int dh, int dout, uint64_t seed, sp_mlp** out);
int sp_mlp_destroy(sp_mlp* q);
int sp_mlp_dims(const sp_mlp* q, int* din, int* dh, int* dout, long long* nparams);
int sp_mlp_params(sp_mlp* q, float* host_out, const float* host_in);
/* Save the network to a file (a small header with the dimensions, then the
 * FP32 parameters in the layout above) / create a network from such a file
 * (`seed` only initialises the optimiser state's generator; the Adam
 * moments start at zero).  SP_EINVAL on I/O errors or a malformed file. */
int sp_mlp_save(sp_mlp* q, const char* path);
int sp_mlp_load(const char* path, uint64_t seed, sp_mlp** out);
int sp_mlp_forward(sp_mlp* q, int count, const float* X, float* Y, void* stream);
int sp_mlp_gradients(sp_mlp* q, int count, const float* X, const float* T, float* grads_host,
                     float* loss_host, void* stream);
int sp_mlp_train(sp_mlp* q, int count, const float* X, const float* T, int epochs, int batch,
                 float lr, float* losses_host, void* stream);

/*
 * Attach a warm-start network (din = 2n inputs (x * x_scale, v), dout = 1 + m
 * outputs (log(t+ / t_scale), u)) to a spectrahedron for SP_MODE_LEARNED
 * walks, or detach it (q = NULL).  The Billiard walk then factors
 * F + sigma0 V at sigma0 = (1 - margin) t^ and runs at most `iters` FP32
 * power iterations from the predicted u; a prediction that fails the
 * certificate (convergence, positive dominant eigenvalue, t+ - sigma0 <
 * sigma0) falls back to the plain stage 1.  The caller keeps ownership of q.
 */
int sp_attach_mlp(sp_spec* s, sp_mlp* q, double x_scale, double t_scale, double margin,
                  int iters);

/*
 * Diagnostic of the reciprocal routines inside the dense kernels (the
 * Cholesky pivots and the inverted diagonal blocks use them instead of the
 * FP64 divide and square root): for each x[c] (device, count float64)
 * out[4c .. 4c+3] (device) = 1/sqrt(x) and 1/x from an FP32 seed refined by
 * two Newton steps in FP64, then the same two in double-float arithmetic
 * (rounded to FP64).  The FP64 versions hold for x in [1e-37, 3e37], the
 * range the Cholesky accepts as pivots (outside it the factorisation reports
 * failure); the double-float ones for x in [2^-62, 2^100] (below, the
 * conversion of an FP64 x to a pair keeps only its FP32 part; above, the low
 * parts of the intermediate products leave the FP32 normal range), far
 * beyond the O(1) to O(10^4) pivots of the workloads here.
 */
int sp_selftest_recip(int count, const double* x, double* out, void* stream);

/* Warm starts accepted / rejected by the last SP_MODE_LEARNED sp_reflect call
 * on `s` (host outputs, may be NULL; synchronises the device). */
int sp_learned_counts(sp_spec* s, int* accepted, int* rejected);

/*
 * Record training tuples during SP_MODE_MIXED / SP_MODE_LEARNED Billiard
 * walks: each segment whose refinement succeeded appends
 *   x_out[k] = (x * x_scale, v)          (2n floats),
 *   y_out[k] = (log(t+ / t_scale), u)    (1 + m floats)
 * with k = atomicAdd(*count, 1) while k < capacity (device buffers; the
 * caller zeroes *count).  x_scale and t_scale are those of sp_attach_mlp
 * (defaults 1).  Pass x_out = NULL to stop recording.
 */
int sp_record_tuples(sp_chains* ch, float* x_out, float* y_out, int capacity, int* count);

/*
 * Sampled record of the boundary-oracle calls (segments) of later walk calls
 * on `ch` (all modes and walks; a measurement aid: what the walk's own
 * Alg. 2 / Alg. 3 evaluations returned on the lines it actually visited).
 * Every segment takes a ticket k from *count (device int32, zeroed by the
 * caller, incremented once per segment); the segment is written to slot
 * k / every when k % every == 0 and k / every < capacity.  buf (device,
 * capacity x (3n + 8) float64) slot layout: p[n] (the start point of the
 * segment), v[n] (its direction), w_hat[n] (unit normal, zeros unless the
 * segment reflected), t_plus, t_minus (-inf for Billiard segments), status
 * (SP_ST_*), reflected (1 if the walk reflected there), the chain's Philox
 * index (chain0 + c), the step number, the segment's index within its
 * step (0 for the first, i after i reflections) and the solver path as
 * bit flags: 1 a shifted factorisation failed and a smaller shift was used,
 * 2 the mixed path's stage 2 fell back to FP64, 4 / 8 the learned warm start
 * was accepted / rejected, 16 an eigen-solve hit its cap, 32 a shift-invert
 * refinement next to the boundary ran.  Slots fill in
 * arrival order (not deterministic across runs).  buf = NULL stops
 * recording.  SP_EINVAL when buf is given without count, capacity >= 1 and
 * every >= 1.
 */
int sp_record_segments(sp_chains* ch, double* buf, int capacity, int every, int* count);

/*
 * Per-kernel timing of later walk calls on `ch` (CUDA events recorded on the
 * walk's stream around each launch; the mixed path reads them between its
 * waves, the FP64 path at the end of the call).  out (host, 13 doubles, may
 * be NULL): [0] FP64 walk kernel ms, [1] its launches, [2] tensor-core
 * formation ms, [3] its launches (digit slicing + GEMM), [4] mixed wave
 * kernel ms, [5] its launches, [6] warm-start network ms, [7] its launches,
 * [8] other launches, [9] tensor-core normal contraction ms (Billiard),
 * [10] its launches (digit slicing + GEMM), [11] reflection finish kernel
 * ms, [12] its launches.  enable: 1 on (counters reset), 0 off (reset), -1
 * read only.
 */
int sp_kernel_timing(sp_chains* ch, int enable, double* out);

/*
 * Stage timers of the mixed path (profiling aid).  timers: device int64
 * array of (number of SMs) x 16 entries, zeroed by the caller, or NULL to
 * switch the timers off.  Block b adds the clock64() cycles it spends in
 * each stage of each segment to timers[16 b + k]: k = 0 stage-1 fill and
 * FP32 Cholesky, 1 FP32 Lanczos, 2 stage-2 fill and factorisation (double-
 * float, or FP64 on the fallback), 3 stage-2 power iterations, 4 FP64
 * Lanczos fallback, 5 normal contraction, 6 bookkeeping; and inside every
 * Lanczos run: 8 operator application, 9 reorthogonalisation, 10
 * convergence checks, 11 final Ritz pairs; and inside the double-float
 * power iterations: 12 L^{-T} solve, 13 product with V, 14 L^{-1} solve,
 * 15 reductions and vector updates.
 */
int sp_set_stage_timers(sp_spec* s, long long* timers);

/* Tuning knobs of the FP64 path (defaults in parentheses):
 *   kmax (96): Lanczos iteration cap; tol (1e-13): relative residual target;
 *   sigma_frac (0.1): after a reflection the next factorisation is taken at
 *   x + sigma v with sigma = sigma_frac * (previous t+), falling back to
 *   sigma = 0 when that point is outside S. */
int sp_set_solver(sp_spec* s, int kmax, double tol, double sigma_frac);

/*
 * Parameters of the mixed-precision path: tol32 (relative residual of the
 * FP32 Lanczos of stage 1, default 1e-4), tol64 (relative residual of the
 * stage-2 power iteration, default 1e-10: t then takes a pencil Rayleigh
 * correction on the exact F and V, summed with error-free transformations,
 * whose error is quadratic in u's), delta1 (stage 2 factors at
 * sigma0 + (t~ - sigma0)(1 - delta1), default 2e-4) and power_iters (its
 * iteration limit before the FP64 fallback, default 8).  SP_EINVAL outside
 * tol32, tol64 in (0, 1), delta1 in (0, 0.5), power_iters in [1, 64].
 */
int sp_set_mixed_solver(sp_spec* s, double tol32, double tol64, double delta1, int power_iters);

#ifdef __cplusplus
}
#endif
#endif /* SPECTRA_GB_H */
