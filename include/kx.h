/*
 * kx.h -- C ABI of the GB300 exponential-Krylov Maxwell solver.
 *
 * Method: Botchev, Hanse & Uppu, "Exponential Krylov time integration for
 * modeling multi-frequency optical response with monochromatic sources"
 * (arXiv:1707.00023).  The library solves the semi-discrete Maxwell system
 *
 *     y'(t) = -A y(t) + sin(Omega t) g,   y(0) = 0          (eq. (ode))
 *
 * on a Yee grid, by exponential Krylov methods: the plain time-restarted
 * method on the system augmented with the source phase, and the asymptotic
 * splitting y = Im(e^{i Omega t} z) - exp(-tA) Im z with z = (A + i Omega I)^{-1} g
 * (eq. (split1)), whose stationary parts for many frequencies share one
 * Krylov basis (Corollary 1).
 *
 * Conventions shared by every entry point:
 *  - Field vectors are CALLER-OWNED DEVICE arrays of n = ncomp * ncell
 *    scalars in the context's precision (double for KX_FP64, float for
 *    KX_FP32).  Layout: component-major [Hx, Hy, Ez] (2D) or
 *    [Hx, Hy, Hz, Ex, Ey, Ez] (3D); within a component x is fastest, then y,
 *    then z.  Nodes on a conducting wall (integer coordinate along a PEC
 *    axis at index 0) are not unknowns: input values there are ignored and
 *    outputs there are 0.
 *  - Small arrays (H, u, omegas, results) may be host or device memory
 *    where stated; the library tells them apart itself.
 *  - Every call is ordered on the CUDA stream given at creation.  Calls
 *    that return host values synchronise that stream.  The context owns all
 *    workspace (allocated at creation); the compute calls allocate nothing.
 *  - Every call returns a kx_status and never aborts or prints; the reason
 *    of the last failure is kept in kx_last_error(ctx).  A context is not
 *    thread-safe: use one per stream.
 */
#ifndef KX_H
#define KX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KX_OK = 0,
  KX_EINVAL = 1,      /* bad argument or descriptor                        */
  KX_ENOMEM = 2,      /* device or host allocation failed (creation only)  */
  KX_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed       */
  KX_ENONFINITE = 4,  /* NaN/Inf met in an input or a reduction            */
  KX_ENOCONV = 5,     /* iteration cap reached; partial result returned    */
  KX_ETIMEOUT = 6     /* a bounded device-side wait ran out                */
} kx_status;

enum { KX_PERIODIC = 0, KX_PEC = 1 };
enum { KX_FP64 = 0, KX_FP32 = 1 };
enum { KX_PLAIN = 0, KX_SPLIT = 1, KX_RSTDIM = 2, KX_SPLIT2 = 3, KX_SPLIT4D = 4 };
/* Form of the Arnoldi process (kx_desc.arnoldi_form).  Both are classical
 * Gram-Schmidt (Sect. 3.2, eq. (Arn)) and agree up to rounding.
 *   KX_ARN_DEFAULT: the single-sweep form for restart in Krylov dimension
 *                   on grids of 3e6 unknowns or more (where it is the
 *                   faster of the two on GB300), the two-pass form
 *                   everywhere else.
 *   KX_ARN_TWOPASS: per step, one pass applies A fused with the dots
 *                   V_j^T A v_j, a second applies the update and the norm;
 *                   the basis is read twice.
 *   KX_ARN_SWEEP:   per step, one pass reads the basis once: it forms the new
 *                   column from the explicit A v_{j-1} and, from A^2 v_{j-1},
 *                   the dots that give the next Hessenberg column through
 *                   the Arnoldi relation and the Gram matrix of the basis.
 *                   A second, light pass applies A to the new column.  Used
 *                   wherever the process carries no augmented source phase:
 *                   restart in Krylov dimension and arnoldi(). */
enum { KX_ARN_DEFAULT = 0, KX_ARN_TWOPASS = 1, KX_ARN_SWEEP = 2 };

/* Problem descriptor.  Grid of n[0] x n[1] (x n[2]) unit cells; the
 * absorbing layer (conductivity ramping linearly from 0 to sigma_max over
 * layer_cells cells at both ends of layer_axis) lies inside the grid.  The
 * conductivity of a node is sigma_max * d / layer_cells with d the depth of
 * the node's own staggered coordinate into the layer (Sect. 2.1 damping
 * terms; a plain lossy layer, no auxiliary PML variable). */
typedef struct {
  int dim;            /* 2 (fields Hx, Hy, Ez) or 3 (Hx, Hy, Hz, Ex, Ey, Ez) */
  int n[3];           /* cells along x, y, z (n[2] ignored when dim == 2); each >= 3 */
  int bc[3];          /* KX_PERIODIC or KX_PEC per axis                      */
  int layer_axis;     /* 0 .. dim-1                                          */
  int layer_cells;    /* >= 1, 2 * layer_cells <= n[layer_axis]              */
  double sigma_max;   /* >= 0                                                */
  int precision;      /* KX_FP64 or KX_FP32 (vectors); projected work is FP64 */
  int krylov_dim;     /* m, 2 <= m <= 64: Arnoldi steps per restart          */
  int max_freqs;      /* largest nfreq of any later call, 1 .. 64            */
  int batch;          /* bases held for concurrent transients, >= 1          */
  int max_checkpoints; /* forward states kept for the adjoint (0: no adjoint;
                          otherwise batch >= 2); one per time sub-step       */
  int rst_samples;    /* time samples of [0, T] per frequency kept by the
                         restart-in-dimension method (0: method unavailable);
                         the workspace is max_freqs * rst_samples * 72
                         bytes plus max_freqs output-plane accumulators      */
  int pml;            /* 0: lossy layer (above).  1: the paper's perfectly
                         matched layer (2D, layer_axis 0 only; Sect. 2.1,
                         eq. (mxw)): fields [Hx, Hy, Ez, P] with P on the Ez
                         nodes, Hy' = dEz/dx - sigma Hy, Ez' = (dHy/dx -
                         dHx/dy)/eps - sigma Ez + P, P' = -(sigma/eps) dHx/dy,
                         sigma = sigma_max (d/L)^2 damping Hy and Ez only.
                         n = 4 ncell; the output plane holds Ez; the adjoint
                         and kx_arnoldi_noalloc reject it                    */
  int arnoldi_form;   /* KX_ARN_DEFAULT, KX_ARN_TWOPASS or KX_ARN_SWEEP (above);
                         kx_arnoldi_noalloc always runs the two-pass form   */
} kx_desc;

typedef struct kx_ctx kx_ctx;

/* Per-context counters since creation (or the last kx_reset_stats). */
typedef struct {
  int64_t matvecs;         /* applications of A (one per Arnoldi step)   */
  int64_t arnoldi_steps;
  int64_t substeps;        /* accepted time sub-steps                     */
  int64_t expm_evals;      /* projected exponentials                      */
  int64_t fom_cycles;      /* restarts of the shifted FOM                 */
  int64_t kernel_launches; /* kernels this library launched               */
} kx_stats;

/* Pass as cuda_stream to have the context create (and destroy) its own
 * non-blocking stream; kx_stream() returns it. */
#define KX_OWN_STREAM ((void*)-1)

/* Create a context.  eps_cell: HOST array of n[0]*n[1](*n[2]) per-cell
 * relative permittivities (> 0, finite), x fastest; mu_r = 1 (Sect. 2.1).
 * The permittivity of an E node is the mean over the cells whose closure
 * holds the node.  stream: a cudaStream_t (NULL = legacy default stream) or
 * KX_OWN_STREAM.
 * All workspace (batch Krylov bases of krylov_dim + 1 vectors, projected
 * matrices, reduction buffers) is allocated here.
 * Errors: KX_EINVAL (descriptor), KX_ENONFINITE (eps), KX_ENOMEM. */
kx_status krylov_expm_create(const kx_desc* desc, const double* eps_cell,
                             void* cuda_stream, kx_ctx** out);

/* Create a context from a material id per cell (the layout Sect. 4.1's
 * media suggest: a few materials, each cell in one of them).
 *   d_mat_id : DEVICE array of n[0]*n[1](*n[2]) material ids (uint8, x
 *              fastest), caller-owned; read during this call only.
 *   eps_table: HOST array of n_mat relative permittivities (> 0, finite);
 *              cell c gets eps_table[d_mat_id[c]].
 *   n_mat    : 1 .. KX_MAX_MATERIALS.
 * Everything else as for krylov_expm_create (the per-cell permittivity is
 * expanded on the device and kept, so kx_set_permittivity and the adjoint's
 * per-cell gradient work as for a context made from eps_cell).
 * Errors: those of krylov_expm_create, and KX_EINVAL when an id is >= n_mat. */
#define KX_MAX_MATERIALS 64
kx_status krylov_expm_create_mat(const kx_desc* desc, const uint8_t* d_mat_id, const double* eps_table,
                                 int n_mat, void* cuda_stream, kx_ctx** out);

/* Release a context and its workspace.  NULL is accepted. */
kx_status krylov_expm_destroy(kx_ctx* ctx);

/* The CUDA stream the context works on (a cudaStream_t). */
void* kx_stream(const kx_ctx* ctx);

/* Number of unknowns n (including wall nodes) of the context's grid. */
int64_t kx_num_unknowns(const kx_ctx* ctx);

/* w = A v (transpose = 0) or w = A^T v (transpose = 1), A the matrix of
 * eq. (ode): H rows sigma H + curl E, E rows (sigma E - curl H) / eps.
 * d_v, d_w: device vectors of n scalars, must not overlap.  Asynchronous. */
kx_status apply_A(kx_ctx* ctx, const void* d_v, void* d_w, int transpose);

/* m steps of the Arnoldi process for K_m(A, v0) (Sect. 3.2, eqs. (Arn),
 * (Arn1)): A V_m = V_{m+1} H, v_1 = v0/||v0||.  Classical Gram-Schmidt,
 * dots fused with the operator application; the descriptor's arnoldi_form
 * picks the two-pass form (KX_ARN_DEFAULT, KX_ARN_TWOPASS) or the
 * single-sweep form (KX_ARN_SWEEP).
 *   d_v0  : device, n scalars (not modified).
 *   m     : 1 .. krylov_dim.
 *   d_V   : device n x (m+1) column-major (leading dim n) receiving the
 *           orthonormal basis, or NULL.
 *   H     : (m+1) x m column-major FP64, host or device, zero-filled then
 *           written.
 *   beta  : host, receives ||v0||.     m_done: host, steps done (< m only
 *           after a lucky breakdown, h_{j+1,j} ~ 0; then columns past
 *           m_done of d_V are zero).
 * Synchronises the stream.  Errors: KX_EINVAL, KX_ENONFINITE (v0 = 0 or
 * non-finite). */
kx_status arnoldi(kx_ctx* ctx, const void* d_v0, int m, void* d_V, double* H,
                  double* beta, int* m_done);

/* Projected solutions (eq. (corr2); Corollary 1).  H: (m+1) x m upper
 * Hessenberg (only the leading m x m block is used), leading dimension
 * ldh >= m, FP64, host or device.
 *   nfreq == 0: u = exp(-tau H_m) beta e_1                   (m values)
 *   nfreq >= 1: u_j = u(tau) of u' = -H_m u + sin(omega_j t) beta e_1,
 *               u(0) = 0, for each omega_j (host array)      (m x nfreq)
 * Evaluated by FP64 scaling-and-squaring Pade (Higham 2005) of the
 * (m+2) x (m+2) matrix that carries the source phase.  u_out: host or
 * device, column-major m x max(1, nfreq).  m <= krylov_dim, nfreq <=
 * max_freqs.  Synchronises the stream. */
kx_status expm_phi_project(kx_ctx* ctx, const double* H, int ldh, int m,
                           double beta, double tau, const double* omegas,
                           int nfreq, double* u_out);

/* Stationary parts z_j = (A + i omega_j I)^{-1} g for all j (eq. (split1)),
 * by restarted shifted FOM on ONE real Krylov basis per restart (the
 * residuals of all shifts stay collinear with v_{m+1}, eq. (Arn1)).
 *   d_g: device n scalars.  omegas: host nfreq (1 .. max_freqs).
 *   rtol: stop when every |rho_j| <= rtol ||g||.  max_matvecs: cap (> 0).
 *   d_z_re, d_z_im: device n x nfreq column-major (leading dim n).
 *   rel_resid: host nfreq, TRUE relative residuals ||g - (A+i w)z||/||g||
 *              (or NULL).  matvecs: host, applications of A used (or NULL).
 * Returns KX_ENOCONV (with the partial z) if the cap is hit first.
 * Synchronises the stream. */
kx_status stationary_solve(kx_ctx* ctx, const void* d_g, const double* omegas,
                           int nfreq, double rtol, int max_matvecs,
                           void* d_z_re, void* d_z_im, double* rel_resid,
                           int* matvecs);

/* y = exp(-T A) y0 (the homogeneous problem eq. (y_homo)) by exponential
 * Krylov restarted in time; each sub-step's length is chosen so that the
 * integrated Lemma 1 residual stays below rtol * ||y0|| * (sub-step / T).
 * d_y0, d_y: device n scalars (may be equal).  err_est: host (or NULL).
 * Synchronises the stream. */
kx_status expm_action(kx_ctx* ctx, const void* d_y0, double T, double rtol,
                      void* d_y, double* err_est);

/* Frequency responses y_j(T) of eq. (ode) (v = 0, alpha = sin(omega_j t)).
 *   method KX_PLAIN: exponential Krylov restarted in time on the system
 *     augmented with the source phase, one frequency at a time.
 *   method KX_SPLIT: eq. (split1) with all stationary parts from one
 *     shifted solve (stationary_solve) and the transients exp(-TA) Im z_j by
 *     expm_action (Fig. alg:spl1 steps 1-3 for each frequency).
 *   method KX_RSTDIM: response_restart_dim with dt_sample = 0 and
 *     max_restarts = 0; err_est receives its resid.
 *   method KX_SPLIT2: source splitting (eq. (split2)): restart in time on
 *     subintervals of one source period dT_j = 2 pi / omega_j.  w2, the
 *     solution from zero over one period (and over the remainder
 *     r = T - K dT_j when T is not a whole number of periods), is found
 *     once per frequency by the plain method; then y <- exp(-dT_j A) y + w2
 *     on every later period (homogeneous problems only).  err_est receives
 *     the summed error estimates of all pieces.
 *   method KX_SPLIT4D: as KX_SPLIT, but the transient of each frequency
 *     after the first comes from the previous one's (eq. (4diff), Fig.
 *     alg:spl1 steps 4-6): yhat_j(T) = yhat_{j-1}(T) + exp(-TA)(Im z_j -
 *     Im z_{j-1}), each difference solved to rtol ||Im z_j|| / nfreq (so the
 *     errors that frequency j accumulates stay within its own budget);
 *     frequencies are taken in the given order (neighbours should be close).
 *   plane: host int[2] = {axis, index}: output plane perpendicular to axis.
 *   d_E_plane: device, nfreq x nE x (plane nodes) scalars (nE = 1 in 2D:
 *     Ez; 3 in 3D: Ex, Ey at the plane, Ez half a cell above), or NULL.
 *   intensity: host nfreq, summed |E|^2 over the plane (or NULL).
 *   err_est: host nfreq, a-posteriori error estimates (or NULL).
 *   d_Y: device n x nfreq full fields y_j(T), or NULL.
 * Synchronises the stream.  KX_ENOCONV if a stationary solve hit its cap. */
kx_status response_at_freqs(kx_ctx* ctx, const void* d_g, const double* omegas,
                            int nfreq, double T, double rtol, int method,
                            const int* plane, void* d_E_plane, double* intensity,
                            double* err_est, void* d_Y);

/* Frequency responses by residual-based restarting in Krylov dimension
 * (Sect. 3.4, eq. (rst), Corollary 2, Fig. alg:rst; regular Krylov
 * variant).  One Arnoldi basis per restart serves every frequency: restart 1
 * starts from g / ||g|| with source alpha(t) = ||g|| sin(omega_j t); after m
 * steps each frequency's projected problem u' = -H_m u + alpha(t) e_1,
 * u(0) = 0 (eq. (corr2)) is integrated over [0, T], y_j(T) += V_m u(T)
 * (eq. (upd1)), and the residual alphahat(t) v_{m+1}, alphahat =
 * -h_{m+1,m} e_m^T u(t) (eq. (resid)), is the next restart's source, from
 * v_{m+1}.  alphahat is stored per frequency at Nt + 1 equally spaced times
 * with its first two derivatives (Fig. alg:rst step 2(b)); the projected
 * problems are integrated exactly for the quintic Hermite interpolant of
 * those samples on each sample interval (matrix exponential and phi
 * functions of the interval, FP64).
 *   rtol       : frequency j stops after the restart whose new residual has
 *                max_t |alphahat(t)| <= rtol * ||g|| (step 2(c)); rtol = 0
 *                runs max_restarts restarts.
 *   dt_sample  : sample spacing (T / Nt rounds it down to fit); 0 picks
 *                T * ||H_m||_1 / Nt = 1 (KX_FP32) or 0.3 (KX_FP64) from the
 *                first restart's Hessenberg matrix.
 *   max_restarts: cap (0: 3 * T * ||H_m||_1 / m + 20).
 *   plane, d_E_plane, intensity, d_Y: as for response_at_freqs.  The plane
 *                values are accumulated in FP64 over the restarts; d_Y in
 *                KX_FP32 through a compensated float pair.
 *   resid      : host nfreq (or NULL): last max_t |alphahat(t)| / ||g||.
 *   restarts   : host nfreq (or NULL): restarts each frequency took.
 * Needs a context with rst_samples >= Nt (KX_EINVAL names the Nt needed);
 * krylov_dim = 64 is advised, smaller m lets intermediate residuals grow.
 * With batch >= 2 the projected work of restart k runs on an auxiliary
 * stream of the context while restart k+1's Arnoldi process runs on the
 * context's stream (so one Arnoldi process may run past the last restart);
 * results are the same bits as with batch = 1.
 * Synchronises the stream.  KX_ENOCONV (with the iterate) when a frequency
 * has not stopped after max_restarts restarts. */
kx_status response_restart_dim(kx_ctx* ctx, const void* d_g, const double* omegas, int nfreq,
                               double T, double rtol, double dt_sample, int max_restarts,
                               const int* plane, void* d_E_plane, double* intensity,
                               double* resid, int* restarts, void* d_Y);

/* Gradient of the summed output-plane intensity
 *     L = sum_j sum_plane |E_j(T)|^2,   E_j from response_at_freqs(KX_PLAIN),
 * with respect to the per-cell permittivity (the paper has no gradient; this
 * is the adjoint of eq. (ode)):
 *     dL/deps_c = -sum_j int_0^T lambda_j(t)^T (dA/deps_c) y_j(t) dt,
 *     lambda_j(t) = exp(-(T - t) A^T) 2 P^T P y_j(T).
 * The forward solution is stored at every time sub-step (at most
 * max_checkpoints of them); backwards, each sub-step's forward Krylov basis
 * is recomputed from its checkpoint and lambda is carried by exponential
 * Krylov on A^T; the time integral is composite Gauss-Legendre quadrature on
 * the exact projected solutions.
 *   d_grad_eps: device, ncell doubles (x fastest), receives dL/deps.
 *   loss: host, receives L.
 * Requires a context created with max_checkpoints > 0 (and batch >= 2).
 * Synchronises the stream.  KX_ENOMEM if the sub-steps exceed the
 * checkpoints. */
kx_status adjoint_response_grad(kx_ctx* ctx, const void* d_g, const double* omegas, int nfreq,
                                double T, double rtol, const int* plane, double* d_grad_eps,
                                double* loss);

/* Replace the per-cell permittivity of a context (host or device array of
 * ncell doubles, each > 0); the grid and workspace stay.  Synchronises. */
kx_status kx_set_permittivity(kx_ctx* ctx, const double* eps_cell);

/* Independent problems in one call (the uneven batch: many scatterer
 * instances of different sizes).  ctxs[i] holds problem i's grid, medium and
 * CUDA stream (use a distinct non-default stream per context); d_g[i] its
 * source; omegas is nctx x nfreq (row i = problem i's frequencies); planes is
 * nctx x 2; intensity and err_est (host, nctx x nfreq, or NULL) as for
 * response_at_freqs.  nthreads host threads take the problems largest-first
 * and drive them concurrently, so their kernels overlap on the GPU (each
 * context's sub-steps replay a captured CUDA graph).  The streams of the
 * contexts must be distinct (KX_OWN_STREAM guarantees it).  Each context must be
 * created with max_freqs >= nfreq; its batch sets how many of its frequencies
 * advance together.  On failure the first error is returned and its text is
 * kx_last_error(NULL). */
kx_status response_at_freqs_multi(kx_ctx* const* ctxs, int nctx, const void* const* d_g,
                                  const double* omegas, int nfreq, double T, double rtol, int method,
                                  const int* planes, double* intensity, double* err_est, int nthreads);

/* Batched restart in Krylov dimension for many independent problems (the
 * uneven batch of Sect. 4's use case: scatterer instances of different sizes,
 * a few frequencies each).  Each problem keeps its own context; the Arnoldi
 * process of every restart (Sect. 3.2) runs for all problems together, one
 * launch per phase whose blocks a table splits between the problems, and
 * each problem's per-frequency projected work (Fig. alg:rst steps (2), (3))
 * runs on its context's auxiliary stream beside the next batched Arnoldi
 * process.  Results equal response_restart_dim on each problem up to the
 * order of the block reductions.
 *
 * kx_batch_create: ctxs are nctx distinct contexts, each 3D, KX_FP32, the
 * lossy layer, n[0] a multiple of 4, batch >= 2, rst_samples > 0, and all
 * with the same krylov_dim; they stay owned by the caller and must outlive
 * the batch, and must not be used by other calls while a batched call runs.
 * cuda_stream: the stream of the batched launches (or KX_OWN_STREAM).
 * Creation allocates a small table and chooses how each launch is split
 * (an autotuner times an Arnoldi process of min(12, krylov_dim) steps of the whole batch for each
 * candidate granularity -- sweep tiles per block 1..16, apply work per thread
 * r = 1, 2, 4 (step 0: r quad rounds; later steps: 2 r planes a thread in the
 * column march) -- and keeps the fastest; the choice is cached per size
 * class, the multiset of the problems' grids, for the rest of the process).
 * The timing runs overwrite basis slot 0 of every context.  The batched
 * Arnoldi process of each basis slot (about 2 m launches) is captured once as a
 * CUDA graph and replayed at every restart; it is captured again when the
 * split or krylov_dim changes, and launched directly while per-launch timing
 * is on (or if a capture fails).
 * Errors: KX_EINVAL (arguments, a context that does not qualify), KX_ENOMEM,
 * KX_ECUDA; text by kx_batch_last_error(NULL). */
typedef struct kx_batch kx_batch;
typedef struct {
  int problems;
  int sweep_tiles_per_block;    /* the autotuner's choice                      */
  int apply_rounds_per_thread;  /* the autotuner's choice                      */
  int sweep_blocks;             /* blocks of one batched sweep launch          */
  int apply_blocks;             /* blocks of one batched apply launch, steps
                                   j >= 1 (the column march)                   */
  int from_cache;               /* 1: the choice came from an earlier batch    */
  double tune_ms;               /* time the timing runs took (0 if cached)     */
  int64_t batched_launches;     /* batched Arnoldi launches so far             */
  double sweep_ms;              /* summed event time of the timed batched sweep
                                   launches (kx_batch_set_timing)              */
  double sweep_bytes;           /* their algorithmic bytes: per problem still
                                   running (j+2) n s + 3 ncell s at step j     */
  int64_t sweep_timed_launches;
  int64_t graph_replays;        /* batched Arnoldi processes launched as one
                                   replay of their captured CUDA graph         */
} kx_batch_info;
kx_status kx_batch_create(kx_ctx* const* ctxs, int nctx, void* cuda_stream, kx_batch** out);
kx_status kx_batch_destroy(kx_batch* batch);
kx_status kx_batch_get_info(const kx_batch* batch, kx_batch_info* out);
/* Per-launch timing of the batched sweep launches (a measurement aid, off by
 * default): with it on, each batched sweep launch is bracketed by CUDA events
 * on the batch's stream, and the totals appear in kx_batch_info after each
 * batched call.  The events break the programmatic overlap between
 * neighbouring launches; leave it off in timed runs. */
kx_status kx_batch_set_timing(kx_batch* batch, int on);
const char* kx_batch_last_error(const kx_batch* batch);

/* Responses of every problem of a batch by restart in Krylov dimension (as
 * response_restart_dim, with dt_sample = 0).
 *   d_g      : nctx device sources (problem i's grid, FP32).
 *   omegas   : host nctx x nfreq, row i = problem i's frequencies
 *              (nfreq <= every context's max_freqs).
 *   planes   : host nctx x 2 output planes {axis, index}.
 *   intensity, resid: host nctx x nfreq (or NULL), as for
 *              response_restart_dim.  restarts: host nctx x nfreq int (or NULL).
 * Synchronises the batch's stream.  KX_ENOCONV when some frequency has not
 * stopped after max_restarts restarts (0: the default cap per problem);
 * KX_ETIMEOUT when a bounded device wait ran out. */
kx_status response_restart_dim_batch(kx_batch* batch, const void* const* d_g, const double* omegas, int nfreq,
                                     double T, double rtol, int max_restarts, const int* planes, double* intensity,
                                     double* resid, int* restarts);

/* Counters; kx_reset_stats zeroes them. */
kx_status kx_get_stats(const kx_ctx* ctx, kx_stats* out);
kx_status kx_reset_stats(kx_ctx* ctx);

/* Per-kernel-class device timing (a measurement aid, off by default).
 * With timing on, every launch of the classes below is bracketed by CUDA
 * events recorded on the context's stream; kx_kernel_times synchronises the
 * stream and returns, per class, the summed event time, the algorithmic
 * bytes those launches must move (the traffic counted in the design notes)
 * and the launch count, then clears the record.  Timing adds host work per
 * launch; leave it off in timed runs. */
enum { KX_K_PASS_A = 0,    /* operator application fused with the Gram-Schmidt dots */
       KX_K_PASS_B = 1,    /* Gram-Schmidt update and norm                          */
       KX_K_RESTART = 2,   /* basis combination y = V_m u and renormalisation       */
       KX_K_PROJ = 3,      /* FP64 projected work (expm, step control, shifted solves) */
       KX_K_ZUPDATE = 4,   /* multi-shift update of the stationary parts            */
       KX_K_APPLY = 5,     /* plain operator application                            */
       KX_K_CASCADE = 6,   /* projected time stepping of restart in dimension       */
       KX_K_SWEEP = 7,     /* single-sweep Arnoldi: update, dots and norms in one pass */
       KX_K_SWAPPLY = 8,   /* single-sweep Arnoldi: A applied to the new column     */
       KX_NKCLASS = 9 };
typedef struct {
  double ms;
  double bytes;
  int64_t launches;
} kx_kernel_time;
kx_status kx_set_timing(kx_ctx* ctx, int on);
kx_status kx_kernel_times(kx_ctx* ctx, kx_kernel_time out[KX_NKCLASS]);

/* Text of the last failure on this context ("" if none).  NULL ctx gives
 * the last creation failure of the calling thread. */
const char* kx_last_error(const kx_ctx* ctx);

/* Check of the device-side failure path (not a paper operation): every wait
 * in this library's kernels is bounded (the single-sweep Arnoldi waits on
 * mbarriers for its basis copies); when a wait runs out the kernel records
 * KX_ETIMEOUT, returns normally and the context stays usable.  This call
 * runs that wait, `rounds` try_wait rounds (1 .. KX_WAIT_SELFTEST_MAX_ROUNDS,
 * the limit of one wait in the library's own kernels), on an mbarrier that
 * nothing completes and no copy targets.  Synchronises the stream.
 * Returns KX_ETIMEOUT (the expected outcome), KX_EINVAL (rounds out of
 * range) or KX_ECUDA. */
#define KX_WAIT_SELFTEST_MAX_ROUNDS (4194304u)
kx_status kx_wait_selftest(kx_ctx* ctx, unsigned rounds);

/* Allocation-free Arnoldi (the paper has no counterpart: this is a
 * deployment convenience).  Some callers cannot allocate device memory at
 * all -- code running inside another runtime's memory pool, plug-ins handed
 * a fixed arena, services that forbid cudaMalloc and cudaFree after
 * start-up -- and so cannot create a context.  This call needs
 * no context and performs no device allocation: the caller passes every
 * input and output, the basis array d_V doubles as the Krylov workspace, and
 * the remaining scratch (block partial sums, column scales, the step state
 * and a completion counter) lives in one fixed device array of
 * KX_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   desc      : grid, boundaries, layer and precision as for
 *               krylov_expm_create (krylov_dim, max_freqs, batch ignored).
 *   d_eps_cell: DEVICE array of the per-cell permittivities (double).
 *   d_v0      : device start vector, n scalars (not modified).
 *   m         : 1 .. 64 Arnoldi steps; larger m is rejected (KX_EINVAL),
 *               the scratch array holds at most 64 columns.
 *   d_V       : device n x (m+1) basis (leading dim n), 16-byte aligned,
 *               with n * sizeof(scalar) a multiple of 16 (KX_EINVAL
 *               otherwise); returned orthonormal as by arnoldi().
 *   d_H       : device (m+1) x m FP64 Hessenberg matrix (column-major).
 *   beta, m_done: host outputs as for arnoldi(); a zero or non-finite v0
 *               is refused (KX_ENONFINITE) before any Arnoldi step runs.
 * Results match arnoldi() on a context with the same descriptor and
 * arnoldi_form KX_ARN_DEFAULT or KX_ARN_TWOPASS (this entry runs the
 * two-pass form whatever the descriptor's arnoldi_form).  The call
 * synchronises cuda_stream.  Its first call on a device takes the device
 * address of the scratch array (set-up), so make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents (each call clears what must start at zero); calls whose GPU work
 * overlaps, on different streams or from unsynchronised host threads, race
 * on it.  Errors are reported by kx_noalloc_last_error(). */
#define KX_NOALLOC_SCRATCH_BYTES (1310720)
kx_status kx_arnoldi_noalloc(const kx_desc* desc, const double* d_eps_cell, const void* d_v0,
                             int m, void* d_V, double* d_H, double* beta, int* m_done,
                             void* cuda_stream);
const char* kx_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KX_H */
