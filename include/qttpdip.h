/*
 * qttpdip.h - C ABI of the GB300 library for QTT-accelerated PDIP Newton solves
 * of the frictional-contact cone complementarity problem (CCP).
 *
 * Method: Corona, Gorsich, Jayakumar, Veerapaneni, "Tensor Train accelerated
 * solvers for nonsmooth rigid body dynamics" (arXiv 1808.02558).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: QP_OK (0) or a negative QP_* code.
 *    No C++ exception crosses this boundary.  qp_status_string() names a code;
 *    qp_last_error() returns the message of the last failure on a context.
 *  - Pointers are DEVICE pointers (memory of the context's device) unless the
 *    parameter name ends in _host.  Input buffers are borrowed for the call
 *    only; the caller keeps ownership.  Buffers reported through output structs
 *    (qp_contacts views, qtt_t handles) are owned by the context and stay
 *    valid until the next ccp_assemble on that context (views) or until
 *    qtt_free / qp_destroy (handles).
 *  - All work is enqueued on the stream given to qp_create.  Functions that
 *    return statistics or sizes to the host synchronise that stream first.
 *  - Unknown layout ("padded layout"): contact c owns rows slots*c + {0: n,
 *    1: t1, 2: t2}; with slots = 4 row 4c+3 is a dummy row.  Rows from
 *    slots*Nc to P-1 (P = 2^L) are dummy rows too.  Dummy rows of every
 *    operator are identity rows (Sec. 3.3, uniform tree of 2^L leaves with
 *    dummy variables); dummy entries of gamma and of right-hand sides are 0.
 *  - Contacts are ordered by the Morton key of their contact point (Sec. 3.3
 *    spatial octree hierarchy), ties broken by (body a, body b).
 */
#ifndef QTTPDIP_H
#define QTTPDIP_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define QP_OK 0
#define QP_INVALID_ARG (-1)   /* bad pointer, size or option               */
#define QP_OOM (-2)           /* device allocation failed                  */
#define QP_CUDA_ERROR (-3)    /* a CUDA runtime call failed                */
#define QP_NOT_CONVERGED (-4) /* iteration cap reached before tolerance    */
#define QP_BREAKDOWN (-5)     /* Krylov breakdown (p'Sp <= 0 or r'z <= 0)  */
#define QP_LINESEARCH_FAIL (-6) /* PDIP backtracking found no step         */
#define QP_TIMEOUT (-7)       /* a bounded device-side wait expired        */
#define QP_NOT_READY (-8)     /* call order violated (e.g. no contacts)    */

typedef enum { QP_F64 = 0, QP_F32 = 1, QP_BF16 = 2 } qp_dtype;

typedef struct qp_ctx* qp_ctx_t;  /* opaque context: device buffers + stream */
typedef struct qp_qtt* qtt_t;     /* opaque QTT matrix owned by a context    */

/* ---- context ----------------------------------------------------------- */

/* Create a context on `device`; `cuda_stream` is a cudaStream_t (NULL = the
 * legacy default stream).  The context allocates its own device buffers.   */
int qp_create(qp_ctx_t* out, int device, void* cuda_stream);
int qp_destroy(qp_ctx_t ctx);
const char* qp_status_string(int status);
/* Copy the last error message (NUL-terminated, truncated to len) to buf_host. */
int qp_last_error(qp_ctx_t ctx, char* buf_host, int len);

/* ---- scene and contact assembly (Sec. 2.2-2.3, 3.3) -------------------- */

typedef struct {
  int M;                    /* number of spheres                                 */
  const double* pos;        /* [3*M] SoA: x[0..M), y[M..2M), z[2M..3M)           */
  const double* vel;        /* [3*M] SoA translational velocity                  */
  const double* omega;      /* [3*M] SoA angular velocity                        */
  const double* radius;     /* [M]                                               */
  const double* inv_mass;   /* [M] 1/m                                           */
  const double* inv_inertia;/* [M] 1/I (solid spheres: isotropic inertia)        */
  double floor_z;           /* static floor plane z = floor_z, normal +z         */
  double gravity[3];        /* body acceleration g (force m g)                   */
  double dt;                /* time step                                         */
  double delta;             /* contact envelope: active iff gap Phi <= delta     */
  double mu;                /* friction coefficient of every contact             */
  int slots;                /* rows per contact in the padded layout: 3 or 4     */
  int nwalls;               /* side walls, 0..4 (an extension for boxed scenes): */
  int wall_axis[4];         /*   static planes x_axis = wall_offset, axis 0..2,  */
  int wall_sign[4];         /*   the box on the side sign = +1 or -1             */
  double wall_offset[4];
} qp_scene;

typedef struct {
  int M, Nc, L, slots;      /* P = 1 << L padded unknowns                        */
  long long P;
  const int* body_a;        /* [Nc] first body; M denotes the static floor       */
  const int* body_b;        /* [Nc] second body                                  */
  const double* phi;        /* [Nc] gap function                                 */
  const double* frame;      /* [9*Nc] SoA: n.x n.y n.z t1.x .. t2.z, each [Nc]   */
  const double* point;      /* [3*Nc] SoA contact point                          */
  const double* arm_a;      /* [3*Nc] SoA p - x_a (0 for the floor)              */
  const double* arm_b;      /* [3*Nc] SoA p - x_b                                */
  const unsigned long long* key; /* [Nc] Morton key                              */
  const double* r;          /* [P] padded r = b + D^T M^-1 k (Eq. rdef)          */
  const int* plane;         /* [Nc] -1 for a sphere pair, 0 the floor, 1 + w side
                               wall w (which static plane body M stands for)     */
} qp_contacts;

/* Active set A(q, delta) (Sec. 2.2): every sphere pair with gap
 * Phi = |x_b - x_a| - r_a - r_b <= delta, every sphere with
 * Phi = z - floor_z - r <= delta, and every sphere with
 * Phi = sign (x_axis - offset) - r <= delta against a side wall (normal
 * sign e_axis, contact point offset + sign Phi/2 on that axis, the floor's
 * rule); floor and walls are the static body M (ties in the order broken by
 * plane: floor, then walls in their order); nwalls outside 0..4, an axis
 * outside 0..2 or a sign other than +-1 is QP_INVALID_ARG.  Builds frames (normal from a to b; t1 =
 * normalize(n x e), e the axis minimising |n_e|; t2 = n x t1), contact points
 * p = x_a + n (r_a + Phi/2), arms, Morton keys (21 bits per axis over the
 * bounding box of the contact points), the ordered list, the body->contact
 * incidence, and r (Eq. rdef, body force = gravity).  Pair list and order are
 * bit-exact with an IEEE evaluation in the documented order.  Replaces the
 * previous contact set of the context (and invalidates earlier views).      */
int ccp_assemble(qp_ctx_t ctx, const qp_scene* scene, qp_contacts* out);

/* ---- PDIP state and the Newton operator (Sec. 2.4, 3.3) ----------------- */

typedef struct {
  double* gamma;   /* [P] padded impulses (gn, g1, g2 per contact), dummies 0    */
  double* lambda;  /* [2*Nc] multipliers: cone constraints, then -gn <= 0       */
  double t;        /* barrier parameter of the current Newton system (output of
                      pdip_step; input of newton_solve/newton_apply rhs)        */
} qp_state;

/* Initial point of Sec. 3.3: gn = gn0 (> 0), gt = 0, lambda_i = -1/f_i.      */
int pdip_init(qp_ctx_t ctx, qp_state* st, double gn0);

/* Warm start from the previous time step (Sec. 3.3: most contacts persist
 * from one step to the next).  prev describes the previous step's contact set:
 * its pairs (body_a, body_b, [Nc] each) and its final impulses gamma (padded,
 * prev->slots rows per contact); all device arrays owned by the caller, who
 * must copy them before the ccp_assemble that replaces the contact set.  Each
 * contact of the current set whose pair (a, b) -- with prev->plane given, and
 * the same static plane (qp_contacts.plane), so that a sphere's floor and wall
 * contacts stay apart -- is in prev takes that impulse
 * moved into its cone's interior: gamma_n = max(gamma_n, gn0), gamma_t scaled
 * to |gamma_t| <= shrink * mu * gamma_n; a new contact takes (gn0, 0, 0);
 * dummy rows 0; lambda_i = -1/f_i (centred at t = 1), t = 1.
 * QP_INVALID_ARG unless gn0 > 0, 0 < shrink <= 1, prev->slots in {3, 4}.    */
typedef struct {
  int Nc;
  int slots;
  const int* body_a;
  const int* body_b;
  const double* gamma;
  const int* plane;  /* [Nc] the previous qp_contacts.plane, or NULL: match by (a, b)
                        alone (enough without walls: a sphere has one floor contact) */
} qp_prev_contacts;
int pdip_init_warm(qp_ctx_t ctx, qp_state* st, const qp_prev_contacts* prev, double gn0, double shrink);

/* The time step around the CCP (Sec. 2.3, Eqs. force_balance_disc and
 * particle_evolution_disc), for the context's current contact set (built by
 * the last ccp_assemble from this scene) and the impulses st->gamma (padded,
 * momentum units):
 *   v' = (v + dt g) + M^-1 D gamma,  omega' = omega + I^-1 (D gamma)_torque,
 *   x' = x + dt v'   (semi-implicit Euler; spheres need no orientation).
 * pos_out, vel_out, omega_out: [3*M] SoA device arrays, written on the
 * context's stream; they may be the scene's own pos/vel/omega (each body is
 * read and written by one thread).  The contact set is left as it is:
 * ccp_assemble on the new positions builds the next step's.
 * QP_INVALID_ARG if scene->M differs from the assembled body count.         */
int ccp_advance(qp_ctx_t ctx, const qp_scene* scene, const qp_state* st, double* pos_out, double* vel_out,
                double* omega_out);


/* y = S x with S = N + blockdiag(H_c(gamma, lambda)) (Schur complement of Eq.
 * qp_Newton_system, Sec. 3.3) and identity dummy rows; st == NULL gives
 * y = N x.  N = D^T M^-1 D is applied in factored form (Eq. Ndef): body
 * gather w = M^-1 D x, then contact projection D^T w, plus the 3x3 block.
 * dtype QP_F64: x, y double[P]; QP_F32: float[P] (operator data rounded to
 * FP32).  x and y must not alias.                                           */
int newton_apply(qp_ctx_t ctx, const qp_state* st, const void* x, void* y, qp_dtype dtype);

/* Newton right-hand side and blocks at (gamma, lambda, t): rhs = -(N gamma + r)
 * + (1/t) sum_i grad f_i / f_i (padded, dummies 0).                         */
int newton_rhs(qp_ctx_t ctx, const qp_state* st, double* rhs);

/* QP_QTT_DIRECT uses X as an approximate direct solver (Sec. 3.3): each
 * refinement step applies X to the FP64 residual, dx += X (rhs - S dx), until
 * tol; it converges when the spectral radius of I - S X is below 1.  max_outer
 * caps the refinements (default 100).                                       */
typedef enum { QP_JACOBI_PCG = 0, QP_QTT_PCG = 1, QP_QTT_DIRECT = 2 } qp_precond;
typedef enum { QP_CG = 0, QP_BICGSTAB = 1 } qp_krylov;

typedef struct {
  qp_precond precond; /* Jacobi (diag S) or the QTT approximate inverse        */
  qtt_t X;            /* QP_QTT_PCG / QP_QTT_DIRECT: approximate S^-1          */
  double tol;         /* stop at ||rhs - S dx||_2 <= tol ||rhs||_2             */
  int maxit;          /* Krylov iteration cap (total inner iterations)         */
  int mixed;          /* 1: FP32 inner PCG + FP64 outer refinement             */
  double inner_tol;   /* mixed: relative tolerance of each inner solve         */
  int max_outer;      /* mixed: refinement cap                                 */
  qp_dtype core_dtype;/* QTT preconditioner core type (QP_F32 or QP_BF16)      */
  qp_krylov krylov;   /* QP_CG (preconditioned CG) or QP_BICGSTAB (the Krylov
                         method of the paper's Sec. 4.2, right-preconditioned;
                         tolerates a nonsymmetric or indefinite preconditioner)  */
} qp_solve_opts;

typedef struct {
  int status;         /* QP_OK / QP_NOT_CONVERGED / QP_BREAKDOWN / QP_TIMEOUT */
  int iters;          /* total Krylov iterations                               */
  int outer;          /* refinement steps (mixed)                              */
  double rel_res;     /* true ||rhs - S dx|| / ||rhs|| in FP64                 */
  double ms;          /* device time of the solve                              */
  int fallback;       /* 1: the QTT-preconditioned solve broke down and the
                         system was solved again with the Jacobi preconditioner */
} qp_solve_stats;

/* Solve S dx = rhs (S at st) by preconditioned CG or BiCGSTAB, run as one
 * persistent cooperative kernel (the whole Krylov loop stays on the device).
 * rhs, dx: double[P].  stats may be NULL.  A breakdown of the QTT-preconditioned
 * solve is followed by a Jacobi-preconditioned solve (stats->fallback = 1).   */
int newton_solve(qp_ctx_t ctx, const qp_state* st, const double* rhs, double* dx,
                 const qp_solve_opts* opts, qp_solve_stats* stats);

/* Batched Newton solves (many independent scenes in one launch): scene i is
 * the current contact set of ctxs[i] with state st[i] (NULL: S = N), solved
 * for rhs[i] -> dx[i] (device, P_i doubles each, not aliased).  The launch is
 * made of clusters of two thread blocks, one job per cluster: a large scene
 * runs on both blocks (hardware cluster barriers, sums through distributed
 * shared memory), small scenes run one per block with block-level
 * synchronisation only (see newton_batch_plan for the grouping).  Each
 * scene's blocks build its Schur blocks and Jacobi diagonal and run FP32
 * Jacobi-PCG to inner_tol inside FP64 iterative refinement to tol; jobs start
 * in decreasing cost.  All contexts must be on one device; the launch goes to
 * ctxs[0]'s stream after the other contexts' streams, and their later work
 * waits for it.
 * block_threads: 128, 256, 512 or 1024, or 0 to pick the fastest of 256, 512
 * and 1024 by timing this batch (the choice is kept per device, batch size
 * class and split mode).  stats[i] (may be NULL): per-scene statistics; *used
 * (may be NULL): the block size used.  Returns QP_OK when every scene
 * converged, else QP_NOT_CONVERGED or QP_BREAKDOWN (first failing scene in
 * stats); QP_INVALID_ARG for a bad block size or split mode.               */
typedef struct {
  double tol;          /* FP64 relative residual target                      */
  int maxit;           /* inner iteration cap per scene                      */
  double inner_tol;    /* FP32 inner relative tolerance (0: 1e-3)            */
  int max_outer;       /* refinement cap (0: 50)                             */
  int block_threads;   /* see above                                          */
  int split;           /* 0: split the scenes whose cost exceeds an even
                          share of the SMs; 1: one block per scene; 2: every
                          scene on two blocks                                */
  const qtt_t* precond;/* NULL: Jacobi for every scene; else n handles, one
                          per scene (NULL entries: Jacobi for that scene), a
                          QTT approximate inverse of the scene's S (or of its
                          Jacobi-scaled form, as qtt_compress makes it with a
                          state) with d = that scene's L; the FP32 inner PCG
                          applies it by one core per pass within the scene's
                          block(s) (Sec. 3.2 mat-vec); a scene whose QTT PCG
                          breaks down (a truncated inverse need not be
                          definite) finishes with Jacobi, stats.fallback = 1 */
  qp_dtype core_dtype; /* cores of the QTT preconditioners: QP_BF16, else FP32 */
  int qtt_tile;        /* tile shape of the QTT passes: 0 the measured table of
                          newton_batch_qtt_tiles; 1 one column item per thread;
                          2 two items per thread sharing the core staged in
                          shared memory where r_{k-1} r_k <= 256 and r_k <= 16 */
} qp_batch_opts;
int newton_solve_batched(int n, const qp_ctx_t* ctxs, const qp_state* const* st, const double* const* rhs,
                         double* const* dx, const qp_batch_opts* opts, qp_solve_stats* stats, int* used);

/* The measured tile shapes of the batched QTT passes for blocks of
 * block_threads (128, 256, 512 or 1024) threads on this context's device:
 * tiles_host[c] (c = 0..3 for input ranks <= 4, <= 8, <= 16, above) is 1 (one
 * column item per thread, inputs in registers) or 2 (two items per thread,
 * the core staged in shared memory), whichever a one-block probe (a d = 14
 * QTT of that interior rank, applied four times) timed faster; measured once
 * per device and block size, then cached.  The automatic tile choice of
 * newton_solve_batched (qtt_tile = 0) uses this table.                      */
int newton_batch_qtt_tiles(qp_ctx_t ctx, int block_threads, int* tiles_host /* [4] */);

/* Host only: the cluster jobs newton_solve_batched launches for scenes with
 * the given costs (cost_host[i] >= 0; the solver uses P_i + Nc_i) on num_sms
 * SMs with the given split mode.  jobs_host (2n ints) receives, per job in
 * launch order, (scene, -2) for a scene run on both blocks or (a, b) for
 * scene a on the first block and scene b on the second (b = -1: none).
 * Scenes are taken in decreasing cost; with split = 0 a scene runs on both
 * blocks when its cost exceeds total / num_sms; the others are paired with
 * their neighbour in that order.  Jobs are ordered by decreasing estimate
 * (half the cost of a split scene, the first scene's cost for a pair), ties
 * in the order made.  Needs no device.                                      */
int newton_batch_plan(int n, const long long* cost_host, int num_sms, int split, int* jobs_host, int* njobs);

typedef struct {
  double nu;          /* t = nu * 2Nc / eta                         (10)       */
  double alpha;       /* sufficient-decrease factor                 (0.01)     */
  double beta;        /* backtracking factor                        (0.5)      */
  double step_frac;   /* fraction of the max dual step              (0.99)     */
  int max_halvings;   /* backtracking cap                           (60)       */
  qp_solve_opts solve;/* Newton solve options                                  */
  int qtt_refresh;    /* 1: compress the Jacobi-scaled S~ = D^-1/2 S D^-1/2
                         (D = diag S) and invert it before the solve; the
                         preconditioner is D^-1/2 X~ D^-1/2.  The new inverse
                         is kept by the context and warm-starts the next
                         refresh (solve.X, when set, is the warm start).
                         0 with a QTT preconditioner and solve.X NULL: reuse
                         the context's last refreshed inverse (re-use across
                         Newton iterations, Sec. 3.3); QP_INVALID_ARG if
                         there is none of this size                          */
  double qtt_eps;     /* TT accuracy of the refresh                            */
  int qtt_rmax;       /* TT rank cap of the refresh                            */
} qp_pdip_opts;

typedef struct {
  int status;
  double eta;         /* surrogate duality gap at the start of the step        */
  double t;           /* barrier parameter used                                */
  double r_dual;      /* ||r_dual|| at the start of the step                   */
  double r_t;         /* ||r_t|| at the start of the step                      */
  double s;           /* accepted step length                                  */
  int halvings;
  qp_solve_stats solve;
  double ms_refresh;  /* QTT compress + invert time (device)                   */
} qp_pdip_stats;

/* One PDIP iteration (Sec. 2.4): eta, t, residuals, Schur blocks and rhs, the
 * Newton solve, dlambda recovery, ratio test, backtracking on feasibility and
 * on ||r_t||, update of (gamma, lambda) in place.  Readings of the steps the
 * paper leaves open follow Boyd and Vandenberghe, Convex Optimization 11.7.  */
int pdip_step(qp_ctx_t ctx, qp_state* st, const qp_pdip_opts* opts, qp_pdip_stats* stats);

/* Surrogate gap and dual residual norm at st (host scalars).                */
int pdip_measure(qp_ctx_t ctx, const qp_state* st, double* eta_host, double* r_dual_host);

/* The PDIP loop (Sec. 2.4; Boyd and Vandenberghe, Alg. 11.2): starting from
 * st, measure eta and ||r_dual||; while eta > gap_tol or ||r_dual|| > dual_tol
 * and fewer than max_iter steps were taken, run pdip_step.  st is updated in
 * place and holds the last iterate in every case.  A Krylov solve that stops
 * at its iteration cap (QP_NOT_CONVERGED) gives an inexact Newton step and the
 * loop goes on; any other step error ends the loop and is returned.
 * Returns QP_OK when both tolerances are met, QP_NOT_CONVERGED after max_iter
 * steps.  stats (may be NULL): the last step's statistics, with eta and r_dual
 * replaced by the final measurement; iters_host (may be NULL): steps taken.  */
int pdip_solve(qp_ctx_t ctx, qp_state* st, const qp_pdip_opts* opts, double gap_tol, double dual_tol, int max_iter,
               qp_pdip_stats* stats, int* iters_host);

/* Failure-detection self-test of the bounded grid barrier of the persistent
 * kernels (no paper counterpart): one cooperative launch (one 128-thread block
 * per SM) in which block absent_block never arrives; every other block's wait
 * expires after `budget` clock ticks and records QP_TIMEOUT, which is written
 * to *device_status (absent_block < 0: all arrive, status QP_OK).  The launch
 * always ends; the context stays usable.  QP_INVALID_ARG unless 0 < budget <=
 * the kernels' own budget (4e9 ticks) and absent_block < the SM count.       */
int qp_selftest_barrier(qp_ctx_t ctx, long long budget, int absent_block, int* device_status);

/* ---- Learned warm start (an extension; the paper has no counterpart) ---- */

/* A message-passing network over the contact graph predicts the impulses the
 * PDIP starts from.  Contacts are the nodes; a message goes from a contact to
 * each of its dynamic bodies and back: m_b = sum of h_c over the contacts of
 * body b, s_c = m_a + m_b (the static floor sends nothing).  With x_c the 8
 * scaled features of contact c (normal n in the world frame, Phi/dt, the
 * relative velocity D_c^T v in the contact frame = r_c - b_c, mu; each times
 * feat_scale[k]):
 *   h0 = relu(W0 x + b0), hl = relu(Wl [h(l-1); s(h(l-1))] + bl), l = 1..3,
 *   o = Wo h3 + bo  (o = impulse / out_scale).
 * params: device float[QP_MPNN_NPARAM], the FP32 master vector [W0 (64x8),
 * b0, W1 (64x128), b1, W2, b2, W3, b3, Wo (3x64), bo], row-major; the passes
 * use its BF16 rounding and FP32 arithmetic.  Activations live in the
 * context (valid until its next mpnn_* call).                               */
#define QP_MPNN_NPARAM 25539

/* out: device float[3*Nc], the network outputs for the current contacts.     */
int mpnn_forward(qp_ctx_t ctx, const float* params, const float* feat_scale_host, float* out);

/* Loss = mean over the 3 Nc entries of (o - target)^2 (target: device
 * float[3*Nc], impulses / out_scale); grad: device float[QP_MPNN_NPARAM]
 * (overwritten) = d loss / d params at the BF16-rounded parameters;
 * *loss_host (may be NULL) after an internal synchronisation.
 * QP_INVALID_ARG without contacts.                                           */
int mpnn_grad(qp_ctx_t ctx, const float* params, const float* feat_scale_host, const float* target, float* grad,
              double* loss_host);

/* One Adam step (Kingma and Ba, 2015) on the FP32 master parameters: m, v
 * device float[QP_MPNN_NPARAM] moment buffers (zero before step 1), step >= 1. */
int mpnn_adam(qp_ctx_t ctx, float* params, float* m, float* v, const float* grad, int step, double lr, double beta1,
              double beta2, double eps);

/* Warm start from network outputs: gamma = out_scale * o moved into the
 * cone's interior (gamma_n >= gn_min, |gamma_t| <= shrink mu gamma_n),
 * dummies 0, lambda_i = -1/f_i (centred at t = 1), t = 1.                   */
int mpnn_warm_start(qp_ctx_t ctx, qp_state* st, const float* out, double out_scale, double gn_min, double shrink);

/* ---- QTT matrices (Sec. 3.1-3.2) --------------------------------------- */

/* Core k (k = 0..d-1) of a QTT matrix is G_k(a, i, j, b), a < r_k, b <
 * r_{k+1}, stored a-major: index ((a*2 + i)*2 + j)*r_{k+1} + b, i.e. the TT
 * core (r_k, 4, r_{k+1}) with mode b_k = 2 i_k + j_k.  Row/column bit i_1 is the
 * most significant bit (Sec. 3.2 tensorisation).                            */

/* Upload cores: ranks_host[d+1] (ranks[0] = ranks[d] = 1), cores_host is the
 * concatenation of the d cores in the layout above (double).                */
int qtt_from_host(qp_ctx_t ctx, int d, const int* ranks_host, const double* cores_host, qtt_t* out);
int qtt_free(qp_ctx_t ctx, qtt_t A);
int qtt_get_dims(qtt_t A, int* d_host, long long* ncore_values_host);
int qtt_get_ranks(qtt_t A, int* ranks_host /* [d+1] */);
int qtt_copy_cores_to_host(qtt_t A, double* cores_host);

/* y = A x, contracting one core at a time (Sec. 3.2 mat-vec, O(r^2 N log N)).
 * core_dtype: QP_F64, QP_F32 or QP_BF16 (cores rounded to that type; BF16 and
 * F32 accumulate in FP32).  vec_dtype: QP_F64 (x, y double[2^d]) or QP_F32
 * (float[2^d]); QP_F64 vectors require QP_F64 cores.                        */
int qtt_apply(qp_ctx_t ctx, qtt_t A, const void* x, void* y, qp_dtype core_dtype, qp_dtype vec_dtype);

/* Which cores qtt_apply contracts on the tensor cores (tcgen05, TF32 products
 * with the FP32 vector split into a TF32 part and a remainder; F32 cores split
 * the same way).  Only FP32 vectors with BF16 or F32 cores, d >= 8, and cores
 * with r_{k-1}, r_k <= 64 qualify.  The result is good to about 1e-5 of the
 * largest entry (the CUDA-core steps: about 4e-7).  mode 0: none; 1 (the
 * default): BF16 cores with r_{k-1} r_k >= 512, where the contraction is
 * dense enough to pay and the cores' own rounding (2^-9) dominates; 2: every
 * core that qualifies, F32 cores included.  Applies to later qtt_apply calls
 * on this context; the Krylov solvers' preconditioner keeps its CUDA-core
 * step.  QP_INVALID_ARG for another mode; a tensor-core step whose wait
 * expires makes qtt_apply return QP_TIMEOUT.                                */
int qtt_set_tensor_cores(qp_ctx_t ctx, int mode);

/* TT rounding: right-to-left QR orthogonalisation then left-to-right
 * truncated SVD in FP64, keeping per split the smallest rank with discarded
 * norm <= eps ||A||_F / sqrt(d-1), capped at rmax (Sec. 3.1 truncation rule,
 * Alg. 1 accuracy split).  For eps >= 1e-7 the factorisations go through Gram
 * matrices (singular values resolved down to about 1e-8 of the largest); for
 * eps < 1e-7 through one-sided Jacobi on the cores themselves (resolved down
 * to FP64 rounding), slower at large ranks.                                 */
int qtt_round(qp_ctx_t ctx, qtt_t A, double eps, int rmax, qtt_t* out);

/* QTT compression of S (st != NULL) or of N (st == NULL) in the padded layout:
 * exact TT-SVD (Alg. 1) of the tensorised sparse matrix, swept right to left
 * over the nonzero block rows of each level, same truncation rule as above.
 * Ranks are capped at min(rmax, 128).  The SVDs go through FP64 Gram matrices,
 * which resolve singular values down to about 1e-8 of the largest one, so eps
 * below about 1e-7 does not reduce the error further (qtt_round does not have
 * this limit).                                                              */
int qtt_compress(qp_ctx_t ctx, const qp_state* st, double eps, int rmax, qtt_t* out);

/* Approximate inverse X ~ S^-1 of a QTT matrix by alternating linear-scheme
 * sweeps with rank adaptation (Sec. 3.2 "TT inversion", two-site variant),
 * warm-started from `warm` (nullable, must have the same d; Sec. 3.3 inverse
 * update).  The result is symmetrised, X <- (X + X^T)/2, and rounded.       */
int qtt_inverse(qp_ctx_t ctx, qtt_t S, double eps, int rmax, int sweeps, qtt_t warm, qtt_t* out);

/* ---- allocation-free QTT mat-vec ---------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc, for example code running inside a host application
 * that owns the device memory pool, or that must keep a fixed device footprint.
 * It needs no context and allocates nothing: the caller passes the cores, x
 * and y, and the two intermediate buffers come from a static device array of
 * 2 * QTT_NOALLOC_MAX_VALUES floats (32 MiB) that every GPU which loads this
 * library holds until the process exits.
 *
 * y = A x as qtt_apply(..., QP_F32, QP_F32) computes it: d = number of cores,
 * ranks_host[d+1] (host, ranks[0] = ranks[d] = 1), cores = device float32
 * values in the core layout above, x and y device float32 [2^d], no aliasing;
 * work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy stream) of the
 * current device.  Returns QP_INVALID_ARG when max_k(r_k) * 2^d exceeds
 * QTT_NOALLOC_MAX_VALUES (e.g. d = 17 allows ranks up to 32, d = 20 up to 4),
 * or for bad pointers/ranks.
 * The first call on a device looks up the device address of the static array
 * (once per device); make that first call before any stream capture.  Every
 * call shares the same array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it; serialise them.                  */
#define QTT_NOALLOC_MAX_VALUES (1LL << 22)
int qtt_apply_f32_noalloc(int d, const int* ranks_host, const float* cores, const float* x, float* y,
                          void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* QTTPDIP_H */
