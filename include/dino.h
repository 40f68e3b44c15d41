/*
 * dino.h -- C ABI of the many-chain surrogate (DINO) mMALA sampler for GB300.
 *
 * One transition of C independent chains of surrogate-driven mMALA with
 * surrogate-only acceptance (the surrogate stage of Algorithm 1 of Cao,
 * O'Leary-Roseberry and Ghattas, "Derivative-informed neural operator acceleration of geometric
 * MCMC for infinite-dimensional Bayesian inverse problems"), with the
 * prior-complement draw of Proposition 5.1 (Sec. 5.3) applied to every
 * proposal so that accepted chains move their full parameter field.
 *
 * Conventions for every entry point
 *   - Every call returns an int status (DINO_OK or a negative error code);
 *     nothing throws or longjmps across the ABI.
 *   - Pointers named host_* or documented as "host" are ordinary host memory.
 *     The library copies what it needs before returning and never retains a
 *     caller pointer.  Matrices are row-major float64 unless stated otherwise.
 *   - The library owns all device memory it allocates for a context
 *     (cudaMalloc on the context's device).  Results are copied into
 *     caller-owned host buffers; a NULL output pointer skips that output.
 *   - On error the call leaves the context usable and records a message that
 *     dino_last_error() returns (valid until the next call on that context).
 *   - A context is internally serialised: concurrent calls from several host
 *     threads are safe but run one at a time.
 *   - Every per-step operation runs in CUDA kernels on the context's stream;
 *     there is no CPU fallback.  If the device cannot be used, dino_init fails
 *     with DINO_ECUDA.
 *
 * Notation (reduced, whitened coordinates, Sec. 5.1):
 *   N = n_grid^2 field nodes, r reduced dimension, d_y observations,
 *   E = Psi_r^* (r x N encoder), D = Psi_r (N x r decoder), E D = I_r,
 *   f = reduced MLP R^r -> R^{d_y}, J = df/dm_r (d_y x r),
 *   Gamma = noise_var I,
 *   Phi(m_r) = |f(m_r) - y|^2 / (2 noise_var),  g = J^T (f - y) / noise_var,
 *   H = J^T J / noise_var,  L L^T = I + H (lower Cholesky, FP64),
 *   hld = (1/2) log det(I + H) = sum_j log L_jj,  s = (4 - dt)/(4 + dt).
 */
#ifndef DINO_H
#define DINO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DINO_OK          0
#define DINO_PENDING     1   /* serving: request not finished yet */
#define DINO_EINVAL     (-1) /* invalid argument (shape, range, NULL) */
#define DINO_ENOMEM     (-2) /* HBM budget or device allocation exceeded */
#define DINO_ECUDA      (-3) /* a CUDA runtime/driver call failed */
#define DINO_EBUSY      (-4) /* serving queue full */
#define DINO_ETIMEOUT   (-5) /* a bounded device or host wait ran out */
#define DINO_ENOTFOUND  (-6) /* unknown surrogate, pool or ticket id */
#define DINO_ENUMERIC   (-7) /* non-SPD input or non-finite setup data */
#define DINO_ESTATE     (-8) /* call not valid in the object's state */

/* ---- enumerations ------------------------------------------------------ */
#define DINO_ACT_IDENTITY 0
#define DINO_ACT_TANH     1
#define DINO_ACT_GELU     2   /* exact x * Phi(x) */

#define DINO_BASIS_KLE      0 /* closed-form Karhunen-Loeve basis (Sec. 4.2) */
#define DINO_BASIS_DIS      1 /* C_pr^-1-orthonormalised Gaussian vectors (DIS stand-in) */
#define DINO_BASIS_EXPLICIT 2 /* caller supplies E (r x N) and D (N x r) */

#define DINO_PREC_FP64 0      /* every step in float64 */
#define DINO_PREC_BF16 1      /* MLP/Jacobian GEMMs on tcgen05 in BF16 (FP32 accum);
                                 Gram matrices and complement projections on
                                 tcgen05 with FP32-level operands (three bf16
                                 slices); Cholesky, solves and log-acceptance
                                 FP64-accurate (double-float); field in FP32 */

/* Proposal noise map (Sec. 5.3, eq:reduced_space_sampling).  Both maps give
 * the proposal law N(mu, (1 - s^2)(I + H)^-1); a given set of normals maps to
 * different samples, so a parity check must use the map the library reports
 * (dino_surrogate_query).
 *   CHOLESKY      zeta = L^-T xi, L L^T = I + H (r normals per proposal);
 *   PERTURBATION  zeta = (I + H)^-1 (xi + K^T xi2), K = J / sigma, with d_y
 *                 further normals xi2: only the d_y x d_y matrix I + K K^T is
 *                 factored (needs d_y < r and d_y <= 192);
 *   EIGEN         zeta = (I + H)^-1/2 xi = P diag((d + 1)^-1/2) P^T xi with
 *                 H = P diag(d) P^T: the paper's eigen form, written with the
 *                 symmetric root so that it does not depend on eigenvector
 *                 signs; the d_y x d_y matrix I + K K^T is eigendecomposed
 *                 per chain (one-sided Jacobi, FP64; needs d_y < r, d_y <= 64);
 *   AUTO          PERTURBATION when it applies, else CHOLESKY. */
#define DINO_NOISE_AUTO         0
#define DINO_NOISE_CHOLESKY     1
#define DINO_NOISE_PERTURBATION 2
#define DINO_NOISE_EIGEN        3

#define DINO_FLAG_TIMING 1u   /* record per-kernel CUDA-event times */
#define DINO_FLAG_NO_DIRECT_HOST 2u /* copy host fields with cudaMemcpy even where
                                       the device reads pageable host memory */

typedef struct dino_ctx dino_ctx;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.
 * hbm_budget_bytes: cap on device memory the context may allocate
 *   (0 = 90% of the device's free memory at init).
 * stream: a cudaStream_t (as void*) to launch on, or NULL for a new
 *   non-blocking stream owned by the context.  A caller stream stays owned by
 *   the caller and must outlive the context.
 * flags: DINO_FLAG_* bits.
 * Errors: EINVAL (out == NULL), ECUDA (no usable device). */
int dino_init(dino_ctx **out, int device, size_t hbm_budget_bytes, void *stream,
              unsigned flags);

/* Wait for the stream, free every device allocation, destroy the context. */
int dino_destroy(dino_ctx *ctx);

/* Last error message of this context ("" if none); owned by the context. */
const char *dino_last_error(const dino_ctx *ctx);

/* ABI version (major*100 + minor). */
int dino_version(void);  /* 101 */

/* Block until all work issued on the context's stream has finished. */
int dino_sync(dino_ctx *ctx);

/* ---- surrogate --------------------------------------------------------- */

/* A reduced-basis neural-operator surrogate G~(m) = V f(Psi_r^* m)
 * (eq:rb_dino, Sec. 4) with its Gaussian prior and data.
 *
 * Prior: n_grid x n_grid interior nodes of the unit square, h = 1/(n_grid+1),
 *   node p = i + n_grid*j; A = prior_delta I - prior_gamma Lap_h (5-point
 *   Dirichlet stencil / h^2); C_pr = A^-2 (Assumption 2, Sec. 2.2).
 * MLP: n_layers affine layers; widths[0] = r, widths[n_layers] = d_y;
 *   W[l] is widths[l+1] x widths[l], b[l] has widths[l+1] entries; the
 *   activation acts on every hidden layer, the output layer is linear.
 * Basis: KLE (E, D built from the closed-form eigenpairs; ties in the KLE
 *   order broken by smaller kx), DIS (basis_gauss = N x r standard normals,
 *   Q = thin QR with positive diag R, D = A^-1 Q, E = Q^T A), or EXPLICIT
 *   (E r x N and D N x r given, E D = I_r required to 1e-8).
 * Data: y (d_y values) and noise_var > 0; y may be NULL and set later with
 *   dino_set_data (chains cannot be created before data is set).
 * precision: DINO_PREC_FP64 or DINO_PREC_BF16.
 * fwd_slices / jac_slices (BF16 only): number of bf16 terms that represent
 *   each operand of the MLP-forward / Jacobian GEMMs (1..3; 0 = default 3 and
 *   2).  k terms use the k(k+1)/2 leading cross products, so 2 is the
 *   "bf16x3" scheme and 3 reaches FP32-level accuracy.
 * noise_map: DINO_NOISE_* (0 = AUTO).
 * Errors: EINVAL (shapes, r > N, NULL arrays, noise_var <= 0, a noise map
 *   that does not apply), ENUMERIC (E D != I, non-finite data), ENOMEM. */
typedef struct {
  int n_grid;
  double prior_gamma, prior_delta;
  int r;
  int n_layers;
  const int *widths;
  int activation;
  const double *const *W;
  const double *const *b;
  int basis_kind;
  const double *basis_gauss;
  const double *E;
  const double *D;
  const double *y;
  double noise_var;
  int precision;
  int fwd_slices;
  int jac_slices;
  int noise_map;
} dino_surrogate_desc;

int dino_load_surrogate(dino_ctx *ctx, const dino_surrogate_desc *desc, int *surrogate_id);

/* What the library made of a loaded surrogate: sizes, precision, the noise
 * map its chains use (DINO_NOISE_CHOLESKY or DINO_NOISE_PERTURBATION),
 * whether the Gram matrices J J^T come from the tensor cores, and the bf16
 * slice counts (0 on the FP64 path).  Errors: ENOTFOUND, EINVAL (NULL). */
typedef struct {
  int N, r, d_y, n_layers, precision;
  int noise_map;
  int gram_on_tensor_cores;
  int fwd_slices, jac_slices;
  int true_model_rank;  /* r_t of an attached true map, 0 if none */
  int jac_forward;      /* 1: the Jacobian is accumulated in forward mode (r < d_y
                           and fewer flops, Sec. 4.3's min{d_y, r} rule), 0: reverse */
} dino_surrogate_info;

int dino_surrogate_query(dino_ctx *ctx, int surrogate_id, dino_surrogate_info *info);

/* Replace the data y (d_y host values) and noise variance of a surrogate.
 * Pools created later use the new data; existing pools are unaffected
 * only if they were created before (they keep a reference to the surrogate,
 * so do not change data while pools of it exist: ESTATE). */
int dino_set_data(dino_ctx *ctx, int surrogate_id, const double *y, double noise_var);

/* Free a surrogate (ESTATE while chain pools of it exist). */
int dino_unload_surrogate(dino_ctx *ctx, int surrogate_id);

/* Copy the reduced basis the library built: E (r x N) and D (N x r), host. */
int dino_read_basis(dino_ctx *ctx, int surrogate_id, double *E, double *D);

/* Evaluate the surrogate and its geometry at n reduced points m_r (n x r,
 * host) with the surrogate's precision path (Sec. 5.1; Algorithm 1):
 *   f (n x d_y), J (n x d_y x r), phi (n), g (n x r),
 *   L (n x r x r, full lower-triangular with zeros above), hld (n).
 * Any output may be NULL.  With y unset, phi and g are not defined. */
int dino_surrogate_eval(dino_ctx *ctx, int surrogate_id, int n, const double *m_r,
                        double *f, double *J, double *phi, double *g, double *L,
                        double *hld);

/* ---- chain pools ------------------------------------------------------- */

/* Create n_chains chains of surrogate `surrogate_id` with step size dt > 0
 * (s = (4 - dt)/(4 + dt), eq:mmala), each at the "Known at m_j" state of
 * Algorithm 1: m_r = Psi_r^* m0 (eq:projector, Sec. 4.1) and the surrogate
 * misfit, gradient and Gauss-Newton factor at m_r (Sec. 5.1).
 * Chain k has global id chain_id_base + k; its random numbers are
 * Philox4x32-10 with key = seed and counter = (block, step, global id,
 * stream), stream 0 = reduced noise xi, 1 = accept uniform, 2 = complement
 * prior draw, 3 = initial prior draw (step 0).  Results therefore do not
 * depend on how chains are grouped into pools.
 * m0: n_chains x N host field values, or NULL for prior draws.
 * The initial state is m_r = E m0 (FP64) and the surrogate geometry at m_r.
 * Where the device reads pageable host memory coherently (cudaDevAttr-
 * PageableMemoryAccess, e.g. Grace over NVLink-C2C) a kernel reads m0 in
 * place instead of a cudaMemcpy, unless the context has
 * DINO_FLAG_NO_DIRECT_HOST; m0 is not used after the call returns either way.
 * Errors: EINVAL, ENOTFOUND, ESTATE (data unset), ENOMEM. */
int dino_chains_create(dino_ctx *ctx, int surrogate_id, int n_chains, double dt,
                       uint64_t seed, uint64_t chain_id_base, const double *m0,
                       int *pool_id);

typedef struct {
  uint64_t proposals;   /* chain-steps performed */
  uint64_t accepts;
  uint64_t nan_rejects; /* proposals rejected because log rho was not finite */
  double sum_alpha;     /* sum over proposals of min(1, rho) (first stage) */
  uint64_t stage1_accepts; /* proposals accepted by the first (surrogate) stage;
                              equals accepts unless the surrogate has a true
                              model (delayed acceptance) */
} dino_step_stats;

/* Advance every chain of the pool by n_steps transitions.  Each transition:
 * reduced proposal m_r^dagger = mu + sqrt(1-s^2) L^-T xi with
 * mu = m_r - (1-s)(I+H)^-1 (m_r + g) (eq:reduced_space_sampling in Cholesky
 * form); surrogate geometry at m_r^dagger; log rho_r^(1) (eq:da_dino_trr_1);
 * complement draw m^dagger = s m + sqrt(1-s^2) M + D (m_r^dagger - s m_r -
 * sqrt(1-s^2) E M) with M a prior draw (Prop. 5.1); accept iff
 * log u <= min(0, log rho) (non-finite log rho rejects).
 * stats (may be NULL) receives the totals of this call (it synchronises). */
int dino_chains_step(dino_ctx *ctx, int pool_id, int n_steps, dino_step_stats *stats);

/* Advance several pools by n_steps transitions each, concurrently: every
 * pool runs on a stream of its own (up to 16, created by the context on
 * first use) after the work already issued on its stream, and its stream
 * waits for the result, so the call returns without synchronising.  The
 * results are those of dino_chains_step on each pool.  Errors: ENOTFOUND,
 * EINVAL (a pool listed twice, a serving pool). */
int dino_chains_step_many(dino_ctx *ctx, int n_pools, const int *pool_ids, int n_steps);

/* Copy the current chain positions m_j of Algorithm 1 to host buffers (any
 * may be NULL): the field m (n_chains x N, row-major), its reduced
 * coordinates m_r = Psi_r^* m (n_chains x r, eq:projector), the surrogate
 * misfit Phi(m_r) (n_chains; Sec. 5.1 with Gamma = noise_var I) and the
 * accepts per chain (n_chains).  Synchronises the pool's stream.
 * Errors: ENOTFOUND; ETIMEOUT if a bounded device wait gave up in an earlier
 * step (the pool state is then invalid and should be destroyed). */
int dino_chains_read(dino_ctx *ctx, int pool_id, double *m, double *m_r, double *phi,
                     uint64_t *accepts);

/* Copy what the last transition computed (any may be NULL): the proposal
 * m_r^dagger (n_chains x r), the proposal mean mu (n_chains x r), log rho,
 * log u and the accept flags (0/1) of each chain. */
int dino_chains_read_last(dino_ctx *ctx, int pool_id, double *b, double *mu,
                          double *log_rho, double *log_u, int *accepted);

/* Test hook: the noise of the pool's NEXT transition from the caller instead
 * of Philox, so that an independent implementation of Algorithm 1 can be
 * fed exactly the same draws (Algorithm 1 lines 1 and 6, Prop. 5.1):
 *   xi    n_chains x r   reduced normals (xi_r);
 *   xi2   n_chains x d_y observation-space normals of the perturbation map
 *                        (EINVAL on a pool with the Cholesky map);
 *   z     n_chains x N   the standard normals of the complement prior draw
 *                        M = sum_q sqrt(lambda_q) z_q eta_q (full KLE, mode
 *                        q = (kx-1) + n_grid (ky-1));
 *   log_u n_chains       the log of the accept uniform (accept iff
 *                        log_u <= min(0, log rho));
 *   log_u2 n_chains      the log of the second-stage uniform of delayed
 *                        acceptance (EINVAL without a true model).
 * Any pointer may be NULL (that stream stays Philox).  Host arrays, copied
 * before return; they apply to exactly one transition, after which every
 * stream is Philox again.  The first call allocates a device buffer of
 * n_chains (r + d_y + N + 2) doubles for the pool.
 * Errors: ENOTFOUND, EINVAL, ENOMEM. */
int dino_chains_set_noise(dino_ctx *ctx, int pool_id, const double *xi, const double *xi2,
                          const double *z, const double *log_u, const double *log_u2);

/* ---- delayed acceptance (Algorithm 1, lines 7-13) ----------------------- */

/* The true parameter-to-observable map of the second stage.  The paper's are
 * PDE solves; this library takes a stand-in of the same role that also sees
 * the field outside the surrogate's reduced basis: G(m) = f_t(E_t m), with
 * E_t an r_t x N encoder (host, row-major, r_t <= N) and f_t an MLP
 * (n_layers affine layers, widths[0] = r_t, widths[n_layers] = d_y, the
 * activation on every hidden layer).  Its data misfit uses the surrogate's
 * data: Phi(m) = |G(m) - y|^2 / (2 noise_var). */
typedef struct {
  int r_t;
  const double *E_t;
  int n_layers;
  const int *widths;
  int activation;
  const double *const *W;
  const double *const *b;
} dino_true_model_desc;

/* Attach a true map to a surrogate (desc == NULL detaches it).  Pools created
 * afterwards run the two-stage transition of Algorithm 1: the first stage
 * tests rho_r^(1) (eq:da_dino_trr_1) as before; a chain that passes draws
 * its complement (only then), evaluates Phi at the full proposal m^dagger
 * (Prop. 5.1) and moves only if log u2 <= min(0, log rho^(2)) with
 * log rho^(2) = Phi(m_j) - Phi(m^dagger) + Phi~(m_r^dagger) - Phi~(m_r,j)
 * (eq:da_dino_trr_2), u2 from its own Philox stream (5).  The chain state
 * adds E_t m and Phi(m).  Copied before return; the precision of the
 * surrogate applies (BF16: three bf16 slices per operand, FP32 accumulation).
 * Errors: ENOTFOUND, ESTATE (pools of the surrogate exist), EINVAL,
 * ENUMERIC, ENOMEM. */
int dino_set_true_model(dino_ctx *ctx, int surrogate_id, const dino_true_model_desc *desc);

/* What the last transition of a delayed-acceptance pool computed in its
 * second stage (any output may be NULL, each n_chains long): Phi(m) of the
 * current state, log rho^(2) (NaN where the first stage rejected), log u2
 * and the first-stage flags (0/1).  Errors: ENOTFOUND, ESTATE (no true model). */
int dino_chains_read_da(dino_ctx *ctx, int pool_id, double *phi_true, double *log_rho2,
                        double *log_u2, int *stage1);

/* ---- derivative-informed subspace from the surrogate ------------------- */

/* The DIS eigenproblem (eq:jtj_eigenvalue) restricted to the span of the
 * surrogate's basis, with the Monte Carlo estimate of the expected ppGNH
 * (eq:mc_ppgnh): at n_samples encoded prior draws m_r,i ~ N(0, I_r) (Philox
 * stream 6, step 0, chain i; Lemma of Sec. 5.3) the surrogate's Jacobians give
 *   H_mc = (1/n) sum_i J(m_r,i)^T J(m_r,i) / noise_var   (r x r),
 * eigendecomposed on the device (one-sided Jacobi) as P diag(lambda) P^T with
 * lambda decreasing.  Outputs (host, any may be NULL): eigvals (r), P (r x
 * r_new, the leading eigenvectors, signs arbitrary), E_new = P^T E (r_new x N)
 * and D_new = D P (N x r_new), a C_pr^-1-orthonormal basis with
 * E_new D_new = I.  A surrogate on the new basis takes the first-layer
 * weights W_1 P (coordinates outside the r_new leading directions set to 0).
 * Errors: ENOTFOUND, EINVAL (n_samples < 1, r_new outside 1..r), ENOMEM. */
int dino_dis_from_surrogate(dino_ctx *ctx, int surrogate_id, int n_samples, uint64_t seed,
                            int r_new, double *eigvals, double *P, double *E_new, double *D_new);

/* ---- chain diagnostics (Sec. 6.2) ---------------------------------------- */

/* A device trajectory of n_chains chains x n_dof degrees of freedom (at most
 * max_samples samples), and the diagnostics the paper uses to assess a pool
 * of chains, computed on the device from it:
 *   ESS% per degree of freedom (eq:ess): 1 / (1 + 2 sum_{t=1}^{2n'+1} MACT(t)),
 *     MACT(t) = 1 - (w - mean_k AC(t, k)) / v with w, v the 1D covariance
 *     estimators and AC(t, k) the lag-t autocovariance of chain k; n' ends the
 *     initial positive sequence (MACT(0) = 1, pairs MACT(2i) + MACT(2i+1) > 0);
 *     returned as a fraction;
 *   the Wasserstein MPSRF Tr(W + V - 2 (W^1/2 V W^1/2)^1/2) of the within-
 *     chain and pooled covariance estimators (eq:covariance_estimator), with
 *     the symmetric square roots from a one-sided Jacobi eigensolver
 *     (n_dof <= 1024);
 *   the mean squared jump MSJ = 1/(n_s - 1) sum_j |x_{j+1} - x_j|^2, averaged
 *     over chains (the acceptance rate comes with dino_chains_step's stats).
 * The trajectory takes n_dof n_chains max_samples doubles of device memory. */
#define DINO_DIAG_REDUCED 0   /* record m_r (n_dof = r) */
#define DINO_DIAG_FIELD   1   /* record the field m (n_dof = N) */

typedef struct {
  int n_samples;
  double ess_median;     /* median over degrees of freedom of ESS% (fraction) */
  double msj;
  double mpsrf_w;        /* NaN unless requested */
  double trace_w, trace_v;
  int jacobi_sweeps;     /* sweeps of the last eigensolve */
} dino_diag_result;

/* Errors: EINVAL (n_chains < 2 or > 6144, n_dof < 1, max_samples < 2), ENOMEM. */
int dino_diag_create(dino_ctx *ctx, int n_chains, int n_dof, int max_samples, int *diag_id);
/* Append the current state of chains chain0 .. chain0 + n_chains - 1 of a
 * pool (what = DINO_DIAG_REDUCED or DINO_DIAG_FIELD), after the work already
 * issued on the pool's stream.  Errors: ENOTFOUND, EINVAL (shape), ENOMEM (full). */
int dino_diag_record(dino_ctx *ctx, int diag_id, int pool_id, int what, int chain0);
/* Append a caller sample (host, n_chains x n_dof, row-major). */
int dino_diag_push(dino_ctx *ctx, int diag_id, const double *sample);
/* Compute the diagnostics of the samples recorded so far; ess (host, n_dof)
 * and result may be NULL.  Errors: ENOTFOUND, ESTATE (< 2 samples), EINVAL. */
int dino_diag_compute(dino_ctx *ctx, int diag_id, int want_mpsrf, double *ess,
                      dino_diag_result *result);
int dino_diag_destroy(dino_ctx *ctx, int diag_id);

/* Free a chain pool's device memory (after its stream has drained); the
 * pool id is invalid afterwards.  Errors: ENOTFOUND. */
int dino_chains_destroy(dino_ctx *ctx, int pool_id);

/* ---- serving: continuous batching of chain ensembles -------------------- */

/* A request: n_chains chains of a loaded surrogate advanced n_steps
 * transitions, exactly as dino_chains_create + dino_chains_step would (same
 * random numbers for the same seed and chain ids), with the results copied
 * into caller buffers when it finishes.  m0 (n_chains x N, host, may be NULL
 * for prior draws) is copied at submit.  The output buffers (any may be NULL)
 * must stay valid until dino_serve_poll returns DINO_OK for the ticket:
 * m_r_out n_chains x r, phi_out n_chains, accepts_out n_chains,
 * m_out n_chains x N. */
typedef struct {
  int surrogate_id;
  int n_chains;
  int n_steps;
  double dt;
  uint64_t seed;
  uint64_t chain_id_base;
  const double *m0;
  double *m_r_out;
  double *phi_out;
  uint64_t *accepts_out;
  double *m_out;
} dino_request;

typedef struct {
  dino_step_stats stats;
  double queue_s;    /* submit -> admitted (device memory reserved) */
  double latency_s;  /* submit -> results in the caller's buffers */
} dino_result;

/* Optional, before the first submit: number of CUDA streams requests are
 * spread over (1..32, default 4), transitions issued per scheduling round
 * (default 8) and the most requests resident at once (default 32).
 * ESTATE once serving has started. */
int dino_serve_config(dino_ctx *ctx, int n_streams, int steps_per_round, int max_active);

/* Queue a request; returns immediately with a ticket.  A background thread
 * admits queued requests as soon as their device footprint (the pool's
 * arena) fits in the HBM budget, so requests arriving while others run are
 * batched with them, each on its own stream.  Among the requests that fit,
 * the one with the least estimated work (chains x steps x per-proposal cost)
 * goes first; a request that has waited longer than 20 s goes before all
 * others, in arrival order, and is not passed over while it does not fit.
 * Of the resident requests, as many as there are streams progress at a time:
 * those with the least remaining work (shortest remaining work first).
 * Errors: ENOTFOUND (surrogate), ESTATE (no data), EINVAL, EBUSY (queue full),
 * ENOMEM (the request alone exceeds the whole budget). */
int dino_serve_submit(dino_ctx *ctx, const dino_request *req, uint64_t *ticket);

/* DINO_PENDING while queued or running; DINO_OK once the outputs are in the
 * caller's buffers (res, may be NULL, gets stats and timings); the request's
 * error code if it failed; ENOTFOUND for an unknown ticket.  Never blocks
 * beyond the context lock. */
int dino_serve_poll(dino_ctx *ctx, uint64_t ticket, dino_result *res);

/* Poll until done or timeout_s seconds have passed (then ETIMEOUT). */
int dino_serve_wait(dino_ctx *ctx, uint64_t ticket, double timeout_s, dino_result *res);

/* Queue length, resident requests, the most resident at once, and device
 * memory in use now and at peak since serving started. */
int dino_serve_status(dino_ctx *ctx, int *queued, int *active, int *peak_active,
                      size_t *hbm_used, size_t *peak_hbm_used);

/* ---- instrumentation --------------------------------------------------- */

/* Measured FP32 fused-multiply-add throughput of the context's device in
 * TFLOP/s (2 flops per FMA; independent FMA chains on every SM, best of three
 * timed launches).  The denominator of the double-float kernels' roofline. */
int dino_measure_fp32_peak(dino_ctx *ctx, double *tflops);

/* Number of kernels this context has launched since creation. */
uint64_t dino_launch_count(const dino_ctx *ctx);

/* Per-kernel CUDA-event timing collected under DINO_FLAG_TIMING.
 * Writes up to `cap` entries: name (NUL-terminated, 48 bytes each in
 * `names`), total milliseconds and launch count.  Returns the number of
 * entries through *n.  reset != 0 clears the accumulators afterwards. */
int dino_kernel_times(dino_ctx *ctx, char *names, double *total_ms, uint64_t *launches,
                      int cap, int *n, int reset);

/* ---- allocation-free evaluation ---------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers of the
 * library rather than the method.
 *
 * Surrogate forward pass f(x) and reduced Jacobian J = df/dx (reverse mode,
 * FP64) at n reduced points, computed without allocating any device memory.
 * It is meant for host code that must not call cudaMalloc: for example a
 * plugin inside a framework that owns every device byte through its own
 * pool, or a latency-critical loop in which the synchronisation that
 * cudaMalloc/cudaFree can imply is not acceptable.  The intermediate
 * d_y x width products live in a fixed device array of
 * DINO_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB) that every GPU loading the
 * library keeps until the process exits.
 *
 * widths: host array of n_layers + 1 entries (widths[0] = r, widths[n_layers]
 *   = d_y), 1 <= n_layers <= 16; activation as in dino_surrogate_desc.
 * W, b: host arrays of n_layers DEVICE pointers; W[l] is widths[l+1] x
 *   widths[l] row-major, b[l] has widths[l+1] entries.
 * x: device, n x r; f: device, n x d_y; J: device, n x d_y x r (row-major).
 *   All buffers belong to the caller; results are written before the kernel
 *   ends on `stream` (a cudaStream_t, or NULL for the legacy default stream).
 * Limit: n * 2 * d_y * (largest hidden width) must not exceed
 *   DINO_NOALLOC_SCRATCH_DOUBLES, and the activations must fit in 200 KB of
 *   shared memory; larger requests are rejected with DINO_ENOMEM (scratch)
 *   or DINO_EINVAL (shared memory, NULL pointers, bad sizes) and nothing runs.
 * The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current, so make that first call
 *   before any stream capture on the device.
 * Every call shares the one array: calls whose kernels can overlap on the GPU
 *   (unordered streams) race on it, so order them on one stream.
 * Returns DINO_OK once the kernel is queued, DINO_ECUDA if the launch fails. */
#define DINO_NOALLOC_SCRATCH_DOUBLES (1u << 20)

int dino_surrogate_jacobian_noalloc(int n, int n_layers, const int *widths, int activation,
                                    const double *const *W, const double *const *b,
                                    const double *x, double *f, double *J, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DINO_H */
