/*
 * pd.h -- C ABI of libpd, a GB300 (sm_103a) implementation of the hot path
 * of polynomial-diagram fitting from "Polynomial diagrams for microstructure
 * modelling" (Bourne, Buze, Gallouet, Merigot).
 *
 * Notation follows the paper:
 *   Omega      the pixel (or voxel) set, |Omega| = P points in [-1,1]^dim;
 *   G          the grain map Omega -> {0..N-1} (0-based here; 1-based in
 *              the paper), given as int32 labels[P];
 *   eta(x)     the tensor-product Legendre design function of degree d
 *              (Sec. 3.3), K = K_d entries;
 *   theta      the parameters, theta[N][K] row-major (grain-major), double;
 *   h_i(x)     = theta_i . eta(x); the diagram is F(x) = argmin_i h_i(x);
 *   Phi        the objective Phi_eps^G of eq. (Phi), always <= 0, which the
 *              fit maximises.
 *
 * Layout conventions
 *   Pixels of a structured grid of extents n[0] x n[1] (x n[2]) have centres
 *   x_a = -1 + (2 k_a + 1) / n[a] (Sec. 2.1 with n = 2M, each axis scaled to
 *   [-1,1] on its own) and linear index j = k_0 + n[0] (k_1 + n[1] k_2).
 *   The multi-indices alpha of A_d are ordered by ascending total degree,
 *   then descending alpha_1, then descending alpha_2 (the paper fixes "an
 *   ordering" without choosing one, Sec. 3.1).  Entries 0..dim of every
 *   theta_i are therefore the constant and the linear terms.
 *
 * Ownership and execution
 *   The caller owns every buffer.  Pointers documented "device" must be
 *   device memory of the current CUDA device; "host" pointers host memory.
 *   Entry points taking a stream enqueue their work on that stream
 *   (a cudaStream_t passed as void*; NULL = the legacy default stream) and
 *   return without synchronising, except where documented "synchronous".
 *   Scratch memory is drawn from the device's stream-ordered memory pool on
 *   the given stream and returned to it on the same stream before the call
 *   returns, so calls on different streams never share scratch.
 *
 * Errors
 *   Every entry point returns PD_OK (0) or a negative PD_E* code and never
 *   aborts or exits.  Arguments are checked on the host before anything is
 *   enqueued; an error return means nothing was enqueued.  Asynchronous
 *   device errors surface at the caller's next synchronisation, as for any
 *   CUDA call.
 */
#ifndef PD_H_
#define PD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PD_OK 0
#define PD_EINVAL (-1)   /* bad argument: N<2, eps<=0, bad dim/d, NULL, P   */
#define PD_ELABEL (-2)   /* a label outside 0..N-1 (checked where stated)    */
#define PD_ENAN (-3)     /* a non-finite objective or parameter was met      */
#define PD_ENOMEM (-4)   /* scratch allocation failed                        */
#define PD_ECUDA (-5)    /* a CUDA runtime call or kernel launch failed      */
#define PD_ETIMEOUT (-6) /* a bounded device wait gave up                    */
#define PD_ENOTSUP (-7)  /* valid but unsupported combination (e.g. degree)  */
#define PD_ESCRATCH (-8) /* needs more scratch than the fixed array of
                            pd_objective_grad_noalloc holds               */

/* ---- precisions of an evaluation --------------------------------------- */
#define PD_FP64 0  /* all arithmetic in double                              */
#define PD_FP32 1  /* logits, exp and per-tile sums in float; log-sum-exp in
                      float; cross-tile and final reductions in double       */
#define PD_BF16 2  /* logits and gradient contraction on tcgen05 tensor cores
                      with bf16 operands and fp32 accumulation; float
                      log-sum-exp; double final reduction                    */
#define PD_BF16X3 3 /* as PD_BF16 with every operand split into three bf16
                      terms (hi+mid+lo), which recovers float-level accuracy
                      on the tensor cores                                     */
/* The tensor-core precisions serve the objective, the gradient and the
 * Hessian-vector product for K <= 32 (2-D d <= 6, 3-D d <= 3) and grid
 * sides <= 2^23; other combinations return PD_ENOTSUP.  The log-sum-exp
 * pass keeps the grains' parameters resident in one SM's shared memory
 * (about 112 bytes a grain at K <= 16 in PD_BF16X3, up to 1536
 * grains); more grains are processed in groups whose partial sums are
 * merged, with a scratch buffer of 8 bytes per pixel and group.  Besides
 * log S per pixel, the scratch holds one float per (128-pixel tile,
 * grain) of centre logits (4 N / 128 bytes per pixel).  Internally the
 * grains are reordered by the Morton code of their label centroids and
 * the passes leave out the (tile, grain block) pairs whose contributions
 * round to zero (underflowing exponentials; probabilities below 2^-26,
 * 2^-32 for the HVP, which the fp16 gradient operand rounds to zero);
 * results are in the caller's grain order.  Setting PD_TC_NO_SKIP=1 in
 * the environment visits every pair in the caller's order.             */

/* ---- supported sizes --------------------------------------------------- */
#define PD_MAX_DEGREE_2D 7
#define PD_MAX_DEGREE_3D 4

/* Pixel set Omega (Sec. 2.1).  coords == NULL: structured grid n[0..dim-1]
 * with P = n[0]*n[1](*n[2]).  coords != NULL: an explicit device point list
 * [P][dim] of doubles in [-1,1]^dim (the paper's "any finite set of sample
 * points"); n is then ignored.  The tensor-core precisions take 128
 * consecutive points as one tile and split each logit at the tile's first
 * point, so their accuracy needs a list ordered along space (e.g. a
 * z-curve order); Phi and its gradient do not depend on the order. */
typedef struct pd_grid {
  int dim;              /* 2 or 3 */
  int64_t n[3];
  const double* coords; /* device, or NULL */
  int64_t P;
} pd_grid;

/* Options of one evaluation. */
typedef struct pd_eval_opts {
  int d;       /* polynomial degree, 1..PD_MAX_DEGREE_{2D,3D}            */
  double eps;  /* regularisation eps > 0 of eq. (p-e)                     */
  int prec;    /* PD_FP64, PD_FP32, PD_BF16, PD_BF16X3                     */
} pd_eval_opts;

/* K_d = |A_d| for dimension dim (Sec. 3.1: (d+1)(d+2)/2 in 2-D; the 3-D
 * tensor product gives (d+1)(d+2)(d+3)/6).  Returns -1 for bad arguments. */
int pd_K(int dim, int d);

/* Writes the exponents of A_d in library order to alpha_out (host,
 * [K][dim] ints).  Returns K, or a negative code. */
int pd_alpha(int dim, int d, int* alpha_out);

/* Human-readable text of a status code (static storage). */
const char* pd_strerror(int code);

/* Design matrix eta(Omega) (Sec. 3.3, eq. h-degree-d-legendre): writes
 * eta_out[j][k] = psi_{alpha_k}(x_j), pixel-major, as double (prec ==
 * PD_FP64) or float (PD_FP32).  eta_out: device, P*K elements.  Used to
 * check the in-register features of the other kernels; those never write
 * eta to memory.  P == 0 is a no-op. */
int pd_features(const pd_grid* grid, int d, int prec, void* eta_out,
                void* stream);

/* Objective and gradient, one fused evaluation (eqs. Phi and grad):
 *   Phi       = (1/P) sum_x log p_{G(x)}(x),
 *   grad_i    = -(1/(eps P)) sum_x (delta_{i G(x)} - p_i(x)) eta(x),
 * with p_i(x) = exp(-h_i(x)/eps) / sum_j exp(-h_j(x)/eps) (eq. p-e).
 * labels: device int32[P], each in 0..N-1 (not checked here; see
 * pd_check_labels).  theta: device double[N][K].  obj_out: device double
 * scalar.  grad_out: device double[N][K], or NULL to skip the gradient.
 * Results are bitwise reproducible run to run (fixed-order reductions). */
int pd_objective_grad(const pd_grid* grid, const int32_t* labels, int N,
                      const double* theta, const pd_eval_opts* opts,
                      double* obj_out, double* grad_out, void* stream);

/* Hessian-vector product from eq. (hess):
 *   (H v)_i = -(1/(eps^2 P)) sum_x p_i(x) (u_i(x) - sum_k p_k(x) u_k(x)) eta(x),
 * u_i(x) = v_i . eta(x).  v, hv_out: device double[N][K].  labels do not
 * enter the Hessian (the call keeps the shape of pd_objective_grad); they
 * may be NULL (the tensor-core precisions take them as a hint for the
 * grain order of their pair skipping).  u_i - ubar of the grain that holds
 * nearly all of a pixel's probability is a small difference of two large
 * terms: PD_FP32 forms it from sums that leave each pixel's arg-max grain
 * out, so that it keeps its relative accuracy where p is close to 1; the
 * tensor-core precisions form the plain difference, whose error is about
 * 2^-24 |u| at such pixels (negligible beside the grain boundaries'
 * terms, except on maps where nearly every pixel has p within 1e-4 of 1).
 * prec: any;
 * the tensor-core precisions scale v by a power of two internally (their
 * fp16 operands need |v| <= 1) and undo it exactly. */
int pd_hvp(const pd_grid* grid, const int32_t* labels, int N,
           const double* theta, const double* v, const pd_eval_opts* opts,
           double* hv_out, void* stream);

/* ---- plans: repeated evaluations on one pixel set and label map -------- */
/* The ascent of Sec. 5.2 evaluates Phi, its gradient and Hessian-vector
 * products hundreds of times on the same pixel set Omega and the same label
 * map G, only theta (and eps, when annealed) changing.  A plan does the
 * parts that depend on Omega and G alone once: it sizes and allocates all
 * scratch of an evaluation up front (one device allocation), and its first
 * evaluation leaves in that scratch the Legendre features of every tile
 * centre (Omega only) and, for the tensor-core precisions, the grain order
 * (Morton order of the label centroids, G only), which later evaluations
 * reuse.  Plan evaluations take no scratch allocation and return results
 * bitwise equal to pd_objective_grad / pd_hvp with the same arguments.
 * Calls that repeat the previous call's arguments (theta, v and output
 * pointers, eps), as the evaluations of a fit do, replay a CUDA graph of
 * the evaluation recorded on the second such call (kept until
 * pd_plan_destroy); tracing (pd_prof_enable) runs every call directly.
 *
 * pd_plan_create: grid, labels, N, d and prec as for pd_objective_grad
 * (N >= 2, P >= 1); flags = 0, or PD_PLAN_HVP to also reserve the scratch of
 * pd_plan_hvp.  The plan keeps a copy of *grid and the pointers grid->coords
 * and labels (device, borrowed): both must stay allocated and unchanged
 * until pd_plan_destroy.  Allocates with cudaMalloc on the current device
 * (PD_ENOMEM when that fails) and writes the handle to *plan_out (host);
 * on failure *plan_out is NULL and nothing is held.
 * pd_plan_objective_grad / pd_plan_hvp: theta (and v) device double[N][K],
 * eps > 0 finite; outputs as for pd_objective_grad (obj_out or grad_out may
 * be NULL, not both) and pd_hvp; pd_plan_hvp on a plan created without
 * PD_PLAN_HVP returns PD_EINVAL.  Calls on one plan share its scratch: they
 * must not overlap on the GPU (one stream, or ordered by the caller) and
 * must not run from several host threads at once.  Calls on different
 * plans are independent.
 * pd_plan_scratch_bytes: the device bytes the plan holds (host *bytes_out).
 * pd_plan_destroy: frees the plan (cudaFree, which waits for the device);
 * NULL is a no-op. */
typedef struct pd_plan pd_plan;
#define PD_PLAN_HVP 1
int pd_plan_create(const pd_grid* grid, const int32_t* labels, int N, int d,
                   int prec, int flags, pd_plan** plan_out);
int pd_plan_objective_grad(pd_plan* plan, const double* theta, double eps,
                           double* obj_out, double* grad_out, void* stream);
int pd_plan_hvp(pd_plan* plan, const double* theta, const double* v,
                double eps, double* hv_out, void* stream);
int pd_plan_scratch_bytes(const pd_plan* plan, size_t* bytes_out);
void pd_plan_destroy(pd_plan* plan);

/* Arg-min assignment F_theta (Sec. 2.1, eq. Li_def), computed in double:
 * labels_out[j] = the smallest i attaining min_i theta_i . eta(x_j).
 * gap_out (device double[P] or NULL): second-smallest minus smallest h.
 * ref_labels (device int32[P] or NULL) with mismatch_out (device int64
 * scalar): the number of pixels with labels_out != ref_labels, i.e.
 * Err^G * P (Sec. 4); mismatch_out is overwritten, not accumulated.
 * P == 0 writes 0 to mismatch_out (if given; ref_labels may then be NULL)
 * and returns. */
int pd_assign(const pd_grid* grid, int N, int d, const double* theta,
              int32_t* labels_out, double* gap_out, const int32_t* ref_labels,
              int64_t* mismatch_out, void* stream);

/* Grain moments for the initialisations of Sec. 5.5.2: counts_out[i] =
 * |G_i| and mom_out[i][k] = sum_{x in G_i} psi_{alpha_k}(x) for the
 * Legendre multi-indices of degree <= dm (1..4).  Accumulated exactly in
 * 64-bit fixed point (resolution 2^-36 per term), so the result is
 * independent of thread order.  mom_out: device double[N][K_dm];
 * counts_out: device int64[N].  Labels must be in range. */
int pd_moments(const pd_grid* grid, const int32_t* labels, int N, int dm,
               double* mom_out, int64_t* counts_out, void* stream);

/* Synchronous: returns PD_ELABEL if any label is outside 0..N-1, else PD_OK. */
int pd_check_labels(const pd_grid* grid, const int32_t* labels, int N,
                    void* stream);

/* Host helper (Sec. 2.3): parameters of an (anisotropic) power diagram,
 * cost |x - y_i|^2_{A_i} - w_i, as Legendre coefficients of degree d.
 * y: host double[N][dim]; w: host double[N]; A: host double[N][dim][dim]
 * symmetric, or NULL for a power diagram (A_i = Id; the quadratic term,
 * common to all grains, is then dropped, so d = 1 suffices).
 * theta_out: host double[N][K_d], higher-degree terms zero. */
int pd_theta_from_apd(int dim, int d, int N, const double* y, const double* w,
                      const double* A, double* theta_out);

/* Host helper (Sec. 2.3, eqs. pd-lr-to-phys and apd-lr-to-phys; Sec. 5.5.3):
 * the physical parameters of fitted Legendre coefficients of degree d = 1
 * (power diagram: seeds y and weights w) or d = 2 (anisotropic power
 * diagram: y, w and metrics A).  theta: host double[N][K_d], in any gauge.
 * The coefficients are written in monomials, then for d = 2 every metric is
 * shifted by the same lambda Id, lambda = max(0, margin - min_i
 * lambda_min(A_i)) -- a common shift of all theta_i, which changes no cell
 * (Lemma 4.2) -- so that every A_i has eigenvalues >= margin > 0, and
 * y_i = -A_i^-1 b_i / 2, w_i = b_i . A_i^-1 b_i / 4 - theta_i,1 (b_i the
 * linear coefficients).  For d = 1, y_i = -b_i / 2, w_i = |b_i|^2 / 4 -
 * theta_i,1 (margin and A unused; the |x|^2 term common to a power diagram
 * is not represented).  Outputs (host): y [N][dim], w [N], A [N][dim][dim]
 * (d = 2), *lambda_out (may be NULL).  PD_ENOTSUP for other degrees,
 * PD_EINVAL for a non-positive margin (d = 2) or NULL pointers, PD_ENAN for
 * non-finite coefficients. */
int pd_theta_to_apd(int dim, int d, int N, const double* theta, double margin, double* y, double* w, double* A,
                    double* lambda_out);

/* Synchronous: the moment heuristic of Sec. 5.5.2 (eqs. centroid-guess to
 * w-guess) as Legendre coefficients of degree d: centroids y', central
 * second moments B' (normalised by |G_i|), A' = B'^-1 (identity for d = 1,
 * for empty grains and for singular B'), w' = sqrt(det A') |G_i| / (P pi)
 * (3-D: / (P 4pi/3)).  theta_out: device double[N][K]. */
int pd_heuristic_init(const pd_grid* grid, const int32_t* labels, int N,
                      int d, double* theta_out, void* stream);

/* ---- the ascent scheme (Sec. 5.2) --------------------------------------- */
#define PD_INIT_GIVEN 0     /* start from theta_io as passed               */
#define PD_INIT_ZERO 1      /* theta = 0, the fully ambiguous state         */
#define PD_INIT_HEURISTIC 2 /* the moment heuristic (pd_heuristic_init)     */

#define PD_METHOD_LBFGS 0     /* L-BFGS, strong-Wolfe line search           */
#define PD_METHOD_NEWTON_CG 1 /* truncated Newton with pd_hvp products      */

typedef struct pd_fit_opts {
  int d;              /* degree                                            */
  double eps;         /* regularisation                                    */
  int init;           /* PD_INIT_*                                         */
  int method;         /* PD_METHOD_*                                       */
  int max_iter;       /* iteration budget of the first phase               */
  int lbfgs_m;        /* L-BFGS memory (10)                                */
  int max_cg;         /* Newton-CG inner iterations (50)                   */
  int prec;           /* precision of the first phase (PD_FP64 ...)        */
  int refine_iter;    /* FP64 iterations after the first phase (0: none)   */
  double gtol;        /* stop a phase when ||grad Phi||_2 <= gtol          */
  double target_phi;  /* stop when Phi >= target_phi (-inf: never); with
                         refine_iter > 0 a target met in a reduced-
                         precision phase must hold in FP64, else the FP64
                         phase continues                                  */
  double switch_rtol; /* leave the first phase when the relative Phi gain
                         of an iteration is below this (0: never)          */
  /* Annealing of eps (Secs. 5.2 and 5.5.4 leave the schedule to future
   * work; this is the library's reading).  With anneal_eps0 > eps the fit
   * runs in stages at eps_k = max(eps, anneal_eps0 * anneal_factor^k),
   * k = 0, 1, ...: every stage above eps runs the first phase for
   * anneal_iter iterations (no refinement, no target) from the parameters
   * the previous stage ended with -- the same diagram, made sharper by the
   * smaller eps (Lemma 4.1) --, and the stage at eps runs the phases as
   * configured above.  With err_stop != 0 the schedule ends after a stage
   * above eps once the hard assignment reconstructs G: when
   * Phi > -log 2 / |Omega| (evaluated in FP64), which certifies Err^G = 0
   * (Cor. 4.10), or else when the double-precision assignment finds no
   * mismatch (report->status 5).  anneal_eps0 <= eps: no annealing. */
  double anneal_eps0;
  double anneal_factor; /* in (0, 1)                                        */
  int anneal_iter;      /* iterations of each stage above eps (>= 1)        */
  int err_stop;         /* stop the schedule once Err^G = 0                 */
} pd_fit_opts;

typedef struct pd_fit_report {
  double phi;         /* final Phi (evaluated in FP64)                     */
  double gnorm;       /* final ||grad Phi||_2 over the free blocks (from
                         the last evaluation with a gradient: a target met in
                         reduced precision is confirmed by the FP64 objective
                         alone)                                              */
  double err;         /* final Err^G (Sec. 4)                              */
  int iters;          /* iterations of both phases                         */
  int iters_phase1;   /* iterations of the first phase                     */
  int64_t evals;      /* objective+gradient evaluations                    */
  int64_t hvps;       /* Hessian-vector products                           */
  int status;         /* 0 budget, 1 gtol, 2 line search stalled, 3 target,
                         5 annealing stopped with Err^G = 0                */
  double seconds;     /* wall time of the call                             */
  double eps_final;   /* eps of the last stage (eps without annealing)     */
  int stages;         /* annealing stages run (1 without annealing)        */
} pd_fit_report;

/* Synchronous: maximise Phi over theta with the gauge theta_{N-1} = 0
 * (Remark 4.3) by the selected method; an optional FP64 refinement phase
 * follows a reduced-precision phase.  theta_io: device double[N][K] (read
 * when init == PD_INIT_GIVEN; always written, gauge-fixed).  report: host.
 * Labels are checked (PD_ELABEL).  Returns PD_OK, or an error code (the
 * report then holds the state reached). */
int pd_fit(const pd_grid* grid, const int32_t* labels, int N,
           const pd_fit_opts* opts, double* theta_io, pd_fit_report* report,
           void* stream);

/* ---- batched evaluation and fitting of many grain maps ----------------- */
/* One grain map of a batch (2-D pixel sets).  Pointers are device pointers
 * owned by the caller and must stay valid while a batch built on them is
 * used.  theta, obj_out and grad_out are read/written by pd_batch_eval;
 * pd_fit_batched ignores them (it uses theta_io).  target_phi is read by
 * pd_fit_batched only: this map's objective target (as pd_fit_opts'
 * target_phi), or NaN to take opts->target_phi. */
typedef struct pd_map {
  pd_grid grid;
  const int32_t* labels; /* [P], each in 0..N-1 */
  int N;
  const double* theta;   /* [N][K] */
  double* obj_out;       /* scalar Phi of this map */
  double* grad_out;      /* [N][K] grad Phi, or NULL */
  double target_phi;     /* pd_fit_batched: per-map target, or NaN */
} pd_map;

typedef struct pd_batch pd_batch;

/* Synchronous: builds a plan that evaluates eq. (Phi) and eq. (grad) of all
 * maps (same degree, eps and precision).
 * PD_FP64 / PD_FP32: one persistent launch per pass, every pass working
 * through a list of (map, pixel block) and (map, pixel chunk, grain tile)
 * items, heaviest maps first; the whole evaluation is captured once as a
 * CUDA graph.  With autotune != 0 the pass-2 chunking and the persistent
 * grid size are chosen by timing five candidates on the first plan of a
 * (degree, precision, batch size, total work) class; the choice is cached
 * for the process.
 * PD_BF16 / PD_BF16X3: every map gets the plan of a single-map evaluation
 * (see pd_plan_create; the first evaluation, run here at theta = 0 into the
 * plan's own buffers, leaves its centre features and grain order), and the
 * evaluations of all maps are captured as one CUDA graph in which the maps
 * run on parallel chains (each map, heaviest first, on the chain with the
 * least pixels x grains so far).  With autotune != 0 the number of chains
 * (1, 2, 4 or 8) is chosen by timing the graph at theta = 0, else 4.  A
 * map's results are bitwise those of pd_objective_grad on that map.
 * The plan owns its scratch (allocated here, freed by pd_batch_destroy).
 * PD_EINVAL for an invalid precision; PD_ENOTSUP for a degree the
 * precision does not support. */
int pd_batch_create(int n_maps, const pd_map* maps, const pd_eval_opts* opts,
                    int autotune, pd_batch** out);
/* Enqueues one replay of the plan's graph on the stream: every active map's
 * Phi and gradient from its current theta.  Replays on one plan must not
 * overlap (they share the plan's scratch).  On the tensor cores, while some
 * map is inactive, the active maps' evaluations are launched directly on
 * the same chains instead of the graph. */
int pd_batch_eval(pd_batch* batch, void* stream);
/* Which maps the next replays evaluate: active[m] != 0 (host int32[n_maps];
 * CUDA cores: copied asynchronously on the stream; tensor cores: read
 * before the call returns).  All maps are active initially. */
int pd_batch_set_active(pd_batch* batch, const int32_t* active, void* stream);
/* The tuning choice of the plan (CUDA cores: chunk factor and occupancy
 * divisor; tensor cores: the number of chains in *chunk_factor, 0 in
 * *occ_div) and the measured milliseconds per replay (0 without tuning). */
int pd_batch_info(const pd_batch* batch, int* chunk_factor, int* occ_div,
                  double* tuned_ms);
/* Synchronises the device and frees the plan. */
void pd_batch_destroy(pd_batch* batch);

/* Synchronous: the ascent scheme of pd_fit (L-BFGS only; a first phase in
 * any precision with optional FP64 refinement; init PD_INIT_ZERO or
 * PD_INIT_GIVEN, e.g. a learned warm start; eps-annealing as in pd_fit, but
 * no Err-aligned stopping: err_stop != 0 is PD_ENOTSUP) for every map at
 * once.  Each map runs its own optimiser
 * on a host thread; their objective/gradient requests are served together,
 * one graph replay per round for all maps that are waiting.  theta_io[m]:
 * device double[N_m][K], in (PD_INIT_GIVEN) and out (gauge-fixed).
 * reports[m] (host) as for pd_fit; seconds is the wall time of the call. */
int pd_fit_batched(int n_maps, const pd_map* maps, double* const* theta_io,
                   const pd_fit_opts* opts, pd_fit_report* reports,
                   void* stream);

/* ---- learned warm start (not from the paper) -------------------------- */
/* A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 that
 * maps the features of a grain (pd_mlp_features) to its parameters, gauge-
 * fixed to zero mean over the grains and scaled to unit root-mean-square
 * norm over the grains.  Weights are kept in fp32 for training and used in
 * bf16 with fp32 accumulation by the forward and backward kernels.
 * Parameters are laid out W1 [h1][in], b1, W2 [h2][h1], b2, W3 [out][h2], b3. */
typedef struct pd_mlp pd_mlp;

/* Synchronous: allocates a network with He-uniform weights drawn from a
 * counter-based generator keyed by seed (zero biases). */
int pd_mlp_create(int n_in, int n_h1, int n_h2, int n_out, uint64_t seed,
                  pd_mlp** out);
void pd_mlp_destroy(pd_mlp* net);
int64_t pd_mlp_num_params(const pd_mlp* net);
/* Synchronous copies of all parameters to/from host float[num_params];
 * rounded != 0 returns the bf16 values the kernels use. */
int pd_mlp_get_params(const pd_mlp* net, float* host, int rounded);
int pd_mlp_set_params(pd_mlp* net, const float* host);
/* Y [B][out] = network(X [B][in]); device pointers. */
int pd_mlp_forward(const pd_mlp* net, const float* X, int B, float* Y,
                   void* stream);
/* Mean squared error of the network on (X, T [B][out]) and its gradient
 * with respect to every parameter (device float[num_params]). */
int pd_mlp_loss_grad(const pd_mlp* net, const float* X, const float* T, int B,
                     float* loss_out, float* grad_out, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on (X, T). */
int pd_mlp_train_step(pd_mlp* net, const float* X, const float* T, int B,
                      float lr, float* loss_out, void* stream);
/* Per-grain inputs of the network: the grain's Legendre moments of degree
 * <= 4 divided by |G_i| (first entry 1), then those of its 8 nearest grains
 * by centroid (the mean pixel), nearest first, ties to the smaller index,
 * padded with the grain's own moments.  feat_out: device float
 * [N][9 K_4] (135 in 2-D). */
int pd_mlp_features(const pd_grid* grid, const int32_t* labels, int N,
                    float* feat_out, void* stream);
/* Training targets of one map from its parameters theta (device double
 * [N][K], K <= 64): (theta_i - mean_j theta_j) / s, s the root-mean-square
 * norm of the centred rows; out: device float[N][K]. */
int pd_mlp_targets(const double* theta, int N, int K, float* out, void* stream);
/* Synchronous: starting parameters for pd_fit (init PD_INIT_GIVEN) from the
 * network's prediction: the prediction is gauge-fixed (theta_{N-1} = 0,
 * Remark 4.3) and scaled by the s in {2^(q/2): q = -16..40} that maximises
 * Phi(s theta) at (d, eps, prec) -- the network predicts the shape of the
 * diagram, not the sharpness that eps asks for (Lemma 4.1).  theta_out:
 * device double[N][K]; scale_out (host, may be NULL) receives s. */
int pd_warm_start(const pd_mlp* net, const pd_grid* grid,
                  const int32_t* labels, int N, int d, double eps, int prec,
                  double* theta_out, double* scale_out, void* stream);

/* ---- tracing of the library's own kernels ------------------------------ */
/* pd_prof_enable(1) clears the record and starts timing every kernel this
 * library launches, with a pair of CUDA events recorded on the launching
 * stream around the launch; pd_prof_enable(0) stops recording (the record
 * is kept).  pd_prof_read synchronises the recorded events and fills, for
 * up to cap distinct kernels, their names (static strings), launch counts
 * and total device milliseconds (host arrays); it returns the number of
 * distinct kernels recorded, or a negative code.  Timing adds two event
 * records per launch and is meant for profiling runs, not production. */
int pd_prof_enable(int on);
int pd_prof_read(int cap, const char** names, int64_t* launches, double* total_ms);

/* Synchronous throughput microbenchmark of one execution unit on the
 * current device, for roofline denominators: kind 0 = FP32 FMA, 1 = MUFU
 * ex2 (approximate base-2 exponential), 2 = FP64 FMA.  Writes operations
 * per second (one FMA or one ex2 = one operation) to *ops_per_s (host). */
int pd_microbench(int kind, double* ops_per_s, void* stream);

/* ---- evaluation without any device allocation -------------------------- */
/* pd_objective_grad allocates its scratch (the scaled parameters, log S per
 * pixel, per-block and per-chunk partial sums) from the device's
 * stream-ordered memory pool.  Some callers cannot let a library allocate:
 * a host whose device memory is entirely reserved up front by another
 * framework's allocator, a latency-bound loop that must not grow or touch
 * a memory pool after start-up, or an embedding that forbids cudaMalloc /
 * cudaMallocAsync outside its own initialisation.  This entry point gives
 * them the same evaluation with all scratch taken from one fixed array of
 * PD_NOALLOC_SCRATCH_BYTES compiled into the library (held on every device
 * that loads the library until the process exits); it calls no cudaMalloc,
 * cudaFree or any allocating routine.  The paper has no counterpart: this
 * is a deployment variant of the objective/gradient call above.
 *
 * Arguments, results and precisions are those of pd_objective_grad, limited
 * to 2-D pixel sets (PD_ENOTSUP otherwise) and PD_FP64 / PD_FP32 (another
 * valid precision: PD_ENOTSUP; an invalid one: PD_EINVAL).  A problem whose
 * scratch does not fit returns PD_ESCRATCH before anything is enqueued: in
 * FP32 about P * (4 + K/16) bytes (log S, and per 128-pixel tile its centre
 * features and reference logit), in FP64 P * 8, plus the scaled parameters
 * and at least one N*K*8-byte gradient partial.  Results equal
 * pd_objective_grad's up to the order of the fixed cross-chunk sum (fewer
 * chunks when scratch is tight).
 *
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, with that device current) and keeps it;
 * make that first call before any stream capture.  pd_release forgets the
 * address of the current device: call it after a reset of the device
 * (cudaDeviceReset), which reloads the library's module, before the next
 * call.  All calls share the one array: calls that overlap on the GPU (on
 * different streams, or from several host threads) race on it and must be
 * serialised by the caller. */
#define PD_NOALLOC_SCRATCH_BYTES (32u << 20)
int pd_objective_grad_noalloc(const pd_grid* grid, const int32_t* labels,
                              int N, const double* theta,
                              const pd_eval_opts* opts, double* obj_out,
                              double* grad_out, void* stream);

/* Synchronous self-test of the failure path of the tensor-core kernels: one
 * CTA waits on an mbarrier phase that nothing completes, with the same kind
 * of bounded wait those kernels use, limited to `seconds` (0 < seconds <=
 * 1).  The wait gives up, the kernel records PD_ETIMEOUT in *status_out
 * (host) and returns normally, so the context stays usable.  Returns PD_OK
 * when the self-test itself ran. */
int pd_selftest_wait_timeout(double seconds, int* status_out, void* stream);

/* Release cached library state on the current device (memory pool
 * reservations are trimmed, the cached device address of the allocation-
 * free entry point's array is forgotten).  Safe to call at any time when no
 * call of this library is in flight. */
void pd_release(void);

#ifdef __cplusplus
}
#endif

#endif /* PD_H_ */
