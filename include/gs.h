/*
 * gs.h -- C ABI of libgs, GPU point-set geodesic shooting with the exact
 * all-pairs flow and its Barnes-Hut approximation (arXiv 1907.04834).
 *
 * The problem (Sec. 2.1): N template points q(0) = q0 in R^3 with initial
 * momenta p(0) = p0 evolve under the Hamiltonian H(q,p) = 1/2 <p, K(q) p>,
 * K's 3x3 blocks G(|q_i - q_j|) I_3 with G(r) = exp(-r^2 / (2 sigma^2)):
 *     dq_i/dt = F_i   = sum_j G(|q_i-q_j|) p_j                      (Eq. 1, 3)
 *     dp_i/dt = Phi_i = sigma^-2 sum_j (p_i.p_j) G(|q_i-q_j|) (q_i-q_j)  (Eq. 1)
 * integrated by explicit Euler over t in [0, 1] with T steps (h = 1/T).  The
 * registration objective (Eq. 2) is
 *     E(p0) = H(q0, p0) + lambda sum_i |q_i(1) - X_i|^2
 * and its gradient with respect to p0 comes from the discrete adjoint of the
 * Euler scheme (the "backward stage" of Sec. 2.2).  In GS_BH mode every
 * forward and backward step evaluates the sums with the octree approximation
 * of Sec. 2.2: nodes whose points all lie farther than thresh_sigmas * sigma
 * from a point act as one source (centroid, total momentum, Eq. 4 and the
 * replacements after it); leaves are summed exactly.
 *
 * Conventions shared by every call:
 *   - Arrays of points are row-major N x 3 float64 (x, y, z per point), i.e.
 *     the layout of a contiguous (N, 3) tensor.  Each pointer may be host or
 *     device memory (detected per pointer with cudaPointerGetAttributes);
 *     device pointers must be on the context's device.  Inputs are only read.
 *   - Point counts N are in [1, 2^30]; an empty set (N = 0) or a larger one
 *     returns GS_ERR_INVALID_ARG before any work is enqueued.
 *     The caller owns all inputs and outputs; the context owns its workspace
 *     (grown on demand, reused across calls, freed by gs_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it.  A call whose outputs are all device
 *     pointers returns without waiting; a call with any host output
 *     synchronises the stream before returning.
 *   - Arithmetic: per-pair sums in FP32 (exp on the MUFU ex2 unit) with
 *     compensated accumulation; point state, Euler update, energies and
 *     reductions in FP64.
 *   - Errors: host-side checks return GS_ERR_INVALID_ARG before any work is
 *     enqueued; CUDA failures return GS_ERR_CUDA / GS_ERR_OOM.  Conditions
 *     detected on the device (non-finite results, a bounded wait that ran
 *     out) are recorded in a device status word that the next synchronising
 *     call, or gs_sync, returns.  gs_last_error gives a message.
 *   - A context is bound to one device and is not thread-safe; use one
 *     context per host thread.
 */
#ifndef GS_H
#define GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter (nothing enqueued) */
  GS_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GS_ERR_OOM = 3,         /* workspace allocation failed */
  GS_ERR_NONFINITE = 4,   /* NaN/Inf in a result (device-detected) */
  GS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  GS_ERR_UNSUPPORTED = 6  /* valid request this build cannot serve */
} gs_status;

typedef enum gs_mode {
  GS_EXACT = 0, /* all pairs, O(N^2) per step (Sec. 2.1) */
  GS_BH = 1,    /* octree / threshold approximation (Sec. 2.2) */
  GS_TRUNC = 2  /* variant, not the paper's approximation: pure truncation --
                   only pairs whose FP32 positions lie within thresh_sigmas *
                   sigma (dx = x_i - x_j per axis, (dx*dx + dy*dy) + dz*dz <=
                   r*r, each operation rounded), the same cut in the adjoint;
                   far nodes are dropped instead of summarised.  rhs counts:
                   {pairs kept, 0} */
} gs_mode;

typedef struct gs_params {
  double sigma;          /* Gaussian kernel width, > 0, same unit as q */
  double lambda;         /* data-term weight of Eq. 2, >= 0 */
  double thresh_sigmas;  /* GS_BH: a node is summarised when all its points
                            lie farther than thresh_sigmas * sigma (paper: 3);
                            GS_TRUNC: the cutoff radius in sigmas; with
                            criterion 1: the opening angle theta */
  int32_t T;             /* Euler steps over t in [0, 1], >= 1 */
  int32_t mode;          /* gs_mode */
  int32_t ckpt_every;    /* gs_shoot_grad: 0 = keep every step's state for the
                            backward pass; k > 0 = keep every k-th state and
                            recompute the others (memory (T/k + k) x N);
                            -1 = k = round(sqrt(T)), which minimises T/k + k */
  uint32_t flags;        /* reserved, must be 0 */
  int32_t leaf_size;     /* GS_BH: 0 or 1 = the paper's rule (a leaf is one
                            point, every near node is opened); L in [2, 32] =
                            leaf-size variant: a node of at most L points that
                            is not far is taken exactly, all its points, instead
                            of being opened (far nodes are still summarised).
                            Changes results; gs_autotune picks L by timing */
  int32_t criterion;     /* GS_BH far test: 0 = the paper's rule (the node's
                            FP32 actual range farther than thresh_sigmas *
                            sigma); 1 = opening-angle variant (classic
                            Barnes-Hut form): summarised iff s*s < theta^2 *
                            d2, s the largest side of the range, d2 the FP32
                            squared distance to its centre (lo + hi) * 0.5,
                            theta = thresh_sigmas in (0, 1] (dimensionless) */
  int32_t sympl_iters;   /* gs_shoot time stepping: 0 = explicit Euler (the
                            scheme of the gradient); M in [1, 64] =
                            semi-implicit symplectic Euler: per step, M
                            fixed-point passes r <- p^k + h Phi(q^k, r) from
                            r = p^k at fixed q^k, then q^{k+1} = q^k + h F(q^k,
                            r), p^{k+1} = p^k + h Phi(q^k, r) (M + 1 right-hand
                            sides per step; the step tends to symplectic Euler
                            as M grows).  gs_shoot, gs_shoot_traj and
                            gs_shoot_grad (the gradient of this scheme: the
                            discrete adjoint of its passes) take it; other
                            entry points need 0 (GS_ERR_UNSUPPORTED
                            otherwise) */
  int32_t reserved;      /* must be 0 */
} gs_params;

typedef struct gs_ctx gs_ctx;

/* Creates a context on CUDA device `device`.  *out receives the handle. */
gs_status gs_create(int device, gs_ctx **out);

/* Frees the context and its workspace (waits for its pending work). */
void gs_destroy(gs_ctx *ctx);

/* Message for the last error of this context ("" if none).  Valid until the
 * next call on the context. */
const char *gs_last_error(const gs_ctx *ctx);

/* Waits for `stream`, then returns and clears the device status word. */
gs_status gs_sync(gs_ctx *ctx, void *stream);

/* Failure-detection self-test.  Runs one kernel whose bounded device-side
 * wait (the one the bulk-copy pipelines use) cannot complete: it waits on a
 * barrier nothing arrives at, gives up after about 2e6 SM clocks (about 1 ms)
 * and records a timeout in the context's status word; the call then
 * synchronises `stream` and returns GS_ERR_TIMEOUT.  The context stays
 * usable: no trap, no fault, the status word is cleared. */
gs_status gs_selftest_timeout(gs_ctx *ctx, void *stream);

/*
 * Geodesic shooting (Sec. 2.1 Eq. 1, Euler with T steps; GS_BH: Sec. 2.2 at
 * every step).  q0, p0: N x 3 inputs.  q1, p1: N x 3 outputs q(1), p(1)
 * (either may be NULL).  H: NULL or 2 doubles receiving H(q0,p0) and
 * H(q(1),p(1)) = 1/2 sum_i p_i . F_i (the energy drift check; the second
 * costs one more right-hand-side evaluation).  N >= 1.
 */
gs_status gs_shoot(gs_ctx *ctx, const double *q0, const double *p0, int64_t N,
                   const gs_params *prm, double *q1, double *p1, double *H,
                   void *stream);

/*
 * Geodesic shooting as gs_shoot (Sec. 2.1 Eq. 1 with T Euler steps, or the
 * semi-implicit variant of sympl_iters; GS_BH: Sec. 2.2 at every step) that
 * also returns the whole discrete path: qtraj, ptraj are NULL or
 * (T + 1) x N x 3 outputs (state k at rows [k N, (k + 1) N), state 0 = q0,
 * p0), at least one of them non-NULL.  The path is what the paper's
 * registrations deform meshes along (Sec. 3.2).  Launches kernel by kernel
 * (no graph replay).
 */
gs_status gs_shoot_traj(gs_ctx *ctx, const double *q0, const double *p0, int64_t N,
                        const gs_params *prm, double *qtraj, double *ptraj,
                        void *stream);

/*
 * Objective of Eq. 2 and its gradient with respect to p0 (discrete adjoint,
 * backward stage of Sec. 2.2).  X: N x 3 targets.  E: 3 doubles {E, H(q0,p0),
 * lambda sum |q(1) - X|^2}.  grad: N x 3 dE/dp0.  q1: NULL or N x 3 q(1).
 * In GS_BH mode the backward steps use the tree approximation as the paper
 * prescribes (summaries of alpha and beta), which is not the derivative of
 * the discontinuous Barnes-Hut forward map.  With prm->sympl_iters = M > 0
 * the objective is that of the semi-implicit scheme and the gradient its
 * discrete adjoint: per step, with r_0 = p^k and r_m = p^k + h Phi(q^k,
 * r_{m-1}), rho_M = h dB[a, b](r_M), rho_{m-1} = h dB[0, rho_m](r_{m-1}),
 * dE/dq^k = a + h dA[a, b](r_M) + sum_{m=1..M} h dA[0, rho_m](r_{m-1}),
 * dE/dp^k = b + sum_{m=0..M} rho_m ([x, y](r): the adjoint right-hand side
 * of gs_adj_rhs at (q^k, r) with alpha = x, beta = y).
 */
gs_status gs_shoot_grad(gs_ctx *ctx, const double *q0, const double *p0,
                        const double *X, int64_t N, const gs_params *prm,
                        double *E, double *grad, double *q1, void *stream);

/*
 * Many independent registrations in one launch per step.  S >= 1 subjects;
 * offsets: host array of S+1 increasing int64, subject s owns rows
 * [offsets[s], offsets[s+1]) of q0, p0, X, grad (each offsets[S] x 3);
 * every subject has >= 1 point.  E: S x 3 doubles as in gs_shoot_grad.
 * All subjects share prm.  Points interact only within their subject.
 */
gs_status gs_shoot_batched(gs_ctx *ctx, int32_t S, const int64_t *offsets,
                           const double *q0, const double *p0,
                           const double *X, const gs_params *prm, double *E,
                           double *grad, void *stream);

/*
 * Fixed-step gradient descent on the initial momenta of S independent
 * registrations (the batched driver; the paper optimises each subject with
 * L-BFGS, Sec. 2.1): `iters` times, (E, grad) as gs_shoot_batched, then
 * p0 <- p0 - step * grad.  p0 (offsets[S] x 3) is read and overwritten with
 * the final momenta.  E_hist: NULL or iters x S x 3 doubles, the energies
 * of each iteration before its update.  The per-iteration step loop is
 * replayed from one captured CUDA graph (see gs_set_option "graphs").
 */
gs_status gs_descend_batched(gs_ctx *ctx, int32_t S, const int64_t *offsets,
                             const double *q0, double *p0, const double *X,
                             const gs_params *prm, double step, int32_t iters,
                             double *E_hist, void *stream);

/*
 * Shooting that also carries M tracer points (mesh vertices, grid nodes)
 * through the dense velocity field of Eq. 3, v(x, t) = sum_i G(|x - q_i(t)|)
 * p_i(t), as the paper does to deform meshes and label maps with the
 * registration.  The tracers take the particles' explicit Euler steps from
 * each step's particle state: x^{k+1} = x^k + h v(x^k; q^k, p^k); they do
 * not act on the particles.  x0, x1: M x 3 (M >= 0; x0, x1 may be NULL when
 * M = 0); q1, p1: NULL or N x 3 particle results.  GS_EXACT: exact sums;
 * GS_BH: the tracers are targets of the Sec. 2.2 traversal of the
 * particles' tree of each step (their FP32 positions decide; leaf_size and
 * criterion apply); GS_TRUNC returns GS_ERR_UNSUPPORTED.
 */
gs_status gs_flow(gs_ctx *ctx, const double *q0, const double *p0, int64_t N,
                  const double *x0, int64_t M, const gs_params *prm,
                  double *q1, double *p1, double *x1, void *stream);

/*
 * L-BFGS on the initial momenta of one registration (Sec. 2.1: the paper
 * minimises Eq. 2 with the L-BFGS of the VNL library): limited-memory BFGS
 * with the m most recent curvature pairs (two-loop recursion), a
 * backtracking line search from the unit step (Armijo condition, constant
 * 1e-4, halving up to 50 times; the first direction is -grad / |grad|), and
 * pairs with s.y <= 1e-12 |s| |y| skipped.  Stops after `iters` iterations,
 * when |grad| <= gtol * max(1, |grad(p0 initial)|), or when the line search
 * fails.  Each objective and gradient is gs_shoot_grad's (prm: mode,
 * checkpointing and all).  p0 (N x 3) is read and overwritten with the last
 * iterate; E_hist: NULL or iters + 1 doubles, E of the initial point and of
 * each accepted iterate (NaN after the last); n_done: NULL or the
 * iterations done.  The vector algebra runs on the device (FP64, fixed-order
 * dot products); the host reads back scalars.  Synchronises the stream.
 */
gs_status gs_lbfgs(gs_ctx *ctx, const double *q0, double *p0, const double *X,
                   int64_t N, const gs_params *prm, int32_t m, int32_t iters,
                   double gtol, double *E_hist, int32_t *n_done, void *stream);

/*
 * Autotuner of the Barnes-Hut leaf size (gs_params.leaf_size) for a state
 * (q, p) of N points (prm: GS_BH, its sigma and thresh_sigmas): times one
 * forward and one adjoint right-hand side (tree build, walk, evaluations, as
 * in a gradient step) for each candidate leaf size with CUDA events on the
 * stream (best of three after a warm-up) and writes the fastest to *best.
 * cand: n_cand candidates in [1, 32], or NULL for {1, 2, 4, 8, 16, 32};
 * ms: NULL or n_cand times in milliseconds.  Leaf sizes above 1 change the
 * approximation (more pairs exact), so the result is a choice for the
 * caller, not applied by the library.  Synchronises the stream.
 */
gs_status gs_autotune(gs_ctx *ctx, const double *q, const double *p, int64_t N,
                      const gs_params *prm, const int32_t *cand, int32_t n_cand,
                      int32_t *best, double *ms, void *stream);

/*
 * Autotuner of the exact kernels' tile shape for a state (q, p) of N points
 * (prm: GS_EXACT and its sigma).  A block of the all-pairs kernels owns 256
 * targets and sweeps 1/J of the sources (512-source tiles); J, the number of
 * source splits, is the one tile dimension chosen at run time.  For each
 * candidate J it times one forward and one adjoint right-hand side (CUDA
 * events on the stream, best of three after a warm-up) and writes the
 * fastest J of each to best[0] (forward) and best[1] (adjoint), as applied:
 * a candidate above the number of source tiles, ceil(N / 512), acts as that
 * number.  cand: n_cand values in [1, 4096] (n_cand <= 64), or NULL for
 * {1, 2, 3, 4, 6, 8, 12, 16, 24, 32}; ms: NULL or 2 x n_cand times in
 * milliseconds (forward, adjoint per candidate).  J changes the order in which
 * the FP32 tile partials are combined, so results move by rounding only; the
 * choice is the caller's (gs_set_option "exact_splits_fwd" and
 * "exact_splits_adj"), never applied by the library.  Synchronises the
 * stream.
 */
gs_status gs_autotune_exact(gs_ctx *ctx, const double *q, const double *p,
                            int64_t N, const gs_params *prm,
                            const int32_t *cand, int32_t n_cand, int32_t *best,
                            double *ms, void *stream);

/* ---- single-step entry points (one right-hand side, for checks) ---------- */

/* Velocity field of Eq. 3 at M >= 1 points x (M x 3): v = sum_i G(|x - q_i|)
 * p_i over the N particles; prm: sigma and mode (GS_EXACT: all pairs;
 * GS_BH: Barnes-Hut over the particles' tree as in gs_flow), FP32 pairs with
 * compensated sums as in gs_rhs.  v: M x 3. */
gs_status gs_velocity(gs_ctx *ctx, const double *q, const double *p, int64_t N,
                      const double *x, int64_t M, const gs_params *prm, double *v,
                      void *stream);

/* One forward right-hand side at state (q, p): F, Phi as in Eq. 1 (GS_BH:
 * Sec. 2.2 summaries).  counts: NULL or 2 int64 {point-point interactions,
 * point-node interactions} (GS_EXACT reports N*N and 0). */
gs_status gs_rhs(gs_ctx *ctx, const double *q, const double *p, int64_t N,
                 const gs_params *prm, double *F, double *Phi, int64_t *counts,
                 void *stream);

/* One adjoint right-hand side: with a = alpha^{k+1}, b = beta^{k+1} given in
 * `al`, `be`, the backward step is alpha^k = a + h dA, beta^k = b + h dB.
 * counts as in gs_rhs. */
gs_status gs_adj_rhs(gs_ctx *ctx, const double *q, const double *p,
                     const double *al, const double *be, int64_t N,
                     const gs_params *prm, double *dA, double *dB,
                     int64_t *counts, void *stream);

/*
 * Octree of Sec. 2.2 for positions q (N x 3), built as the GS_BH steps build
 * it.  codes: N uint32 30-bit Morton codes per input point (bit 3b+2 = x bit
 * b, 3b+1 = y, 3b = z, of the 10-bit quantised coordinates of the FP32
 * position within the FP32 bounding box).  order: N int32, points sorted
 * stably by code.  nodes: up to `cap` records of 4 int32 {depth, first,
 * count, skip} in depth-first preorder: cells holding >= 2 points that have
 * >= 2 non-empty child cells (or sit at depth 10), and single-point leaves
 * (depth = -1); members are order[first .. first+count); skip = preorder
 * index after the node's subtree.  range: NULL or cap x 6 float {lo, hi} of
 * each node's FP32 "actual range".  *n_nodes receives the node count
 * (N + internal nodes).  Any of codes/order/nodes/range may be NULL.
 */
gs_status gs_tree(gs_ctx *ctx, const double *q, int64_t N, uint32_t *codes,
                  int32_t *order, int32_t *nodes, float *range, int64_t cap,
                  int64_t *n_nodes, void *stream);

/*
 * Per-target record of the Barnes-Hut decisions (Sec. 2.2, the three cases
 * and the summaries of Eq. 4) on the tree of positions q (N x 3): the walk
 * of every GS_BH step, with its decisions recorded instead of listed.  prm:
 * mode GS_BH with its sigma, thresh_sigmas, leaf_size and criterion (other
 * modes: GS_ERR_UNSUPPORTED).  tally: N x 5 int64, row i (input order) =
 * {point interactions of target i, node interactions, sum over the points
 * it takes exactly of mix(key), the same sum over the nodes it summarises,
 * nodes of >= 2 points the traversal reaches for target i (tests: summarised,
 * opened or taken whole; gs_tree's nodes, so a cell whose points all lie in
 * one child cell is counted once)}, sums modulo 2^64 (bit patterns in
 * int64), mix = the splitmix64 output function (Steele, Lea and Flood,
 * OOPSLA 2014) of the 64-bit state key, key = (sorted position of the
 * source's first member << 32) | member count, sorted = the stable Morton
 * order of gs_tree.  Two records agree exactly when the targets took the
 * same sources, in any order; the totals of gs_rhs's counts are the column
 * sums of the first two columns, and points + nodes reached are the
 * traversal's node visits.  stats: NULL or 2 int64 {iterations of the
 * warp-cooperative walk (all warps), interaction-list entries it emits}.
 */
gs_status gs_bh_tally(gs_ctx *ctx, const double *q, int64_t N, const gs_params *prm,
                      int64_t *tally, int64_t *stats, void *stream);

/*
 * Sums over each node of the octree of gs_tree (same nodes, same preorder)
 * for state (q, p) and, if given, the adjoint variables (al, be): sums is
 * NULL or cap x 12 doubles per node {sum q (3), sum p (3), sum alpha (3),
 * sum beta (3)} over its members (a leaf: its point), in input units --
 * the statistics of Sec. 2.2 from which the summaries of Eq. 4 (centroid
 * sum q / n, P = sum p) and of the backward stage (A = sum alpha, B / n)
 * are formed.  al, be: both N x 3 or both NULL (sums of alpha and beta are
 * then 0).  The sums are the library's compensated FP32-pair sums of the
 * FP32-rounded values, converted to FP64.  *n_nodes (may be NULL)
 * receives the node count.  Synchronises the stream.
 */
gs_status gs_tree_sums(gs_ctx *ctx, const double *q, const double *p, const double *al,
                       const double *be, int64_t N, double *sums, int64_t cap,
                       int64_t *n_nodes, void *stream);

/* ---- diagnostics ---------------------------------------------------------- */

/* Tuning options of a context:
 *   "bh_list_cap": interaction-list storage of the Barnes-Hut walk, in
 *   entries per walk list on average (up to eight walk lists per 32 points,
 *   one pool per kept step); 0 = default (a budget of up to 24 GB, at most a
 *   quarter of the free memory, shared by the kept steps).  Slices whose
 *   lists do not fit are evaluated by a slower fused walk-and-evaluate pass
 *   that gives bit-identical results.
 *   "bh_walk_split": walk lists per slice of the Barnes-Hut walk (each group
 *   of 32 points has four slices): 1, 2 or 4, or 0 (default) = 2 for trees
 *   of fewer than 48 x (SM count) groups, else 1.  Splitting spreads a small
 *   tree's walk over more warps; results are bit-identical either way.
 *   "trunc_grid": 1 = GS_TRUNC on one point set searches its pairs with a
 *   uniform cell grid instead of the octree: cells of side 0.51 r (r =
 *   thresh_sigmas * sigma; doubled while there would be more than 8 N + 4096
 *   cells), points sorted stably by cell, and each warp of 32 consecutive
 *   points sweeps the cells within two of its own.  The kept pairs, and so
 *   the counts, are the same as the octree's; sums differ by rounding order
 *   only.  Batched calls keep the octree.  0 (default) = the octree.
 *   "exact_splits_fwd", "exact_splits_adj": source splits J of the exact
 *   single-point-set forward and adjoint kernels (gs_autotune_exact), in
 *   [1, 4096], capped at ceil(N / 512); 0 (default) = the built-in choice
 *   (the J that fills whole waves of blocks over the SMs).  Partial sums
 *   take J x 9 x N x 8 bytes of workspace.
 *   "graphs": 1 (default) = gs_shoot, gs_shoot_grad, gs_shoot_batched and
 *   gs_descend_batched capture their step loop (every launch between the
 *   input staging and the result copies) into a CUDA graph the first time
 *   they see a set of sizes, parameters and device addresses, and replay it
 *   while those stay the same; 0 = launch kernel by kernel.  Graphs are not
 *   used while gs_timing is on.  Results are identical either way. */
gs_status gs_set_option(gs_ctx *ctx, const char *name, int64_t value);

/* Kernel classes timed by gs_timing. */
enum {
  GS_K_EXACT_FWD = 0,  /* exact forward pair kernel */
  GS_K_EXACT_ADJ = 1,  /* exact adjoint pair kernel */
  GS_K_TREE_BUILD = 2, /* octree build: bbox, Morton, sort, nodes, aggregates */
  GS_K_BH_FWD = 3,     /* Barnes-Hut forward evaluation of the interaction lists */
  GS_K_BH_ADJ = 4,     /* Barnes-Hut adjoint evaluation of the interaction lists */
  GS_K_BH_WALK = 5,    /* Barnes-Hut tree walk (decisions, interaction lists) */
  GS_K_COUNT = 6
};

/* enable != 0: subsequent calls bracket each launch group of the classes
 * above with CUDA events on the call's stream (small overhead per group). */
gs_status gs_timing(gs_ctx *ctx, int enable);

/* Waits for the recorded events and returns, per class, the number of timed
 * launch groups (launches[GS_K_COUNT]) and their summed device time in ms
 * (ms[GS_K_COUNT]) since the previous read; total_launches (may be NULL)
 * receives the number of kernels this library launched (all kinds, this
 * process) since the previous read. */
gs_status gs_timing_read(gs_ctx *ctx, int64_t *launches, double *ms,
                         int64_t *total_launches);

/* Measured device-wide issue rates of the units the pair kernels use, in
 * lane-operations per second: out[0] scalar FP32 FMA, out[1] FP32 operations
 * through packed f32x2 FMA (two per lane per instruction), out[2] MUFU ex2.
 * Runs short synthetic kernels on `device` (about 10 ms); no context needed. */
gs_status gs_alu_peaks(int device, double *out);

/* ---- allocation-free variant -------------------------------------------- */

/* Largest N that gs_rhs_exact_noalloc accepts. */
#define GS_RHS_NOALLOC_MAX_N 16384

/*
 * The exact forward right-hand side of gs_rhs (GS_EXACT: F and Phi at state
 * (q, p)) computed without allocating any device memory.  The paper has no
 * counterpart: it serves callers that cannot call cudaMalloc -- applications
 * whose device memory is owned entirely by their own pool allocator, which
 * forbids other allocations, and latency-critical loops in which an
 * allocation's implicit device synchronisation is not acceptable.
 *
 * q, p, F, Phi: N x 3 float64 device buffers on the current CUDA device
 * (host buffers are rejected with GS_ERR_INVALID_ARG); sigma > 0;
 * 1 <= N <= GS_RHS_NOALLOC_MAX_N, larger N returns GS_ERR_INVALID_ARG.  No
 * context is needed.  Work is enqueued on `stream` and the call returns
 * without waiting; device-side conditions are not reported by this call: if
 * a bounded wait of the kernel's copy pipeline gives up (it cannot complete
 * only when the GPU is failing; the context-based entry points report it as
 * GS_ERR_TIMEOUT, and gs_selftest_timeout exercises that wait), F and Phi
 * are undefined and nothing tells the caller.
 *
 * Scratch: one fixed array of about 6.4 MiB of device memory that every GPU
 * on which the library's device code has been loaded (see the first call,
 * below) holds until the process exits.  Every call on that
 * GPU shares it and it keeps the previous call's contents (the call clears
 * what must start at zero); calls whose GPU work overlaps -- on different
 * streams or from concurrent host threads -- race on it, so serialise them.
 * The first call on a device looks up the array's device address and sets
 * up the kernel, with that device current.  Under CUDA's default lazy
 * module loading (CUDA_MODULE_LOADING=LAZY) that first call is also when
 * the driver loads this library's device code and commits the array: it
 * takes device memory and may synchronise, and it fails if the caller's
 * pool has already reserved all of the GPU's memory.  So make one warm-up
 * call at initialisation, before the pool reserves its memory and before
 * any stream capture; later calls take no memory.
 */
gs_status gs_rhs_exact_noalloc(const double *q, const double *p, int64_t N,
                               double sigma, double *F, double *Phi,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
