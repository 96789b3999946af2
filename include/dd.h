/*
 * dd.h — C ABI of the GB300 library for entropic domain decomposition of
 * optimal transport between two 2D images (Bonafini & Schmitzer, "Domain
 * decomposition for entropy regularized optimal transport").
 *
 * The library solves min ε·KL(π|K) over couplings π of μ and ν with
 * K = exp(−c/ε)·(μ⊗ν) and c(x,y) = |x−y|² on pixel centres in [0,1]²
 * (§2.2 eq. EntropicOTPrimal, §3 eq. Problem, §7.1 "Test data"), by
 * Algorithm 2 (§6.1) inside the multi-scale / ε-scaling driver of §6.4.
 *
 * Conventions for every entry point:
 *  - Images are n×n, row-major, pixel (i,j) has flat index i·n+j and centre
 *    ((i+½)h, (j+½)h), h = 1/n at the finest level. Level l of L has
 *    n_l = n/2^(L−1−l) pixels per side; level 0 is the coarsest.
 *  - A basic cell is a b×b block of pixels (§7.1 "Basic and composite
 *    partitions"); basic cells are numbered row-major over the n_l/b × n_l/b
 *    grid of cells ("natural order"). Partition A (= 0) groups them in 2×2
 *    blocks; partition B (= 1) is A shifted by one basic cell.
 *  - All pointer arguments are HOST pointers. The library copies what it
 *    reads; the caller keeps ownership of its buffers. Device memory is owned
 *    by the context and freed by dd_destroy.
 *  - Every call returns a dd_status. On failure the context keeps the state
 *    it had before the call and dd_last_error() describes the problem. After
 *    a CUDA error the context is unusable and later calls return
 *    DD_ERR_STATE. No call aborts the process or throws.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_ctx dd_ctx;

typedef enum {
  DD_OK = 0,
  DD_ERR_ARG = 1,          /* invalid argument (sizes, NaN, negative mass, …)  */
  DD_ERR_CUDA = 2,         /* a CUDA call failed                               */
  DD_ERR_OOM = 3,          /* device allocation failed                         */
  DD_ERR_CAPACITY = 4,     /* a caller buffer is too small (see *nnz)          */
  DD_ERR_NUMERIC = 5,      /* a cell solve produced a non-finite value         */
  DD_ERR_STATE = 6,        /* context unusable or call out of order            */
  DD_ERR_NOT_CONVERGED = 7 /* an iterative solve missed its tolerance: a host
                              solve, or cell solves still at max_iter after the
                              safeguard (the call completed; state feasible)  */
} dd_status;

/* Image size and number of multi-scale levels (§6.4, §7.1 "Multi-scale"). */
typedef struct {
  int32_t n;       /* finest image side in pixels                              */
  int32_t levels;  /* ≥ 1; n/2^(levels−1) must be a multiple of 2·b            */
} dd_grid;

/* One step of the ε schedule: `sweeps` sweeps (A then B half-sweep each) at
 * regularisation `eps` ([0,1]² units, same units as c) on `level`. Levels must
 * be non-decreasing; entering a new level refines the state by eq.
 * FineBasicMarginals (§6.4). When ε changes, ε·log u is kept (§6.4, last
 * paragraph). */
typedef struct {
  double eps;
  int32_t sweeps;
  int32_t level;
} dd_eps_step;

typedef struct {
  double err_tol;        /* Err of §6.2: a cell solve stops after the first
                            Y-iteration whose X-marginal L1 error is
                            ≤ ‖μ_J‖·err_tol. Default 1e-6.                     */
  double trunc;          /* Truncate threshold on ν_i entries (§7.1), absolute
                            mass. Default 1e-15.                               */
  int32_t max_iter;      /* cap on Sinkhorn Y-iterations per cell solve.
                            Default 2000.                                      */
  int32_t threads_per_cell; /* CUDA threads per composite cell (32, 64, 128
                            or 256); 0 = library choice. Default 0.            */
  int32_t max_cluster_cells; /* at most this many of the cells with the
                            largest predicted work (≥ an eighth of one SM's
                            share) are solved by a cluster of 8 CTAs each;
                            0 = none, −1 = library default (256).              */
  int32_t x_newton;      /* ≥ 1: a cell of at most 64 pixels whose X-iteration
                            contracts slowly switches to Newton X-iterations
                            (same fixed point, same stopping rule): at
                            iteration 6 when the contraction over iterations
                            3–6 predicts more than x_newton − 1 further plain
                            iterations (1: whenever it is slow), later when 16
                            iterations reduce the error less than tenfold.
                            0: plain Sinkhorn X-iterations only. Default 1.    */
  int32_t warm;          /* warm start of the cell solves. 0: the duals of the
                            cell's previous solve (Algorithm 2 input u_{C,J}).
                            1: with a network attached (dd_attach_mlp), 8×8
                            cells also get a predicted dual at the first sweep
                            on a new level, and start from whichever of the
                            two has the smaller X-marginal error after one
                            Y-iteration. 2: the same also at the first sweep
                            after a change of ε. 3: at every half-sweep.
                            Default 0.                                         */
  int32_t dual_refine;   /* duals at a new level. 0: both partitions start
                            from the last partition's duals refined cell by
                            cell (first-order, within each coarse cell).
                            1 (hybrid): A as 0; B from the glued coarse dual
                            of both partitions (§6.3, on the GPU; on the host
                            beyond 256 A cells per side) interpolated
                            linearly (§6.4). Default 0.                        */
  int32_t mode;          /* 0: every half-sweep as separate launches with a host
                            check in between. 1: per-CTA cell solves as one
                            persistent wave of CTAs that take cells in launch
                            order from a counter, and every sweep at the same
                            (level, ε) as the previous one replayed from one
                            captured CUDA graph (A and B half-sweeps, no host
                            synchronisation inside); the state buffers then
                            hold twice the current entries. Default 0.         */
  void* stream;          /* cudaStream_t to run on; NULL = a stream owned by
                            the context.                                       */
  uint64_t debug_flags;  /* bit 0: synchronise and check after every kernel;
                            bit 1: time the gather and cell-solve kernels with
                            CUDA events (see dd_get_profile).
                            Fault injection on the host (for tests; no GPU
                            fault is involved):
                            bit 2: graph-replayed sweeps (mode 1) get an
                            output buffer of half the current entries, so the
                            sweep overflows and is run again with per-kernel
                            launches (dd_profile.graph_reruns counts it);
                            bit 3: the main solve of every cell stops after
                            one iteration, so the safeguard re-solves it;
                            bit 4: the first growth of the half-sweep
                            workspace fails as a failed cudaMalloc would
                            (DD_ERR_OOM, state untouched; one shot).
                            bit 5: the hybrid refinement (dual_refine = 1)
                            glues on the host at every size, as it does
                            beyond 256 A cells per side (for comparing the
                            two paths).
                            Bits 0 and 1 turn the graph replay of mode 1
                            off.                                               */
  int32_t safeguard;     /* 1: a cell whose solve stops at max_iter, or
                            stagnates (its X-error falls by less than 0.1 %
                            over 128 iterations), with an X-error above
                            10·Err·‖μ_J‖ is solved again, warm-started from
                            where it stopped (the local safeguard of §7.3,
                            "temporarily increasing ε"): at 4ε, then at ε from
                            that result (4ε again if ε fails), otherwise at
                            16ε, 64ε, … 4096ε, keeping the first solve that
                            converges. A kept solve at a larger ε sets bit 3
                            of the cell's status and counts in
                            cells_escalated. Cells still not converged
                            afterwards (also those just above their
                            tolerance) make the call return
                            DD_ERR_NOT_CONVERGED after completing it. 0: off
                            (the half-sweep keeps the cut-off solves).
                            Default 1.                                         */
} dd_options;

/* Counters of the work done by a context since creation or the last
 * dd_reset_profile (the peaks are maxima over the same period). Kernel times
 * are filled only with debug_flags bit 1. */
typedef struct {
  int64_t launches;          /* CUDA kernels launched by the context            */
  int64_t half_sweeps;       /* half-sweeps run                                 */
  int64_t solve_launches;    /* launches of the cell-solve kernel               */
  double solve_ms;           /* their summed duration (CUDA events)             */
  int64_t gather_launches;   /* launches of the Y-marginal gather kernel        */
  double gather_ms;          /* their summed duration (CUDA events)             */
  double cluster_ms;         /* summed duration of the cluster cell solves,
                                which run beside the per-CTA solves (events)    */
  double kernel_evals;       /* Σ over cell solves of |X_J|·N_y(J)·(iterations+1):
                                kernel entries exp(…) evaluated                  */
  double sinkhorn_iters;     /* Σ over cell solves of the Sinkhorn iterations   */
  int64_t cells;             /* cell solves                                     */
  int64_t newton_steps;      /* X-iterations taken as Newton steps (cells of at
                                most 64 pixels whose iteration converges slowly) */
  double hessian_fma;        /* FMAs of their Hessian accumulations,
                                Σ over steps of 64²·N_y(J)                       */
  int64_t learned_cells;     /* cell solves that started from the predicted
                                duals (warm ≠ 0)                                 */
  int64_t compared_cells;    /* cell solves whose prediction was compared with
                                the previous duals                               */
  int64_t rescued_cells;     /* cells re-solved by the safeguard                 */
  int64_t graph_reruns;      /* graph-replayed sweeps whose output did not fit
                                and that ran again with per-kernel launches      */
  int64_t peak_nnz;          /* largest number of stored entries of (ν_i)        */
  int64_t peak_state_bytes;  /* largest device memory of the two CSR buffers of
                                (ν_i): column, fixed-point value, row pointers   */
  int64_t peak_work_bytes;   /* largest device memory of the half-sweep buffers
                                that scale with the entries (gathered supports,
                                stabilisers, extracted rows)                     */
  int64_t escalated_cells;   /* cell solves that the safeguard kept at a larger
                                ε than the half-sweep's (status bit 3)           */
} dd_profile;

/* Statistics of the last sweep run by dd_sweep / dd_run_schedule. */
typedef struct {
  int32_t level;          /* level of the last half-sweep                     */
  int32_t partition;      /* 0 = A, 1 = B                                     */
  double eps;             /* ε of the last half-sweep                         */
  int64_t nnz;            /* entries stored in (ν_i) after it                 */
  int32_t max_iters;      /* largest Sinkhorn iteration count over its cells  */
  double mean_iters;      /* mean Sinkhorn iteration count over its cells     */
  int32_t cells_not_converged; /* cells still at max_iter after the safeguard   */
  int64_t sweeps_done;    /* total sweeps since dd_create                     */
  int32_t cells_rescued;  /* cells of the last half-sweep that the safeguard
                             solved again                                     */
  int32_t cells_escalated; /* of these, cells whose kept solve is at a larger
                             ε (4ε … 4096ε; status bit 3)                     */
} dd_sweep_stats;

/* Fill *opt with the defaults listed above. */
void dd_options_default(dd_options* opt);

/* Create a context for transporting μ to ν.
 * mu, nu: n×n host arrays of finite non-negative FP64 masses (n = grid->n).
 *   They are normalised to mass 1; their masses must agree to 1e-9 relative.
 *   Every basic cell of the finest level must carry positive μ-mass (Def. 3.1).
 * b: basic cell side in pixels (2, 4 or 8).
 * schedule, n_steps: the ε schedule (copied). n_steps ≥ 1, first level 0.
 * opt: NULL for defaults.
 * The context starts at level 0 with the product coupling ν_i = ‖μ_i‖·ν
 * (§6.4) and α = ε·log u = 0 on both partitions (Algorithm 2 inputs).
 * On success *out receives the context. */
dd_status dd_create(const double* mu, const double* nu, const dd_grid* grid, int32_t b,
                    const dd_eps_step* schedule, int32_t n_steps,
                    const dd_options* opt, dd_ctx** out);

/* Replace the state at the context's current level with the inputs of
 * Algorithm 2 (§6.1): feasible basic Y-marginals (ν_i) and the scaling u as
 * α = ε·log u, one value per pixel.
 * row_ptr: n_basic+1 offsets (natural order of basic cells), col: Y pixel
 *   indices at this level, strictly increasing within each row, val: masses
 *   (FP64, ≥ 0) in the normalisation of dd_create (total mass 1).
 * alpha_A, alpha_B: n_l×n_l FP64 arrays or NULL for zero.
 * Returns DD_ERR_ARG for unsorted / out-of-range / negative input. */
dd_status dd_set_state(dd_ctx* ctx, const int64_t* row_ptr, const int32_t* col,
                       const double* val, const double* alpha_A, const double* alpha_B);

/* One iteration of Algorithm 2 on `partition` (0 = A, 1 = B) at the current
 * level with regularisation eps: for every composite cell J, gather
 * ν_cell = Σ_{i∈J} ν_i, solve the cell by log-domain Sinkhorn warm-started
 * from u_{C,J} (stop rule of §6.2), extract ν_i = P_Y(π_cell|X_i×Y),
 * BalanceMeasures, Truncate. Does not advance the schedule. */
dd_status dd_half_sweep(dd_ctx* ctx, int32_t partition, double eps);

/* Move the state one level finer (§6.4) without sweeping: the basic
 * marginals by eq. FineBasicMarginals, the duals as dd_options.dual_refine
 * says. dd_sweep then continues the schedule; its steps on coarser levels run
 * on the current level. DD_ERR_STATE at the finest level. */
dd_status dd_refine(dd_ctx* ctx);

/* Run n_sweeps sweeps (A then B) following the schedule, refining when the
 * schedule enters a new level. After the last step of the schedule the
 * remaining sweeps stay at its ε and level. stats may be NULL. */
dd_status dd_sweep(dd_ctx* ctx, int32_t n_sweeps, dd_sweep_stats* stats);

/* Run every remaining sweep of the schedule. stats may be NULL. */
dd_status dd_run_schedule(dd_ctx* ctx, dd_sweep_stats* stats);

/* FP64 summaries of the coupling of the last half-sweep, π = Σ_J π_J with
 * π_J the final cell plans: cost = Σ c·π (transport cost ⟨c,π⟩),
 * err_x = Σ_x |P_X π(x) − μ(x)|, err_y = Σ_y |Σ_i ν_i(y) − ν(y)| (L1 errors of
 * the marginals, Table 1 "L1 X/Y-marginal error"). Any pointer may be NULL. */
dd_status dd_cost(dd_ctx* ctx, double* cost, double* err_x, double* err_y);

/* Copy the basic Y-marginals (ν_i) at the current level to host memory as
 * CSR in natural order of basic cells: row_ptr[n_basic+1], col (Y pixel
 * index), val (FP64 mass). Call with col = val = NULL (row_ptr may be NULL)
 * to get *nnz; cap is the capacity of col/val in entries
 * (DD_ERR_CAPACITY if smaller than *nnz). */
dd_status dd_get_basic_marginals(dd_ctx* ctx, int64_t* nnz, int64_t* row_ptr,
                                 int32_t* col, double* val, int64_t cap);

/* Pixel-level coupling of the partition solved last (§6.1 item (iv): the
 * partial couplings are recovered from the scalings): on every composite
 * cell, f from u_{C,J} and one Y-iteration against ν_cell, so P_Y π = ν.
 * CSR with one row per X pixel (n_l² rows), entries > trunc only.
 * Two-call pattern as in dd_get_basic_marginals. */
dd_status dd_get_plan(dd_ctx* ctx, double trunc, int64_t* nnz, int64_t* row_ptr,
                      int32_t* col, double* val, int64_t cap);

/* Objective of a coupling π, summed cell by cell as §6.3 describes: with
 * partition = -1 the coupling of dd_get_plan (the partition solved last, at
 * its ε; eps is ignored), with partition 0 (A) or 1 (B) the coupling that
 * the current basic marginals and that partition's α give at ε = eps (on
 * every cell f from α and one Y-iteration against ν_cell). K = e^{−c/ε}·μ⊗ν:
 *   primal  = KL(π|K) − ‖K‖ = Σ π·(log π − log K − 1), the primal score of
 *             eq. RelPDGap (Lemma 4.2 evaluates it from the scalings);
 *   gap     = Σ_J gap_J and gap_abs = Σ_J |gap_J|, where gap_J =
 *             KL(π_J|K_J) − J_J(u_J, v_J) is the primal-dual gap of the cell
 *             problem on X_J × supp ν_cell with marginals μ_J and ν_cell
 *             (J_J: eq. EntropicOTDualObjective, Prop. 2.5). π_J meets ν_cell
 *             exactly and μ_J only approximately (up to the Sinkhorn
 *             tolerance after a solve), so gap_J has no fixed sign; it is
 *             zero at the cell's optimum and does not
 *             depend on the per-cell constants of the duals beyond
 *             (‖ν_cell‖ − ‖μ_J‖)·constant/ε, the mass lost to Truncate.
 * Entries are FP32 exponentials (as in dd_get_plan), logs and sums FP64. The
 * global primal-dual gap of eq. RelPDGap needs the glued duals of §6.3:
 * dd_relative_pd_gap. Allocates (and frees) 16 bytes per composite cell of
 * device memory; synchronises the stream; leaves the state and the
 * statistics of the last half-sweep as they were. Any output pointer may be
 * NULL.
 * DD_ERR_STATE for partition -1 before the first half-sweep of a level;
 * DD_ERR_ARG for another partition or a non-positive eps. */
dd_status dd_objective(dd_ctx* ctx, int32_t partition, double eps, double* primal, double* gap,
                       double* gap_abs);

/* The glued X-dual of §6.3 ("Estimating the primal-dual gap") of the
 * context's current level, computed on the GPU from the duals of both
 * partitions at the current ε: per basic cell i the μ-weighted means s±_i =
 * log ⨍_i exp(±(α_A − α_B)/ε) dμ; every ordered pair (i, i') of distinct
 * basic cells of one B cell is an edge between the A cells holding them with
 * log q = s⁺_i + s⁻_{i'}; the potential V on the A cells minimises
 * Σ_e ((V(j1) − V(j2)) + log q_e)² with Σ V = 0 (conjugate gradients,
 * Jacobi-preconditioned, relative residual 1e-13, at most 100 000
 * iterations); α̂ = α_A + ε·V[A cell]. The same construction as
 * dd_glue_duals_host, whose results it reproduces up to rounding.
 * Outputs (host, each may be NULL): alpha_hat (n_l² FP64, absolute frame as
 * dd_get_duals, 0 on pixels without mass), V ((n_l/2b)² FP64, row-major over
 * the A cells), *cg_iters, *rel_residual. Allocates and frees device scratch
 * (8 bytes per pixel and 16 per basic cell); synchronises the stream; leaves
 * the state as it was. DD_ERR_CAPACITY when the A cells exceed 256 per side
 * (the CG runs on one cluster of 8 CTAs that holds at most 256 rows of 256
 * cells); DD_ERR_NOT_CONVERGED (outputs written) when the CG stopped at its
 * iteration limit. */
dd_status dd_glue_duals(dd_ctx* ctx, double* alpha_hat, double* V, int32_t* cg_iters, double* rel_residual);

/* eq. RelPDGap on the GPU for the coupling of the last partition (the one
 * dd_get_plan and dd_objective reconstruct: support X_J × supp ν_cell per
 * cell, entries from the stored duals and one Y-iteration) and the glued
 * X-dual α̂ of dd_glue_duals: with K = e^{−c/ε}·μ⊗ν (masses normalised to 1),
 *   *primal = KL(π|K) − ‖K‖ (dd_objective's primal),
 *   v̂(y) = 1/S(y), S(y) = Σ_{x: π(x,y) > 0} û(x) μ(x) e^{−c(x,y)/ε}, the Y-dual
 *            that maximises J(û, ·) for the kernel restricted to supp π,
 *   *gap = KL(π|K) − J(û, v̂) = primal − (⟨μ, log û⟩ − ⟨ν, log S⟩ − Σ_{y
 *            covered} ν(y)),
 *   *rel = gap / primal.
 * The same quantities as dd_relative_pd_gap_host on dd_get_plan's coupling
 * (with no truncation) and dd_glue_duals_host's α̂. Logs and sums FP64,
 * exponentials of the inner sums FP32 after an FP64 shift by their maximum
 * (the precision of the coupling's entries); S is accumulated with atomic
 * additions, so the last digits may vary from call to call. Outputs may be
 * NULL. Allocates and frees device scratch (24 bytes per pixel, 8 per
 * gathered support point and 16 per composite cell); synchronises the
 * stream; leaves the state as it was.
 * DD_ERR_STATE before the first half-sweep of a level or when a pixel with
 * ν > 0 carries no entry of the coupling; DD_ERR_CAPACITY and
 * DD_ERR_NOT_CONVERGED as dd_glue_duals. */
dd_status dd_relative_pd_gap(dd_ctx* ctx, double* rel, double* gap, double* primal);

/* The least-squares step of the dual gluing (§6.3, "Estimating the
 * primal-dual gap"): on a graph of n_nodes vertices (the cells of partition
 * A) with n_edges directed edges (j1[e], j2[e]) carrying the values logq[e]
 * (log of the edge weights q), V[n_nodes] minimises
 *     Σ_e ((V[j1[e]] − V[j2[e]]) + logq[e])²
 * and has mean zero on every connected component (on a connected graph the
 * gauge Σ V = 0). The sign in front of logq makes the result agree with the
 * section's path-product construction (û_J = Π q along a path · u_{A,J}), so
 * that û_J = exp(V[J])·u_{A,J}. Edges with j1 = j2 are ignored. Solved by
 * conjugate gradients on the graph Laplacian with degree (Jacobi)
 * preconditioning until ‖residual‖ ≤ tol·‖right-hand side‖ or max_iter
 * iterations; *iters and *rel_residual (either may be NULL) report the run.
 * Host code, FP64; needs no GPU and no context. DD_ERR_ARG for indices out
 * of range, non-finite logq or negative sizes; DD_ERR_NOT_CONVERGED (V then
 * holds the last iterate) when the tolerance was not reached; DD_ERR_OOM when
 * host memory runs out. */
dd_status dd_glue_potential(int32_t n_nodes, int64_t n_edges, const int32_t* j1, const int32_t* j2,
                            const double* logq, double tol, int32_t max_iter, double* V,
                            int32_t* iters, double* rel_residual);

/* The glued X-dual of §6.3 from the duals of both partitions, on the host:
 * n×n pixels, b×b basic cells (n/b even), μ and α_A, α_B = ε·log u per pixel
 * (n² FP64 each, as dd_get_duals returns them; μ in any normalisation). For
 * every basic cell i the μ-weighted means of exp(±(α_A − α_B)/ε) over its
 * pixels give the edge values log q = s⁺_i + s⁻_{i'} of the ordered pairs
 * of distinct basic cells (i, i') of each B cell (the A cells containing
 * them are the vertices); V = dd_glue_potential(…) (tolerance 1e-13) and
 * alpha_hat = α_A + ε·V[A cell] (n² FP64; 0 on pixels without mass).
 * V (may be NULL) receives the (n/2b)² potentials in row-major order of the
 * A cells. Host code; needs no GPU and no context. DD_ERR_ARG for bad sizes,
 * non-finite or negative input, or a basic cell without mass;
 * DD_ERR_NOT_CONVERGED / DD_ERR_OOM from the solve. */
dd_status dd_glue_duals_host(int32_t n, int32_t b, const double* mu, const double* alpha_A,
                             const double* alpha_B, double eps, double* alpha_hat, double* V);

/* Dual refinement of §6.4 on the host: alpha_c (n_coarse² FP64, a glued
 * dual α̂ = ε·log û of one level) interpolated linearly onto the level
 * twice as fine, alpha_f ((2·n_coarse)² FP64). Fine pixel I sits at
 * t = I/2 − 1/4 in coarse index units (bilinear weights 1/4 and 3/4; linear
 * extrapolation over the outermost quarter step), so affine α is reproduced
 * exactly. Host code; no GPU, no context. DD_ERR_ARG for n_coarse < 2 or a
 * NULL pointer. */
dd_status dd_interpolate_dual_host(int32_t n_coarse, const double* alpha_c, double* alpha_f);

/* Relative primal-dual gap of eq. RelPDGap on the host, for a coupling π
 * given as the CSR of dd_get_plan (row_ptr[n²+1] over X pixels, col = Y
 * pixel, val = mass, total 1) and an X-dual alpha_hat (n² FP64, e.g. from
 * dd_glue_duals_host) on an n×n level with pixel spacing 1/n (c = |x−y|²,
 * K = e^{−c/ε}·μ⊗ν; μ, ν (n² FP64, ≥ 0) are normalised to mass 1 here).
 * The Y-dual is the one that maximises J(û, ·) for the kernel restricted
 * to the support of π: v̂(y) = 1 / Σ_{x: π(x,y)>0} û(x) μ(x) e^{−c/ε}.
 * Outputs (each may be NULL): *primal = KL(π|K) − ‖K‖, *gap = KL(π|K) −
 * J(û, v̂), *rel = gap / primal. Host code; no GPU, no context. DD_ERR_ARG
 * for bad sizes, negative or non-finite input, an entry of π where ν = 0 or
 * a y with ν(y) > 0 that π does not reach. */
dd_status dd_relative_pd_gap_host(int32_t n, const double* mu, const double* nu, double eps,
                                  const int64_t* row_ptr, const int32_t* col, const double* val,
                                  const double* alpha_hat, double* rel, double* gap, double* primal);

/* Colour image of a coupling (§7.2): rgb[3·y + k] = Σ_i colours[3·i + k] ·
 * ν_i(y) / ν(y) with ν(y) = Σ_i ν_i(y), for basic Y-marginals given as the
 * CSR of dd_get_basic_marginals (row_ptr[n_basic+1], col < n², val ≥ 0);
 * pixels that no ν_i reaches are black. colours: n_basic × 3 floats (e.g. a
 * checkerboard); rgb: n² × 3 floats, written. Host code; no GPU, no context.
 * DD_ERR_ARG for bad sizes, indices or values. */
dd_status dd_coupling_image_host(int32_t n, int32_t n_basic, const int64_t* row_ptr, const int32_t* col,
                                 const double* val, const float* colours, float* rgb);

/* The colour image of §7.2 for the context's current basic marginals,
 * computed on the GPU: rgb[3·y + k] = Σ_i colours[3·i + k]·ν_i(y)/ν(y), ν(y) =
 * Σ_i ν_i(y), black where no ν_i reaches y (the same image as
 * dd_coupling_image_host, summed with FP64 atomics in an unspecified order).
 * colours: n_basic × 3 floats (HOST, finite); rgb: n_l² × 3 floats (HOST,
 * written). Allocates and frees scratch of 40 bytes per pixel; synchronises
 * the stream. DD_ERR_ARG for NULL or non-finite colours. */
dd_status dd_coupling_image(dd_ctx* ctx, const float* colours, float* rgb);

/* α = ε·log u_{C,J} of `partition` on every pixel of the current level, up to
 * one additive constant per composite cell (the gauge of Prop. 2.3 (ii)). */
dd_status dd_get_duals(dd_ctx* ctx, int32_t partition, double* alpha);

/* Current level, its side n_l, its number of basic cells (n_l/b)², the ε of
 * the last half-sweep and the number of stored entries of (ν_i). Any output
 * pointer may be NULL. */
dd_status dd_get_info(dd_ctx* ctx, int32_t* level, int32_t* n_level, int32_t* n_basic,
                      double* eps, int64_t* nnz);

/* Per composite cell of the last half-sweep (in the cell order of its
 * partition: row-major over the grid of composite cells): Sinkhorn
 * iterations, final X-marginal L1 error, support size N_y of ν_cell, a
 * status word (bit 0: stopped at max_iter or stagnated, bit 1: non-finite,
 * bit 2: workspace overflow, bit 3: the safeguard kept a solve at a larger ε),
 * the transport
 * cost ⟨c, π_J⟩ of the cell's plan (FP64; the terms of dd_cost's cost) and
 * whether its main solve ran on a cluster of CTAs (1) or one CTA (0). Any
 * array may be NULL; cap is their length; *n_cells receives the number of
 * cells. */
dd_status dd_get_cell_stats(dd_ctx* ctx, int32_t* iters, double* err_x, int32_t* n_y,
                            int32_t* status, double* cost, int32_t* cluster, int32_t cap,
                            int32_t* n_cells);

/* Copy the context's counters to *out. */
dd_status dd_get_profile(dd_ctx* ctx, dd_profile* out);

/* Reset the context's counters to zero. */
dd_status dd_reset_profile(dd_ctx* ctx);

/* Solve one composite cell without allocating any memory (no counterpart in
 * the paper: this is a library facility). Some callers cannot call
 * cudaMalloc when they need a solve: hosts whose device memory belongs to
 * another runtime or memory pool that forbids allocations behind its back
 * (for example a plug-in that only receives pre-allocated buffers), and
 * latency-critical loops that must not stall on the allocator (cudaMalloc can
 * synchronise the device). This entry point runs the same cell solve as a
 * half-sweep (Sinkhorn with the §6.2 stop rule, extraction, BalanceMeasures,
 * Truncate) with all scratch memory in one fixed-size array that the library
 * holds on every device that loads it, from load until process exit (about
 * 1.9 MB).
 *
 * The cell is a 2b×2b block of 4 basic cells of b×b pixels with pixel
 * spacing `spacing` ([0,1]² units). All array arguments are DEVICE pointers
 * owned by the caller:
 *   mu        (2b)² FP64, μ of the cell's pixels, row-major;
 *   y_row, y_col  n_y int32 offsets of the support points of ν_cell from the
 *             cell's top-left pixel, distinct, sorted row-major, each in
 *             (−2048, 2048);
 *   nu        n_y FP64 masses ν_cell(y) > 0 (all masses are fractions of a
 *             total mass 1, as in dd_create). BalanceMeasures needs the cell's
 *             two masses to agree: |Σ nu − Σ mu| ≤ 1e-9·Σ mu + 4·n_y·trunc
 *             (the second term allows for mass that Truncate removed);
 *   alpha     (2b)² FP64, in: warm-start α = ε·log u (any constant offset),
 *             out: the cell's new α (up to a constant);
 *   nu_basic  4·n_y FP64 output, row k = basic cell k (row-major in the 2×2
 *             block): its new Y-marginal on the support points, 0 where
 *             truncated.
 * eps, err_tol (Err), max_iter and trunc as in dd_options. stream: the
 * cudaStream_t to run on (NULL = the legacy default stream). The call
 * returns after the solve has finished on that stream.
 *
 * Limits: b ∈ {2,4,8}; 1 ≤ n_y ≤ 16384; larger inputs are rejected with
 * DD_ERR_ARG before any work is queued, and dd_last_error(NULL) says why.
 * The first call on a device does a one-time set-up with that device
 * current: it resolves the device address of the scratch array
 * (cudaGetSymbolAddress) and raises the cell-solve kernel's shared-memory
 * limit (cudaFuncSetAttribute); make that first call before any stream
 * capture begins. Every call reuses the same array and leaves its own data in
 * it; calls that overlap on the GPU (other streams or host threads) race on
 * it and must be serialised by the caller.
 * Errors: DD_ERR_ARG (sizes, NULL, unsorted or out-of-range support, masses
 * of μ and ν that disagree; for the last two the solve is skipped and alpha
 * and nu_basic are left as they were), DD_ERR_NOT_CONVERGED (the solve
 * stopped at max_iter before its X-error reached ‖μ_J‖·err_tol; alpha and
 * nu_basic hold its result, which is feasible: Σ_k nu_basic[k] = nu),
 * DD_ERR_NUMERIC, DD_ERR_CUDA. */
dd_status dd_solve_cell_noalloc(const double* mu, int32_t b, double spacing, int32_t n_y,
                                const int32_t* y_row, const int32_t* y_col, const double* nu,
                                double eps, double err_tol, int32_t max_iter, double trunc,
                                double* alpha, double* nu_basic, void* stream);

/* Autotuner of the launch schedule (no counterpart in the paper). Runs
 * `rounds` × 9 sweeps of the schedule (real sweeps: they advance the state
 * like dd_sweep), one per candidate of threads_per_cell ∈ {64, 128, 256} ×
 * max_cluster_cells ∈ {0, 64, 256} in turn, times each with CUDA events,
 * scores it by time per unit of algorithmic work (2 FMAs per kernel entry,
 * 64·65/2 per support point of a Newton step) and keeps the best candidate in
 * the context's options (reported in threads, clusters; nullable).
 * 1 ≤ rounds ≤ 16. */
dd_status dd_autotune(dd_ctx* ctx, int32_t rounds, int32_t* threads, int32_t* clusters);

/* ---- learned warm start (no counterpart in the paper) -------------------
 * A network of 1089 inputs, two hidden layers of 256 (ReLU) and 64 outputs,
 * y = W3·relu(W2·relu(W1·x + b1) + b2) + b3, with bfloat16 weights (rounded
 * to nearest even from the FP32 master copy) and FP32 sums. Its input for a
 * cell of 8×8 pixels: 64·μ(x)/‖μ_J‖ on the cell's pixels (row-major),
 * 1024·ν_cell(y)/‖ν_cell‖ on the 32×32 pixel window whose centre pixel (16,16)
 * is the rounded centroid of ν_cell, and log(ε/Δ²). Its output: the cell's
 * dual α in the frame of that centroid (anchor a = round(centroid − 3.5);
 * α̃(i,j) = α − 2Δ²((r₀ − a_r)·i + (c₀ − a_c)·j)), divided by ε, mean zero.
 * Parameters are one FP32 vector: W1 (256×1089 row-major), b1 (256),
 * W2 (256×256), b2, W3 (64×256), b3 (64): dd_mlp_num_params() floats.
 * A network is not thread-safe; calls on one network are serialised. Errors
 * are reported by the status and dd_last_error(NULL). */
typedef struct dd_mlp dd_mlp;

int64_t dd_mlp_num_params(void);
/* New network on the current device from host parameters (copied). */
dd_status dd_mlp_create(const float* params, dd_mlp** out);
void dd_mlp_destroy(dd_mlp* m);
dd_status dd_mlp_get_params(dd_mlp* m, float* params);
dd_status dd_mlp_set_params(dd_mlp* m, const float* params);
/* y[n·64] = network(x[n·1089]); DEVICE pointers, run on `stream`, returns
 * after it finished. 1 ≤ n ≤ 2^24. */
dd_status dd_mlp_forward(dd_mlp* m, const float* x, int64_t n, float* y, void* stream);
/* Mean squared error over the n·64 outputs against t[n·64] and its gradient
 * with respect to the parameters (grad: HOST, dd_mlp_num_params() floats, or
 * NULL). x, t: DEVICE. The rounding of the weights is taken as the identity
 * in the derivative. */
dd_status dd_mlp_loss_grad(dd_mlp* m, const float* x, const float* t, int64_t n, double* loss, float* grad,
                           void* stream);
/* One Adam step (β = 0.9, 0.999, ε = 1e-8) on the mean squared error of the
 * batch; loss (nullable) receives the loss before the step. */
dd_status dd_mlp_train_step(dd_mlp* m, const float* x, const float* t, int64_t n, float lr, double* loss,
                            void* stream);
/* Attach a network to a context (NULL detaches); used when options.warm ≠ 0.
 * The context does not own it: keep it alive while attached. */
dd_status dd_attach_mlp(dd_ctx* ctx, dd_mlp* m);
/* Training pairs of the last half-sweep, one per composite cell of its
 * partition (n_cells of them): features (DEVICE, n_cells·1089 floats) from
 * the ν_cell the cells were solved with, targets (DEVICE, n_cells·64) from
 * the duals the solves returned, ok (DEVICE, n_cells int32) = 1 for cells of
 * 8×8 pixels (the others are not written). cap: rows the buffers hold. */
dd_status dd_cell_training_pairs(dd_ctx* ctx, float* features, float* targets, int32_t* ok, int64_t cap,
                                 int64_t* n_cells);

/* Checkpoint and resume (no counterpart in the paper). dd_save writes the
 * context's state to the file `path`: the images (finest level, fixed point),
 * the schedule and its position, the options (without stream), the basic
 * marginals (ν_i) and the duals of both partitions at the current level, and
 * the iteration counts of the last solves (which order the next launch). An
 * attached network is not saved. The file is in host byte order.
 * dd_load creates a new context (*out) on the current device from such a
 * file; opt = NULL takes the saved options (stream NULL), otherwise *opt.
 * Sweeps after dd_load give the state that the saved context would have
 * reached with the same sweeps, bit for bit.
 * Errors: DD_ERR_ARG for a path that cannot be opened, a failed write, or a
 * file that is not a checkpoint of this library or is truncated or
 * inconsistent (checked before any device memory is allocated); DD_ERR_CUDA /
 * DD_ERR_OOM from the device; dd_last_error(NULL) describes a dd_load
 * failure. */
dd_status dd_save(dd_ctx* ctx, const char* path);
dd_status dd_load(const char* path, const dd_options* opt, dd_ctx** out);

/* Free the context and all device memory it owns. NULL is allowed. */
void dd_destroy(dd_ctx* ctx);

/* Description of the last failure on ctx (never NULL; "" after success).
 * With ctx == NULL: the last failure of dd_create in this thread. */
const char* dd_last_error(const dd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
