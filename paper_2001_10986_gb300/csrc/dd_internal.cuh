// Internal declarations shared by the kernels and the C-ABI host code.
//
// Mass representation: every mass (μ, ν, ν_i entries) is an unsigned 64-bit
// fixed-point number with one unit = 2^-62 of the total mass (total = 2^62).
// Integer sums make Σ_i ν_i(y) = ν(y) exact through gather and extraction,
// which the paper needs after every half-sweep (§6.2: the Y-marginal must be
// reproduced exactly) and which FP64 arithmetic would do only up to rounding
// — at 1/64 of the FP32 rate on this GPU.
//
// Potentials are FP32 in a per-cell frame (see k_sinkhorn): with x = x0 + ξ on
// the cell and y = y_a + η around an anchor pixel y_a, and D = x0 − y_a,
//   c(x,y) = Δ²|D + ξ − η|² = Δ²|D|² + 2Δ²D·ξ − 2Δ²D·η + Δ²|ξ − η|²,
// so f(x) + g(y) − c(x,y) = f̃(ξ) + g̃(η) − Δ²|ξ − η|² with f̃ = f − 2Δ²D·ξ and
// g̃ = g + 2Δ²D·η − Δ²|D|². Only the small quantities f̃, g̃ and |ξ−η|² are held
// in FP32. The stored dual of a cell is α̃(ξ) = α(x) − 2Δ²D·ξ + const together
// with its anchor y_a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ddk {

constexpr int kFixShift = 62;                       // one unit = 2^-62 of the mass
constexpr double kFixOne = 4611686018427387904.0;   // 2^62
constexpr float kFixToFloat = 2.168404344971009e-19f;  // 2^-62

struct LevelView {
  int n;                  // pixels per side at this level
  int nb;                 // basic cells per side
  int b;                  // basic cell side (pixels)
  double spacing;         // Δ: pixel spacing in [0,1]² units
  const uint64_t* mu_q;   // n·n fixed-point μ
  const uint64_t* nu_q;   // n·n fixed-point ν
  const float* mu_f;      // μ as float (true mass)
  const float* log2mu;    // log2 μ
  const uint64_t* M_q;    // nb·nb fixed-point basic-cell masses ‖μ_i‖
};

// geometry of a composite cell (§7.1): a rectangle of nbr×nbc basic cells
struct CellGeom {
  int bi0, bj0;   // first basic cell (row, col)
  int nbr, nbc;   // basic cells per column / row of the cell (1 or 2)
  int r0, c0;     // corner pixel
  int H, W;       // size in pixels
};

// support point of a cell relative to its anchor pixel: two int16 in one word
__device__ __forceinline__ int32_t pack_eta(int r, int c) {
  return (int32_t)((uint32_t)(r & 0xffff) | ((uint32_t)(c & 0xffff) << 16));
}
__device__ __forceinline__ int eta_r(int32_t p) { return (int)(int16_t)(p & 0xffff); }
__device__ __forceinline__ int eta_c(int32_t p) { return (int)(int16_t)((uint32_t)p >> 16); }

__host__ __device__ inline int num_cells(int part, int nb) {
  int m = part == 0 ? nb / 2 : nb / 2 + 1;
  return m * m;
}

__host__ __device__ inline CellGeom cell_geom(int part, int J, int nb, int b) {
  CellGeom g;
  if (part == 0) {
    int m = nb / 2;
    int a = J / m, c = J - (J / m) * m;
    g.bi0 = 2 * a; g.bj0 = 2 * c; g.nbr = 2; g.nbc = 2;
  } else {
    int m = nb / 2 + 1;
    int a = J / m, c = J - (J / m) * m;
    int r_lo = 2 * a - 1 < 0 ? 0 : 2 * a - 1;
    int r_hi = 2 * a > nb - 1 ? nb - 1 : 2 * a;
    int c_lo = 2 * c - 1 < 0 ? 0 : 2 * c - 1;
    int c_hi = 2 * c > nb - 1 ? nb - 1 : 2 * c;
    g.bi0 = r_lo; g.bj0 = c_lo; g.nbr = r_hi - r_lo + 1; g.nbc = c_hi - c_lo + 1;
  }
  g.r0 = g.bi0 * b; g.c0 = g.bj0 * b; g.H = g.nbr * b; g.W = g.nbc * b;
  return g;
}

// composite cell of `part` that contains basic cell (bi, bj)
__host__ __device__ inline int cell_of_basic(int part, int bi, int bj, int nb) {
  if (part == 0) return (bi / 2) * (nb / 2) + bj / 2;
  return ((bi + 1) / 2) * (nb / 2 + 1) + (bj + 1) / 2;
}

// state of one half-sweep
struct SweepArgs {
  LevelView L;
  int part;                 // 0 = A, 1 = B
  int ncells;
  float eps;                // ε ([0,1]² units)
  float err_tol;            // Err
  int max_iter;
  uint64_t trunc_q;         // Truncate threshold in fixed-point units
  // input CSR (natural order)
  const int64_t* rp;
  const int32_t* col;
  const uint64_t* val;
  // workspace (capacity ws_cap entries; cell J owns [cell_off[J], +L_J))
  int64_t ws_cap;
  unsigned long long* ws_counter;
  int64_t* cell_off;
  int32_t* cell_ny;
  int2* anchor_new;
  int32_t* ws_ytmp;
  uint64_t* ws_vtmp;
  int32_t* ws_eta;          // packed (ηr, ηc) int16 pair
  uint64_t* ws_nu;          // ν_cell fixed point
  float* ws_lognu;          // log2 ν_cell (true mass)
  float* ws_g;              // stabiliser / potential G(η) in log2 units
  // dual state of the partition
  float* alpha;             // α̃ per pixel ([0,1]² units)
  int2* anchor;             // anchor pixel per cell
  // outputs (tmp capacity 4·ws_cap)
  int32_t* tmp_col;
  uint64_t* tmp_val;
  int32_t* row_cnt;         // per basic row (natural order)
  int64_t* row_src;         // offset of the row's entries in tmp
  double* cell_cost;
  double* cell_errx;
  int32_t* cell_iters;
  int32_t* cell_newton;     // Newton X-iterations of each cell solve (nullable)
  int newton;               // Newton X-iterations allowed
  int32_t* cell_learned;    // per cell: 1 learned duals used, 0 compared and not used,
                            // −1 not compared (nullable: no prediction this half-sweep)
  int32_t* cell_status;     // bit0 not converged, bit1 non-finite, bit2 workspace overflow,
                            // bit3 converged only at a larger ε in the safeguard
  int escalate;             // the safeguard's launch: solves at 4ε, 16ε, … up to 4^escalate·ε until
                            // one converges (see k_sinkhorn_safeguard); unused elsewhere
  int* err_flag;
  const int32_t* order;     // launch order of the cells (NULL: natural order)
  const int* nbig;          // the first *nbig cells of `order` are solved by clusters (NULL: none)
  int* work_next;           // persistent per-CTA solves: next position of `order` to take
                            // (NULL: one CTA per cell)
  const int* ncells_dev;    // persistent per-CTA solves: number of cells in `order`, read on the
                            // device (NULL: ncells); the safeguard's re-solves use it
  const int* rescued_dev;   // cells re-solved by the safeguard in this half-sweep (NULL: none)
  int max_big;              // upper limit for *nbig (≤ 256)
  int32_t* iters_hist;      // iterations of each cell's last solve in this partition
  int trace_cell;           // debug: cell whose per-iteration error is recorded (-1: none)
  float* trace;             // debug: 2×512 floats (relative X-error, ω) per iteration
  unsigned long long* cell_times;  // debug: per cell [start, end] in ns (NULL: off)
};

// kernel launchers (dd_kernels.cu)
cudaError_t launch_gather(const SweepArgs& a, cudaStream_t s);
cudaError_t launch_order(const SweepArgs& a, int32_t* order, int* nbig, cudaStream_t s);
cudaError_t launch_sinkhorn_cluster(const SweepArgs& a, cudaStream_t s);
// per-CTA cell solves; persistent: one wave of CTAs that take cells from
// a.work_next (which must be 0 at launch) until none are left
cudaError_t launch_sinkhorn(const SweepArgs& a, int threads, cudaStream_t s, bool persistent = false);
// the safeguard's re-solves (a.escalate attempts with growing ε, see
// k_sinkhorn_safeguard) of the cells a.order[0 .. *a.ncells_dev) as one
// persistent wave; a.work_next must be 0 at launch
cudaError_t launch_sinkhorn_safeguard(const SweepArgs& a, int threads, cudaStream_t s);
// exclusive scan of the row lengths into rp_out[0..nrows]; skipped when
// *err_flag (nullable) is non-zero
cudaError_t launch_row_scan(const int32_t* cnt, int64_t* rp_out, int64_t* tile_sum, int nrows, cudaStream_t s,
                            const int* err_flag = nullptr);
// rp_out[i] = tile_off[tile] + prefix within the tile; with tmp_col != NULL the
// kept entries of each row are copied to col_out/val_out (capacity cap_out)
cudaError_t launch_compact(const int32_t* cnt, const int64_t* src, const int64_t* tile_off,
                           int64_t* rp_out, const int32_t* tmp_col, const uint64_t* tmp_val,
                           int32_t* col_out, uint64_t* val_out, int64_t cap_out, int nrows,
                           int* err_flag, cudaStream_t s);
cudaError_t launch_init_product(LevelView L, int64_t* rp, int32_t* col, uint64_t* val, int imax,
                                cudaStream_t s);

struct SweepTotals {
  double cost, errx;
  double kernel_evals;       // Σ_J |X_J|·N_y·(iterations + 1)
  double hessian_fma;        // Σ_J Newton steps · 64²·N_y
  long long iters_sum;
  long long newton_steps;
  int iters_max, not_converged, nonfinite, overflow;
  int learned;               // cells started from the learned duals
  int compared;              // cells whose prediction was compared
  int rescued;               // cells re-solved by the safeguard
  int escalated;             // cells whose plan is that of a larger ε (status bit 3)
};
cudaError_t launch_reduce_cells(const SweepArgs& a, SweepTotals* out_dev, cudaStream_t s);
// §7.2 image of basic marginals (CSR, nrows rows, Y pixels < n2): rgb[3y+k]
// = Σ_i colours[3i+k]·ν_i(y) / Σ_i ν_i(y) (0 where no row reaches y); acc
// (3·n2 doubles) and mass (n2) are scratch
cudaError_t launch_coupling_image(const int64_t* rp, const int32_t* col, const uint64_t* val, int nrows, int n2,
                                  const float* colours, double* acc, unsigned long long* mass, float* rgb,
                                  cudaStream_t s);
// the cells of the half-sweep in `a` whose solve stopped at max_iter (status
// bit 0) with an X-error above min_err·‖μ_J‖ into list[0..*count), for the
// safeguard's re-solves
cudaError_t launch_collect_failed(const SweepArgs& a, int32_t* list, int* count, double min_err, cudaStream_t s);
cudaError_t launch_y_error(LevelView L, const int64_t* rp, const int32_t* col, const uint64_t* val,
                           int nrows, unsigned long long* scratch, double* out_dev, cudaStream_t s);

// refinement (§6.4): fine rows from coarse rows
struct RefineArgs {
  LevelView C, F;           // coarse and fine level (same b)
  const int64_t* rp_c;
  const int32_t* col_c;
  const uint64_t* val_c;
  const int64_t* rp_f;      // after scan
  int32_t* cnt_f;
  int32_t* col_f;
  uint64_t* val_f;
};
cudaError_t launch_refine_count(const RefineArgs& r, cudaStream_t s);
cudaError_t launch_refine_write(const RefineArgs& r, cudaStream_t s);
// dual refinement: coarse α̃/anchors of partition `cpart` → fine α̃/anchors of `fpart`
cudaError_t launch_refine_duals(LevelView C, LevelView F, int cpart, const float* alpha_c,
                                const int2* anchor_c, int fpart, float* alpha_f, int2* anchor_f,
                                cudaStream_t s);

// plan reconstruction: counts per X pixel, then values
// objective of the last partition's coupling: per cell (primal, gap) into
// cell_obj[2·ncells], then out[3] = {Σ primal, Σ gap, Σ |gap|}
cudaError_t launch_objective(const SweepArgs& a, double* cell_obj, double* out, cudaStream_t s);
cudaError_t launch_plan(const SweepArgs& a, float trunc, const int64_t* xrp, int32_t* xcnt,
                        int32_t* pcol, double* pval, int write, cudaStream_t s);

// ---- learned warm start (cells of 8×8 pixels) ----
constexpr int kMlpIn = 1089, kMlpHidden = 256, kMlpOut = 64;
// features of every 8×8 cell of the half-sweep in `a` (after the gather):
// feat[J·1089 + …], the anchor of the ν_cell centroid frame, ok[J] ∈ {0, 1}
cudaError_t launch_cell_features(const SweepArgs& a, float* feat, int2* fanchor, int32_t* ok,
                                 cudaStream_t s);
// targets of the same cells from the duals after the solve: tgt[J·64 + …]
cudaError_t launch_cell_targets(const SweepArgs& a, const int2* fanchor, const int32_t* ok, float* tgt,
                                cudaStream_t s);
// comparison: per 8×8 cell, the X-error after one Y-iteration from the current
// duals and from the prediction pred[J·64 + …]; the better one is written to
// a.alpha and a.cell_learned[J] records the choice
cudaError_t launch_warm_compare(const SweepArgs& a, const float* pred, const int2* fanchor, const int32_t* ok,
                         cudaStream_t s);

// ---- dual gluing (§6.3) and eq. RelPDGap (dd_gluing.cu) ----
struct GlueInfo {
  int iters;            // CG iterations run
  int converged;        // 1 if the relative residual reached the tolerance
  double rel_residual;  // ‖L V + Dᵀ log q‖ / ‖Dᵀ log q‖ at the end
};
// largest side na of the A-cell grid that the one-cluster CG holds
int glue_max_cells_per_side();
// s±_i of every basic cell (sp, sm: nb² doubles) from the duals of both
// partitions, then the potential V (na² doubles, mean zero) of the gluing
// graph by preconditioned CG to ‖residual‖ ≤ tol·‖rhs‖ or max_iter
// iterations; cudaErrorInvalidValue when na exceeds glue_max_cells_per_side()
cudaError_t launch_glue_potential(LevelView L, const float* alpha_A, const int2* anchor_A, const float* alpha_B,
                                  const int2* anchor_B, double eps, double tol, int max_iter, double* sp,
                                  double* sm, double* V, GlueInfo* info, cudaStream_t s);
// α̂ = α_A + ε·V[A cell] (absolute frame, n² doubles); pixels without mass
// get 0, or with fill_massless the affine fit of their A cell's α̂
cudaError_t launch_glue_apply(LevelView L, const float* alpha_A, const int2* anchor_A, const double* V, double eps,
                              int fill_massless, double* alpha_hat, cudaStream_t s);
// α̂ (n_c² doubles) interpolated linearly onto level F (n_f = 2·n_c) and
// written into the cell frames (α̃, anchors) of partition fpart of F
cudaError_t launch_glue_frames(int n_c, const double* alpha_c, LevelView F, int fpart, float* alpha_f,
                               int2* anchor_f, cudaStream_t s);
// eq. RelPDGap's dual terms for the coupling of the half-sweep in `a`
// (after its gather) and the glued X-dual α̂: out[4] = {Σ_x μ α̂/ε,
// −Σ_y ν log S(y), Σ_{y: S > 0} ν(y), #{y: ν(y) > 0, S(y) = 0}}; tws (one
// double per support entry), Mkey and St (n² each) and part (4·nparts) are
// scratch
cudaError_t launch_gap(const SweepArgs& a, const double* alpha_hat, double* tws, long long* Mkey, double* St,
                       double* part, int nparts, double* out, cudaStream_t s);

}  // namespace ddk

struct dd_mlp;
namespace ddk {
// network output y[n·64] for inputs x[n·1089] (device), on stream s
cudaError_t mlp_forward(dd_mlp* m, const float* x, int64_t n, float* y, cudaStream_t s);
}  // namespace ddk

// sets the message returned by dd_last_error(NULL) in this thread
void dd_set_noalloc_error(const char* msg);
