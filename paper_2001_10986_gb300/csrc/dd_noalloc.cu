// dd_solve_cell_noalloc: one composite-cell solve that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a
// solve: hosts whose device memory belongs to another runtime or pool that
// forbids allocations behind its back (a plug-in inside a framework that
// hands out only pre-allocated buffers), and latency-critical loops that must
// not stall on cudaMalloc, which can synchronise the device and take locks.
// For them this entry point runs the library's cell solve (the same
// k_sinkhorn kernel as a half-sweep) with all of its scratch memory in one
// file-scope __device__ array of fixed size. The caller passes device
// pointers for every input and output.
//
// The scratch array is a single buffer per device, held from library load to
// process exit. Its device address is resolved once per device, by the first
// call on that device (cudaGetSymbolAddress with that device current); that
// first call should come before any stream capture begins. Every call uses
// the array and leaves its own data in it; the kernels below rewrite what
// they read before reading it. Calls that overlap on the GPU (from different
// streams or host threads) race on it; callers serialise them.
#include "dd.h"
#include "dd_internal.cuh"

#include <cstdio>
#include <mutex>
#include <string>

using namespace ddk;

namespace {

// ---- the virtual level the cell is placed in -------------------------------
// The solve kernel indexes pixels, basic cells and composite cells of a
// level. The cell is placed at pixel (kCorner, kCorner) of a virtual level of
// kSide×kSide pixels, and every array the kernel touches is a view whose
// origin is shifted so that the few indices the cell uses fall inside the
// scratch array. Support points may lie up to kCorner pixels away from the
// cell corner in each direction.
constexpr int kSide = 4096;
constexpr int kCorner = 2048;
constexpr int kMaxNy = 16384;                       // support points per call
constexpr int kMaxB = 8;
constexpr int kXSpan = (2 * kMaxB - 1) * kSide + 2 * kMaxB;  // pixel indices of one cell
constexpr int kBasicSpan = kSide / 2 + 2;           // basic-cell indices of one cell (b ≥ 2)

struct Scratch {
  float mu_f[kXSpan];
  float log2mu[kXSpan];
  float alpha[kXSpan];
  uint64_t M_q[kBasicSpan];
  int64_t row_src[kBasicSpan];
  int32_t row_cnt[kBasicSpan];
  int32_t ws_eta[kMaxNy];
  uint64_t ws_nu[kMaxNy];
  float ws_g[kMaxNy];
  int32_t tmp_col[4 * kMaxNy];
  uint64_t tmp_val[4 * kMaxNy];
  int64_t cell_off;
  double cell_cost, cell_errx;
  int2 anchor, anchor_new;
  int2 flags;               // {err_flag, cell_status}: read back together
  int32_t cell_ny, cell_iters, order;
  unsigned long long ws_counter;
};

__device__ __align__(256) Scratch g_noalloc_scratch;

std::mutex g_mutex;
Scratch* g_scratch_addr[64] = {nullptr};

struct Geometry {
  int b, nb, J, bi_base, p_base;
};

__host__ __device__ inline Geometry geometry(int b) {
  Geometry q;
  q.b = b;
  q.nb = kSide / b;
  q.J = (kCorner / (2 * b)) * (q.nb / 2) + kCorner / (2 * b);
  q.bi_base = (kCorner / b) * q.nb + kCorner / b;
  q.p_base = kCorner * kSide + kCorner;
  return q;
}

__device__ double block_sum_d(double v, double* ws) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
  __syncthreads();
  return t;
}

// inputs → scratch: masses in fixed point, anchor, frame of the duals. A
// rejected input (err_flag 16: support; 32: masses of μ and ν disagree) sets
// cell_off = −1, so the solve kernel returns at once and k_noalloc_finish
// leaves the caller's buffers untouched.
__global__ void k_noalloc_prep(Scratch* S, int b, double spacing, const double* mu, int n_y,
                               const int32_t* y_row, const int32_t* y_col, const double* nu,
                               const double* alpha, double trunc) {
  __shared__ double ws[32];
  __shared__ int s_anchor[2];
  __shared__ unsigned long long s_mq[4];
  const Geometry q = geometry(b);
  const int H = 2 * b;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S->flags = make_int2(0, 0);
    S->cell_off = 0;
    S->cell_ny = n_y;
    S->order = q.J;
    S->ws_counter = 0;
  }
  // basic-cell masses and per-pixel μ
  for (int x = tid; x < H * H; x += blockDim.x) {
    const int ar = x / H, ac = x % H;
    const double m = mu[x];
    const int p = ar * kSide + ac;
    S->mu_f[p] = (float)m;
    S->log2mu[p] = m > 0.0 ? (float)log2(m) : -1.0e30f;
  }
  for (int i = tid; i < 4; i += blockDim.x) {
    const int kr = i / 2, kc = i % 2;
    unsigned long long s = 0;
    for (int r = 0; r < b; ++r)
      for (int c = 0; c < b; ++c) s += __double2ull_rn(mu[(kr * b + r) * H + kc * b + c] * kFixOne);
    const int slot = kr * q.nb + kc;
    S->M_q[slot] = s;
    s_mq[i] = s;
  }
  // support: fixed-point ν, validity, centroid
  double sw = 0.0, sr = 0.0, sc = 0.0, sq = 0.0;
  int bad = 0;
  for (int k = tid; k < n_y; k += blockDim.x) {
    const int yr = y_row[k], yc = y_col[k];
    const double v = nu[k];
    if (yr <= -kCorner || yr >= kCorner || yc <= -kCorner || yc >= kCorner || !(v > 0.0)) bad = 1;
    if (k > 0 && (y_row[k - 1] > yr || (y_row[k - 1] == yr && y_col[k - 1] >= yc))) bad = 1;
    S->ws_nu[k] = __double2ull_rn(v * kFixOne);
    sq += (double)S->ws_nu[k];
    sw += v;
    sr += v * yr;
    sc += v * yc;
  }
  if (bad) atomicOr(&S->flags.x, 16);
  sw = block_sum_d(sw, ws);
  sr = block_sum_d(sr, ws);
  sc = block_sum_d(sc, ws);
  sq = block_sum_d(sq, ws);
  if (tid == 0) {
    // BalanceMeasures needs ‖ν_cell‖ = ‖μ_J‖; Truncate may have removed up to
    // trunc per entry of the four basic marginals from a previous solve
    const double mq = (double)s_mq[0] + (double)s_mq[1] + (double)s_mq[2] + (double)s_mq[3];
    if (!(fabs(sq - mq) <= 1e-9 * mq + 4.0 * n_y * trunc * kFixOne)) atomicOr(&S->flags.x, 32);
    if (S->flags.x & (16 | 32)) S->cell_off = -1;
    const double cr = sw > 0 ? sr / sw : 0.0, cc = sw > 0 ? sc / sw : 0.0;
    s_anchor[0] = kCorner + (int)lrint(cr - 0.5 * (H - 1));
    s_anchor[1] = kCorner + (int)lrint(cc - 0.5 * (H - 1));
    S->anchor = make_int2(s_anchor[0], s_anchor[1]);
    S->anchor_new = S->anchor;
  }
  __syncthreads();
  const int ar0 = s_anchor[0], ac0 = s_anchor[1];
  for (int k = tid; k < n_y; k += blockDim.x) {
    const int er = kCorner + y_row[k] - ar0, ec = kCorner + y_col[k] - ac0;
    S->ws_eta[k] = (int32_t)((uint32_t)(er & 0xffff) | ((uint32_t)(ec & 0xffff) << 16));
  }
  // α in the cell frame: α̃(ξ) = α(x) − α(corner) − 2Δ²D·ξ, D = corner − anchor
  const double d2 = spacing * spacing;
  const int Dr = kCorner - ar0, Dc = kCorner - ac0;
  const double a00 = alpha[0];
  for (int x = tid; x < H * H; x += blockDim.x) {
    const int ar = x / H, ac = x % H;
    S->alpha[ar * kSide + ac] = (float)(alpha[x] - a00 - 2.0 * d2 * ((double)Dr * ar + (double)Dc * ac));
  }
}

// scratch → outputs: dense basic marginals on the support, α in the caller's frame
__global__ void k_noalloc_finish(Scratch* S, int b, double spacing, int n_y, const int32_t* y_row,
                                 const int32_t* y_col, double* alpha, double* nu_basic) {
  const Geometry q = geometry(b);
  const int H = 2 * b;
  if (S->flags.x & (16 | 32)) return;   // rejected input: outputs untouched
  for (int e = threadIdx.x; e < 4 * n_y; e += blockDim.x) nu_basic[e] = 0.0;
  __syncthreads();
  for (int i = 0; i < 4; ++i) {
    const int slot = (i / 2) * q.nb + (i % 2);
    const int cnt = S->row_cnt[slot];
    const int64_t src = S->row_src[slot];
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int code = S->tmp_col[src + e];
      const int yr = code / kSide - kCorner, yc = code % kSide - kCorner;
      int lo = 0, hi = n_y;
      while (lo < hi) {   // first support point not before (yr, yc)
        const int m = (lo + hi) >> 1;
        if (y_row[m] < yr || (y_row[m] == yr && y_col[m] < yc)) lo = m + 1; else hi = m;
      }
      if (lo < n_y && y_row[lo] == yr && y_col[lo] == yc)
        nu_basic[(int64_t)i * n_y + lo] = (double)S->tmp_val[src + e] * (1.0 / kFixOne);
    }
  }
  const double d2 = spacing * spacing;
  const int Dr = kCorner - S->anchor.x, Dc = kCorner - S->anchor.y;
  for (int x = threadIdx.x; x < H * H; x += blockDim.x) {
    const int ar = x / H, ac = x % H;
    alpha[x] = (double)S->alpha[ar * kSide + ac] + 2.0 * d2 * ((double)Dr * ar + (double)Dc * ac);
  }
}

dd_status fail(const std::string& m, dd_status st = DD_ERR_ARG) {
  dd_set_noalloc_error(m.c_str());
  return st;
}

}  // namespace

extern "C" dd_status dd_solve_cell_noalloc(const double* mu, int32_t b, double spacing, int32_t n_y,
                                           const int32_t* y_row, const int32_t* y_col, const double* nu,
                                           double eps, double err_tol, int32_t max_iter, double trunc,
                                           double* alpha, double* nu_basic, void* stream) {
  if (!mu || !y_row || !y_col || !nu || !alpha || !nu_basic) return fail("NULL argument");
  if (b != 2 && b != 4 && b != 8) return fail("b must be 2, 4 or 8");
  if (n_y < 1 || n_y > kMaxNy)
    return fail("n_y must be in [1, " + std::to_string(kMaxNy) + "] (fixed scratch size of this entry point)");
  if (!(eps > 0) || !(spacing > 0) || !(err_tol > 0) || max_iter < 1 || !(trunc >= 0))
    return fail("eps, spacing and err_tol must be positive, max_iter >= 1, trunc >= 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail("no current CUDA device", DD_ERR_CUDA);
  Scratch* S = nullptr;
  {
    // first call on a device: resolve the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), DD_ERR_CUDA);
      g_scratch_addr[dev] = (Scratch*)p;
    }
    S = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const Geometry q = geometry(b);

  k_noalloc_prep<<<1, 256, 0, st>>>(S, b, spacing, mu, n_y, y_row, y_col, nu, alpha, trunc);

  // views: shift each array so that the cell's level indices land in S
  SweepArgs a{};
  a.L.n = kSide;
  a.L.nb = q.nb;
  a.L.b = b;
  a.L.spacing = spacing;
  a.L.mu_q = nullptr;
  a.L.nu_q = nullptr;
  a.L.mu_f = S->mu_f - q.p_base;
  a.L.log2mu = S->log2mu - q.p_base;
  a.L.M_q = S->M_q - q.bi_base;
  a.part = 0;
  a.ncells = 1;
  a.eps = (float)eps;
  a.err_tol = (float)err_tol;
  a.max_iter = max_iter;
  const double tq = trunc * kFixOne;
  a.trunc_q = tq >= 1.8e19 ? ~0ull : (uint64_t)tq;
  a.ws_cap = kMaxNy;
  a.ws_counter = &S->ws_counter;
  a.cell_off = &S->cell_off - q.J;
  a.cell_ny = &S->cell_ny - q.J;
  a.anchor_new = &S->anchor_new - q.J;
  a.ws_eta = S->ws_eta;
  a.ws_nu = S->ws_nu;
  a.ws_g = S->ws_g;
  a.alpha = S->alpha - q.p_base;
  a.anchor = &S->anchor - q.J;
  a.tmp_col = S->tmp_col;
  a.tmp_val = S->tmp_val;
  a.row_cnt = S->row_cnt - q.bi_base;
  a.row_src = S->row_src - q.bi_base;
  a.cell_cost = &S->cell_cost - q.J;
  a.cell_errx = &S->cell_errx - q.J;
  a.cell_iters = &S->cell_iters - q.J;
  a.newton = 1;
  a.cell_status = &S->flags.y - q.J;
  a.err_flag = &S->flags.x;
  a.order = &S->order;
  a.nbig = nullptr;
  a.max_big = 0;
  a.iters_hist = nullptr;
  a.trace_cell = -1;
  a.trace = nullptr;
  a.cell_times = nullptr;
  cudaError_t e = launch_sinkhorn(a, 128, st);
  if (e != cudaSuccess) return fail(std::string("launch: ") + cudaGetErrorString(e), DD_ERR_CUDA);
  k_noalloc_finish<<<1, 256, 0, st>>>(S, b, spacing, n_y, y_row, y_col, alpha, nu_basic);
  int2 flags = make_int2(0, 0);   // {err_flag, cell_status}
  e = cudaMemcpyAsync(&flags, &S->flags, sizeof(int2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(std::string("CUDA: ") + cudaGetErrorString(e), DD_ERR_CUDA);
  if (flags.x & 16) return fail("support points must be distinct, row-major sorted, within 2047 pixels of the corner, with nu > 0");
  if (flags.x & 32) return fail("the masses of mu and nu over the cell must agree (1e-9 relative + 4 n_y trunc)");
  if (flags.x & 2) return fail("the cell solve produced a non-finite value", DD_ERR_NUMERIC);
  if (flags.y & 1) return fail("the cell solve stopped at max_iter before reaching err_tol", DD_ERR_NOT_CONVERGED);
  dd_set_noalloc_error("");
  return DD_OK;
}
