// CUDA kernels of one half-sweep of Algorithm 2 (§6.1) and of the
// multi-scale driver (§6.4), written for sm_103a.
//
//   k_gather    ν_cell = Σ_{i∈J} ν_i: sorted union of ≤4 sparse rows by
//               merge-path ranks, then duplicate folding (Algorithm 2).
//   k_sinkhorn  cell Sinkhorn in log2 form with the §6.2 stop rule, then
//               extraction ν_i = P_Y(π_cell|X_i×Y), BalanceMeasures and
//               Truncate with in-row stream compaction.
//   k_scan_*    prefix sums of the kept row lengths → new row offsets.
//   k_compact   copies kept entries into the new CSR.
//   k_refine_*  eq. FineBasicMarginals and the dual initialisation at the
//               next level.
//
// All kernels are plain launches; none of them waits on another CTA.
#include <algorithm>
#include <atomic>
#include "dd_internal.cuh"

#include <cooperative_groups.h>

#include <cfloat>
#include <cstdint>

namespace cg = cooperative_groups;

namespace ddk {

namespace {

constexpr float kLn2 = 0.69314718055994530942f;
constexpr float kNegBig = -1.0e30f;

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// packed pairs of FP32 values and the f32x2 arithmetic of sm_100-class GPUs
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}


// exclusive scan of one int per thread over the block; returns the prefix,
// writes the block total. `ws` holds ≥ 32 ints.
__device__ int block_exscan(int v, int* ws, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  __syncthreads();
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) ws[lane] = w;
  }
  __syncthreads();
  int before = warp > 0 ? ws[warp - 1] : 0;
  total = ws[nw - 1];
  __syncthreads();
  return before + x - v;
}

template <typename T>
__device__ T block_sum(T v, T* ws) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  T t = 0;
  for (int w = 0; w < nw; ++w) t += ws[w];
  __syncthreads();
  return t;
}

// block sum with one barrier: ws holds two buffers of 32 used alternately, so
// a buffer is rewritten only after every thread has passed the barrier of the
// following call
__device__ __forceinline__ float block_sum1(float v, float* ws, int& phase) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  float* buf = ws + 32 * phase;
  if (lane == 0) buf[warp] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < nw; ++w) t += buf[w];
  phase ^= 1;
  return t;
}

// number of elements < y (strict) or <= y in a sorted int row
__device__ __forceinline__ int64_t lower_bound_row(const int32_t* a, int64_t n, int y) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if (a[m] < y) lo = m + 1; else hi = m;
  }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_row(const int32_t* a, int64_t n, int y) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    if (a[m] <= y) lo = m + 1; else hi = m;
  }
  return lo;
}

__device__ __forceinline__ uint64_t frac_to_u64(float f) {
  // f in [0,1] → round-down fixed point of f·2^64, clamped below 2^64
  if (!(f > 0.0f)) return 0ull;
  if (f >= 1.0f) return 0xffffffffffffffffull;
  return __float2ull_rz(f * 18446744073709551616.0f);
}

}  // namespace

// ---------------------------------------------------------------------------
// S1: gather ν_cell = Σ_{i∈J} ν_i (Algorithm 2)
// ---------------------------------------------------------------------------
constexpr int kGatherStage = 3072;   // entries of a cell's rows staged in shared memory
constexpr int kGatherThreads = 256;  // threads of a gather CTA

__global__ void __launch_bounds__(kGatherThreads) k_gather(SweepArgs a) {
  const int J = blockIdx.x;
  if (*a.err_flag) return;
  const LevelView& L = a.L;
  const CellGeom g = cell_geom(a.part, J, L.nb, L.b);
  __shared__ int64_t rs[4];
  __shared__ int64_t rl[4];
  __shared__ int64_t rb[4];   // start of each row in the staged copy
  __shared__ int32_t s_col[kGatherStage];
  __shared__ uint64_t s_val[kGatherStage];
  __shared__ int nrows;
  __shared__ int64_t s_off, s_tot;
  __shared__ int s_anchor[2];
  __shared__ float fred[32];
  __shared__ int iws[32];

  if (threadIdx.x == 0) {
    int k = 0;
    int64_t tot = 0;
    for (int kr = 0; kr < g.nbr; ++kr)
      for (int kc = 0; kc < g.nbc; ++kc) {
        int bi = (g.bi0 + kr) * L.nb + g.bj0 + kc;
        rs[k] = a.rp[bi];
        rl[k] = a.rp[bi + 1] - a.rp[bi];
        rb[k] = tot;
        tot += rl[k];
        ++k;
      }
    nrows = k;
    unsigned long long off = atomicAdd(a.ws_counter, (unsigned long long)tot);
    int64_t o = (int64_t)off;
    if (o + tot > a.ws_cap) {
      o = -1;
      atomicOr(a.err_flag, 4);
    }
    s_off = o;
    s_tot = tot;
    a.cell_off[J] = o;
  }
  __syncthreads();
  const int64_t off = s_off, tot = s_tot;
  if (off < 0) return;
  // the rows, concatenated, in shared memory when they fit: the binary
  // searches below then read shared memory instead of L2
  const bool staged = tot <= kGatherStage;
  if (staged) {
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      int r = 0;
      int64_t k = e;
      while (k >= rl[r]) { k -= rl[r]; ++r; }
      s_col[e] = a.col[rs[r] + k];
      s_val[e] = a.val[rs[r] + k];
    }
    __syncthreads();
  }

  // merge-path rank of every element of the ≤4 sorted rows; staged: the
  // merged order replaces the staged copy in shared memory
  float sw = 0.f, sr = 0.f, sc = 0.f;
  auto rank_of = [&](int64_t e, int& y, uint64_t& v) {
    int r = 0;
    int64_t k = e;
    while (k >= rl[r]) { k -= rl[r]; ++r; }
    y = staged ? s_col[e] : a.col[rs[r] + k];
    v = staged ? s_val[e] : a.val[rs[r] + k];
    int64_t rank = k;
    for (int r2 = 0; r2 < nrows; ++r2) {
      if (r2 == r) continue;
      const int32_t* row = staged ? s_col + rb[r2] : a.col + rs[r2];
      rank += (r2 < r) ? upper_bound_row(row, rl[r2], y) : lower_bound_row(row, rl[r2], y);
    }
    const float vf = (float)v * kFixToFloat;
    const int yr = y / L.n, yc = y - (y / L.n) * L.n;
    sw += vf;
    sr += vf * (float)yr;
    sc += vf * (float)yc;
    return rank;
  };
  if (staged) {
    constexpr int kPer = kGatherStage / kGatherThreads;
    int my_y[kPer], my_rank[kPer];
    uint64_t my_v[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t e = threadIdx.x + (int64_t)q * kGatherThreads;
      my_rank[q] = -1;
      if (e < tot) my_rank[q] = (int)rank_of(e, my_y[q], my_v[q]);
    }
    __syncthreads();   // every search of the staged rows is done
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (my_rank[q] >= 0) {
        s_col[my_rank[q]] = my_y[q];
        s_val[my_rank[q]] = my_v[q];
      }
  } else {
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      int y;
      uint64_t v;
      const int64_t rank = rank_of(e, y, v);
      a.ws_ytmp[off + rank] = y;
      a.ws_vtmp[off + rank] = v;
    }
  }
  sw = block_sum(sw, fred);
  sr = block_sum(sr, fred);
  sc = block_sum(sc, fred);
  if (threadIdx.x == 0) {
    // anchor so that η ≈ ξ for the bulk of the cell's mass
    float cr = sw > 0.f ? sr / sw : (float)g.r0;
    float cc = sw > 0.f ? sc / sw : (float)g.c0;
    s_anchor[0] = __float2int_rn(cr - 0.5f * (float)(g.H - 1));
    s_anchor[1] = __float2int_rn(cc - 0.5f * (float)(g.W - 1));
    a.anchor_new[J] = make_int2(s_anchor[0], s_anchor[1]);
  }
  __syncthreads();
  const int ya = s_anchor[0], yc0 = s_anchor[1];

  // fold duplicates, keep sorted order
  int carry = 0;
  for (int64_t base = 0; base < tot; base += blockDim.x) {
    const int64_t p = base + threadIdx.x;
    int head = 0;
    int y = 0;
    const int32_t* my = staged ? s_col : a.ws_ytmp + off;
    const uint64_t* mv = staged ? s_val : a.ws_vtmp + off;
    if (p < tot) {
      y = my[p];
      head = (p == 0) || (my[p - 1] != y);
    }
    int chunk_total;
    int u = block_exscan(head, iws, chunk_total);
    if (head) {
      uint64_t s = mv[p];
      for (int64_t q = p + 1; q < tot && my[q] == y; ++q) s += mv[q];
      const int64_t w = off + carry + u;
      const int yr = y / L.n, yc = y - (y / L.n) * L.n;
      a.ws_eta[w] = pack_eta(yr - ya, yc - yc0);
      a.ws_nu[w] = s;
      a.ws_lognu[w] = log2f((float)s * kFixToFloat);
    }
    carry += chunk_total;
  }
  if (threadIdx.x == 0) a.cell_ny[J] = carry;
}

// ---------------------------------------------------------------------------
// S2-S5: cell Sinkhorn + extraction + BalanceMeasures + Truncate
// ---------------------------------------------------------------------------
// Stabilised Sinkhorn with absorption (the log-domain stabilisation that the
// paper takes from its reference implementation, §7.3 "Numerical
// stability"): the plan of a cell is
//     π(x,y) = u(x) · K̃(x,y) · v(y),   K̃(x,y) = 2^(F(ξ) + Gs(η) − κ|ξ−η|²),
// with log2-unit stabilisers F (per pixel, from the stored dual α̃) and Gs
// (per support point), κ = Δ²/(ε ln 2), and scalings u, v near 1.
//   Y-iteration: s(y) = Σ_x K̃ u, v(y) = ν(y)/s(y);
//   X-marginal:  P_X π(x) = u(x) Σ_y K̃ v;   X-iteration: u ← u·μ/P_X π.
// The stabilisers stay fixed while u, v stay in [2^-16, 2^16], so K̃ is
// recomputed bit-identically in every pass and the scalings converge to FP32
// precision; a scaling that leaves that band is absorbed into its stabiliser.
// The first pass of a solve sets Gs = −max_x(F − κc̃) and absorbs v.
//
// Thread layout: each support point y is handled by a group of G consecutive
// threads; thread g of the group owns RPT = 16/W pixel rows (16 pixels) of
// the H×W cell.

constexpr int kMaxHW = 256;
constexpr int kTraceLen = 512;
constexpr int kStagnationPeriod = 128;     // iterations between stagnation checks (a power of 2)
constexpr float kStagnationRatio = 0.999f;  // error ratio over one period that counts as stagnation
constexpr float kSafeguardFactor = 4.0f;   // ε factor of each safeguard attempt
constexpr int kClusterCTAs = 8;    // CTAs sharing one large cell
constexpr int kMaxBig = 256;       // cells solved by clusters per launch
constexpr int kStageSmall = 1408;  // support points staged in shared memory per CTA (per-CTA solves)
constexpr int kStageBig = 3840;    // … and per CTA of a cluster
constexpr int kNewtonN = 64;       // pixels of a cell that takes Newton steps
constexpr int kNewtonLd = kNewtonN + 1;
// shared floats of the Newton step: the 64×65 matrix C, then M; a batch of
// up to 64 rows z_y; the right-hand side / step
constexpr int kNewtonZ = kNewtonN * kNewtonLd;
// row stride of the batch rows z_y: 72 floats puts the 32 lanes of every
// tensor-core fragment load on 32 distinct shared-memory banks
constexpr int kZs = kNewtonN + 8;
constexpr int kNewtonB = kNewtonZ + 64 * kZs;
constexpr int kNewtonFloats = kNewtonB + kNewtonN + 1;
// largest |δ| of one Newton step in log u; a longer step is scaled down
constexpr float kNewtonMaxStep = 4.0f;
// Newton steps start only once the X-error is below this fraction of ‖μ_J‖
constexpr float kNewtonNear = 0.05f;
constexpr float kTwoTau = 65536.0f;   // scalings leave the band [2^-16, 2^16] → absorb

struct SinkSmem {
  alignas(16) float WT[kMaxHW];   // 2^res·u of the separable split
  float F[kMaxHW];
  float u[kMaxHW];
  float l2mu[kMaxHW];
  float mu[kMaxHW];
  float PX[kMaxHW];
  float PXp[kMaxHW];     // this CTA's partial Σ_y K̃ v (read by the other CTAs of a cluster)
  float red[8][kMaxHW];
  float fws[32];
  float fws2[64];      // two buffers for single-barrier block sums
  int iws[32];
  unsigned long long uws[32];
  double dws[32];
  uint64_t q64[4];
  uint64_t w64[4];
  int nsur, ndef;
  int sur[4], def[4];
};

// lanes tid % 32 rounded down to a multiple of G … +G−1 form one group; a
// group may take a branch the rest of the warp does not, so the shuffles name
// only the group's lanes
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G >= 32) {
    return 0xffffffffu;
  } else {
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(G - 1));
  }
}
template <int G>
__device__ __forceinline__ float group_sum(float v) {
  const unsigned mask = group_mask<G>();
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ float group_max(float v) {
  const unsigned mask = group_mask<G>();
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o));
  return v;
}

// Sum v[0..N) over the lanes of a warp that share lane % G (all lanes take
// part). Afterwards the lane holds ScatterShape<N, G>::nv fully reduced values,
// for thread-local indices base + j; where fewer values than lanes remain,
// several lanes hold the same values and only ScatterShape::writer lanes
// store them.
template <int M, int CNT, int G, int N>
__device__ __forceinline__ void reduce_scatter_stage(float (&v)[N], int lane, int& base) {
  if constexpr (M >= G) {
    if constexpr (CNT > 1) {
      constexpr int half = CNT / 2;
      const bool up = (lane & M) != 0;
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float send = up ? v[j] : v[j + half];
        const float keep = up ? v[j + half] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, M);
      }
      if (up) base += half;
      reduce_scatter_stage<M / 2, half, G, N>(v, lane, base);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], M);
      reduce_scatter_stage<M / 2, 1, G, N>(v, lane, base);
    }
  }
}
template <int N, int G>
__device__ __forceinline__ int warp_reduce_scatter(float (&v)[N], int lane) {
  int base = 0;
  reduce_scatter_stage<16, N, G, N>(v, lane, base);
  return base;
}
constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
template <int N, int G>
struct ScatterShape {
  static constexpr int stages = 5 - ilog2c(G);
  static constexpr int lgN = ilog2c(N);
  static constexpr int plain = stages > lgN ? stages - lgN : 0;
  static constexpr int nv = stages >= lgN ? 1 : (N >> stages);
  __device__ static bool writer(int lane) { return ((lane / G) & ((1 << plain) - 1)) == 0; }
};

// largest |res| of the separable split of the stabiliser for which the
// factorised kernel is used (see sinkhorn_cell)
constexpr float kResMax = 24.0f;

__device__ __forceinline__ uint32_t f2tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Σ_y z_y z_yᵀ over a batch of nys rows z_y (64 floats each, row stride kZs
// at nbuf + kNewtonZ; nys a multiple of 8) added into C (stride kNewtonLd at
// nbuf), on the tensor cores (mma.sync m16n8k8, TF32 inputs, FP32 sums):
// A = Zᵀ (16 rows of C per tile), B = Z (8 columns per tile). Only the 20
// tiles of 16×8 that touch the lower triangle are formed (the diagonal 16×16
// blocks in full); the upper triangle is mirrored after the pass. The Newton
// step needs its Hessian only approximately: its right-hand side (μ − P_X π)
// is exact in FP32, so the step keeps the fixed point and the stopping rule,
// and a Hessian with relative errors of about 1e-3 still contracts fast.
__device__ __forceinline__ void hess_batch_mma(float* nbuf, int nys, int tid, int nthreads) {
  const int lane = tid & 31, warp = tid >> 5, nw = nthreads >> 5;
  const int g = lane >> 2, t = lane & 3;
  const float* Z = nbuf + kNewtonZ;
  for (int p = warp; p < 20; p += nw) {
    // tile p → row block mt (16 rows), column block nt ≤ 2·mt + 1 (8 columns)
    const int mt = p < 2 ? 0 : p < 6 ? 1 : p < 12 ? 2 : 3;
    const int nt = p - mt * (mt + 1);
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    for (int k0 = 0; k0 < nys; k0 += 8) {
      const float* z0 = Z + (k0 + t) * kZs;
      const float* z4 = Z + (k0 + t + 4) * kZs;
      const uint32_t a0 = f2tf32(z0[16 * mt + g]), a1 = f2tf32(z0[16 * mt + g + 8]);
      const uint32_t a2 = f2tf32(z4[16 * mt + g]), a3 = f2tf32(z4[16 * mt + g + 8]);
      const uint32_t b0 = f2tf32(z0[8 * nt + g]), b1 = f2tf32(z4[8 * nt + g]);
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    float* cp = nbuf + (16 * mt + g) * kNewtonLd + 8 * nt + 2 * t;
    cp[0] += c0;
    cp[1] += c1;
    cp[8 * kNewtonLd] += c2;
    cp[8 * kNewtonLd + 1] += c3;
  }
}

// H×W: the cell's shape in pixels. CS > 1: a cluster of CS CTAs shares one
// cell; CTA `rank` takes a contiguous chunk of the support points, the
// X-marginal is summed over the cluster through distributed shared memory,
// every CTA applies the same X-iteration, and rank 0 alone runs the epilogue.
// XI: pixels of the cell each thread updates in the X-iteration (≥ 256/NT)
template <int H, int W, int CS, int XI>
__device__ void sinkhorn_cell(const SweepArgs& a, const int J, const CellGeom& g, SinkSmem& sm,
                              const int rank, float4* ys, const int ycap, float* nbuf) {
  // iterations: a thread holds RM whole rows (at most 64 pixels) of the cell
  // for one support point at a time; GM threads share a point
  constexpr int RM = (H < 64 / W) ? H : 64 / W;
  constexpr int GM = H / RM;
  constexpr int PT = RM * W;
  constexpr int WP = W / 2;
  const LevelView& L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NT = blockDim.x;
  const int HW = H * W;

  const int64_t off = a.cell_off[J];
  if (off < 0) {
    if (tid == 0) a.cell_status[J] = 4;
    return;
  }
  const int ny = a.cell_ny[J];
  if (ny <= 0) {
    if (tid == 0 && rank == 0) {
      a.cell_status[J] = 2;
      atomicOr(a.err_flag, 2);
    }
    return;
  }
  const int2 anc_old = a.anchor[J];
  const int2 anc = a.anchor_new[J];
  const float d2 = (float)(L.spacing * L.spacing);
  const float inv_eln2 = 1.0f / (a.eps * kLn2);
  const float kappa = (float)(L.spacing * L.spacing / ((double)a.eps * 0.69314718055994530942));
  const int Dr = g.r0 - anc.x, Dc = g.c0 - anc.y;
  const int shr = anc.x - anc_old.x, shc = anc.y - anc_old.y;

  // stabiliser F in the new frame, scalings u = 1
  for (int x = tid; x < HW; x += NT) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    const float l2 = L.log2mu[p];
    const float at = a.alpha[p] + 2.0f * d2 * (float)(shr * ar + shc * ac);
    sm.F[x] = at * inv_eln2 + l2;
    sm.u[x] = 1.0f;
    sm.l2mu[x] = l2;
    sm.mu[x] = L.mu_f[p];
  }
  float mu_part = 0.f, nu_part = 0.f;
  for (int x = tid; x < HW; x += NT) mu_part += L.mu_f[(g.r0 + x / g.W) * L.n + g.c0 + x % g.W];
  for (int k = tid; k < ny; k += NT) nu_part += (float)a.ws_nu[off + k] * kFixToFloat;
  const float muJ = block_sum(mu_part, sm.fws);
  const float nuJ = block_sum(nu_part, sm.fws);
  const float tol = a.err_tol * muJ;
  // Truncate leaves ‖ν_cell‖ ≤ ‖μ_J‖: the stopping test compares P_X π with μ
  // rescaled to ‖ν_cell‖ (the §6.2 rule when nothing was truncated)
  const float mscale = muJ > 0.f ? nuJ / muJ : 1.f;
  // over-relaxation state, identical in every thread
  float omega = 1.0f, e3 = 0.f, emin = 3.0e38f, e_stag = 3.0e38f;
  bool relax_off = false;
  int phase = 0;
  // Newton steps for the X-iteration (cells of at most 64 pixels, CTAs of 128
  // or 256 threads, at most 64 support points per pass, nbuf given):
  // `newton` = this pass also accumulates the Hessian and the X-iteration
  // after it is a Newton step. A cell of fewer pixels uses the leading HW
  // rows and columns of the 64×64 system, the rest being the identity.
  constexpr bool kNewtonShape = (H * W <= kNewtonN);
  constexpr int GJ = H / ((H < 16 / W) ? H : 16 / W);   // threads per point in the unsplit pass
  const bool newton_ok = kNewtonShape && a.newton && nbuf != nullptr && (NT == 256 || (CS == 1 && NT == 128)) &&
                         NT / GJ <= 64;
  bool newton = false, newton_off = false;
  float ep_before = 0.f, e_mark = 0.f;
  const int newton_min = a.newton - 1;   // see the X-iteration's Newton decision

  // This CTA's share of the support: all of it, or a contiguous chunk per
  // cluster rank. When it fits, the share is staged once in shared memory as
  // {η, ν, G, −} per point (one 128-bit load per point in every pass); G
  // changes only at absorptions, which also write it to global memory.
  int ylo = 0, yhi = ny;
  if constexpr (CS > 1) {
    const int chunk = (ny + CS - 1) / CS;
    ylo = min(ny, rank * chunk);
    yhi = min(ny, ylo + chunk);
  }
  const bool staged = (yhi - ylo) <= ycap;
  if (staged) {
    for (int k = ylo + tid; k < yhi; k += NT)
      ys[k - ylo] = make_float4(__int_as_float(a.ws_eta[off + k]), (float)a.ws_nu[off + k] * kFixToFloat,
                                0.f, 0.f);
  }
  __syncthreads();

  const int gm = tid % GM, slm = tid / GM, YSM = NT / GM;
  const int row0 = gm * RM;
  // Separable split of the stabiliser: F(r,c) = fr(r) + fc(c) + res(r,c) with
  // fr(r) = F(r,c₀), fc(c) = F(r₀,c) − F(r₀,c₀). Because the cost is a sum of
  // a row and a column term, the kernel entry 2^(F + G − κ|ξ−η|²) of a support
  // point y factorises as 2^res(r,c) · ρ_y(r) · γ_y(c) with
  //   γ_y(c) = 2^(fc(c) − κ(c−η_c)² − m_y),  m_y = max_c (fc(c) − κ(c−η_c)²),
  //   ρ_y(r) = 2^(fr(r) + G(y) − κ(r−η_r)² + m_y),
  // so a point costs H + W exponentials and two FMAs per pixel instead of H·W
  // exponentials. Every term keeps the centred form (r−η_r)², (c−η_c)², so the
  // rounding of the exponents is that of the unsplit form. The split is used
  // while |res| ≤ kResMax on the whole cell: with the scalings u, v held in
  // [2^-16, 2^16] the exponent of F + G − κ|ξ−η|² stays below 32, hence
  // ρ_y ≤ 2^(32+kResMax), γ_y ≤ 1, and entries lost to an underflow of γ_y lie
  // below 2^-78 of the largest entry of their row. Otherwise the iteration
  // evaluates every entry with its own exponential.
  int it = 0;
  constexpr int rc0 = (H - 1) / 2, cc0 = (W - 1) / 2;
  unsigned long long FC2[WP];        // fc, pairs of neighbouring columns
  float FR[RM];                      // fr of the thread's rows
  bool fact = false;
  // 2^res·u into shared memory and the decision for this pass; F and u are
  // final for the pass; contains the barrier before the Y-iteration
  auto prepare = [&]() {
    const float f00 = sm.F[rc0 * W + cc0];
    bool ok = true;
    for (int x = tid; x < HW; x += NT) {
      const int r = x / W, c = x % W;
      const float fc = sm.F[rc0 * W + c] - f00;
      const float res = (sm.F[x] - sm.F[r * W + cc0]) - fc;
      ok = ok && fabsf(res) <= kResMax;   // false on NaN
      sm.WT[x] = ex2(res) * sm.u[x];
    }
    fact = __syncthreads_and(ok) != 0;
#pragma unroll
    for (int j = 0; j < WP; ++j)
      FC2[j] = pk2(sm.F[rc0 * W + 2 * j] - f00, sm.F[rc0 * W + 2 * j + 1] - f00);
#pragma unroll
    for (int r = 0; r < RM; ++r) FR[r] = sm.F[(row0 + r) * W + cc0];
  };
  prepare();
  const unsigned long long NK2 = pk2(-kappa, -kappa);
  const unsigned long long K2 = pk2(kappa, kappa);

  // the unsplit pass: G threads per support point, RPT whole rows (at most
  // 16 pixels) each, the entries of K̃ one exponential each
  constexpr int RPT = (H < 16 / W) ? H : 16 / W;
  constexpr int G = H / RPT;
  constexpr int PJ = RPT * W;
  const int gid = tid % G, slot = tid / G, YS = NT / G;

  // a support point's record {η, ν, G} from the staging buffer or memory
  auto load_y = [&](int kk, int32_t& e, float& nuy, float& g_pre) {
    if (staged) {
      const float4 yd = ys[kk - ylo];
      e = __float_as_int(yd.x);
      nuy = yd.y;
      g_pre = yd.z;
    } else {
      e = a.ws_eta[off + kk];
      nuy = (float)a.ws_nu[off + kk] * kFixToFloat;
      g_pre = it > 0 ? a.ws_g[off + kk] : 0.f;
    }
  };
  // a new stabiliser, or a scaling outside the band: G ← G + log2 v
  auto store_g = [&](int k, float gs, float v) {
    const float gn = gs + log2f(v);
    a.ws_g[off + k] = gn;
    if (staged) ys[k - ylo].z = gn;
  };

  bool stepped = false;
  int nsteps = 0, nfail = 0;
  float ncap = kNewtonMaxStep;   // largest |δ| of the next Newton step
  // Newton direction from the C of the last pass (each CTA's partial in its
  // nbuf): every CTA of the cluster sums the partials in the same order and
  // solves the same system, so all hold the same δ (in nbuf after the
  // matrix). Returns the step length in (0, 1], or −1 if a pivot is not
  // positive or δ is not finite.
  auto newton_x_step = [&](float px_own, float cap) -> float {
    if constexpr (kNewtonShape) {
      float* M = nbuf;
      float* bv = nbuf + kNewtonB;
      const float lam = nuJ / (float)(HW * HW);
      const int tc = NT == 256 ? 4 : 8, tjn = kNewtonN / tc;
      const int ti = tid / tjn, tj = tid % tjn;
      if constexpr (CS > 1) {
        // C summed over the CTAs of the cluster, tile by tile, in rank order
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        float ct[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) ct[q] = 0.f;
#pragma unroll 1
        for (int rr = 0; rr < CS; ++rr) {
          const float* pb = cl.map_shared_rank(nbuf, rr);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) ct[4 * r + c] += pb[(4 * ti + r) * kNewtonLd + 4 * tj + c];
        }
        cl.sync();
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = 4 * ti + r, j = 4 * tj + c;
            M[i * kNewtonLd + j] = (i >= HW || j >= HW) ? (i == j ? 1.f : 0.f)
                                   : (i == j) ? 0.f : lam - ct[4 * r + c];
          }
      } else {
        __syncthreads();
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < tc; ++c) {
            const int i = 4 * ti + r, j = tc * tj + c;
            M[i * kNewtonLd + j] = (i >= HW || j >= HW) ? (i == j ? 1.f : 0.f)
                                   : (i == j) ? 0.f : lam - M[i * kNewtonLd + j];
          }
      }
      __syncthreads();
      if (tid < HW) {
        // diagonal Σ_{j≠x} C(x,j) (C's row sums are P_X π), gauge λ, and a
        // small regulariser for pixels that receive almost no mass
        float rs = 0.f;
        for (int j = 0; j < HW; ++j)
          if (j != tid) rs += lam - M[tid * kNewtonLd + j];
        M[tid * kNewtonLd + tid] = rs + lam + 1e-4f * px_own + 1e-7f * nuJ / (float)HW;
        bv[tid] = sm.mu[tid] * mscale - px_own;
      } else if (tid < kNewtonN) {
        bv[tid] = 0.f;
      }
      __syncthreads();
      // LDLᵀ, right-looking: afterwards M(k,k) = D(k), M(i,k) = L(i,k)·D(k)
      // for i > k. The lower triangle is held in registers as 4×4 blocks
      // (136 of them; thread t owns blocks t and t + NT). At step k the owners
      // of column k (final after step k − 1) write it to shared memory; after
      // one barrier every thread applies the rank-1 update M(i,j) −=
      // M(i,k)·M(j,k)/D(k) to its elements with j > k. One barrier per column.
      constexpr int kNBlk = (kNewtonN / 4) * (kNewtonN / 4 + 1) / 2;
      float R[2][16];
      int qbi[2], qbj[2];
      bool has[2];
#pragma unroll
      for (int sb = 0; sb < 2; ++sb) {
        const int q = tid + sb * NT;
        has[sb] = q < kNBlk;
        int bi = 0;
        if (has[sb])
          while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
        qbi[sb] = bi;
        qbj[sb] = has[sb] ? q - bi * (bi + 1) / 2 : 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) R[sb][r] = 0.f;
        if (has[sb]) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) R[sb][4 * r + c] = M[(4 * qbi[sb] + r) * kNewtonLd + 4 * qbj[sb] + c];
        }
      }
      bool ok = true;
#pragma unroll 1
      for (int k = 0; k < kNewtonN; ++k) {
#pragma unroll
        for (int sb = 0; sb < 2; ++sb) {
          if (has[sb] && qbj[sb] == (k >> 2)) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int i = 4 * qbi[sb] + r;
              float v = R[sb][4 * r];
#pragma unroll
              for (int c = 1; c < 4; ++c) v = (k & 3) == c ? R[sb][4 * r + c] : v;
              if (i >= k) M[i * kNewtonLd + k] = v;
            }
          }
        }
        __syncthreads();
        const float d = M[k * kNewtonLd + k];
        ok = d > 0.f;   // the same d in every thread: a uniform exit
        if (!ok) break;
        const float dinv = 1.0f / d;
#pragma unroll
        for (int sb = 0; sb < 2; ++sb) {
          if (has[sb] && 4 * qbj[sb] + 3 > k) {
            float ci[4], cj[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              ci[r] = M[(4 * qbi[sb] + r) * kNewtonLd + k] * dinv;
              cj[r] = M[(4 * qbj[sb] + r) * kNewtonLd + k];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int i = 4 * qbi[sb] + r, j = 4 * qbj[sb] + c;
                if (j > k && j <= i) R[sb][4 * r + c] -= ci[r] * cj[c];
              }
          }
        }
      }
      __syncthreads();
      if (ok && warp == 0) {
        for (int k = 0; k < kNewtonN; ++k) {
          const float zk = bv[k] / M[k * kNewtonLd + k];
          __syncwarp();
          for (int i = lane; i < kNewtonN; i += 32)
            if (i > k) bv[i] -= M[i * kNewtonLd + k] * zk;
          __syncwarp();
        }
        for (int i = lane; i < kNewtonN; i += 32) bv[i] /= M[i * kNewtonLd + i];
        __syncwarp();
        for (int k = kNewtonN - 1; k >= 0; --k) {
          const float dk = bv[k];
          __syncwarp();
          for (int i = lane; i < k; i += 32) bv[i] -= (M[k * kNewtonLd + i] / M[i * kNewtonLd + i]) * dk;
          __syncwarp();
        }
        // step length: the whole step scaled so that max |δ| ≤ kNewtonMaxStep
        float m = 0.f;
        bool fin = true;
        for (int i = lane; i < kNewtonN; i += 32) {
          const float d = bv[i];
          fin = fin && d == d && fabsf(d) < 1e30f;
          m = fmaxf(m, fabsf(d));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        fin = __all_sync(0xffffffffu, fin);
        if (lane == 0) bv[kNewtonN] = fin ? fminf(1.0f, cap / fmaxf(m, 1e-30f)) : -1.0f;
      }
      __syncthreads();
      return ok ? bv[kNewtonN] : -1.0f;
    } else {
      (void)px_own;
      (void)cap;
      return -1.0f;
    }
  };
  float errx = 0.f;
  bool converged = false, bad = false;
  for (;;) {
    // ---- Y-iteration and X-marginal of the new plan ----
    if (fact && !newton) {
      unsigned long long A2[RM * WP];
#pragma unroll
      for (int q = 0; q < RM * WP; ++q) A2[q] = 0ull;
      for (int k0 = ylo; k0 < yhi; k0 += YSM) {
        const int k = k0 + slm;
        const bool valid = k < yhi;
        int32_t e;
        float nuy, g_pre;
        load_y(valid ? k : yhi - 1, e, nuy, g_pre);
        const float erf = (float)eta_r(e), ecf = (float)eta_c(e);
        const unsigned long long EC2 = pk2(ecf, ecf);
        // stabiliser G from the largest exponent over the cell (with the
        // scalings u after the first pass)
        auto restab = [&](bool with_u) {
          float m = kNegBig;
#pragma unroll 1
          for (int r = 0; r < RM; ++r) {
            const float tr = (float)(row0 + r) - erf;
#pragma unroll
            for (int c = 0; c < W; ++c) {
              const float tc = (float)c - ecf;
              const int x = (row0 + r) * W + c;
              const float ev = sm.F[x] - kappa * tr * tr - kappa * tc * tc;
              const float uu = sm.u[x];
              m = fmaxf(m, with_u ? (uu > 0.f ? ev + lg2(uu) : kNegBig) : ev);
            }
          }
          return -group_max<GM>(m);
        };
        float Gs = (it == 0) ? restab(false) : g_pre;
        bool absorb = (it == 0);
        unsigned long long GA2[WP];
        float rho[RM];
        // s = Σ_x K̃(x,y) u(x) from the factors
        auto fact_sum = [&](float gs) {
          float ce[W];
          float mc = kNegBig;
#pragma unroll
          for (int j = 0; j < WP; ++j) {
            const unsigned long long t2 = sub2(pk2((float)(2 * j), (float)(2 * j + 1)), EC2);
            upk2(fma2(mul2(NK2, t2), t2, FC2[j]), ce[2 * j], ce[2 * j + 1]);
            mc = fmaxf(mc, fmaxf(ce[2 * j], ce[2 * j + 1]));
          }
#pragma unroll
          for (int j = 0; j < WP; ++j) GA2[j] = pk2(ex2(ce[2 * j] - mc), ex2(ce[2 * j + 1] - mc));
          const float cy = gs + mc;
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int r = 0; r < RM; ++r) {
            const float tr = (float)(row0 + r) - erf;
            rho[r] = ex2(FR[r] + cy - kappa * tr * tr);
            unsigned long long T2 = 0ull;
            if constexpr (W >= 4) {
              const float4* wr = reinterpret_cast<const float4*>(&sm.WT[(row0 + r) * W]);
#pragma unroll
              for (int j4 = 0; j4 < W / 4; ++j4) {
                const float4 w4 = wr[j4];
                T2 = fma2(pk2(w4.x, w4.y), GA2[2 * j4], T2);
                T2 = fma2(pk2(w4.z, w4.w), GA2[2 * j4 + 1], T2);
              }
            } else {
              const float2 w2 = reinterpret_cast<const float2*>(&sm.WT[(row0 + r) * W])[0];
              T2 = fma2(pk2(w2.x, w2.y), GA2[0], T2);
            }
            float t0, t1;
            upk2(T2, t0, t1);
            if (r & 1) s1 = fmaf(rho[r], t0 + t1, s1);
            else s0 = fmaf(rho[r], t0 + t1, s0);
          }
          return group_sum<GM>(s0 + s1);
        };
        // one call site, so that the factor arrays stay in registers; a
        // second attempt when the stabiliser is too far off for this y,
        // restarted from the running maximum
        float s;
#pragma unroll 1
        for (int attempt = 0;; ++attempt) {
          s = fact_sum(Gs);
          if ((s > 1e-30f && s < 1e30f) || attempt == 1) break;
          Gs = restab(true);
          absorb = true;
        }
        // v = ν/s with IEEE division: the iteration map itself uses correctly
        // rounded arithmetic; only the frozen kernel K̃ uses ex2.approx
        const float v = valid ? nuy / s : 0.f;
        if (valid && gm == 0 && (absorb || v > kTwoTau || v < 1.0f / kTwoTau)) store_g(k, Gs, v);
        // Σ_y v ρ_y(r) γ_y(c); the factor 2^res·u is applied once per pass
#pragma unroll
        for (int r = 0; r < RM; ++r) {
          const float vr = v * rho[r];
          const unsigned long long VR2 = pk2(vr, vr);
#pragma unroll
          for (int j = 0; j < WP; ++j) A2[r * WP + j] = fma2(VR2, GA2[j], A2[r * WP + j]);
        }
      }
      // P_X π on the thread's pixels, partial over its support points:
      // (2^res·u)·Σ_y v ρ γ
      float acc[PT];
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int j = 0; j < WP; ++j) {
          const int x = (row0 + r) * W + 2 * j;
          upk2(mul2(A2[r * WP + j], pk2(sm.WT[x], sm.WT[x + 1])), acc[r * W + 2 * j], acc[r * W + 2 * j + 1]);
        }
      using SS = ScatterShape<PT, GM>;
      const int base = warp_reduce_scatter<PT, GM>(acc, lane);
      if (SS::writer(lane)) {
#pragma unroll
        for (int j = 0; j < SS::nv; ++j) sm.red[warp][gm * PT + base + j] = acc[j];
      }
    } else {
      const int rj0 = gid * RPT;
      unsigned long long F2[RPT * WP], U2[RPT * WP], P2[RPT * WP], A2[RPT * WP];
      if constexpr (kNewtonShape) {
        if (newton) {
          // C = Σ_y z_y z_yᵀ starts at zero; each thread clears its own tile
          const int tc = NT == 256 ? 4 : 8, tjn = kNewtonN / tc;
          const int ti = tid / tjn, tj = tid % tjn;
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < tc; ++c) nbuf[(4 * ti + r) * kNewtonLd + tc * tj + c] = 0.f;
          // the rows z_y have no entries beyond the cell's pixels
          if constexpr (H * W < kNewtonN) {
            constexpr int pad = kNewtonN - H * W;
            for (int q = tid; q < 64 * pad; q += NT) nbuf[kNewtonZ + (q / pad) * kZs + H * W + q % pad] = 0.f;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int j = 0; j < WP; ++j) {
          const int x = (rj0 + r) * W + 2 * j;
          F2[r * WP + j] = pk2(sm.F[x], sm.F[x + 1]);
          U2[r * WP + j] = pk2(sm.u[x], sm.u[x + 1]);
          A2[r * WP + j] = 0ull;
        }
      for (int k0 = ylo; k0 < yhi; k0 += YS) {
        const int k = k0 + slot;
        const bool valid = k < yhi;
        int32_t e;
        float nuy, g_pre;
        load_y(valid ? k : yhi - 1, e, nuy, g_pre);
        const float erf = (float)eta_r(e), ecf = (float)eta_c(e);
        // κ(c − η_c)² for the pairs of columns, κ(a − η_r)² for the rows
        unsigned long long CC2[WP];
        const unsigned long long EC2 = pk2(ecf, ecf);
#pragma unroll
        for (int j = 0; j < WP; ++j) {
          const unsigned long long t2 = sub2(pk2((float)(2 * j), (float)(2 * j + 1)), EC2);
          CC2[j] = mul2(mul2(K2, t2), t2);
        }
        float Rq[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const float t = (float)(rj0 + r) - erf;
          Rq[r] = kappa * t * t;
        }
        auto row_max = [&](bool with_u) {
          float m = kNegBig;
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const unsigned long long R2 = pk2(-Rq[r], -Rq[r]);
#pragma unroll
            for (int j = 0; j < WP; ++j) {
              float e0, e1;
              upk2(sub2(add2(F2[r * WP + j], R2), CC2[j]), e0, e1);
              if (with_u) {
                float u0, u1;
                upk2(U2[r * WP + j], u0, u1);
                e0 = u0 > 0.f ? e0 + lg2(u0) : kNegBig;
                e1 = u1 > 0.f ? e1 + lg2(u1) : kNegBig;
              }
              m = fmaxf(m, fmaxf(e0, e1));
            }
          }
          return -group_max<G>(m);
        };
        float Gs = (it == 0) ? row_max(false) : g_pre;
        bool absorb = (it == 0);
        auto kernel_row = [&](float gs) {
          unsigned long long S2 = 0ull;
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const unsigned long long RA2 = pk2(gs - Rq[r], gs - Rq[r]);
#pragma unroll
            for (int j = 0; j < WP; ++j) {
              const int q = r * WP + j;
              float e0, e1;
              upk2(sub2(add2(F2[q], RA2), CC2[j]), e0, e1);
              P2[q] = pk2(ex2(e0), ex2(e1));
              S2 = fma2(P2[q], U2[q], S2);
            }
          }
          float s0, s1;
          upk2(S2, s0, s1);
          return group_sum<G>(s0 + s1);
        };
        // one call site (see the split pass); a second attempt from the
        // running maximum when the stabiliser is too far off for this y
        float s;
#pragma unroll 1
        for (int attempt = 0;; ++attempt) {
          s = kernel_row(Gs);
          if ((s > 1e-30f && s < 1e30f) || attempt == 1) break;
          Gs = row_max(true);
          absorb = true;
        }
        const float v = valid ? nuy / s : 0.f;
        if (valid && gid == 0 && (absorb || v > kTwoTau || v < 1.0f / kTwoTau)) store_g(k, Gs, v);
        const unsigned long long V2 = pk2(v, v);
#pragma unroll
        for (int q = 0; q < RPT * WP; ++q) A2[q] = fma2(V2, P2[q], A2[q]);
        if constexpr (kNewtonShape) {
          if (newton) {
            // z_y(x) = √ν(y)·K̃(x,y)u(x)/s(y), so that Σ_y z_y(x) z_y(x') =
            // Σ_y π(x,y)π(x',y)/ν(y); one row per support point of the batch
            const float w = valid ? sqrtf(nuy) / s : 0.f;
            const unsigned long long W2 = pk2(w, w);
            unsigned long long* zrow =
                reinterpret_cast<unsigned long long*>(nbuf + kNewtonZ + slot * kZs + gid * PJ);
#pragma unroll
            for (int q = 0; q < RPT * WP; ++q) zrow[q] = mul2(mul2(P2[q], U2[q]), W2);
            __syncthreads();
            hess_batch_mma(nbuf, YS, tid, NT);
            __syncthreads();
          }
        }
      }
      if constexpr (kNewtonShape) {
        if (newton) {
          // the upper triangle of C outside the diagonal 16×16 blocks from the
          // lower one (read after the barrier that ends the pass)
          for (int q = tid; q < kNewtonN * kNewtonN; q += NT) {
            const int i = q / kNewtonN, j = q % kNewtonN;
            if (j >= 16 * ((i >> 4) + 1)) nbuf[i * kNewtonLd + j] = nbuf[j * kNewtonLd + i];
          }
        }
      }
      // u·Σ_y K̃ v
      float acc[PJ];
#pragma unroll
      for (int q = 0; q < RPT * WP; ++q) upk2(mul2(A2[q], U2[q]), acc[2 * q], acc[2 * q + 1]);
      using SS = ScatterShape<PJ, G>;
      const int base = warp_reduce_scatter<PJ, G>(acc, lane);
      if (SS::writer(lane)) {
#pragma unroll
        for (int j = 0; j < SS::nv; ++j) sm.red[warp][gid * PJ + base + j] = acc[j];
      }
    }
    __syncthreads();
    // X-marginal P_X π(x) for the pixels this thread updates
    // (x = tid + i·NT), kept in registers until the X-iteration
    const int nw = NT >> 5;
    float pxl[XI];
    float ep = 0.f;
    if constexpr (CS > 1) {
      for (int x = tid; x < HW; x += NT) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += sm.red[w][x];
        sm.PXp[x] = t;
      }
      cg::this_cluster().sync();
      cg::cluster_group cl = cg::this_cluster();
#pragma unroll
      for (int i = 0; i < XI; ++i) {
        const int x = tid + i * NT;
        if (x < HW) {
          float t = 0.f;
#pragma unroll
          for (int r = 0; r < CS; ++r) t += cl.map_shared_rank(sm.PXp, r)[x];
          pxl[i] = t;
          ep += fabsf(pxl[i] - sm.mu[x] * mscale);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < XI; ++i) {
        const int x = tid + i * NT;
        if (x < HW) {
          float t = 0.f;
          for (int w = 0; w < nw; ++w) t += sm.red[w][x];
          pxl[i] = t;
          ep += fabsf(pxl[i] - sm.mu[x] * mscale);
        }
      }
    }
    ep = block_sum1(ep, sm.fws2, phase);
    ++it;
    // every thread takes the same decisions from the same ep
    int stop = 0;
    // A solve whose error stays above 10·Err·‖μ_J‖ and falls by less than
    // 0.1 % over 128 iterations (contraction above 0.999992 per iteration)
    // stops as one at max_iter would: such a cell needs far more iterations
    // than any max_iter allows (its support lies so far from the cell that
    // c/ε differs by thousands between its pixels and the cell problem is an
    // assignment problem in all but name), and the safeguard's larger ε,
    // which takes exactly the cells above 10·Err·‖μ_J‖, is what solves it.
    bool stagnant = false;
    if ((it & (kStagnationPeriod - 1)) == 0) {
      stagnant = it >= 2 * kStagnationPeriod && ep > 10.0f * tol && ep > kStagnationRatio * e_stag;
      e_stag = ep;
    }
    if (!(ep == ep) || isinf(ep)) stop = 2;
    else if (ep <= tol) stop = 1;
    else if (it >= a.max_iter || stagnant) stop = 3;
    // Over-relaxed X-iteration u ← u·(μ/P_X π)^ω (same fixed point, same
    // stopping rule, always ending on a Y-iteration). ω follows from the
    // contraction ρ of the plain iteration measured over iterations 3..6,
    // ω = 2/(1+√(1−ρ)) capped at 1.8, and falls back to 1 for good when the
    // error grows well above its running minimum.
    if (it == 3) e3 = ep;
    float rho6 = 0.f;
    if (it == 6 && e3 > 0.f) {
      const float rho = cbrtf(ep / e3);
      rho6 = rho;
      if (!relax_off && rho > 0.5f && rho < 1.0f) omega = fminf(1.8f, 2.0f / (1.0f + sqrtf(1.0f - rho)));
    }
    if (ep > 1.5f * emin && omega != 1.0f) {
      omega = 1.0f;
      relax_off = true;
    }
    emin = fminf(emin, ep);
    if (tid == 0 && rank == 0 && J == a.trace_cell && a.trace && it <= kTraceLen) {
      // relative error; ω + 10·(Newton steps so far) + 1000 while Newton
      // X-iterations are on + 2000 once they are off for this solve
      a.trace[2 * (it - 1)] = ep / muJ;
      a.trace[2 * (it - 1) + 1] = omega + 10.0f * (float)nsteps + (newton ? 1000.f : 0.f) +
                                  (newton_off ? 2000.f : 0.f);
    }
    if (stop) {
      // the reported error is the unscaled Σ_x |P_X π − μ|
      float erp = 0.f;
#pragma unroll
      for (int i = 0; i < XI; ++i) {
        const int x = tid + i * NT;
        if (x < HW) erp += fabsf(pxl[i] - sm.mu[x]);
      }
      errx = block_sum1(erp, sm.fws2, phase);
      converged = stop == 1;
      bad = stop == 2;
      break;
    }
    // ---- Newton X-iteration ----
    // With the Y-iteration exact, P_X π depends on the scalings u alone, and
    // its Jacobian in log u is M = diag(P_X π) − Σ_y π(·,y)π(·,y)ᵀ/ν(y), a
    // graph Laplacian (M·1 = 0). The step solves (M + λ11ᵀ) δ = μ‖ν_cell‖/‖μ_J‖
    // − P_X π and sets u ← u·e^δ. It has the plain iteration's fixed point and
    // stopping rule, and converges in a few steps where the plain iteration
    // needs hundreds (cells whose support spreads far). The decision to take
    // it: an error below 5 % of ‖μ_J‖ and a contraction ρ > 0.75 over
    // iterations 3..6 or less than a tenfold error reduction over 16
    // iterations. A step longer than the cap (kNewtonMaxStep in log u at
    // first) is scaled down; after a step that does not lower the error the
    // cap is quartered, and after three such steps the solve continues with
    // the plain iteration.
    bool newton_step = false;
    float step_len = 0.f;
    if constexpr (kNewtonShape) {
      if (newton) {
        bool take = true;
        if (stepped && ep > ep_before) {
          // the last step raised the error: shorter steps from here, and
          // the plain iteration after three such steps
          ncap *= 0.25f;
          if (++nfail >= 3) {
            newton = false;
            newton_off = true;
            take = false;
          }
        }
        if (take) {
          step_len = newton_x_step(pxl[0], ncap);
          newton_step = step_len > 0.f;
          if (newton_step) {
            ep_before = ep;
            stepped = true;
            ++nsteps;
          } else {
            newton = false;
            newton_off = true;
          }
        }
      }
    }
    if (!newton_step && newton_ok && !newton_off && !newton) {
      const bool near = ep < kNewtonNear * muJ;   // Newton steps only close to the solution
      // at iteration 6 only when the plain iteration, contracting by rho6 per
      // iteration, would need more than newton_min further iterations:
      // ln(tol/ep) < newton_min·ln(rho6) (a Newton step costs as much as
      // several plain iterations)
      if (it == 6 && rho6 > 0.75f && near &&
          (newton_min <= 0 || logf(tol / ep) < (float)newton_min * logf(rho6)))
        newton = true;
      if (it > 6 && (it & 15) == 0) {
        if (ep > 0.1f * e_mark && near) newton = true;
        e_mark = ep;
      }
      if (it == 6) e_mark = ep;
      stepped = false;
    }
    if (newton_step) {
      if (tid < HW) {
        // log2 of the new scaling, absorbed into F when it leaves the band
        const float lu = log2f(sm.u[tid]) + step_len * nbuf[kNewtonB + tid] * (1.0f / kLn2);
        if (fabsf(lu) > 16.0f) {
          sm.F[tid] += lu;
          sm.u[tid] = 1.0f;
        } else {
          sm.u[tid] = exp2f(lu);
        }
      }
    }
    // ---- X-iteration u ← u·(μ/P_X π)^ω, absorbing large scalings into F ----
#pragma unroll
    for (int i = 0; i < XI && !newton_step; ++i) {
      const int x = tid + i * NT;
      if (x >= HW) continue;
      const float px = pxl[i];
      if (px > 1e-37f && px < 1e37f) {
        const float ratio = sm.mu[x] / px;
        if (omega == 1.0f) {
          const float un = sm.u[x] * ratio;
          if (un > kTwoTau || un < 1.0f / kTwoTau) {
            sm.F[x] += log2f(un);
            sm.u[x] = 1.0f;
          } else {
            sm.u[x] = un;
          }
        } else {
          // over-relaxed: in log2, so that (μ/P_X π)^ω cannot overflow
          const float lu = log2f(sm.u[x]) + omega * log2f(ratio);
          if (fabsf(lu) > 16.0f) {
            sm.F[x] += lu;
            sm.u[x] = 1.0f;
          } else {
            sm.u[x] = exp2f(lu);
          }
        }
      } else {
        // no mass reached this x: full log-sum-exp over the support with the
        // current stabilisers
        const int ar = x / g.W, ac = x - (x / g.W) * g.W;
        float m = kNegBig;
        for (int k = 0; k < ny; ++k) {
          const int32_t e = a.ws_eta[off + k];
          const float tr = (float)(ar - eta_r(e)), tc = (float)(ac - eta_c(e));
          m = fmaxf(m, a.ws_g[off + k] - kappa * (tr * tr + tc * tc));
        }
        float s = 0.f;
        for (int k = 0; k < ny; ++k) {
          const int32_t e = a.ws_eta[off + k];
          const float tr = (float)(ar - eta_r(e)), tc = (float)(ac - eta_c(e));
          s += ex2(a.ws_g[off + k] - kappa * (tr * tr + tc * tc) - m);
        }
        sm.F[x] = sm.l2mu[x] - (m + lg2(s));
        sm.u[x] = 1.0f;
      }
    }
    // the whole cluster syncs here: the reads of PXp above are complete
    // before any CTA overwrites it in the next iteration
    if constexpr (CS > 1) {
      cg::this_cluster().sync();
    } else {
      __syncthreads();
    }
    prepare();
  }
  if constexpr (CS > 1) {
    // the stabilisers G written by the other CTAs must be visible to rank 0
    __threadfence();
    cg::this_cluster().sync();
    if (rank != 0) return;
  }

  // ---- epilogue: final plan → fractions per basic cell, transport cost ----
  // The plan of the last Y-iteration, π(x,y) = ν(y)·p(x,y)/Σ_x p(x,y) with
  // p = K̃·u: per support point the fractions of its mass in each basic cell
  // and the cost Σ_x p·|x−y|²/Σ_x p (in pixel² units).
  const int nbas = g.nbr * g.nbc;
  const int64_t tbase = 4 * off;
  double cost_acc = 0.0;
  // one support point's results: fixed-point fractions into the extraction
  // buffer (the largest takes the rounding remainder), cost into cost_acc
  auto emit = [&](int k, int er, int ec, const float (&q)[4], float s, float cst) {
    const uint64_t nuq = a.ws_nu[off + k];
    const float S = q[0] + q[1] + q[2] + q[3];
    int imax = 0;
    for (int i = 1; i < nbas; ++i)
      if (q[i] > q[imax]) imax = i;
    uint64_t rest = nuq;
    const int y = (anc.x + er) * L.n + (anc.y + ec);
    const float invS = S > 0.f ? 1.0f / S : 0.f;
    for (int i = 0; i < nbas; ++i) {
      if (i == imax) continue;
      const uint64_t vq = __umul64hi(nuq, frac_to_u64(q[i] * invS));
      rest -= vq;
      a.tmp_val[tbase + (int64_t)i * ny + k] = vq;
      a.tmp_col[tbase + (int64_t)i * ny + k] = y;
    }
    a.tmp_val[tbase + (int64_t)imax * ny + k] = rest;
    a.tmp_col[tbase + (int64_t)imax * ny + k] = y;
    const double nuf = (double)nuq * (1.0 / kFixOne);
    if (s > 0.f) cost_acc += (double)cst * (nuf / (double)s);
  };
  if (fact) {
    // the separable split of the last pass (F, u and 2^res·u unchanged since
    // its prepare): p = 2^res·u(x) · ρ_y(r) · γ_y(c), so a point costs H + W
    // exponentials. Basic rows split at br, basic columns at bc.
    const int br = g.nbr == 2 ? L.b : H, bc = g.nbc == 2 ? L.b : W;
    for (int k0 = 0; k0 < ny; k0 += YSM) {
      const int k = k0 + slm;
      const bool valid = k < ny;
      const int kk = valid ? k : 0;
      const int32_t e = a.ws_eta[off + kk];
      const int er = eta_r(e), ec = eta_c(e);
      const float Gs = a.ws_g[off + kk];
      float ce[W], GA[W], GD[W];
      float mc = kNegBig;
#pragma unroll
      for (int j = 0; j < WP; ++j) {
        float f0, f1;
        upk2(FC2[j], f0, f1);
        const float t0 = (float)(2 * j) - (float)ec, t1 = (float)(2 * j + 1) - (float)ec;
        ce[2 * j] = f0 - kappa * t0 * t0;
        ce[2 * j + 1] = f1 - kappa * t1 * t1;
        mc = fmaxf(mc, fmaxf(ce[2 * j], ce[2 * j + 1]));
      }
#pragma unroll
      for (int c = 0; c < W; ++c) {
        GA[c] = ex2(ce[c] - mc);
        const float w = (float)(Dc + c - ec);
        GD[c] = GA[c] * (w * w);
      }
      float q[4] = {0.f, 0.f, 0.f, 0.f};
      float s = 0.f, cst = 0.f;
#pragma unroll
      for (int r = 0; r < RM; ++r) {
        const int row = row0 + r;
        const float tr = (float)(row - er);
        const float rho = ex2(FR[r] + Gs + mc - kappa * tr * tr);
        float t0 = 0.f, t1 = 0.f, tD = 0.f;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const float wt = sm.WT[row * W + c];
          if (c < bc) t0 = fmaf(wt, GA[c], t0);
          else t1 = fmaf(wt, GA[c], t1);
          tD = fmaf(wt, GD[c], tD);
        }
        const float wr = (float)(Dr + row - er);
        const float t = t0 + t1;
        const int i0 = (row >= br ? 1 : 0) * g.nbc;
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] += i == i0 ? rho * t0 : (i == i0 + 1 ? rho * t1 : 0.f);
        s = fmaf(rho, t, s);
        cst = fmaf(rho, fmaf(wr * wr, t, tD), cst);
      }
      s = group_sum<GM>(s);
      cst = group_sum<GM>(cst);
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = group_sum<GM>(q[i]);
      if (valid && gm == 0) emit(k, er, ec, q, s, cst);
    }
  } else {
    // unsplit: G threads per support point (the mapping of the unsplit pass),
    // one exponential per kernel entry
    int arow[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) arow[r] = gid * RPT + r;
    float Fr[RPT * W], ur[RPT * W];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const bool ok = arow[r] < g.H;
        Fr[r * W + c] = ok ? sm.F[arow[r] * W + c] : kNegBig;
        ur[r * W + c] = ok ? sm.u[arow[r] * W + c] : 0.f;
      }
    const int bsh = __ffs(L.b) - 1;  // b is a power of two
    for (int k0 = 0; k0 < ny; k0 += YS) {
      const int k = k0 + slot;
      const bool valid = k < ny;
      const int kk = valid ? k : 0;
      const int32_t e = a.ws_eta[off + kk];
      const int er = eta_r(e), ec = eta_c(e);
      const float Gs = a.ws_g[off + kk];
      float Cc[W], Dcc[W];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float t = (float)(c - ec);
        Cc[c] = kappa * t * t;
        const float w = (float)(Dc + c - ec);
        Dcc[c] = w * w;
      }
      float q[4] = {0.f, 0.f, 0.f, 0.f};
      float cst = 0.f, s = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const float tr = (float)(arow[r] - er);
        const float Ra = Gs - kappa * tr * tr;
        const float wr = (float)(Dr + arow[r] - er);
        const float Drr = wr * wr;
        const int kb_r = (arow[r] >> bsh) * g.nbc;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const float p = ex2(Fr[r * W + c] + Ra - Cc[c]) * ur[r * W + c];
          s += p;
          cst = fmaf(p, Drr + Dcc[c], cst);
          if (arow[r] < g.H) {
            const int kb = kb_r + (c >> bsh);
            if (kb == 0) q[0] += p; else if (kb == 1) q[1] += p; else if (kb == 2) q[2] += p; else q[3] += p;
          }
        }
      }
      s = group_sum<G>(s);
      cst = group_sum<G>(cst);
#pragma unroll
      for (int i = 0; i < 4; ++i) q[i] = group_sum<G>(q[i]);
      if (valid && gid == 0) emit(k, er, ec, q, s, cst);
    }
  }
  __syncthreads();

  // ---- BalanceMeasures: proportional transfer from surplus to deficit ----
  unsigned long long msum[4] = {0, 0, 0, 0};
  for (int k = tid; k < ny; k += NT)
    for (int i = 0; i < nbas; ++i) msum[i] += a.tmp_val[tbase + (int64_t)i * ny + k];
  for (int i = 0; i < nbas; ++i) msum[i] = block_sum<unsigned long long>(msum[i], sm.uws);
  if (tid == 0) {
    long long d[4];
    long long dtot = 0;
    sm.nsur = 0;
    sm.ndef = 0;
    for (int i = 0; i < nbas; ++i) {
      const int bi = (g.bi0 + i / g.nbc) * L.nb + g.bj0 + (i % g.nbc);
      d[i] = (long long)(msum[i] - L.M_q[bi]);
      if (d[i] > 0 && msum[i] > 0) {
        sm.sur[sm.nsur] = i;
        sm.q64[sm.nsur] = (uint64_t)fmin((double)d[i] / (double)msum[i] * 18446744073709551616.0,
                                         18446744073709549568.0);
        sm.nsur++;
      } else if (d[i] < 0) {
        sm.def[sm.ndef++] = i;
        dtot += -d[i];
      }
    }
    for (int j = 0; j < sm.ndef; ++j) {
      const int i = sm.def[j];
      sm.w64[j] = (uint64_t)fmin((double)(-d[i]) / (double)dtot * 18446744073709551616.0,
                                 18446744073709549568.0);
    }
  }
  __syncthreads();
  if (sm.nsur > 0 && sm.ndef > 0) {
    for (int k = tid; k < ny; k += NT) {
      uint64_t T = 0;
      for (int j = 0; j < sm.nsur; ++j) {
        const int64_t idx = tbase + (int64_t)sm.sur[j] * ny + k;
        const uint64_t vq = a.tmp_val[idx];
        const uint64_t t = __umul64hi(vq, sm.q64[j]);
        a.tmp_val[idx] = vq - t;
        T += t;
      }
      uint64_t rem = T;
      for (int j = 0; j + 1 < sm.ndef; ++j) {
        const int64_t idx = tbase + (int64_t)sm.def[j] * ny + k;
        const uint64_t t = __umul64hi(T, sm.w64[j]);
        a.tmp_val[idx] += t;
        rem -= t;
      }
      a.tmp_val[tbase + (int64_t)sm.def[sm.ndef - 1] * ny + k] += rem;
    }
  }
  __syncthreads();

  // ---- Truncate + in-row compaction ----
  for (int i = 0; i < nbas; ++i) {
    const int64_t rb = tbase + (int64_t)i * ny;
    int carry = 0;
    for (int k0 = 0; k0 < ny; k0 += NT) {
      const int k = k0 + tid;
      uint64_t vq = 0;
      int y = 0;
      int keep = 0;
      if (k < ny) {
        vq = a.tmp_val[rb + k];
        y = a.tmp_col[rb + k];
        keep = vq > a.trunc_q;
      }
      int tot;
      const int pos = block_exscan(keep, sm.iws, tot);  // contains the barrier
      if (keep) {
        a.tmp_val[rb + carry + pos] = vq;
        a.tmp_col[rb + carry + pos] = y;
      }
      carry += tot;
      __syncthreads();
    }
    if (tid == 0) {
      const int bi = (g.bi0 + i / g.nbc) * L.nb + g.bj0 + (i % g.nbc);
      a.row_cnt[bi] = carry;
      a.row_src[bi] = rb;
    }
  }

  // ---- duals of the cell, statistics ----
  const float eln2 = a.eps * kLn2;
  for (int x = tid; x < HW; x += NT) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    // a pixel without mass has no potential (F = log2 μ = −∞): α = 0 there
    a.alpha[p] = sm.mu[x] > 0.f ? (sm.F[x] + lg2(sm.u[x]) - sm.l2mu[x]) * eln2 : 0.f;
  }
  double cs = block_sum<double>(cost_acc, sm.dws);
  if (tid == 0) {
    a.anchor[J] = anc;
    a.cell_cost[J] = cs * (double)L.spacing * (double)L.spacing;
    a.cell_errx[J] = (double)errx;
    a.cell_iters[J] = it;
    if (a.cell_newton) a.cell_newton[J] = nsteps;
    a.cell_status[J] = (converged ? 0 : 1) | (bad ? 2 : 0);
    if (a.iters_hist) a.iters_hist[J] = it;
    if (bad) atomicOr(a.err_flag, 2);
  }
}

// the cell shape picks the instantiation (A cells share one shape, B has
// corner and edge shapes)
template <int CS, int XI>
__device__ void solve_cell(const SweepArgs& a, int J, SinkSmem& sm, int rank, float4* ys, int ycap,
                           float* nbuf) {
  const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
  const int W = g.W, H = g.H;
  // b ∈ {2, 4, 8}: cells are b or 2b pixels high and wide
  if (H == 2) {
    if (W == 2) sinkhorn_cell<2, 2, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else sinkhorn_cell<2, 4, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
  } else if (H == 4) {
    if (W == 2) sinkhorn_cell<4, 2, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else if (W == 4) sinkhorn_cell<4, 4, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else sinkhorn_cell<4, 8, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
  } else if (H == 8) {
    if (W == 4) sinkhorn_cell<8, 4, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else if (W == 8) sinkhorn_cell<8, 8, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else sinkhorn_cell<8, 16, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
  } else {
    if (W == 8) sinkhorn_cell<16, 8, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
    else sinkhorn_cell<16, 16, CS, XI>(a, J, g, sm, rank, ys, ycap, nbuf);
  }
}

// one CTA per cell, for the cells after the first nbig of the launch order
__global__ void __maxnreg__(168) k_sinkhorn(SweepArgs a) {
  __shared__ SinkSmem sm;
  __shared__ int s_pos, s_stop;
  // the arguments, once per CTA in shared memory: the cell solve takes them
  // by reference, and a reference to the kernel parameter itself would give
  // every thread a copy in local memory, which does not fit in the L1 that
  // the shared-memory carve-out leaves
  __shared__ SweepArgs s_args;
  extern __shared__ float4 ys_small[];
  if (threadIdx.x == 0) s_args = a;
  __syncthreads();
  const int nbig = a.nbig ? *a.nbig : 0;
  const int ncells = a.ncells_dev ? *a.ncells_dev : a.ncells;
  // one cell per CTA, or (persistent) cells taken in launch order from a
  // counter until none are left. The capacity bits of err_flag (4: workspace,
  // set by the gather; 8: output, set by an earlier compaction) do not change
  // while this kernel runs: every thread reads the same value.
  for (int round = 0;; ++round) {
    int pos, stop;
    if (a.work_next) {
      if (threadIdx.x == 0) {
        s_pos = atomicAdd(a.work_next, 1);
        s_stop = *a.err_flag & (4 | 8);
      }
      __syncthreads();
      pos = nbig + s_pos;
      stop = s_stop;
      __syncthreads();   // every thread has read s_pos before it is overwritten
    } else {
      if (round > 0) break;
      pos = nbig + blockIdx.x;
      stop = *a.err_flag & (4 | 8);
    }
    if (pos >= ncells || stop) break;
    const int J = a.order ? a.order[pos] : pos;
    if (a.cell_times && threadIdx.x == 0) a.cell_times[2 * J] = globaltimer();
    // dynamic shared memory: the staged support points, then the Newton buffer
    solve_cell<1, kMaxHW / 32>(s_args, J, sm, 0, ys_small, kStageSmall,
                               reinterpret_cast<float*>(ys_small + kStageSmall));
    if (a.cell_times && threadIdx.x == 0) a.cell_times[2 * J + 1] = globaltimer();
    __syncthreads();     // the cell's shared memory is free for the next one
  }
}

// The safeguard of §7.3 (a persistent wave over the cells in `order`): per
// cell, solves at 4ε, 16ε, … up to 4^escalate·ε, each warm-started from the
// duals the last one ended with, until one converges. After a solve converged
// at 4ε the cell is solved at ε from that result, and again at 4ε if that
// fails; a kept solve at a larger ε sets status bit 3. The attempts at 16ε
// and above stop after max_iter/4 iterations. A kernel
// of its own, so that the attempt loop leaves the main solve kernel's
// registers alone.
__global__ void __maxnreg__(168) k_sinkhorn_safeguard(SweepArgs a) {
  __shared__ SinkSmem sm;
  __shared__ int s_pos, s_stop, s_step, s_phase, s_more;
  __shared__ float s_f;
  __shared__ SweepArgs s_args;   // see k_sinkhorn
  extern __shared__ float4 ys_small[];
  if (threadIdx.x == 0) s_args = a;
  __syncthreads();
  const int ncells = a.ncells_dev ? *a.ncells_dev : a.ncells;
  for (;;) {
    if (threadIdx.x == 0) {
      s_pos = atomicAdd(a.work_next, 1);
      s_stop = *a.err_flag & (4 | 8);
    }
    __syncthreads();
    const int pos = s_pos, stop = s_stop;
    __syncthreads();   // every thread has read s_pos before it is overwritten
    if (pos >= ncells || stop) break;
    const int J = a.order[pos];
    // The attempt state lives in shared memory and is advanced by thread 0,
    // so that nothing stays live in registers across the solve.
    if (threadIdx.x == 0) {
      s_f = kSafeguardFactor;
      s_step = 1;
      s_phase = 0;   // 0: escalating; 1: at ε after 4ε converged; 2: 4ε again
      s_args.eps = a.eps * s_f;
      s_args.max_iter = a.max_iter;
    }
    __syncthreads();
    for (;;) {
      // dynamic shared memory: the staged support points, then the Newton buffer
      solve_cell<1, kMaxHW / 32>(s_args, J, sm, 0, ys_small, kStageSmall,
                                 reinterpret_cast<float*>(ys_small + kStageSmall));
      __syncthreads();   // the status written by thread 0; the cell's shared memory is free
      if (threadIdx.x == 0) {
        bool more = false, keep = false;
        const bool ok = (a.cell_status[J] & 7) == 0;
        if (s_phase == 0) {
          if (ok && s_step == 1) {
            s_phase = 1;
            s_f = 1.0f;
            more = true;
          } else if (ok) {
            keep = true;
          } else if (++s_step <= a.escalate) {
            s_f *= kSafeguardFactor;
            more = true;
          }
        } else if (s_phase == 1 && !ok) {
          s_phase = 2;
          s_f = kSafeguardFactor;
          more = true;
        } else if (s_phase == 2) {
          keep = ok;
        }
        if (keep) a.cell_status[J] |= 8;
        s_args.eps = more ? a.eps * s_f : a.eps;
        // the attempts at 16ε and above get a quarter of max_iter: a solve
        // that needs more at a larger ε is better taken one factor further,
        // and the attempts of one cell run one after another in one CTA, at
        // the tail of the launch (the repeat at 4ε starts from the failed
        // solve at ε and gets all of max_iter, as the first solve at 4ε did)
        s_args.max_iter = (more && s_step > 1) ? max(a.max_iter / 4, 64) : a.max_iter;
        s_more = more;
      }
      __syncthreads();
      if (!s_more) break;
    }
    __syncthreads();     // the cell's shared memory is free for the next one
  }
}

// a cluster of kClusterCTAs CTAs per cell, for the first nbig cells of the
// launch order (largest predicted work)
__global__ void __cluster_dims__(kClusterCTAs, 1, 1) __launch_bounds__(256, 2) k_sinkhorn_cluster(SweepArgs a) {
  __shared__ SinkSmem sm;
  __shared__ SweepArgs s_args;   // see k_sinkhorn
  const int c = blockIdx.x / kClusterCTAs;
  if (c >= *a.nbig) return;   // uniform over the cluster
  const int rank = (int)cg::this_cluster().block_rank();
  const int J = a.order[c];
  if (*a.err_flag & (4 | 8)) return;
  extern __shared__ float4 ys_big[];
  if (threadIdx.x == 0) s_args = a;
  __syncthreads();
  if (a.cell_times && threadIdx.x == 0 && rank == 0) a.cell_times[2 * J] = globaltimer();
  // dynamic shared memory: the staged support points, then the Newton buffer
  solve_cell<kClusterCTAs, 1>(s_args, J, sm, rank, ys_big, kStageBig, reinterpret_cast<float*>(ys_big + kStageBig));
  if (a.cell_times && threadIdx.x == 0 && rank == 0) a.cell_times[2 * J + 1] = globaltimer();
}

// ---------------------------------------------------------------------------
// launch order of the cells: largest predicted work first (Sinkhorn
// iterations of the cell's previous solve × support size × pixels), so that
// slowly converging cells do not start last and stretch the launch. Counting
// sort over 32 logarithmic buckets, one CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_order(SweepArgs a, int32_t* order, int* nbig) {
  if (*a.err_flag) return;   // an earlier step failed: nothing to order
  // buckets [0, 64): cells for clusters, [64, 128): cells for one CTA each;
  // half-octave buckets of predicted work inside each class, heaviest first
  constexpr int NB = 128;
  __shared__ int cnt[NB];
  __shared__ int off[NB];
  __shared__ double dws[32];
  __shared__ double s_thr;
  const int nc = a.ncells;
  for (int k = threadIdx.x; k < NB; k += blockDim.x) cnt[k] = 0;
  // FP32 work estimates and logarithms: this kernel runs on one SM, where
  // FP64 arithmetic would dominate its time
  auto work = [&](int J) {
    if (a.cell_off[J] < 0) return 1.0f;
    const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
    const int it = a.iters_hist ? max(a.iters_hist[J], 1) : 1;
    return (float)it * (float)max(a.cell_ny[J], 1) * (float)(g.H * g.W);
  };
  double tot = 0.0;
  for (int J = threadIdx.x; J < nc; J += blockDim.x) tot += (double)work(J);
  tot = block_sum<double>(tot, dws);
  // an eighth of one SM's fair share: a single CTA runs such a cell long
  // enough to stretch the launch
  if (threadIdx.x == 0) s_thr = a.max_big > 0 ? tot / (8.0 * 152.0) : 3.0e300;
  __syncthreads();
  const float thr = (float)fmin(s_thr, 3.0e38);
  auto bucket = [&](float w) {
    const int b2 = min(63, (int)(2.0f * log2f(fmaxf(w, 1.0f))));
    return (w >= thr ? 0 : 64) + 63 - b2;
  };
  // counts and positions with one shared-memory atomic per bucket and warp
  // (most cells fall into a few buckets: per-cell atomics serialise)
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < nc; base += blockDim.x) {
    const int J = base + threadIdx.x;
    const int bk = J < nc ? bucket(work(J)) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bk);
    if (bk >= 0 && (peers & lt) == 0) atomicAdd(&cnt[bk], __popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < NB; ++k) {
      off[k] = s;
      s += cnt[k];
      if (k == 63) *nbig = min(s, min(kMaxBig, a.max_big));
    }
  }
  __syncthreads();
  for (int base = 0; base < nc; base += blockDim.x) {
    const int J = base + threadIdx.x;
    const int bk = J < nc ? bucket(work(J)) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bk);
    const int leader = __ffs(peers) - 1;
    int pos0 = 0;
    if (bk >= 0 && lane == leader) pos0 = atomicAdd(&off[bk], __popc(peers));
    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
    if (bk >= 0) order[pos0 + __popc(peers & lt)] = J;
  }
}

// ---------------------------------------------------------------------------
// S6: prefix sums of the kept row lengths and compaction into the new CSR
// ---------------------------------------------------------------------------
constexpr int kScanTile = 1024;

__global__ void __launch_bounds__(kScanTile) k_scan_tiles(const int32_t* cnt, int64_t* tile_sum, int n,
                                                          const int* err_flag) {
  if (err_flag && *err_flag) return;   // an earlier step failed: the rows stay as they are
  __shared__ long long ws[32];
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  long long v = i < n ? cnt[i] : 0;
  v = block_sum<long long>(v, ws);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kScanTile) k_scan_top(int64_t* tile_sum, int ntiles, int64_t* rp_out,
                                                        int nrows, const int* err_flag) {
  if (err_flag && *err_flag) return;
  __shared__ long long lws[32];
  long long carry = 0;
  for (int t0 = 0; t0 < ntiles; t0 += kScanTile) {
    const int t = t0 + threadIdx.x;
    long long v = t < ntiles ? tile_sum[t] : 0;
    // 64-bit exclusive scan via warp shuffles
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) lws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long w = lws[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      lws[lane] = w;
    }
    __syncthreads();
    const long long before = warp > 0 ? lws[warp - 1] : 0;
    const long long chunk = lws[31];
    if (t < ntiles) tile_sum[t] = carry + before + x - v;
    carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) rp_out[nrows] = carry;
}

__global__ void __launch_bounds__(kScanTile) k_compact(const int32_t* cnt, const int64_t* src,
                                                       const int64_t* tile_off, int64_t* rp_out,
                                                       const int32_t* tmp_col, const uint64_t* tmp_val,
                                                       int32_t* col_out, uint64_t* val_out,
                                                       int64_t cap_out, int nrows, int* err_flag) {
  __shared__ int iws[32];
  __shared__ int64_t s_start[kScanTile];
  if (*err_flag) {
    // an earlier step failed (for example the other half-sweep of a
    // graph-replayed sweep overflowed its output): leave the output rows
    // alone, and mark the compaction as skipped so that k_copy_rows, which
    // copies on after an overflow of its own compaction (bit 8 alone), does
    // not write rows of a stale layout into this output
    if (threadIdx.x == 0) atomicOr(err_flag, 64);
    return;
  }
  const int i = blockIdx.x * kScanTile + threadIdx.x;
  const int c = i < nrows ? cnt[i] : 0;
  int tot;
  const int pre = block_exscan(c, iws, tot);
  const int64_t start = tile_off[blockIdx.x] + pre;
  if (i < nrows) rp_out[i] = start;
  s_start[threadIdx.x] = start;
  __syncthreads();
  if (tmp_col == nullptr) return;
  // warp-cooperative copies, one row per warp at a time
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < kScanTile; r += kScanTile / 32) {
    const int row = blockIdx.x * kScanTile + r;
    if (row >= nrows) break;
    const int len = cnt[row];
    const int64_t dst = s_start[r];
    if (dst + len > cap_out) {
      if (lane == 0) atomicOr(err_flag, 8);
      continue;
    }
    const int64_t s0 = src[row];
    for (int k = lane; k < len; k += 32) {
      col_out[dst + k] = tmp_col[s0 + k];
      val_out[dst + k] = tmp_val[s0 + k];
    }
  }
}

// one warp per row: copy the row's kept entries into the output CSR at the
// row start the scan gave (rp_out)
__global__ void __launch_bounds__(256) k_copy_rows(const int32_t* cnt, const int64_t* src, const int64_t* rp_out,
                                                   const int32_t* tmp_col, const uint64_t* tmp_val,
                                                   int32_t* col_out, uint64_t* val_out, int64_t cap_out,
                                                   int nrows, int* err_flag) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nrows || (*err_flag & ~8)) return;
  const int len = cnt[row];
  const int64_t dst = rp_out[row];
  if (dst + len > cap_out) {
    if (lane == 0) atomicOr(err_flag, 8);
    return;
  }
  const int64_t s0 = src[row];
  for (int k = lane; k < len; k += 32) {
    col_out[dst + k] = tmp_col[s0 + k];
    val_out[dst + k] = tmp_val[s0 + k];
  }
}

// ---------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_reduce_cells(SweepArgs a, SweepTotals* out) {
  __shared__ double dws[32];
  __shared__ long long lws[32];
  __shared__ int iws[32];
  double c = 0.0, e = 0.0, ev = 0.0, hf = 0.0;
  long long its = 0, nst = 0;
  int mx = 0, nc = 0, nf = 0, ov = 0, nl = 0, nj = 0, nesc = 0;
  for (int J = threadIdx.x; J < a.ncells; J += blockDim.x) {
    const int st = a.cell_status[J];
    if (a.cell_learned) {
      nl += a.cell_learned[J] == 1 ? 1 : 0;
      nj += a.cell_learned[J] >= 0 ? 1 : 0;
    }
    if (st & 4) { ++ov; continue; }
    const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
    ev += (double)(g.H * g.W) * (double)a.cell_ny[J] * (double)(a.cell_iters[J] + 1);
    c += a.cell_cost[J];
    e += a.cell_errx[J];
    its += a.cell_iters[J];
    if (a.cell_newton) {
      nst += a.cell_newton[J];
      hf += (double)a.cell_newton[J] * (double)(kNewtonN * kNewtonN) * (double)a.cell_ny[J];
    }
    mx = max(mx, a.cell_iters[J]);
    nc += (st & 1) ? 1 : 0;
    nf += (st & 2) ? 1 : 0;
    nesc += (st & 8) ? 1 : 0;
  }
  c = block_sum<double>(c, dws);
  e = block_sum<double>(e, dws);
  ev = block_sum<double>(ev, dws);
  its = block_sum<long long>(its, lws);
  nst = block_sum<long long>(nst, lws);
  hf = block_sum<double>(hf, dws);
  nc = block_sum<int>(nc, iws);
  nf = block_sum<int>(nf, iws);
  ov = block_sum<int>(ov, iws);
  nl = block_sum<int>(nl, iws);
  nj = block_sum<int>(nj, iws);
  nesc = block_sum<int>(nesc, iws);
  // max via shuffles
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) iws[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, iws[w]);
    out->cost = c;
    out->errx = e;
    out->kernel_evals = ev;
    out->iters_sum = its;
    out->newton_steps = nst;
    out->hessian_fma = hf;
    out->iters_max = m;
    out->not_converged = nc;
    out->nonfinite = nf;
    out->overflow = ov;
    out->learned = nl;
    out->compared = nj;
    out->rescued = a.rescued_dev ? *a.rescued_dev : 0;
    out->escalated = nesc;
  }
}

__global__ void __launch_bounds__(1024) k_collect_failed(SweepArgs a, int32_t* list, int* count, double min_err) {
  __shared__ int s_n;
  if (*a.err_flag) {   // an earlier step failed: the statuses are not this half-sweep's
    if (threadIdx.x == 0) *count = 0;
    return;
  }
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  // stopped at max_iter with a finite result, and still far from the
  // tolerance: an X-error above min_err·‖μ_J‖ (a cell that stalls just above
  // its tolerance is at the FP32 floor of its sums and gains nothing)
  for (int J = threadIdx.x; J < a.ncells; J += blockDim.x) {
    if ((a.cell_status[J] & 7) != 1) continue;
    const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
    uint64_t m = 0;
    for (int kr = 0; kr < g.nbr; ++kr)
      for (int kc = 0; kc < g.nbc; ++kc) m += a.L.M_q[(g.bi0 + kr) * a.L.nb + g.bj0 + kc];
    if (a.cell_errx[J] > min_err * ((double)m * (1.0 / kFixOne))) list[atomicAdd(&s_n, 1)] = J;
  }
  __syncthreads();
  if (threadIdx.x == 0) *count = s_n;
}

__global__ void k_scatter_rows(const int64_t* rp, int nrows, const int32_t* col, const uint64_t* val,
                               unsigned long long* dense) {
  const int64_t nnz = rp[nrows];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(dense + col[e], (unsigned long long)val[e]);
}

__global__ void k_y_error(const unsigned long long* dense, const uint64_t* nu, int n2, double* out) {
  __shared__ double dws[32];
  double s = 0.0;
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n2; y += gridDim.x * blockDim.x) {
    const long long d = (long long)(dense[y] - nu[y]);
    s += (double)(d < 0 ? -d : d);
  }
  s = block_sum<double>(s, dws);
  if (threadIdx.x == 0) atomicAdd(out, s * (1.0 / kFixOne));
}

// ---------------------------------------------------------------------------
// initial coupling μ⊗ν on the coarsest level (§6.4)
// ---------------------------------------------------------------------------
__global__ void k_init_product(LevelView L, int64_t* rp, int32_t* col, uint64_t* val, int imax) {
  const int n2 = L.n * L.n, nr = L.nb * L.nb;
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y < nr + 1 && y <= nr) rp[y] = (int64_t)y * n2;
  if (y >= n2) return;
  const uint64_t nu = L.nu_q[y];
  uint64_t rest = nu;
  for (int i = 0; i < nr; ++i) {
    col[(int64_t)i * n2 + y] = y;
    if (i == imax) continue;
    const uint64_t m = L.M_q[i];
    const uint64_t m4 = m >= (1ull << 62) ? 0xffffffffffffffffull : (m << 2);
    const uint64_t v = __umul64hi(nu, m4);   // ν(y)·M_i / 2^62
    val[(int64_t)i * n2 + y] = v;
    rest -= v;
  }
  val[(int64_t)imax * n2 + y] = rest;
}

// ---------------------------------------------------------------------------
// refinement (§6.4, eq. FineBasicMarginals)
// ---------------------------------------------------------------------------
__global__ void k_refine_count(RefineArgs r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nbf = r.F.nb, nbc = r.C.nb;
  if (i >= nbf * nbf) return;
  const int R = i / nbf, S = i - (i / nbf) * nbf;
  const int j = (R >> 1) * nbc + (S >> 1);
  r.cnt_f[i] = (int32_t)(4 * (r.rp_c[j + 1] - r.rp_c[j]));
}

__global__ void __launch_bounds__(128) k_refine_write(RefineArgs r) {
  const int i = blockIdx.x;
  const int nbf = r.F.nb, nbc = r.C.nb, nc = r.C.n, nf = r.F.n;
  const int R = i / nbf, S = i - (i / nbf) * nbf;
  const int j = (R >> 1) * nbc + (S >> 1);
  const int64_t c0 = r.rp_c[j];
  const int64_t len = r.rp_c[j + 1] - c0;
  const int32_t* row = r.col_c + c0;
  const int64_t o = r.rp_f[i];
  const double wmass = (double)r.F.M_q[i] / (double)r.C.M_q[j];
  for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
    const int yh = row[k];
    const int pi = yh / nc, pj = yh - (yh / nc) * nc;
    const int64_t k0 = lower_bound_row(row, len, pi * nc);
    const int64_t k1 = lower_bound_row(row, len, (pi + 1) * nc);
    const double vh = (double)r.val_c[c0 + k];
    const double nuh = (double)r.C.nu_q[yh];
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj) {
        const int y = (2 * pi + di) * nf + 2 * pj + dj;
        const int64_t pos = 4 * k0 + di * 2 * (k1 - k0) + 2 * (k - k0) + dj;
        const double v = vh * ((double)r.F.nu_q[y] / nuh) * wmass;
        r.col_f[o + pos] = y;
        r.val_f[o + pos] = (uint64_t)__double2ull_rn(v);
      }
  }
}

// α of the coarse level at coarse pixel (pr, pc), FP64, from the reduced
// storage of the cell of `cpart` containing it
__device__ double coarse_alpha(const LevelView& C, int cpart, const float* alpha_c, const int2* anchor_c,
                               int pr, int pc, CellGeom& gK) {
  const int K = cell_of_basic(cpart, pr / C.b, pc / C.b, C.nb);
  gK = cell_geom(cpart, K, C.nb, C.b);
  const int2 an = anchor_c[K];
  const double d2 = C.spacing * C.spacing;
  const int Dr = gK.r0 - an.x, Dc = gK.c0 - an.y;
  return (double)alpha_c[pr * C.n + pc] + 2.0 * d2 * ((double)Dr * (pr - gK.r0) + (double)Dc * (pc - gK.c0));
}

// first-order refinement of α inside the coarse cell (finite differences)
__device__ double fine_alpha(const LevelView& C, int cpart, const float* alpha_c, const int2* anchor_c,
                             int R, int S) {
  const int pr = R >> 1, pc = S >> 1;
  CellGeom gK;
  const double a0 = coarse_alpha(C, cpart, alpha_c, anchor_c, pr, pc, gK);
  CellGeom tmp;
  double dr = 0.0, dc = 0.0;
  if (gK.H > 1) {
    const int lr = pr - gK.r0;
    if (lr == 0) dr = coarse_alpha(C, cpart, alpha_c, anchor_c, pr + 1, pc, tmp) - a0;
    else if (lr == gK.H - 1) dr = a0 - coarse_alpha(C, cpart, alpha_c, anchor_c, pr - 1, pc, tmp);
    else
      dr = 0.5 * (coarse_alpha(C, cpart, alpha_c, anchor_c, pr + 1, pc, tmp) -
                  coarse_alpha(C, cpart, alpha_c, anchor_c, pr - 1, pc, tmp));
  }
  if (gK.W > 1) {
    const int lc = pc - gK.c0;
    if (lc == 0) dc = coarse_alpha(C, cpart, alpha_c, anchor_c, pr, pc + 1, tmp) - a0;
    else if (lc == gK.W - 1) dc = a0 - coarse_alpha(C, cpart, alpha_c, anchor_c, pr, pc - 1, tmp);
    else
      dc = 0.5 * (coarse_alpha(C, cpart, alpha_c, anchor_c, pr, pc + 1, tmp) -
                  coarse_alpha(C, cpart, alpha_c, anchor_c, pr, pc - 1, tmp));
  }
  const double orr = (R & 1) ? 0.25 : -0.25;
  const double occ = (S & 1) ? 0.25 : -0.25;
  return a0 + orr * dr + occ * dc;
}

__global__ void k_refine_duals(LevelView C, LevelView F, int cpart, const float* alpha_c,
                               const int2* anchor_c, int fpart, float* alpha_f, int2* anchor_f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= F.n * F.n) return;
  const int R = x / F.n, S = x - (x / F.n) * F.n;
  const int Jf = cell_of_basic(fpart, R / F.b, S / F.b, F.nb);
  const CellGeom gf = cell_geom(fpart, Jf, F.nb, F.b);
  // anchor: same physical displacement as the coarse cell holding the corner
  const int pr0 = gf.r0 >> 1, pc0 = gf.c0 >> 1;
  const int K0 = cell_of_basic(cpart, pr0 / C.b, pc0 / C.b, C.nb);
  const CellGeom gK0 = cell_geom(cpart, K0, C.nb, C.b);
  const int2 anK = anchor_c[K0];
  const int Dfr = 2 * (gK0.r0 - anK.x), Dfc = 2 * (gK0.c0 - anK.y);
  const double d2f = F.spacing * F.spacing;
  const double af = fine_alpha(C, cpart, alpha_c, anchor_c, R, S);
  const double acorner = fine_alpha(C, cpart, alpha_c, anchor_c, gf.r0, gf.c0);
  const int xr = R - gf.r0, xc = S - gf.c0;
  const double at = af - acorner - 2.0 * d2f * ((double)Dfr * xr + (double)Dfc * xc);
  alpha_f[x] = (float)at;
  if (xr == 0 && xc == 0) anchor_f[Jf] = make_int2(gf.r0 - Dfr, gf.c0 - Dfc);
}

// ---------------------------------------------------------------------------
// coupling of the last partition: one Y-iteration per cell (dd_get_plan)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_plan(SweepArgs a, float trunc, const int64_t* xrp, int32_t* xcnt,
                                              int32_t* pcol, double* pval, int write) {
  const int J = blockIdx.x;
  const LevelView& L = a.L;
  const CellGeom g = cell_geom(a.part, J, L.nb, L.b);
  const int64_t off = a.cell_off[J];
  if (off < 0) return;
  const int ny = a.cell_ny[J];
  const int2 anc_old = a.anchor[J], anc = a.anchor_new[J];
  const float d2 = (float)(L.spacing * L.spacing);
  const float inv_eln2 = 1.0f / (a.eps * kLn2);
  const float kappa = (float)(L.spacing * L.spacing / ((double)a.eps * 0.69314718055994530942));
  const int shr = anc.x - anc_old.x, shc = anc.y - anc_old.y;
  const int HW = g.H * g.W;
  __shared__ float F[kMaxHW];
  __shared__ int iws[32];
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    F[x] = (a.alpha[p] + 2.0f * d2 * (float)(shr * ar + shc * ac)) * inv_eln2 + L.log2mu[p];
  }
  __syncthreads();
  if (!write) {
    // G(y) = log2 ν(y) − LSE_x(F − κc̃): written to ws_g
    for (int k = threadIdx.x; k < ny; k += blockDim.x) {
      const int32_t e = a.ws_eta[off + k];
      const int er = eta_r(e), ec = eta_c(e);
      float m = kNegBig;
      for (int x = 0; x < HW; ++x) {
        const float tr = (float)(x / g.W - er), tc = (float)(x % g.W - ec);
        m = fmaxf(m, F[x] - kappa * (tr * tr + tc * tc));
      }
      float s = 0.f;
      for (int x = 0; x < HW; ++x) {
        const float tr = (float)(x / g.W - er), tc = (float)(x % g.W - ec);
        s += ex2(F[x] - kappa * (tr * tr + tc * tc) - m);
      }
      a.ws_g[off + k] = a.ws_lognu[off + k] - m - lg2(s);
    }
    __syncthreads();
  }
  for (int x = 0; x < HW; ++x) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    int carry = 0;
    for (int k0 = 0; k0 < ny; k0 += blockDim.x) {
      const int k = k0 + threadIdx.x;
      float v = 0.f;
      int y = 0;
      int keep = 0;
      if (k < ny) {
        const int32_t e = a.ws_eta[off + k];
        const int er = eta_r(e), ec = eta_c(e);
        const float tr = (float)(ar - er), tc = (float)(ac - ec);
        v = ex2(F[x] + a.ws_g[off + k] - kappa * (tr * tr + tc * tc));
        y = (anc.x + er) * L.n + anc.y + ec;
        keep = v > trunc;
      }
      int tot;
      const int pos = block_exscan(keep, iws, tot);
      if (write && keep) {
        pcol[xrp[p] + carry + pos] = y;
        pval[xrp[p] + carry + pos] = (double)v;
      }
      carry += tot;
    }
    if (!write && threadIdx.x == 0) xcnt[p] = carry;
  }
}

// ---------------------------------------------------------------------------
// objective of the last partition's coupling, cell by cell (dd_objective)
// ---------------------------------------------------------------------------
// π_J from the stored duals and one Y-iteration (the coupling of k_plan),
// written as π_J = u ⊗ v · K with K = e^{−c/ε}·μ⊗ν and the true cost c. In
// the cell's frame (pixel x = (r0+ar, c0+ac), support point y = anchor +
// (er, ec), D = corner − anchor) the kernel evaluates 2^(F + G − κ c̃) with
// c̃ = (ar−er)² + (ac−ec)², while c/(ε ln 2) = κ((D_r+ar−er)² + (D_c+ac−ec)²);
// the difference is a term in x plus a term in y, so
//   log2 u(x) = F(x) − log2 μ(x) + κ(D_r² + D_c² + 2D_r·ar + 2D_c·ac),
//   log2 v(y) = G(y) − log2 ν(y) − 2κ(D_r·er + D_c·ec).
// Per cell (Lemma 4.2 on the cell, §6.3):
//   primal_J = ⟨P_X π_J, log u⟩ + ⟨P_Y π_J, log v⟩ − ‖π_J‖
//            = Σ π_J (log π_J − log K − 1),
//   gap_J    = ⟨P_X π_J − μ_J, log u⟩ + ⟨P_Y π_J − ν_cell, log v⟩
//            = KL(π_J|K_J) − J_J(u, v)   (eq. EntropicOTDualObjective).
// log u is shifted by its μ-weighted mean and log v by the opposite amount
// (a change of gauge: primal_J is unchanged, gap_J moves by the mean times
// ‖ν_cell‖ − ‖μ_J‖, the mass lost to Truncate), so that the residuals
// multiply the spread of log u rather than its level. Entries are FP32
// exponentials as in k_plan; logs, residuals and sums are FP64.
__global__ void __launch_bounds__(256) k_objective(SweepArgs a, double* cell_obj) {
  const int J = blockIdx.x;
  const LevelView& L = a.L;
  const CellGeom g = cell_geom(a.part, J, L.nb, L.b);
  const int64_t off = a.cell_off[J];
  if (off < 0) {
    if (threadIdx.x == 0) {
      cell_obj[2 * (int64_t)J] = 0.0;
      cell_obj[2 * (int64_t)J + 1] = 0.0;
    }
    return;
  }
  const int ny = a.cell_ny[J];
  const int2 anc_old = a.anchor[J], anc = a.anchor_new[J];
  const float d2 = (float)(L.spacing * L.spacing);
  const float inv_eln2 = 1.0f / (a.eps * kLn2);
  const float kappa = (float)(L.spacing * L.spacing / ((double)a.eps * 0.69314718055994530942));
  const double kap = L.spacing * L.spacing / ((double)a.eps * 0.69314718055994530942);
  const double ln2 = 0.69314718055994530942;
  const double fix = 1.0 / kFixOne;
  const int shr = anc.x - anc_old.x, shc = anc.y - anc_old.y;
  const int Dr = g.r0 - anc.x, Dc = g.c0 - anc.y;
  const int HW = g.H * g.W;
  __shared__ float F[kMaxHW];
  __shared__ double lu[kMaxHW];
  __shared__ double dws[32];
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    F[x] = (a.alpha[p] + 2.0f * d2 * (float)(shr * ar + shc * ac)) * inv_eln2 + L.log2mu[p];
  }
  __syncthreads();
  // Y-iteration: G(y) = log2 ν_cell(y) − LSE_x(F − κc̃), into ws_g
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const int er = eta_r(e), ec = eta_c(e);
    float m = kNegBig;
    for (int x = 0; x < HW; ++x) {
      const float tr = (float)(x / g.W - er), tc = (float)(x % g.W - ec);
      m = fmaxf(m, F[x] - kappa * (tr * tr + tc * tc));
    }
    float s = 0.f;
    for (int x = 0; x < HW; ++x) {
      const float tr = (float)(x / g.W - er), tc = (float)(x % g.W - ec);
      s += ex2(F[x] - kappa * (tr * tr + tc * tc) - m);
    }
    a.ws_g[off + k] = a.ws_lognu[off + k] - m - lg2(s);
  }
  // log u in the true frame (natural log; 0 on pixels without mass), gauge
  double wl = 0.0, wm = 0.0;
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    const double mu = (double)L.mu_q[p] * fix;
    const double l = mu > 0.0 ? ln2 * ((double)F[x] - (double)L.log2mu[p] +
                                       kap * (double)(Dr * Dr + Dc * Dc + 2 * Dr * ar + 2 * Dc * ac))
                              : 0.0;
    lu[x] = l;
    wl += mu * l;
    wm += mu;
  }
  wl = block_sum<double>(wl, dws);   // contains the barriers after lu and ws_g
  wm = block_sum<double>(wm, dws);
  const double lbar = wm > 0.0 ? wl / wm : 0.0;
  double prim = 0.0, gap = 0.0;
  // the support points: P_Y π(y) and log v(y)
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const int er = eta_r(e), ec = eta_c(e);
    const float G = a.ws_g[off + k];
    const double nuc = (double)a.ws_nu[off + k] * fix;
    const int y = (anc.x + er) * L.n + anc.y + ec;
    const double nuy = (double)L.nu_q[y] * fix;
    if (!(nuc > 0.0 && nuy > 0.0)) continue;   // no coupling mass at y
    double sy = 0.0;
    for (int x = 0; x < HW; ++x) {
      const float tr = (float)(x / g.W - er), tc = (float)(x % g.W - ec);
      sy += (double)ex2(F[x] + G - kappa * (tr * tr + tc * tc));
    }
    const double lv = ln2 * ((double)G - log2(nuy) - 2.0 * kap * (double)(Dr * er + Dc * ec)) + lbar;
    prim += sy * lv;
    gap += (sy - nuc) * lv;
  }
  // the pixels: P_X π(x) and log u(x)
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int ar = x / g.W, ac = x - (x / g.W) * g.W;
    const int p = (g.r0 + ar) * L.n + g.c0 + ac;
    const double mu = (double)L.mu_q[p] * fix;
    if (!(mu > 0.0)) continue;   // π(x, ·) = 0 and log u = 0
    double sx = 0.0;
    for (int k = 0; k < ny; ++k) {
      const int32_t e = a.ws_eta[off + k];
      const float tr = (float)(ar - eta_r(e)), tc = (float)(ac - eta_c(e));
      sx += (double)ex2(F[x] + a.ws_g[off + k] - kappa * (tr * tr + tc * tc));
    }
    const double l = lu[x] - lbar;
    prim += sx * l - sx;
    gap += (sx - mu) * l;
  }
  prim = block_sum<double>(prim, dws);
  gap = block_sum<double>(gap, dws);
  if (threadIdx.x == 0) {
    cell_obj[2 * (int64_t)J] = prim;
    cell_obj[2 * (int64_t)J + 1] = gap;
  }
}

// Σ_J primal_J, Σ_J gap_J and Σ_J |gap_J| in a fixed order (one block)
__global__ void __launch_bounds__(1024) k_objective_sum(const double* cell_obj, int ncells, double* out) {
  __shared__ double dws[32];
  double p = 0.0, gs = 0.0, ga = 0.0;
  for (int J = threadIdx.x; J < ncells; J += blockDim.x) {
    p += cell_obj[2 * (int64_t)J];
    gs += cell_obj[2 * (int64_t)J + 1];
    ga += fabs(cell_obj[2 * (int64_t)J + 1]);
  }
  p = block_sum<double>(p, dws);
  gs = block_sum<double>(gs, dws);
  ga = block_sum<double>(ga, dws);
  if (threadIdx.x == 0) {
    out[0] = p;
    out[1] = gs;
    out[2] = ga;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_gather(const SweepArgs& a, cudaStream_t s) {
  k_gather<<<a.ncells, kGatherThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_order(const SweepArgs& a, int32_t* order, int* nbig, cudaStream_t s) {
  k_order<<<1, 1024, 0, s>>>(a, order, nbig);
  return cudaGetLastError();
}

// opt in to more than 48 KB of shared memory per CTA, once per device (a
// repeated or concurrent call only sets the same value again)
template <typename K>
static cudaError_t ensure_dyn_smem(K kernel, int bytes, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < 64;
  if (cached && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && cached) done[dev].store(true, std::memory_order_release);
  return e;
}

// resident CTAs of `kernel` on the whole GPU for a block size, queried once
// per device (so that a launch inside a stream capture makes no query)
template <typename K>
static cudaError_t resident_wave(K kernel, int threads, int smem, std::atomic<int> (*cache)[4], int& w) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int ti = threads == 32 ? 0 : threads == 64 ? 1 : threads == 128 ? 2 : 3;
  w = (dev >= 0 && dev < 64) ? cache[dev][ti].load() : 0;
  if (w > 0) return cudaSuccess;
  int sms = 0, per_sm = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
  w = sms * std::max(per_sm, 1);
  if (dev >= 0 && dev < 64) cache[dev][ti].store(w);
  return cudaSuccess;
}

cudaError_t launch_sinkhorn_safeguard(const SweepArgs& a, int threads, cudaStream_t s) {
  static std::atomic<bool> done[64];
  static std::atomic<int> wave[64][4];
  if (threads != 32 && threads != 64 && threads != 128 && threads != 256) threads = 128;
  if (!a.work_next || !a.order) return cudaErrorInvalidValue;
  const int smem = (int)(kStageSmall * sizeof(float4) + kNewtonFloats * sizeof(float));
  cudaError_t e = ensure_dyn_smem(k_sinkhorn_safeguard, smem, done);
  if (e != cudaSuccess) return e;
  int w = 0;
  if ((e = resident_wave(k_sinkhorn_safeguard, threads, smem, wave, w)) != cudaSuccess) return e;
  k_sinkhorn_safeguard<<<std::max(1, std::min(a.ncells, w)), threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sinkhorn(const SweepArgs& a, int threads, cudaStream_t s, bool persistent) {
  static std::atomic<bool> done[64];
  if (threads != 32 && threads != 64 && threads != 128 && threads != 256) threads = 128;
  const int smem = (int)(kStageSmall * sizeof(float4) + kNewtonFloats * sizeof(float));
  cudaError_t e = ensure_dyn_smem(k_sinkhorn, smem, done);
  if (e != cudaSuccess) return e;
  int grid = a.ncells;
  if (persistent) {
    // resident CTAs on the whole GPU, per device and block size, queried once
    // (so that a launch inside a stream capture makes no query)
    static std::atomic<int> wave[64][4];
    if (!a.work_next) return cudaErrorInvalidValue;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    const int ti = threads == 32 ? 0 : threads == 64 ? 1 : threads == 128 ? 2 : 3;
    int w = (dev >= 0 && dev < 64) ? wave[dev][ti].load() : 0;
    if (w <= 0) {
      int sms = 0, per_sm = 0;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sinkhorn, threads, smem)) != cudaSuccess)
        return e;
      w = sms * std::max(per_sm, 1);
      if (dev >= 0 && dev < 64) wave[dev][ti].store(w);
    }
    grid = std::max(1, std::min(a.ncells, w));
  } else {
    SweepArgs b = a;
    b.work_next = nullptr;
    k_sinkhorn<<<grid, threads, smem, s>>>(b);
    return cudaGetLastError();
  }
  k_sinkhorn<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sinkhorn_cluster(const SweepArgs& a, cudaStream_t s) {
  static std::atomic<bool> done[64];
  const int smem = (int)(kStageBig * sizeof(float4) + kNewtonFloats * sizeof(float));
  const cudaError_t e = ensure_dyn_smem(k_sinkhorn_cluster, smem, done);
  if (e != cudaSuccess) return e;
  k_sinkhorn_cluster<<<kMaxBig * kClusterCTAs, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_row_scan(const int32_t* cnt, int64_t* rp_out, int64_t* tile_sum, int nrows,
                            cudaStream_t s, const int* err_flag) {
  const int ntiles = (nrows + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<ntiles, kScanTile, 0, s>>>(cnt, tile_sum, nrows, err_flag);
  k_scan_top<<<1, kScanTile, 0, s>>>(tile_sum, ntiles, rp_out, nrows, err_flag);
  return cudaGetLastError();
}

cudaError_t launch_compact(const int32_t* cnt, const int64_t* src, const int64_t* tile_off,
                           int64_t* rp_out, const int32_t* tmp_col, const uint64_t* tmp_val,
                           int32_t* col_out, uint64_t* val_out, int64_t cap_out, int nrows,
                           int* err_flag, cudaStream_t s) {
  const int ntiles = (nrows + kScanTile - 1) / kScanTile;
  // row starts per tile, then the copies with one warp per row (enough CTAs
  // to cover the GPU)
  k_compact<<<ntiles, kScanTile, 0, s>>>(cnt, src, tile_off, rp_out, nullptr, nullptr, col_out, val_out, cap_out,
                                         nrows, err_flag);
  if (tmp_col != nullptr) {
    const int blocks = (int)(((int64_t)nrows * 32 + 255) / 256);
    k_copy_rows<<<blocks, 256, 0, s>>>(cnt, src, rp_out, tmp_col, tmp_val, col_out, val_out, cap_out, nrows,
                                       err_flag);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_product(LevelView L, int64_t* rp, int32_t* col, uint64_t* val, int imax,
                                cudaStream_t s) {
  const int n2 = L.n * L.n;
  k_init_product<<<(n2 + 255) / 256, 256, 0, s>>>(L, rp, col, val, imax);
  return cudaGetLastError();
}

// §7.2 colour image of the basic marginals: every entry ν_i(y) adds
// colour_i·ν_i(y) to pixel y (FP64 atomics) and ν_i(y) to its mass (64-bit
// fixed point, exact); the image is the mass-weighted mean colour
__global__ void __launch_bounds__(256) k_image_scatter(const int64_t* rp, const int32_t* col, const uint64_t* val,
                                                       int nrows, const float* colours, double* acc,
                                                       unsigned long long* mass) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < nrows; i += warps) {
    const float c0 = colours[3 * i], c1 = colours[3 * i + 1], c2 = colours[3 * i + 2];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
      const int y = col[e];
      const uint64_t v = val[e];
      const double m = (double)v * (1.0 / kFixOne);
      atomicAdd(acc + 3 * (int64_t)y, (double)c0 * m);
      atomicAdd(acc + 3 * (int64_t)y + 1, (double)c1 * m);
      atomicAdd(acc + 3 * (int64_t)y + 2, (double)c2 * m);
      atomicAdd(mass + y, (unsigned long long)v);
    }
  }
}

__global__ void k_image_finish(const double* acc, const unsigned long long* mass, int n2, float* rgb) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n2; y += gridDim.x * blockDim.x) {
    const double m = (double)mass[y] * (1.0 / kFixOne);
#pragma unroll
    for (int k = 0; k < 3; ++k) rgb[3 * (int64_t)y + k] = m > 0.0 ? (float)(acc[3 * (int64_t)y + k] / m) : 0.f;
  }
}

cudaError_t launch_coupling_image(const int64_t* rp, const int32_t* col, const uint64_t* val, int nrows, int n2,
                                  const float* colours, double* acc, unsigned long long* mass, float* rgb,
                                  cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)n2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(mass, 0, sizeof(unsigned long long) * (size_t)n2, s);
  if (e != cudaSuccess) return e;
  k_image_scatter<<<std::max(1, std::min((nrows + 7) / 8, 152 * 16)), 256, 0, s>>>(rp, col, val, nrows, colours,
                                                                                   acc, mass);
  k_image_finish<<<std::max(1, std::min((n2 + 255) / 256, 152 * 16)), 256, 0, s>>>(acc, mass, n2, rgb);
  return cudaGetLastError();
}

cudaError_t launch_collect_failed(const SweepArgs& a, int32_t* list, int* count, double min_err, cudaStream_t s) {
  k_collect_failed<<<1, 1024, 0, s>>>(a, list, count, min_err);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cells(const SweepArgs& a, SweepTotals* out_dev, cudaStream_t s) {
  k_reduce_cells<<<1, 1024, 0, s>>>(a, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_y_error(LevelView L, const int64_t* rp, const int32_t* col, const uint64_t* val,
                           int nrows, unsigned long long* scratch, double* out_dev, cudaStream_t s) {
  const int n2 = L.n * L.n;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)n2, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out_dev, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_scatter_rows<<<1216, 256, 0, s>>>(rp, nrows, col, val, scratch);
  const int blocks = (n2 + 255) / 256 < 1216 ? (n2 + 255) / 256 : 1216;
  k_y_error<<<blocks, 256, 0, s>>>(scratch, L.nu_q, n2, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_refine_count(const RefineArgs& r, cudaStream_t s) {
  const int nr = r.F.nb * r.F.nb;
  k_refine_count<<<(nr + 255) / 256, 256, 0, s>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_refine_write(const RefineArgs& r, cudaStream_t s) {
  k_refine_write<<<r.F.nb * r.F.nb, 128, 0, s>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_refine_duals(LevelView C, LevelView F, int cpart, const float* alpha_c,
                                const int2* anchor_c, int fpart, float* alpha_f, int2* anchor_f,
                                cudaStream_t s) {
  const int n2 = F.n * F.n;
  k_refine_duals<<<(n2 + 255) / 256, 256, 0, s>>>(C, F, cpart, alpha_c, anchor_c, fpart, alpha_f,
                                                  anchor_f);
  return cudaGetLastError();
}

cudaError_t launch_objective(const SweepArgs& a, double* cell_obj, double* out, cudaStream_t s) {
  k_objective<<<a.ncells, 256, 0, s>>>(a, cell_obj);
  k_objective_sum<<<1, 1024, 0, s>>>(cell_obj, a.ncells, out);
  return cudaGetLastError();
}

cudaError_t launch_plan(const SweepArgs& a, float trunc, const int64_t* xrp, int32_t* xcnt,
                        int32_t* pcol, double* pval, int write, cudaStream_t s) {
  k_plan<<<a.ncells, 256, 0, s>>>(a, trunc, xrp, xcnt, pcol, pval, write);
  return cudaGetLastError();
}

}  // namespace ddk
