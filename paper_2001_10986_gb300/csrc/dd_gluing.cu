// Dual gluing (§6.3, "Estimating the primal-dual gap"), eq. RelPDGap and the
// §6.4 interpolation of a glued dual into the cell frames of the next level,
// on the GPU.
//
//   k_glue_sides   per basic cell i: s±_i = log ⨍_i exp(±(α_A − α_B)/ε) dμ
//                  (μ-weighted means over the cell's pixels with mass).
//   k_glue_cg      the least-squares potential V on the cells of A: one
//                  cluster of 8 CTAs runs Jacobi-preconditioned conjugate
//                  gradients on the gluing graph's Laplacian, each CTA on a
//                  band of A-cell rows, the halo rows of the search direction
//                  copied from the neighbouring bands through distributed
//                  shared memory.
//   k_glue_apply   α̂ = α_A + ε·V[A cell]; pixels without mass get 0 or the
//                  affine least-squares fit of their A cell's α̂.
//   k_glue_frames  α̂ of a level interpolated linearly onto the level twice as
//                  fine and written into the cell frames of one partition
//                  there (per cell: the anchor from the slope of the affine
//                  fit, the fit's corner value removed).
//   k_gap_*        eq. RelPDGap for the coupling of the last partition.
//
// The gluing graph (§6.3): one vertex per A cell; every B cell meets at most
// four A cells, one basic cell each, and each ordered pair (i, i') of its
// distinct basic cells is an edge (A(i), A(i')) with value log q = s⁺_i +
// s⁻_{i'}. V minimises Σ_e ((V(j1) − V(j2)) + log q_e)² with Σ V = 0, i.e.
// L V = −Dᵀ log q with the Laplacian L = DᵀD of the edges. On the grid of
// A cells each pair of 4-neighbours shares two B cells and each pair of
// diagonal neighbours one, so L is the 9-point stencil with weight 4 on the
// 4-neighbours, 2 on the diagonal ones and the sum of the present weights on
// the diagonal — no edge list is stored.
//
// Nothing here waits on another CTA except through the cluster barrier of
// k_glue_cg, whose CTAs are co-scheduled by the hardware.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "dd_internal.cuh"

namespace cg = cooperative_groups;

namespace ddk {

namespace {

constexpr int kGlueCTAs = 8;          // CTAs of the CG cluster
constexpr int kGlueThreads = 512;     // threads per CTA
constexpr int kGlueNodesPerThread = 16;
constexpr int kGlueMaxHW = 256;       // pixels of the largest composite cell (b = 8)
constexpr double kLog2e = 1.4426950408889634074;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the block in a fixed order; ws holds ≥ 32 doubles
__device__ double block_sum_d(double v, double* ws) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += ws[w];
  __syncthreads();
  return t;
}

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// α = ε·log u of partition `part` at pixel (r, c), absolute frame, from the
// stored cell-frame dual (the conversion of dd_get_duals)
__device__ __forceinline__ double abs_dual(const LevelView& L, int part, const float* alpha, const int2* anchor,
                                           int r, int c) {
  const int J = cell_of_basic(part, r / L.b, c / L.b, L.nb);
  const CellGeom g = cell_geom(part, J, L.nb, L.b);
  const int2 an = anchor[J];
  const double d2 = L.spacing * L.spacing;
  return (double)alpha[(size_t)r * L.n + c] +
         2.0 * d2 * ((double)(g.r0 - an.x) * (r - g.r0) + (double)(g.c0 - an.y) * (c - g.c0));
}

// least-squares affine fit a0 + sr·i + sc·j from the sums over the fitted
// pixels (i, j centred at (ci, cj)); a ridge of 1e-12 of the trace on the
// slopes gives a block whose pixels lie on one line no slope across it
__device__ void affine_solve(double s1, double si, double sj, double sii, double sij, double sjj, double sa,
                             double sia, double sja, double ci, double cj, double& a0, double& sr, double& sc) {
  a0 = 0.0;
  sr = sc = 0.0;
  if (s1 == 0.0) return;
  const double rg = 1e-12 * (s1 + sii + sjj);
  const double A00 = s1, A01 = si, A02 = sj, A11 = sii + rg, A12 = sij, A22 = sjj + rg;
  // symmetric 3×3 system by cofactors
  const double c00 = A11 * A22 - A12 * A12, c01 = A02 * A12 - A01 * A22, c02 = A01 * A12 - A02 * A11;
  const double det = A00 * c00 + A01 * c01 + A02 * c02;
  if (det == 0.0) {
    a0 = sa / s1;
    return;
  }
  const double c11 = A00 * A22 - A02 * A02, c12 = A01 * A02 - A00 * A12, c22 = A00 * A11 - A01 * A01;
  const double m = (c00 * sa + c01 * sia + c02 * sja) / det;
  sr = (c01 * sa + c11 * sia + c12 * sja) / det;
  sc = (c02 * sa + c12 * sia + c22 * sja) / det;
  a0 = m - sr * ci - sc * cj;   // the fit's value at (0, 0)
}

// affine fit over the pixels of an H×W block that have mass; v[x] the values
// (row-major in the block), has[x] whether pixel x has mass; whole block
__device__ void block_affine_fit(const double* v, const unsigned char* has, int H, int W, double* ws, double& a0,
                                 double& sr, double& sc) {
  const double ci = 0.5 * (H - 1), cj = 0.5 * (W - 1);
  double s1 = 0, si = 0, sj = 0, sii = 0, sij = 0, sjj = 0, sa = 0, sia = 0, sja = 0;
  for (int x = threadIdx.x; x < H * W; x += blockDim.x) {
    if (!has[x]) continue;
    const double i = x / W - ci, j = x % W - cj, a = v[x];
    s1 += 1; si += i; sj += j; sii += i * i; sij += i * j; sjj += j * j;
    sa += a; sia += i * a; sja += j * a;
  }
  s1 = block_sum_d(s1, ws); si = block_sum_d(si, ws); sj = block_sum_d(sj, ws);
  sii = block_sum_d(sii, ws); sij = block_sum_d(sij, ws); sjj = block_sum_d(sjj, ws);
  sa = block_sum_d(sa, ws); sia = block_sum_d(sia, ws); sja = block_sum_d(sja, ws);
  affine_solve(s1, si, sj, sii, sij, sjj, sa, sia, sja, ci, cj, a0, sr, sc);
}

// order-preserving integer key of a double (for atomicMax)
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffll;
}
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffll);
}

}  // namespace

// ---------------------------------------------------------------------------
// s±_i per basic cell: one warp per cell
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_glue_sides(LevelView L, const float* alpha_A, const int2* anchor_A,
                                                    const float* alpha_B, const int2* anchor_B, double eps,
                                                    double* sp, double* sm) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= L.nb * L.nb) return;
  const int bi = i / L.nb, bj = i - (i / L.nb) * L.nb;
  const int bb = L.b * L.b;
  const double fix = 1.0 / kFixOne;
  double mp = -INFINITY, mm = -INFINITY;
  double dv[2];
  double wv[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = lane + 32 * k;
    dv[k] = 0.0;
    wv[k] = 0.0;
    if (x < bb) {
      const int r = bi * L.b + x / L.b, c = bj * L.b + x % L.b;
      const double w = (double)L.mu_q[(size_t)r * L.n + c] * fix;
      if (w > 0.0) {
        const double d = (abs_dual(L, 0, alpha_A, anchor_A, r, c) - abs_dual(L, 1, alpha_B, anchor_B, r, c)) / eps;
        dv[k] = d;
        wv[k] = w;
        mp = fmax(mp, d);
        mm = fmax(mm, -d);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
    mm = fmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
  }
  double tp = 0.0, tm = 0.0, mass = 0.0;
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (wv[k] > 0.0) {
      tp += wv[k] * exp(dv[k] - mp);
      tm += wv[k] * exp(-dv[k] - mm);
      mass += wv[k];
    }
  tp = warp_sum(tp);
  tm = warp_sum(tm);
  mass = warp_sum(mass);
  if (lane == 0) {
    // every basic cell has mass (Def. 3.1); NaN marks a violation
    sp[i] = mass > 0.0 ? mp + log(tp / mass) : NAN;
    sm[i] = mass > 0.0 ? mm + log(tm / mass) : NAN;
  }
}

// ---------------------------------------------------------------------------
// the potential V: preconditioned CG on one cluster
// ---------------------------------------------------------------------------
// CTA k owns the A-cell rows [k·rpc, min(na, (k+1)·rpc)). Its search
// direction p lives in shared memory with one halo row above and below
// ((rpc + 2)·na doubles, then rpc·na for the preconditioner's diagonal), copied from the neighbouring CTAs through
// distributed shared memory once per iteration, so that the stencil reads
// only local shared memory; the residual r and L p stay in registers (at
// most kGlueNodesPerThread nodes per thread), the iterate x in V. Scalars are reduced per CTA, exchanged through
// shared-memory slots and summed in rank order, so every CTA takes the same
// decisions. Cluster barriers per iteration: after the p·Lp partials, after
// the residual partials, after the update of p.
__global__ void __cluster_dims__(kGlueCTAs, 1, 1) __launch_bounds__(kGlueThreads, 1)
    k_glue_cg(int na, int nb, const double* sp, const double* sm, double tol, int max_iter, double* V,
              GlueInfo* info) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double glue_smem[];
  __shared__ double ws0[32], ws1[32];
  // one exchange slot per reduction site: a slot is written again only after
  // a later cluster barrier, which every CTA reaches after its reads of it
  __shared__ double slotA[2], slotB[2], slotC[2], bcast[2];
  const int rpc = (na + kGlueCTAs - 1) / kGlueCTAs;
  const int row0 = rank * rpc;
  const int rows = max(0, min(na, row0 + rpc) - row0);
  const int nloc = rows * na;
  double* p_h = glue_smem;        // row −1 of the band
  double* p_s = glue_smem + na;   // rows 0 … rows−1, then row `rows`
  double* dinv_s = glue_smem + (size_t)(rpc + 2) * na;   // 1/degree per node of the band
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // the sum over the cluster of two per-thread values, in rank order
  auto cluster_sum = [&](double v0, double v1, double* slot, double& s0, double& s1) {
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      ws0[warp] = v0;
      ws1[warp] = v1;
    }
    __syncthreads();
    if (warp == 0) {
      double a = lane < kGlueThreads / 32 ? ws0[lane] : 0.0;
      double b = lane < kGlueThreads / 32 ? ws1[lane] : 0.0;
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        slot[0] = a;
        slot[1] = b;
      }
    }
    cluster.sync();
    if (warp == 0) {
      double a = 0.0, b = 0.0;
      if (lane < kGlueCTAs) {
        const double* rs = cluster.map_shared_rank(slot, lane);
        a = rs[0];
        b = rs[1];
      }
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        bcast[0] = a;
        bcast[1] = b;
      }
    }
    __syncthreads();
    s0 = bcast[0];
    s1 = bcast[1];
  };
  // halo rows of p from the CTAs owning rows row0 − 1 and row0 + rows
  auto fetch_halo = [&]() {
    if (rows > 0) {
      if (row0 > 0) {
        const int o = (row0 - 1) / rpc;
        const double* src = cluster.map_shared_rank(p_s, o) + (size_t)(row0 - 1 - o * rpc) * na;
        for (int c = threadIdx.x; c < na; c += blockDim.x) p_h[c] = src[c];
      }
      if (row0 + rows < na) {
        const int o = (row0 + rows) / rpc;
        const double* src = cluster.map_shared_rank(p_s, o) + (size_t)(row0 + rows - o * rpc) * na;
        for (int c = threadIdx.x; c < na; c += blockDim.x) p_s[(size_t)rows * na + c] = src[c];
      }
    }
    __syncthreads();
  };
  auto degree = [&](int R, int C) -> double {
    const bool up = R > 0, dn = R < na - 1, lf = C > 0, rt = C < na - 1;
    return 4.0 * (up + dn + lf + rt) + 2.0 * ((up && lf) + (up && rt) + (dn && lf) + (dn && rt));
  };
  auto sidx = [&](int bi, int bj) { return (size_t)bi * nb + bj; };

  // right-hand side b = −Dᵀ log q, built from the B cells at the four
  // corners of each A cell; x = 0, r = b, p = z = b/deg
  double rreg[kGlueNodesPerThread];
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
    const double d = degree(row0 + l / na, l % na);
    dinv_s[l] = d > 0.0 ? 1.0 / d : 0.0;   // the preconditioner's diagonal
  }
  __syncthreads();
  auto dinv = [&](int l) { return dinv_s[l]; };
  double bb = 0.0, rz = 0.0;
#pragma unroll
  for (int k = 0; k < kGlueNodesPerThread; ++k) {
    const int l = threadIdx.x + k * kGlueThreads;
    rreg[k] = 0.0;
    if (l < nloc) {
      const int R = row0 + l / na, C = l % na;
      double b = 0.0;
      for (int dr = 0; dr < 2; ++dr)
        for (int dc = 0; dc < 2; ++dc) {
          const int Rb = R + dr, Cb = C + dc;                 // B cell (Rb, Cb)
          const int mi = 2 * R + dr, mj = 2 * C + dc;         // this A cell's basic cell in it
          const double spJ = sp[sidx(mi, mj)], smJ = sm[sidx(mi, mj)];
          for (int ei = 2 * Rb - 1; ei <= 2 * Rb; ++ei)
            for (int ej = 2 * Cb - 1; ej <= 2 * Cb; ++ej) {
              if (ei < 0 || ei >= nb || ej < 0 || ej >= nb || (ei == mi && ej == mj)) continue;
              b += sp[sidx(ei, ej)] + smJ - spJ - sm[sidx(ei, ej)];
            }
        }
      const double di = dinv(l);
      rreg[k] = b;
      p_s[l] = b * di;
      V[(size_t)R * na + C] = 0.0;
      bb += b * b;
      rz += b * b * di;
    }
  }
  cluster_sum(bb, rz, slotB, bb, rz);
  const double bnorm = sqrt(bb);
  double rnorm = bnorm;
  int it = 0;
  int converged = !(bnorm > 0.0);
  double qreg[kGlueNodesPerThread];
  if (!converged) {
    fetch_halo();
    for (; it < max_iter; ++it) {
      // q = L p on the band (row −1 at p_h, row `rows` after the band)
      double pq = 0.0;
#pragma unroll
      for (int k = 0; k < kGlueNodesPerThread; ++k) {
        const int l = threadIdx.x + k * kGlueThreads;
        qreg[k] = 0.0;
        if (l < nloc) {
          const int lr = l / na, C = l - (l / na) * na, R = row0 + lr;
          const double* up = lr > 0 ? p_s + (size_t)(lr - 1) * na : p_h;
          const double* mid = p_s + (size_t)lr * na;
          const double* dn = mid + na;
          const bool hu = R > 0, hd = R < na - 1, hl = C > 0, hr = C < na - 1;
          const double pc = mid[C];
          double nb4 = (hl ? mid[C - 1] : 0.0) + (hr ? mid[C + 1] : 0.0);
          double nb2 = 0.0;
          if (hu) {
            nb4 += up[C];
            nb2 += (hl ? up[C - 1] : 0.0) + (hr ? up[C + 1] : 0.0);
          }
          if (hd) {
            nb4 += dn[C];
            nb2 += (hl ? dn[C - 1] : 0.0) + (hr ? dn[C + 1] : 0.0);
          }
          const double q = degree(R, C) * pc - 4.0 * nb4 - 2.0 * nb2;
          qreg[k] = q;
          pq += pc * q;
        }
      }
      double dummy;
      cluster_sum(pq, 0.0, slotA, pq, dummy);
      if (!(pq > 0.0)) break;
      const double a = rz / pq;
      double rr = 0.0, rzn = 0.0;
#pragma unroll
      for (int k = 0; k < kGlueNodesPerThread; ++k) {
        const int l = threadIdx.x + k * kGlueThreads;
        if (l < nloc) {
          const size_t v = (size_t)(row0 + l / na) * na + l % na;
          V[v] += a * p_s[l];
          rreg[k] -= a * qreg[k];
          rr += rreg[k] * rreg[k];
          rzn += rreg[k] * rreg[k] * dinv(l);
        }
      }
      cluster_sum(rr, rzn, slotB, rr, rzn);
      rnorm = sqrt(rr);
      if (rnorm <= tol * bnorm) {
        converged = 1;
        ++it;
        break;
      }
      const double beta = rzn / rz;
      rz = rzn;
#pragma unroll
      for (int k = 0; k < kGlueNodesPerThread; ++k) {
        const int l = threadIdx.x + k * kGlueThreads;
        if (l < nloc) p_s[l] = rreg[k] * dinv(l) + beta * p_s[l];
      }
      cluster.sync();   // the neighbouring bands' new p is complete
      fetch_halo();
    }
  }
  // mean zero (the grid graph is connected: the gauge Σ V = 0)
  double xs = 0.0;
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) xs += V[(size_t)(row0 + l / na) * na + l % na];
  double dummy;
  cluster_sum(xs, 0.0, slotC, xs, dummy);
  const double mean = xs / ((double)na * na);
  for (int l = threadIdx.x; l < nloc; l += blockDim.x) V[(size_t)(row0 + l / na) * na + l % na] -= mean;
  if (rank == 0 && threadIdx.x == 0) {
    info->iters = it;
    info->converged = converged;
    info->rel_residual = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  }
  cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// α̂ on the pixels of each A cell
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_glue_apply(LevelView L, const float* alpha_A, const int2* anchor_A,
                                                    const double* V, double eps, int fill_massless,
                                                    double* alpha_hat) {
  const int J = blockIdx.x;
  const CellGeom g = cell_geom(0, J, L.nb, L.b);
  __shared__ double v[kGlueMaxHW];
  __shared__ unsigned char has[kGlueMaxHW];
  __shared__ double ws[32];
  const int HW = g.H * g.W;
  const double shift = eps * V[J];
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int r = g.r0 + x / g.W, c = g.c0 + x % g.W;
    has[x] = L.mu_q[(size_t)r * L.n + c] != 0;
    v[x] = has[x] ? abs_dual(L, 0, alpha_A, anchor_A, r, c) + shift : 0.0;
  }
  __syncthreads();
  double a0 = 0.0, sr = 0.0, sc = 0.0;
  if (fill_massless) block_affine_fit(v, has, g.H, g.W, ws, a0, sr, sc);
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int i = x / g.W, j = x % g.W;
    alpha_hat[(size_t)(g.r0 + i) * L.n + g.c0 + j] = has[x] ? v[x] : (fill_massless ? a0 + sr * i + sc * j : 0.0);
  }
}

// ---------------------------------------------------------------------------
// §6.4: α̂ of level C interpolated onto level F (twice as fine), written into
// the cell frames of partition `fpart` of F
// ---------------------------------------------------------------------------
// Fine pixel I sits at t = I/2 − 1/4 in coarse index units, between coarse
// centres k₀ = ⌊t⌋ (clamped to [0, n_c − 2]) and k₀ + 1 with weight t − k₀
// per axis (1/4 or 3/4; −1/4 or 5/4 over the outermost quarter step, the
// linear extrapolation), so affine α is reproduced exactly.
__global__ void __launch_bounds__(256) k_glue_frames(int n_c, const double* alpha_c, LevelView F, int fpart,
                                                     float* alpha_f, int2* anchor_f) {
  const int J = blockIdx.x;
  const CellGeom g = cell_geom(fpart, J, F.nb, F.b);
  __shared__ double v[kGlueMaxHW];
  __shared__ unsigned char has[kGlueMaxHW];
  __shared__ double ws[32];
  const int HW = g.H * g.W;
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int I = g.r0 + x / g.W, Jc = g.c0 + x % g.W;
    const double ti = 0.5 * I - 0.25, tj = 0.5 * Jc - 0.25;
    const int ki = min(max((int)floor(ti), 0), n_c - 2), kj = min(max((int)floor(tj), 0), n_c - 2);
    const double wi = ti - ki, wj = tj - kj;
    const double* a = alpha_c + (size_t)ki * n_c + kj;
    const double top = a[0] * (1.0 - wj) + a[1] * wj;
    const double bot = a[n_c] * (1.0 - wj) + a[n_c + 1] * wj;
    v[x] = top * (1.0 - wi) + bot * wi;
    has[x] = F.mu_q[(size_t)I * F.n + Jc] != 0;
  }
  __syncthreads();
  double a0, sr, sc;
  block_affine_fit(v, has, g.H, g.W, ws, a0, sr, sc);
  const double d2 = F.spacing * F.spacing;
  const int Dr = (int)llround(sr / (2.0 * d2)), Dc = (int)llround(sc / (2.0 * d2));
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const int i = x / g.W, j = x % g.W;
    alpha_f[(size_t)(g.r0 + i) * F.n + g.c0 + j] =
        has[x] ? (float)(v[x] - a0 - 2.0 * d2 * ((double)Dr * i + (double)Dc * j)) : 0.f;
  }
  if (threadIdx.x == 0) anchor_f[J] = make_int2(g.r0 - Dr, g.c0 - Dc);
}

// ---------------------------------------------------------------------------
// eq. RelPDGap: the Y-side of J(û, v̂)
// ---------------------------------------------------------------------------
// For the coupling of the last partition (support X_J × supp ν_cell per
// cell J, after the gather of that half-sweep) and the glued X-dual α̂:
//   S(y) = Σ_{J: y ∈ supp ν_cell(J)} Σ_{x ∈ X_J, μ(x) > 0} û(x) μ(x) e^{−c(x,y)/ε},
// the Y-dual that maximises J(û, ·) for the kernel restricted to the
// support is v̂(y) = 1/S(y). Pass 0: t_J(y) = log of the inner sum (FP64
// arguments shifted by their maximum, FP32 exponentials, as the coupling's
// entries) into tws and the running maximum M(y) over the cells; pass 1:
// S̃(y) += e^{t_J(y) − M(y)}, so that log S(y) = M(y) + log S̃(y).
__global__ void __launch_bounds__(256) k_gap_cells(SweepArgs a, const double* alpha_hat, double* tws,
                                                   long long* Mkey, double* St, int pass) {
  const int J = blockIdx.x;
  const LevelView& L = a.L;
  const int64_t off = a.cell_off[J];
  if (off < 0) return;
  const int ny = a.cell_ny[J];
  const int2 anc = a.anchor_new[J];
  if (pass == 1) {
    for (int k = threadIdx.x; k < ny; k += blockDim.x) {
      const int32_t e = a.ws_eta[off + k];
      const size_t y = (size_t)(anc.x + eta_r(e)) * L.n + anc.y + eta_c(e);
      atomicAdd(&St[y], exp(tws[off + k] - dkey_inv(Mkey[y])));
    }
    return;
  }
  const CellGeom g = cell_geom(a.part, J, L.nb, L.b);
  const int HW = g.H * g.W;
  __shared__ double Fx[kGlueMaxHW];
  const double inv_eps = 1.0 / (double)a.eps;
  const double kap = L.spacing * L.spacing * inv_eps;
  for (int x = threadIdx.x; x < HW; x += blockDim.x) {
    const size_t p = (size_t)(g.r0 + x / g.W) * L.n + g.c0 + x % g.W;
    const double mu = (double)L.mu_q[p] / kFixOne;
    Fx[x] = mu > 0.0 ? alpha_hat[p] * inv_eps + log(mu) : -INFINITY;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const int yr = anc.x + eta_r(e), yc = anc.y + eta_c(e);
    double m = -INFINITY;
    for (int x = 0; x < HW; ++x) {
      const double dr = (double)(g.r0 + x / g.W - yr), dc = (double)(g.c0 + x % g.W - yc);
      m = fmax(m, Fx[x] - kap * (dr * dr + dc * dc));
    }
    float s = 0.f;
    for (int x = 0; x < HW; ++x) {
      const double dr = (double)(g.r0 + x / g.W - yr), dc = (double)(g.c0 + x % g.W - yc);
      s += ex2f((float)((Fx[x] - kap * (dr * dr + dc * dc) - m) * kLog2e));
    }
    const double t = m + log((double)s);
    tws[off + k] = t;
    atomicMax(&Mkey[(size_t)yr * L.n + yc], dkey(t));
  }
}

// per block: Σ_x μ α̂/ε, −Σ_y ν (M + log S̃), Σ_{y covered} ν, #{y: ν > 0, S = 0}
__global__ void __launch_bounds__(256) k_gap_pixels(LevelView L, const double* alpha_hat, double eps,
                                                    const long long* Mkey, const double* St, double* part) {
  __shared__ double ws[32];
  const size_t n2 = (size_t)L.n * L.n;
  double dmu = 0.0, dnu = 0.0, cov = 0.0, miss = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n2; p += (size_t)gridDim.x * blockDim.x) {
    const double mu = (double)L.mu_q[p] / kFixOne, nu = (double)L.nu_q[p] / kFixOne;
    if (mu > 0.0) dmu += mu * alpha_hat[p] / eps;
    if (nu > 0.0) {
      if (St[p] > 0.0) {
        dnu -= nu * (dkey_inv(Mkey[p]) + log(St[p]));
        cov += nu;
      } else {
        miss += 1.0;
      }
    }
  }
  dmu = block_sum_d(dmu, ws);
  dnu = block_sum_d(dnu, ws);
  cov = block_sum_d(cov, ws);
  miss = block_sum_d(miss, ws);
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x] = dmu;
    part[4 * blockIdx.x + 1] = dnu;
    part[4 * blockIdx.x + 2] = cov;
    part[4 * blockIdx.x + 3] = miss;
  }
}

__global__ void __launch_bounds__(256) k_gap_final(const double* part, int nparts, double* out) {
  __shared__ double ws[32];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int k = 0; k < 4; ++k) s[k] += part[4 * b + k];
  for (int k = 0; k < 4; ++k) {
    const double t = block_sum_d(s[k], ws);
    if (threadIdx.x == 0) out[k] = t;
  }
}

__global__ void k_fill_ll(long long* p, size_t n, long long v) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int glue_max_cells_per_side() {
  // rpc·na ≤ threads × nodes per thread with rpc = ⌈na/8⌉
  int m = 0;
  for (int na = 1; na <= 4096; ++na)
    if ((size_t)((na + kGlueCTAs - 1) / kGlueCTAs) * na <= (size_t)kGlueThreads * kGlueNodesPerThread) m = na;
  return m;
}

cudaError_t launch_glue_potential(LevelView L, const float* alpha_A, const int2* anchor_A, const float* alpha_B,
                                  const int2* anchor_B, double eps, double tol, int max_iter, double* sp,
                                  double* sm, double* V, GlueInfo* info, cudaStream_t s) {
  const int nbasic = L.nb * L.nb;
  k_glue_sides<<<(nbasic * 32 + 255) / 256, 256, 0, s>>>(L, alpha_A, anchor_A, alpha_B, anchor_B, eps, sp, sm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int na = L.nb / 2;
  if (na > glue_max_cells_per_side()) return cudaErrorInvalidValue;
  const int rpc = (na + kGlueCTAs - 1) / kGlueCTAs;
  const size_t smem = sizeof(double) * (size_t)(2 * rpc + 2) * na;
  e = cudaFuncSetAttribute(k_glue_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_glue_cg<<<kGlueCTAs, kGlueThreads, smem, s>>>(na, L.nb, sp, sm, tol, max_iter, V, info);
  return cudaGetLastError();
}

cudaError_t launch_glue_apply(LevelView L, const float* alpha_A, const int2* anchor_A, const double* V, double eps,
                              int fill_massless, double* alpha_hat, cudaStream_t s) {
  const int na = L.nb / 2;
  k_glue_apply<<<na * na, 256, 0, s>>>(L, alpha_A, anchor_A, V, eps, fill_massless, alpha_hat);
  return cudaGetLastError();
}

cudaError_t launch_glue_frames(int n_c, const double* alpha_c, LevelView F, int fpart, float* alpha_f,
                               int2* anchor_f, cudaStream_t s) {
  k_glue_frames<<<num_cells(fpart, F.nb), 256, 0, s>>>(n_c, alpha_c, F, fpart, alpha_f, anchor_f);
  return cudaGetLastError();
}

cudaError_t launch_gap(const SweepArgs& a, const double* alpha_hat, double* tws, long long* Mkey, double* St,
                       double* part, int nparts, double* out, cudaStream_t s) {
  const size_t n2 = (size_t)a.L.n * a.L.n;
  k_fill_ll<<<1024, 256, 0, s>>>(Mkey, n2, (long long)0x8000000000000000ull);
  cudaError_t e = cudaMemsetAsync(St, 0, sizeof(double) * n2, s);
  if (e != cudaSuccess) return e;
  k_gap_cells<<<a.ncells, 256, 0, s>>>(a, alpha_hat, tws, Mkey, St, 0);
  k_gap_cells<<<a.ncells, 256, 0, s>>>(a, alpha_hat, tws, Mkey, St, 1);
  k_gap_pixels<<<nparts, 256, 0, s>>>(a.L, alpha_hat, (double)a.eps, Mkey, St, part);
  k_gap_final<<<1, 256, 0, s>>>(part, nparts, out);
  return cudaGetLastError();
}

}  // namespace ddk
