// Dual gluing (§6.3, "Estimating the primal-dual gap"): the least-squares
// step that turns the edge values log q of the gluing graph into a potential
// V on its vertices (a discrete Helmholtz decomposition: the gradient part of
// the edge values). Host code in FP64; the graph has one vertex per cell of
// partition A (16 384 at 1024² with 4×4 basic cells) and at most 12 edges
// per B cell, so one solve costs well under a millisecond per iteration.
//
// Normal equations: with D the edge–vertex incidence matrix (row e has +1 at
// j1_e and −1 at j2_e), V minimises ‖D V + log q‖², i.e. L V = −Dᵀ log q with
// the graph Laplacian L = DᵀD (edge multiplicities counted). The right-hand
// side lies in the range of L, so conjugate gradients (Jacobi-preconditioned
// by the vertex degrees) converge; the solution is then shifted to mean zero
// on every connected component, which is the minimum-norm least-squares
// solution and, on a connected graph, the gauge Σ V = 0.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "dd.h"

namespace {

int find_root(std::vector<int32_t>& parent, int32_t v) {
  while (parent[v] != v) {
    parent[v] = parent[parent[v]];
    v = parent[v];
  }
  return v;
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

}  // namespace

extern "C" dd_status dd_glue_potential(int32_t n_nodes, int64_t n_edges, const int32_t* j1, const int32_t* j2,
                                       const double* logq, double tol, int32_t max_iter, double* V,
                                       int32_t* iters, double* rel_residual) {
  if (n_nodes < 1 || n_edges < 0 || !V || !(tol >= 0.0) || max_iter < 0) return DD_ERR_ARG;
  if (n_edges > 0 && (!j1 || !j2 || !logq)) return DD_ERR_ARG;
  for (int64_t e = 0; e < n_edges; ++e)
    if (j1[e] < 0 || j1[e] >= n_nodes || j2[e] < 0 || j2[e] >= n_nodes || !std::isfinite(logq[e]))
      return DD_ERR_ARG;
  const size_t n = (size_t)n_nodes;
  try {
    std::vector<double> b(n, 0.0), deg(n, 0.0), x(n, 0.0), r, z(n), p(n), q(n);
    // a loop edge (j1 = j2) has the constant residual log q and adds nothing
    for (int64_t e = 0; e < n_edges; ++e) {
      if (j1[e] == j2[e]) continue;
      b[j1[e]] -= logq[e];
      b[j2[e]] += logq[e];
      deg[j1[e]] += 1.0;
      deg[j2[e]] += 1.0;
    }
    auto laplacian = [&](const std::vector<double>& v, std::vector<double>& out) {
      std::fill(out.begin(), out.end(), 0.0);
      for (int64_t e = 0; e < n_edges; ++e) {
        if (j1[e] == j2[e]) continue;
        const double d = v[j1[e]] - v[j2[e]];
        out[j1[e]] += d;
        out[j2[e]] -= d;
      }
    };
    auto precondition = [&](const std::vector<double>& in, std::vector<double>& out) {
      for (size_t i = 0; i < n; ++i) out[i] = deg[i] > 0.0 ? in[i] / deg[i] : 0.0;
    };
    r = b;
    const double bnorm = std::sqrt(dot(b, b));
    double rnorm = bnorm;
    int32_t it = 0;
    bool converged = bnorm == 0.0;
    if (!converged) {
      precondition(r, z);
      p = z;
      double rz = dot(r, z);
      for (; it < max_iter; ++it) {
        laplacian(p, q);
        const double pq = dot(p, q);
        if (!(pq > 0.0)) break;
        const double a = rz / pq;
        for (size_t i = 0; i < n; ++i) {
          x[i] += a * p[i];
          r[i] -= a * q[i];
        }
        rnorm = std::sqrt(dot(r, r));
        if (rnorm <= tol * bnorm) {
          converged = true;
          ++it;
          break;
        }
        precondition(r, z);
        const double rz_new = dot(r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      }
    }
    // mean zero on every connected component
    std::vector<int32_t> parent(n);
    std::iota(parent.begin(), parent.end(), 0);
    for (int64_t e = 0; e < n_edges; ++e) {
      const int32_t ra = find_root(parent, j1[e]), rb = find_root(parent, j2[e]);
      if (ra != rb) parent[ra] = rb;
    }
    std::vector<double> csum(n, 0.0), ccount(n, 0.0);
    for (size_t i = 0; i < n; ++i) {
      const int32_t root = find_root(parent, (int32_t)i);
      csum[root] += x[i];
      ccount[root] += 1.0;
    }
    for (size_t i = 0; i < n; ++i) {
      const int32_t root = find_root(parent, (int32_t)i);
      V[i] = x[i] - csum[root] / ccount[root];
    }
    if (iters) *iters = it;
    if (rel_residual) *rel_residual = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    return converged ? DD_OK : DD_ERR_NOT_CONVERGED;
  } catch (...) {
    return DD_ERR_OOM;
  }
}

// The glued X-dual of §6.3 on an n×n grid with b×b basic cells, from the
// duals of both partitions (α = ε·log u, FP64, as dd_get_duals returns them).
// A cell of A and a cell of B meet in at most one basic cell i; on it
//   s⁺_i = log ⨍_i exp((α_A − α_B)/ε) dμ,   s⁻_i = log ⨍_i exp((α_B − α_A)/ε) dμ
// (μ-weighted means), and every ordered pair (i, i') of distinct basic cells
// of one B cell gives the edge (A(i), A(i')) with log q = s⁺_i + s⁻_{i'}.
// Then V = dd_glue_potential(edges) and α̂ = α_A + ε·V on every A cell (0 on
// pixels without mass).
extern "C" dd_status dd_glue_duals_host(int32_t n, int32_t b, const double* mu, const double* alpha_A,
                                        const double* alpha_B, double eps, double* alpha_hat, double* V) {
  if (n < 2 || b < 1 || n % b != 0 || (n / b) % 2 != 0 || !mu || !alpha_A || !alpha_B || !alpha_hat ||
      !(eps > 0.0) || !std::isfinite(eps))
    return DD_ERR_ARG;
  const int nb = n / b, na = nb / 2, nbB = nb / 2 + 1;
  const size_t n2 = (size_t)n * n;
  for (size_t p = 0; p < n2; ++p)
    if (!std::isfinite(mu[p]) || mu[p] < 0.0 || !std::isfinite(alpha_A[p]) || !std::isfinite(alpha_B[p]))
      return DD_ERR_ARG;
  try {
    // per basic cell: log of the μ-weighted means of exp(±(α_A − α_B)/ε)
    std::vector<double> sp((size_t)nb * nb), sm((size_t)nb * nb);
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = 0; bj < nb; ++bj) {
        double mp = -INFINITY, mm = -INFINITY, mass = 0.0;
        for (int r = bi * b; r < (bi + 1) * b; ++r)
          for (int c = bj * b; c < (bj + 1) * b; ++c) {
            const size_t p = (size_t)r * n + c;
            if (!(mu[p] > 0.0)) continue;
            const double d = (alpha_A[p] - alpha_B[p]) / eps;
            mp = std::fmax(mp, d);
            mm = std::fmax(mm, -d);
            mass += mu[p];
          }
        if (!(mass > 0.0)) return DD_ERR_ARG;   // a basic cell needs positive mass (Def. 3.1)
        double tp = 0.0, tm = 0.0;
        for (int r = bi * b; r < (bi + 1) * b; ++r)
          for (int c = bj * b; c < (bj + 1) * b; ++c) {
            const size_t p = (size_t)r * n + c;
            if (!(mu[p] > 0.0)) continue;
            const double d = (alpha_A[p] - alpha_B[p]) / eps;
            tp += mu[p] * std::exp(d - mp);
            tm += mu[p] * std::exp(-d - mm);
          }
        sp[(size_t)bi * nb + bj] = mp + std::log(tp / mass);
        sm[(size_t)bi * nb + bj] = mm + std::log(tm / mass);
      }
    // edges through the cells of B (B cell (R, C) holds basic rows 2R−1, 2R
    // and columns 2C−1, 2C that exist)
    std::vector<int32_t> j1, j2;
    std::vector<double> lq;
    for (int R = 0; R < nbB; ++R)
      for (int Cc = 0; Cc < nbB; ++Cc) {
        int cells[4], k = 0;
        for (int di = 0; di < 2; ++di)
          for (int dj = 0; dj < 2; ++dj) {
            const int bi = 2 * R - 1 + di, bj = 2 * Cc - 1 + dj;
            if (bi >= 0 && bi < nb && bj >= 0 && bj < nb) cells[k++] = bi * nb + bj;
          }
        for (int u = 0; u < k; ++u)
          for (int w = 0; w < k; ++w) {
            if (u == w) continue;
            const int iu = cells[u], iw = cells[w];
            j1.push_back((iu / nb / 2) * na + (iu % nb) / 2);
            j2.push_back((iw / nb / 2) * na + (iw % nb) / 2);
            lq.push_back(sp[iu] + sm[iw]);
          }
      }
    std::vector<double> pot((size_t)na * na);
    const dd_status st = dd_glue_potential(na * na, (int64_t)j1.size(), j1.data(), j2.data(), lq.data(), 1e-13,
                                           100000, pot.data(), nullptr, nullptr);
    if (st != DD_OK) return st;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        const size_t p = (size_t)r * n + c;
        const int ja = (r / b / 2) * na + (c / b) / 2;
        alpha_hat[p] = mu[p] > 0.0 ? alpha_A[p] + eps * pot[ja] : 0.0;
      }
    if (V)
      for (int j = 0; j < na * na; ++j) V[j] = pot[j];
    return DD_OK;
  } catch (...) {
    return DD_ERR_OOM;
  }
}

// Linear interpolation in log space (on α = ε·log û) from an n_c×n_c level to
// the 2n_c×2n_c level (§6.4): fine pixel I lies at t = I/2 − 1/4 in coarse
// index units, between coarse centres k₀ = ⌊t⌋ and k₀ + 1 with weight t − k₀
// (1/4 or 3/4) per axis; the outermost fine pixels lie a quarter step
// outside the outermost centres and take the linear extrapolation of the
// last two (weights −1/4 and 5/4). Affine α is reproduced exactly.
extern "C" dd_status dd_interpolate_dual_host(int32_t n_coarse, const double* alpha_c, double* alpha_f) {
  if (n_coarse < 2 || !alpha_c || !alpha_f) return DD_ERR_ARG;
  const int nc = n_coarse, nf = 2 * n_coarse;
  try {
    std::vector<int> k0(nf);
    std::vector<double> w(nf);
    for (int I = 0; I < nf; ++I) {
      const double t = 0.5 * I - 0.25;
      int k = (int)std::floor(t);
      k = k < 0 ? 0 : (k > nc - 2 ? nc - 2 : k);
      k0[I] = k;
      w[I] = t - k;
    }
    std::vector<double> rows((size_t)nf * nc);   // interpolated along the rows first
    for (int I = 0; I < nf; ++I)
      for (int c = 0; c < nc; ++c)
        rows[(size_t)I * nc + c] = alpha_c[(size_t)k0[I] * nc + c] * (1.0 - w[I]) +
                                   alpha_c[(size_t)(k0[I] + 1) * nc + c] * w[I];
    for (int I = 0; I < nf; ++I)
      for (int J = 0; J < nf; ++J)
        alpha_f[(size_t)I * nf + J] = rows[(size_t)I * nc + k0[J]] * (1.0 - w[J]) +
                                      rows[(size_t)I * nc + k0[J] + 1] * w[J];
    return DD_OK;
  } catch (...) {
    return DD_ERR_OOM;
  }
}

// eq. RelPDGap for a coupling π (sparse, one row per X pixel: the output of
// dd_get_plan) and a glued X-dual α̂ = ε·log û on an n×n level (pixel
// spacing 1/n, c = |x − y|²). K = e^{−c/ε}·μ⊗ν with μ, ν normalised to mass 1.
//   primal = KL(π|K) − ‖K‖ = Σ_entries π (log π − log K − 1);
//   v̂(y)  = 1 / S(y), S(y) = Σ_{x: π(x,y) > 0} û(x) μ(x) e^{−c(x,y)/ε}, the
//           Y-dual that maximises J(û, ·) for the kernel restricted to the
//           support of π (every y with ν(y) > 0 carries entries of π);
//   J − ‖K‖ = ⟨μ, log û⟩ + ⟨ν, log v̂⟩ − Σ_{supp π} û v̂ K
//           = Σ_x μ α̂/ε − Σ_y ν log S(y) − Σ_{y covered} ν(y);
//   gap = primal − (J − ‖K‖), rel = gap / primal.
extern "C" dd_status dd_relative_pd_gap_host(int32_t n, const double* mu, const double* nu, double eps,
                                             const int64_t* row_ptr, const int32_t* col, const double* val,
                                             const double* alpha_hat, double* rel, double* gap, double* primal) {
  if (n < 1 || !mu || !nu || !row_ptr || !alpha_hat || !(eps > 0.0) || !std::isfinite(eps)) return DD_ERR_ARG;
  const size_t n2 = (size_t)n * n;
  if (row_ptr[0] != 0) return DD_ERR_ARG;
  for (size_t x = 0; x < n2; ++x)
    if (row_ptr[x + 1] < row_ptr[x]) return DD_ERR_ARG;
  const int64_t nnz = row_ptr[n2];
  if (nnz > 0 && (!col || !val)) return DD_ERR_ARG;
  double smu = 0.0, snu = 0.0;
  for (size_t p = 0; p < n2; ++p) {
    if (!std::isfinite(mu[p]) || mu[p] < 0.0 || !std::isfinite(nu[p]) || nu[p] < 0.0) return DD_ERR_ARG;
    smu += mu[p];
    snu += nu[p];
  }
  if (!(smu > 0.0) || !(snu > 0.0)) return DD_ERR_ARG;
  for (int64_t e = 0; e < nnz; ++e)
    if (col[e] < 0 || (size_t)col[e] >= n2 || !std::isfinite(val[e]) || val[e] < 0.0) return DD_ERR_ARG;
  try {
    const double h2 = 1.0 / ((double)n * n);
    auto cost_over_eps = [&](size_t x, int32_t y) {
      const double dr = (double)((long)(x / n) - (long)(y / n)), dc = (double)((long)(x % n) - (long)(y % n));
      return h2 * (dr * dr + dc * dc) / eps;
    };
    // S(y) in log form: the largest exponent per y, then the sum
    std::vector<double> m(n2, -INFINITY), s(n2, 0.0);
    double pr = 0.0, dual_mu = 0.0;
    for (size_t x = 0; x < n2; ++x) {
      const double mx = mu[x] / smu;
      if (!(mx > 0.0)) continue;
      dual_mu += mx * alpha_hat[x] / eps;
      for (int64_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
        if (!(val[e] > 0.0)) continue;
        const int32_t y = col[e];
        const double ny = nu[y] / snu;
        if (!(ny > 0.0)) return DD_ERR_ARG;   // π has mass where ν has none
        const double coe = cost_over_eps(x, y);
        pr += val[e] * (std::log(val[e]) + coe - std::log(mx) - std::log(ny) - 1.0);
        m[y] = std::fmax(m[y], alpha_hat[x] / eps + std::log(mx) - coe);
      }
    }
    for (size_t x = 0; x < n2; ++x) {
      const double mx = mu[x] / smu;
      if (!(mx > 0.0)) continue;
      for (int64_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
        if (!(val[e] > 0.0)) continue;
        const int32_t y = col[e];
        s[y] += std::exp(alpha_hat[x] / eps + std::log(mx) - cost_over_eps(x, y) - m[y]);
      }
    }
    double dual_nu = 0.0, covered = 0.0;
    for (size_t y = 0; y < n2; ++y) {
      const double ny = nu[y] / snu;
      if (!(ny > 0.0)) continue;
      if (!(s[y] > 0.0)) return DD_ERR_ARG;    // ν(y) > 0 but no entry of π at y
      dual_nu -= ny * (m[y] + std::log(s[y]));
      covered += ny;
    }
    const double dual_minus_K = dual_mu + dual_nu - covered;
    const double g = pr - dual_minus_K;
    if (primal) *primal = pr;
    if (gap) *gap = g;
    if (rel) *rel = g / pr;
    return DD_OK;
  } catch (...) {
    return DD_ERR_OOM;
  }
}

// Visualisation of a coupling through its basic Y-marginals (§7.2): every
// basic cell i has a colour col_i, and pixel y of the Y image gets
// Σ_i col_i · ν_i(y) / ν(y), ν(y) = Σ_i ν_i(y). A deterministic coupling
// (a Monge map T) paints T(X_i) in col_i; overlapping ν_i mix their colours
// in proportion to their masses.
extern "C" dd_status dd_coupling_image_host(int32_t n, int32_t n_basic, const int64_t* row_ptr, const int32_t* col,
                                           const double* val, const float* colours, float* rgb) {
  if (n < 1 || n_basic < 1 || !row_ptr || !colours || !rgb || row_ptr[0] != 0) return DD_ERR_ARG;
  const size_t n2 = (size_t)n * n;
  for (int32_t i = 0; i < n_basic; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return DD_ERR_ARG;
  const int64_t nnz = row_ptr[n_basic];
  if (nnz > 0 && (!col || !val)) return DD_ERR_ARG;
  for (int64_t e = 0; e < nnz; ++e)
    if (col[e] < 0 || (size_t)col[e] >= n2 || !std::isfinite(val[e]) || val[e] < 0.0) return DD_ERR_ARG;
  try {
    std::vector<double> acc(3 * n2, 0.0), mass(n2, 0.0);
    for (int32_t i = 0; i < n_basic; ++i)
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const size_t y = (size_t)col[e];
        for (int k = 0; k < 3; ++k) acc[3 * y + k] += (double)colours[3 * (size_t)i + k] * val[e];
        mass[y] += val[e];
      }
    for (size_t y = 0; y < n2; ++y)
      for (int k = 0; k < 3; ++k) rgb[3 * y + k] = mass[y] > 0.0 ? (float)(acc[3 * y + k] / mass[y]) : 0.f;
    return DD_OK;
  } catch (...) {
    return DD_ERR_OOM;
  }
}
