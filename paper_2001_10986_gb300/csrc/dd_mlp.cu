// Learned warm start of the cell solves (not in the paper, whose cells start
// from the duals of their previous solve, Algorithm 2 input u_{C,J}):
//
// * features of an 8×8 cell: 64·μ/‖μ_J‖ on its pixels, 1024·ν_cell/‖ν_cell‖
//   on the 32×32 window centred on the rounded centroid of ν_cell, log(ε/Δ²);
// * a network 1089 → 256 → 256 → 64 (ReLU, bfloat16 weights, FP32 sums) that
//   predicts the cell's dual in the frame of that centroid, scaled by 1/ε;
// * its training (forward, backward, Adam) on pairs logged from solves;
// * the comparison: the X-marginal error after one Y-iteration from the previous
//   duals and from the prediction; the cell starts from the better one, so
//   the plain warm start is both the fallback and the referee.
//
// Target of a cell: with the anchor a = round(centroid − (3.5, 3.5)), the
// stored dual α̃_a(ξ) = α(x) − 2Δ²(x₀ − a)·ξ divided by ε, minus its mean.
// Translating ν_cell by t moves α by −2⟨x,t⟩ + const, which the frame removes.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "dd.h"
#include "dd_internal.cuh"

namespace ddk {

namespace {

constexpr int kIn = kMlpIn, kH = kMlpHidden, kOut = kMlpOut;
constexpr int kCellPx = 64;     // 8×8 cells
constexpr int kWin = 32;        // histogram window side
constexpr float kLn2f = 0.69314718055994530942f;
// flat parameter layout: W1 (256×1089), b1, W2 (256×256), b2, W3 (64×256), b3
constexpr int64_t oW1 = 0, ob1 = oW1 + (int64_t)kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + (int64_t)kH * kH,
                  oW3 = ob2 + kH, ob3 = oW3 + (int64_t)kOut * kH, kNParams = ob3 + kOut;

// ---------------------------------------------------------------------------
// features, targets, comparison
// ---------------------------------------------------------------------------
__device__ double block_sum_d(double v, double* ws) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
  return t;
}

__global__ void __launch_bounds__(256) k_cell_features(SweepArgs a, float log_eps_d2, float* feat, int2* fanc,
                                                      int32_t* ok) {
  __shared__ double dws[32];
  __shared__ float hist[kWin * kWin];
  const int J = blockIdx.x;
  const LevelView& L = a.L;
  const CellGeom g = cell_geom(a.part, J, L.nb, L.b);
  const int64_t off = a.cell_off[J];
  const int ny = a.cell_ny[J];
  if (g.H != 8 || g.W != 8 || off < 0 || ny <= 0) {
    if (threadIdx.x == 0) ok[J] = 0;
    return;
  }
  const int2 anc = a.anchor_new[J];
  // centroid of ν_cell in pixel indices, FP64 from the fixed-point masses
  double sw = 0.0, sr = 0.0, sc = 0.0;
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const double v = (double)a.ws_nu[off + k];
    sw += v;
    sr += v * (double)(anc.x + eta_r(e));
    sc += v * (double)(anc.y + eta_c(e));
  }
  sw = block_sum_d(sw, dws);
  sr = block_sum_d(sr, dws);
  sc = block_sum_d(sc, dws);
  const double cr = sr / sw, cc = sc / sw;
  const int wr = __double2int_rn(cr) - kWin / 2, wc = __double2int_rn(cc) - kWin / 2;
  for (int q = threadIdx.x; q < kWin * kWin; q += blockDim.x) hist[q] = 0.f;
  __syncthreads();
  // the support points are distinct pixels: one store per bin
  const double hscale = 1024.0 / sw;
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const int hr = anc.x + eta_r(e) - wr, hc = anc.y + eta_c(e) - wc;
    if (hr >= 0 && hr < kWin && hc >= 0 && hc < kWin) hist[hr * kWin + hc] = (float)((double)a.ws_nu[off + k] * hscale);
  }
  // μ patch
  double mloc = 0.0;
  for (int x = threadIdx.x; x < kCellPx; x += blockDim.x)
    mloc += (double)L.mu_q[(int64_t)(g.r0 + x / 8) * L.n + g.c0 + (x % 8)];
  const double msum = block_sum_d(mloc, dws);
  float* f = feat + (int64_t)J * kIn;
  for (int x = threadIdx.x; x < kCellPx; x += blockDim.x)
    f[x] = (float)(64.0 * (double)L.mu_q[(int64_t)(g.r0 + x / 8) * L.n + g.c0 + (x % 8)] / msum);
  for (int q = threadIdx.x; q < kWin * kWin; q += blockDim.x) f[kCellPx + q] = hist[q];
  if (threadIdx.x == 0) {
    f[kIn - 1] = log_eps_d2;
    fanc[J] = make_int2(__double2int_rn(cr - 3.5), __double2int_rn(cc - 3.5));
    ok[J] = 1;
  }
}

// target from the duals after the solve (stored in the frame a.anchor[J])
__global__ void __launch_bounds__(64) k_cell_targets(SweepArgs a, const int2* fanc, const int32_t* ok, float* tgt) {
  __shared__ float ws[2];
  const int J = blockIdx.x;
  if (!ok[J]) return;
  const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
  const int x = threadIdx.x, i = x / 8, j = x % 8;
  const int2 an = a.anchor[J], fa = fanc[J];
  const double d2 = a.L.spacing * a.L.spacing;
  const double v = ((double)a.alpha[(int64_t)(g.r0 + i) * a.L.n + g.c0 + j] +
                    2.0 * d2 * ((double)(fa.x - an.x) * i + (double)(fa.y - an.y) * j)) / (double)a.eps;
  float t = (float)v;
  float s = t;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((x & 31) == 0) ws[x >> 5] = s;
  __syncthreads();
  tgt[(int64_t)J * kOut + x] = t - (ws[0] + ws[1]) / 64.0f;
}

// X-marginal L1 error, after one Y-iteration from the duals alpha_old (frame
// anc_old) of one 8×8 cell; the rescaled error of the stopping rule
__device__ float x_error_after_y(const SweepArgs& a, const CellGeom& g, int64_t off, int ny, const float* al,
                             int2 anc_old, int2 anc_new, float mscale, float* Fs, float* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float d2 = (float)(a.L.spacing * a.L.spacing);
  const float inv_eln2 = 1.0f / (a.eps * kLn2f);
  const float kappa = (float)(a.L.spacing * a.L.spacing / ((double)a.eps * 0.69314718055994530942));
  const int shr = anc_new.x - anc_old.x, shc = anc_new.y - anc_old.y;
  if (tid < kCellPx) {
    const int i = tid / 8, j = tid % 8;
    const int64_t p = (int64_t)(g.r0 + i) * a.L.n + g.c0 + j;
    Fs[tid] = (al[tid] + 2.0f * d2 * (float)(shr * i + shc * j)) * inv_eln2 + a.L.log2mu[p];
  }
  __syncthreads();
  float px[kCellPx];
#pragma unroll
  for (int x = 0; x < kCellPx; ++x) px[x] = 0.f;
  for (int k = tid; k < ny; k += blockDim.x) {
    const int32_t e = a.ws_eta[off + k];
    const float er = (float)eta_r(e), ec = (float)eta_c(e);
    const float nu = (float)a.ws_nu[off + k] * kFixToFloat;
    float E[kCellPx];
    float m = -3.0e38f;
#pragma unroll
    for (int x = 0; x < kCellPx; ++x) {
      const float tr = (float)(x / 8) - er, tc = (float)(x % 8) - ec;
      E[x] = Fs[x] - kappa * (tr * tr + tc * tc);
      m = fmaxf(m, E[x]);
    }
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < kCellPx; ++x) {
      E[x] = exp2f(E[x] - m);
      s += E[x];
    }
    const float w = nu / s;
#pragma unroll
    for (int x = 0; x < kCellPx; ++x) px[x] = fmaf(w, E[x], px[x]);
  }
  // sum over the threads: warps by shuffles, then across warps
#pragma unroll
  for (int x = 0; x < kCellPx; ++x) {
    float v = px[x];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp * kCellPx + x] = v;
  }
  __syncthreads();
  float err = 0.f;
  if (tid < kCellPx) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w * kCellPx + tid];
    const int64_t p = (int64_t)(g.r0 + tid / 8) * a.L.n + g.c0 + tid % 8;
    err = fabsf(t - a.L.mu_f[p] * mscale);
  }
  for (int o = 16; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o);
  __syncthreads();
  if (lane == 0) red[warp] = err;
  __syncthreads();
  float tot = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

__global__ void __launch_bounds__(128) k_warm_compare(SweepArgs a, const float* pred, const int2* fanc, const int32_t* ok) {
  __shared__ float Fs[kCellPx];
  __shared__ float red[4 * kCellPx];
  __shared__ float cand[2][kCellPx];
  __shared__ float sums[2];
  const int J = blockIdx.x;
  const int tid = threadIdx.x;
  if (!ok[J]) {
    if (tid == 0 && a.cell_learned) a.cell_learned[J] = -1;
    return;
  }
  const CellGeom g = cell_geom(a.part, J, a.L.nb, a.L.b);
  const int64_t off = a.cell_off[J];
  const int ny = a.cell_ny[J];
  const int2 anc_old = a.anchor[J], anc_new = a.anchor_new[J], fa = fanc[J];
  const float d2 = (float)(a.L.spacing * a.L.spacing);
  if (tid < kCellPx) {
    const int i = tid / 8, j = tid % 8;
    cand[0][tid] = a.alpha[(int64_t)(g.r0 + i) * a.L.n + g.c0 + j];
    // prediction → dual in the frame of the previous anchor
    cand[1][tid] = a.eps * pred[(int64_t)J * kOut + tid] + 2.0f * d2 * (float)((anc_old.x - fa.x) * i +
                                                                                (anc_old.y - fa.y) * j);
  }
  // ‖ν_cell‖/‖μ_J‖ of the stopping rule
  float nl = 0.f;
  for (int k = tid; k < ny; k += blockDim.x) nl += (float)a.ws_nu[off + k] * kFixToFloat;
  float ml = 0.f;
  if (tid < kCellPx) ml = a.L.mu_f[(int64_t)(g.r0 + tid / 8) * a.L.n + g.c0 + tid % 8];
  for (int o = 16; o > 0; o >>= 1) {
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
    ml += __shfl_xor_sync(0xffffffffu, ml, o);
  }
  if ((tid & 31) == 0) {
    red[tid >> 5] = nl;
    red[4 + (tid >> 5)] = ml;
  }
  __syncthreads();
  if (tid == 0) {
    sums[0] = red[0] + red[1] + red[2] + red[3];
    sums[1] = red[4] + red[5] + red[6] + red[7];
  }
  __syncthreads();
  const float mscale = sums[1] > 0.f ? sums[0] / sums[1] : 1.f;
  const float e0 = x_error_after_y(a, g, off, ny, cand[0], anc_old, anc_new, mscale, Fs, red);
  const float e1 = x_error_after_y(a, g, off, ny, cand[1], anc_old, anc_new, mscale, Fs, red);
  const bool use = e1 < e0;   // NaN in e1 keeps the previous duals
  if (use && tid < kCellPx)
    a.alpha[(int64_t)(g.r0 + tid / 8) * a.L.n + g.c0 + tid % 8] = cand[1][tid];
  if (tid == 0 && a.cell_learned) a.cell_learned[J] = use ? 1 : 0;
}

// ---------------------------------------------------------------------------
// the network
// ---------------------------------------------------------------------------
// C(m,n) = Σ_k A(m,k)·B(k,n), A FP32 with strides (sam, sak), B FP32 or
// bfloat16 with strides (sbk, sbn); 64×64 tiles, 16-deep slices.
// EPI 0: C = acc (+ bias[n]);  EPI 1: C = acc + bias[n], C2 = max(C, 0);
// EPI 2: C = acc · [mask(m,n) > 0] (mask with row stride ldc).
template <typename TB>
struct GemmArgs {
  const float* A;
  int64_t sam, sak;
  const TB* B;
  int64_t sbk, sbn;
  float* C;
  int64_t ldc;
  float* C2;
  const float* bias;
  const float* mask;
  int M, N, K;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs<TB> g) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int t = threadIdx.x;
  const int tm = t / 16, tn = t % 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;
      int m, k;
      if (g.sak == 1) {
        k = e % BK;
        m = e / BK;
      } else {
        m = e % BM;
        k = e / BM;
      }
      const int gm = m0 + m, gk = k0 + k;
      As[k][m] = (gm < g.M && gk < g.K) ? g.A[gm * g.sam + gk * g.sak] : 0.f;
      int n, kb;
      if (g.sbn == 1) {
        n = e % BN;
        kb = e / BN;
      } else {
        kb = e % BK;
        n = e / BK;
      }
      const int gn = n0 + n, gkb = k0 + kb;
      Bs[kb][n] = (gn < g.N && gkb < g.K) ? to_f(g.B[gkb * g.sbk + gn * g.sbn]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][4 * tm + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][4 * tn + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + 4 * tm + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + 4 * tn + j;
      if (n >= g.N) continue;
      float v = acc[i][j];
      if (EPI == 0) {
        if (g.bias) v += g.bias[n];
        g.C[(int64_t)m * g.ldc + n] = v;
      } else if (EPI == 1) {
        v += g.bias[n];
        g.C[(int64_t)m * g.ldc + n] = v;
        g.C2[(int64_t)m * g.ldc + n] = fmaxf(v, 0.f);
      } else {
        g.C[(int64_t)m * g.ldc + n] = g.mask[(int64_t)m * g.ldc + n] > 0.f ? v : 0.f;
      }
    }
  }
}

template <typename TB, int EPI>
cudaError_t gemm(const GemmArgs<TB>& g, cudaStream_t s) {
  const dim3 grid((g.N + 63) / 64, (g.M + 63) / 64);
  k_gemm<TB, EPI><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* wb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// dY = 2(Y − T)/(n·64) and Σ (Y − T)² (FP64, one atomic per block)
__global__ void __launch_bounds__(256) k_mse(const float* Y, const float* T, int64_t cnt, float* dY, double* loss) {
  __shared__ double ws[8];
  double acc = 0.0;
  const float sc = 2.0f / (float)cnt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = sc * d;
    acc += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    atomicAdd(loss, t);
  }
}

// out[m] = Σ_n D[n·ld + m]
__global__ void k_colsum(const float* D, int64_t n, int m, int64_t ld, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  float s = 0.f;
  for (int64_t r = 0; r < n; ++r) s += D[r * ld + c];
  out[c] = s;
}

__global__ void k_adam(float* p, const float* g, float* m1, float* m2, int64_t n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

}  // namespace

cudaError_t launch_cell_features(const SweepArgs& a, float* feat, int2* fanchor, int32_t* ok, cudaStream_t s) {
  const float le = (float)std::log((double)a.eps / (a.L.spacing * a.L.spacing));
  k_cell_features<<<a.ncells, 256, 0, s>>>(a, le, feat, fanchor, ok);
  return cudaGetLastError();
}

cudaError_t launch_cell_targets(const SweepArgs& a, const int2* fanchor, const int32_t* ok, float* tgt,
                                cudaStream_t s) {
  k_cell_targets<<<a.ncells, 64, 0, s>>>(a, fanchor, ok, tgt);
  return cudaGetLastError();
}

cudaError_t launch_warm_compare(const SweepArgs& a, const float* pred, const int2* fanchor, const int32_t* ok,
                         cudaStream_t s) {
  k_warm_compare<<<a.ncells, 128, 0, s>>>(a, pred, fanchor, ok);
  return cudaGetLastError();
}

}  // namespace ddk

using namespace ddk;

// the network's parameters, optimiser state and activation buffers
struct dd_mlp {
  float* p = nullptr;             // FP32 master parameters (flat layout)
  __nv_bfloat16* wb = nullptr;    // bfloat16 copies of W1, W2, W3 (same offsets as in p)
  float* grad = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  int64_t steps = 0;
  int64_t cap = 0;                // rows of the activation buffers
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dz = nullptr;
  double* loss = nullptr;
  bool wb_fresh = false;
  std::mutex mu;                  // one call at a time per network
};

namespace {

thread_local std::string g_mlp_error;

struct MlpError {
  dd_status st;
  std::string msg;
};

#define MLP_CUDA(x)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) throw MlpError{DD_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

template <typename F>
dd_status mlp_guard(F&& f) {
  try {
    f();
    g_mlp_error.clear();
    return DD_OK;
  } catch (const MlpError& e) {
    g_mlp_error = e.msg;
    dd_set_noalloc_error(e.msg.c_str());
    return e.st;
  } catch (const std::bad_alloc&) {
    g_mlp_error = "out of host memory";
    dd_set_noalloc_error(g_mlp_error.c_str());
    return DD_ERR_OOM;
  }
}

template <typename T>
void mlp_alloc(T*& p, int64_t count) {
  if (cudaMalloc((void**)&p, sizeof(T) * (size_t)count) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    throw MlpError{DD_ERR_OOM, "cudaMalloc failed for the network buffers"};
  }
}

void mlp_reserve(dd_mlp* m, int64_t n) {
  if (n <= m->cap) return;
  const int64_t c = std::max<int64_t>(n, 1024);
  float** bufs[] = {&m->z1, &m->h1, &m->z2, &m->h2, &m->y, &m->dy, &m->dz};
  for (float** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  mlp_alloc(m->z1, c * kH);
  mlp_alloc(m->h1, c * kH);
  mlp_alloc(m->z2, c * kH);
  mlp_alloc(m->h2, c * kH);
  mlp_alloc(m->y, c * kOut);
  mlp_alloc(m->dy, c * kOut);
  mlp_alloc(m->dz, c * kH);
  m->cap = c;
}

void refresh_bf16(dd_mlp* m, cudaStream_t s) {
  k_to_bf16<<<512, 256, 0, s>>>(m->p, m->wb, kNParams);
  MLP_CUDA(cudaGetLastError());
  m->wb_fresh = true;
}

// Z1,H1 = X W1ᵀ + b1, relu; Z2,H2 likewise; Y = H2 W3ᵀ + b3
void forward(dd_mlp* m, const float* X, int64_t n, float* Y, cudaStream_t s) {
  if (!m->wb_fresh) refresh_bf16(m, s);
  GemmArgs<__nv_bfloat16> g1{X, kIn, 1, m->wb + oW1, 1, kIn, m->z1, kH, m->h1, m->p + ob1, nullptr, (int)n, kH, kIn};
  MLP_CUDA((gemm<__nv_bfloat16, 1>(g1, s)));
  GemmArgs<__nv_bfloat16> g2{m->h1, kH, 1, m->wb + oW2, 1, kH, m->z2, kH, m->h2, m->p + ob2, nullptr, (int)n, kH, kH};
  MLP_CUDA((gemm<__nv_bfloat16, 1>(g2, s)));
  GemmArgs<__nv_bfloat16> g3{m->h2, kH, 1, m->wb + oW3, 1, kH, Y, kOut, nullptr, m->p + ob3, nullptr, (int)n, kOut, kH};
  MLP_CUDA((gemm<__nv_bfloat16, 0>(g3, s)));
}

// loss and gradient of the mean squared error into m->grad (forward first)
void loss_grad(dd_mlp* m, const float* X, const float* T, int64_t n, double* loss_host, cudaStream_t s) {
  forward(m, X, n, m->y, s);
  MLP_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
  k_mse<<<256, 256, 0, s>>>(m->y, T, n * kOut, m->dy, m->loss);
  MLP_CUDA(cudaGetLastError());
  // layer 3: dW3 = dYᵀ H2, db3 = Σ dY, dZ2 = (dY W3)·[Z2 > 0]
  GemmArgs<float> w3{m->dy, 1, kOut, m->h2, kH, 1, m->grad + oW3, kH, nullptr, nullptr, nullptr, kOut, kH, (int)n};
  MLP_CUDA((gemm<float, 0>(w3, s)));
  k_colsum<<<1, kOut, 0, s>>>(m->dy, n, kOut, kOut, m->grad + ob3);
  GemmArgs<__nv_bfloat16> d2{m->dy, kOut, 1, m->wb + oW3, kH, 1, m->dz, kH, nullptr, nullptr, m->z2, (int)n, kH, kOut};
  MLP_CUDA((gemm<__nv_bfloat16, 2>(d2, s)));
  // layer 2: dW2 = dZ2ᵀ H1, db2 = Σ dZ2, dZ1 = (dZ2 W2)·[Z1 > 0] (into h2, free now)
  GemmArgs<float> w2{m->dz, 1, kH, m->h1, kH, 1, m->grad + oW2, kH, nullptr, nullptr, nullptr, kH, kH, (int)n};
  MLP_CUDA((gemm<float, 0>(w2, s)));
  k_colsum<<<1, kH, 0, s>>>(m->dz, n, kH, kH, m->grad + ob2);
  GemmArgs<__nv_bfloat16> d1{m->dz, kH, 1, m->wb + oW2, kH, 1, m->h2, kH, nullptr, nullptr, m->z1, (int)n, kH, kH};
  MLP_CUDA((gemm<__nv_bfloat16, 2>(d1, s)));
  // layer 1: dW1 = dZ1ᵀ X, db1 = Σ dZ1
  GemmArgs<float> w1{m->h2, 1, kH, X, kIn, 1, m->grad + oW1, kIn, nullptr, nullptr, nullptr, kH, kIn, (int)n};
  MLP_CUDA((gemm<float, 0>(w1, s)));
  k_colsum<<<1, kH, 0, s>>>(m->h2, n, kH, kH, m->grad + ob1);
  MLP_CUDA(cudaGetLastError());
  if (loss_host) {
    double l = 0.0;
    MLP_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaStreamSynchronize(s));
    *loss_host = l / (double)(n * kOut);
  }
}

}  // namespace

namespace ddk {
cudaError_t mlp_forward(dd_mlp* m, const float* x, int64_t n, float* y, cudaStream_t s) {
  try {
    std::lock_guard<std::mutex> lk(m->mu);
    mlp_reserve(m, n);
    forward(m, x, n, y, s);
    return cudaSuccess;
  } catch (const MlpError& e) {
    dd_set_noalloc_error(e.msg.c_str());
    return cudaErrorUnknown;
  }
}
}  // namespace ddk

extern "C" {

int64_t dd_mlp_num_params(void) { return kNParams; }

dd_status dd_mlp_create(const float* params, dd_mlp** out) {
  if (!out || !params) {
    dd_set_noalloc_error("dd_mlp_create: NULL argument");
    return DD_ERR_ARG;
  }
  *out = nullptr;
  dd_mlp* m = new dd_mlp();
  const dd_status st = mlp_guard([&] {
    mlp_alloc(m->p, kNParams);
    mlp_alloc(m->wb, kNParams);
    mlp_alloc(m->grad, kNParams);
    mlp_alloc(m->m1, kNParams);
    mlp_alloc(m->m2, kNParams);
    mlp_alloc(m->loss, 1);
    MLP_CUDA(cudaMemcpy(m->p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    MLP_CUDA(cudaMemset(m->m1, 0, sizeof(float) * kNParams));
    MLP_CUDA(cudaMemset(m->m2, 0, sizeof(float) * kNParams));
    refresh_bf16(m, 0);
    MLP_CUDA(cudaDeviceSynchronize());
  });
  if (st != DD_OK) {
    dd_mlp_destroy(m);
    return st;
  }
  *out = m;
  return DD_OK;
}

void dd_mlp_destroy(dd_mlp* m) {
  if (!m) return;
  void* bufs[] = {m->p, m->wb, m->grad, m->m1, m->m2, m->z1, m->h1, m->z2, m->h2, m->y, m->dy, m->dz, m->loss};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete m;
}

dd_status dd_mlp_get_params(dd_mlp* m, float* params) {
  if (!m || !params) return DD_ERR_ARG;
  return mlp_guard([&] {
    std::lock_guard<std::mutex> lk(m->mu);
    MLP_CUDA(cudaDeviceSynchronize());
    MLP_CUDA(cudaMemcpy(params, m->p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  });
}

dd_status dd_mlp_set_params(dd_mlp* m, const float* params) {
  if (!m || !params) return DD_ERR_ARG;
  return mlp_guard([&] {
    std::lock_guard<std::mutex> lk(m->mu);
    MLP_CUDA(cudaDeviceSynchronize());
    MLP_CUDA(cudaMemcpy(m->p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    m->wb_fresh = false;
  });
}

dd_status dd_mlp_forward(dd_mlp* m, const float* x, int64_t n, float* y, void* stream) {
  if (!m || !x || !y || n <= 0 || n > (int64_t)1 << 24) {
    dd_set_noalloc_error("dd_mlp_forward: bad argument");
    return DD_ERR_ARG;
  }
  return mlp_guard([&] {
    std::lock_guard<std::mutex> lk(m->mu);
    const cudaStream_t s = (cudaStream_t)stream;
    mlp_reserve(m, n);
    forward(m, x, n, y, s);
    MLP_CUDA(cudaStreamSynchronize(s));
  });
}

dd_status dd_mlp_loss_grad(dd_mlp* m, const float* x, const float* t, int64_t n, double* loss, float* grad,
                           void* stream) {
  if (!m || !x || !t || n <= 0 || n > (int64_t)1 << 24) {
    dd_set_noalloc_error("dd_mlp_loss_grad: bad argument");
    return DD_ERR_ARG;
  }
  return mlp_guard([&] {
    std::lock_guard<std::mutex> lk(m->mu);
    const cudaStream_t s = (cudaStream_t)stream;
    mlp_reserve(m, n);
    double l = 0.0;
    loss_grad(m, x, t, n, &l, s);
    if (loss) *loss = l;
    if (grad) {
      MLP_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, s));
      MLP_CUDA(cudaStreamSynchronize(s));
    }
  });
}

dd_status dd_mlp_train_step(dd_mlp* m, const float* x, const float* t, int64_t n, float lr, double* loss,
                            void* stream) {
  if (!m || !x || !t || n <= 0 || n > (int64_t)1 << 24 || !(lr > 0.f)) {
    dd_set_noalloc_error("dd_mlp_train_step: bad argument");
    return DD_ERR_ARG;
  }
  return mlp_guard([&] {
    std::lock_guard<std::mutex> lk(m->mu);
    const cudaStream_t s = (cudaStream_t)stream;
    mlp_reserve(m, n);
    loss_grad(m, x, t, n, loss, s);
    ++m->steps;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, (double)m->steps);
    const float c2 = 1.f - (float)std::pow((double)b2, (double)m->steps);
    k_adam<<<512, 256, 0, s>>>(m->p, m->grad, m->m1, m->m2, kNParams, lr, b1, b2, c1, c2, 1e-8f);
    MLP_CUDA(cudaGetLastError());
    refresh_bf16(m, s);
    if (!loss) MLP_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"
