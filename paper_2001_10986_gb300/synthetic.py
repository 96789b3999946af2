"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the domain-decomposition method. It only
produces problem data:

* Gaussian-mixture images standing in for the paper's test images (§7.1,
  test data: sums of Gaussian blobs whose widths and heights are drawn at
  random). The images themselves are not available, so the recipe below is
  used instead (isotropic or anisotropic blobs plus a floor, normalised to
  mass 1).
* A feasible starting state (basic Y-marginals whose sums reproduce ν and whose
  masses match μ), the input that Algorithm 2 takes besides μ and ν. It is used
  for sampled comparisons at full size, where the coarse-to-fine run of the
  oracle would take too long.
* ε schedules of the paper's multi-scale protocol (§7.1, multi-scale and
  ε-scaling) in [0,1]² units: the protocol of the Table 1 runs, and a variant
  that ends at ε = 2h² on the finest level.

Pixel (i, j) of an n×n image has centre ((i+½)h, (j+½)h) with h = 1/n; the
flat index is i·n + j.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_mixture(n: int, n_blobs: int, seed: int, *, anisotropic: bool = False,
                     floor: float = 1e-3, sigma_range=(0.05, 0.2),
                     max_condition: float = 10.0) -> np.ndarray:
    """n×n FP64 image: Σ_k a_k·exp(−½(x−m_k)ᵀΣ_k⁻¹(x−m_k)) + floor·max, mass 1.

    m_k ~ U[0,1]², a_k ~ U[0.5,1]. Isotropic blobs have σ ~ U[σ_lo, σ_hi].
    Anisotropic blobs have Σ = R(θ)·diag(σ1², σ2²)·R(θ)ᵀ with σ1 ~ U[σ_lo, σ_hi],
    σ2 = σ1/√κ, κ ~ U[1, max_condition], θ ~ U[0, π).
    """
    rng = _rng(seed)
    h = 1.0 / n
    t = (np.arange(n) + 0.5) * h
    xi, xj = np.meshgrid(t, t, indexing="ij")
    img = np.zeros((n, n), dtype=np.float64)
    for _ in range(n_blobs):
        m = rng.uniform(0.0, 1.0, size=2)
        a = rng.uniform(0.5, 1.0)
        s1 = rng.uniform(*sigma_range)
        if anisotropic:
            kappa = rng.uniform(1.0, max_condition)
            s2 = s1 / math.sqrt(kappa)
            th = rng.uniform(0.0, math.pi)
        else:
            s2, th = s1, 0.0
        c, s = math.cos(th), math.sin(th)
        di, dj = xi - m[0], xj - m[1]
        u = c * di + s * dj
        v = -s * di + c * dj
        img += a * np.exp(-0.5 * ((u / s1) ** 2 + (v / s2) ** 2))
    img += floor * img.max()
    img /= img.sum()
    return img


@dataclass(frozen=True)
class Workload:
    """One named problem recipe (image size, blobs, cell size, levels)."""
    name: str
    n: int
    blobs: int
    b: int
    levels: int
    anisotropic: bool = False
    floor: float = 1e-3


WORKLOADS = {
    # two 32×32 images of 3 isotropic blobs, one level, 4×4 basic cells
    "gm32_b4": Workload("gm32_b4", 32, 3, 4, 1),
    # 256×256, 5 blobs, 4×4 cells, 64²→128²→256²
    "gm256_b4_l3": Workload("gm256_b4_l3", 256, 5, 4, 3),
    # 1024×1024, 8 anisotropic blobs, 4×4 cells, layers 8²→…→1024² as in §7.1
    "gm1024_b4": Workload("gm1024_b4", 1024, 8, 4, 8, anisotropic=True),
    # same images with 8×8 basic cells, 16²→…→1024²
    "gm1024_b8": Workload("gm1024_b8", 1024, 8, 8, 7, anisotropic=True),
    # 512×512, 6 blobs, 8²→…→512²
    "gm512_b4": Workload("gm512_b4", 512, 6, 4, 7),
    # 2048×2048, 12 blobs, floor 1e-4, 5 levels 128²→…→2048²
    "gm2048_b4_l5": Workload("gm2048_b4_l5", 2048, 12, 4, 5, floor=1e-4),
}


def image_pair(w: Workload | str, k: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Pair k of a workload: μ from seed 2k, ν from seed 2k+1."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    mu = gaussian_mixture(w.n, w.blobs, 2 * k, anisotropic=w.anisotropic, floor=w.floor)
    nu = gaussian_mixture(w.n, w.blobs, 2 * k + 1, anisotropic=w.anisotropic, floor=w.floor)
    return mu, nu


def paper_schedule(n: int, levels: int, final_sweeps: int, *, coarse_sweeps=(2, 1, 1),
                   eps_start: float = 2.0 / 64, start_sweeps: int = 1):
    """ε schedule of the multi-scale protocol in [0,1]² units.

    At a coarse level with pixel spacing Δ the paper runs 4 iterations at ε=2Δ²,
    then 2 at Δ², then 2 at Δ²/2, then refines (one A+B sweep = 2 iterations).
    At the finest level (Δ = h = 1/n) the run stays at ε = 2h² for
    `final_sweeps` sweeps. The paper's coarsest layer is 8×8, where the first ε
    is 2·(1/8)² = eps_start; when level 0 is finer than that, ε is first halved
    from eps_start down to 2Δ₀² on level 0 (`start_sweeps` sweeps each), so
    that the product coupling is never solved at a small ε. Returns a list of
    (eps, sweeps, level), level 0 being the coarsest.
    """
    h = 1.0 / n
    steps = []
    d0 = h * 2 ** (levels - 1)
    e = float(eps_start)
    while e > 2.0 * d0 * d0 * (1 + 1e-12):
        steps.append((e, int(start_sweeps), 0))
        e *= 0.5
    for lev in range(levels):
        d = h * 2 ** (levels - 1 - lev)
        if lev < levels - 1:
            for f, s in zip((2.0, 1.0, 0.5), coarse_sweeps):
                steps.append((f * d * d, int(s), lev))
        else:
            steps.append((2.0 * d * d, int(final_sweeps), lev))
    return steps


def table1_schedule(n: int):
    """The iteration protocol of the paper's quantitative runs (§7.1, Table 1)
    in [0,1]² units: layers from 8×8 up to n×n; on each layer with pixel
    spacing Δ, 2 sweeps at ε = 2Δ², 1 at Δ², 1 at Δ²/2; on the finest layer 1
    more sweep at Δ²/4 — (log2 n − 2)·8 + 2 half-sweeps in all. Returns
    (schedule, levels) with schedule a list of (eps, sweeps, level)."""
    levels = int(round(math.log2(n))) - 2
    steps = []
    d = 1.0 / 8
    for lev in range(levels):
        d = 1.0 / (8 * 2 ** lev)
        steps += [(2.0 * d * d, 2, lev), (d * d, 1, lev), (0.5 * d * d, 1, lev)]
    steps.append((0.25 * d * d, 1, levels - 1))
    return steps, levels


def halving_schedule(eps_start: float, eps_end: float, sweeps_each: int, level: int = 0):
    """ε = eps_start, eps_start/2, … down to eps_end (inclusive), same sweeps each."""
    steps = []
    e = float(eps_start)
    while e >= eps_end * (1 - 1e-12):
        steps.append((e, int(sweeps_each), level))
        e *= 0.5
    return steps


def feasible_state(mu: np.ndarray, b: int, seed: int, *, shift_px: float = 6.0,
                   blur_px: float = 2.0, radius_px: int = 7):
    """A feasible set of basic Y-marginals and the ν it induces.

    Every b×b basic cell i (mass M_i) sends its mass to a Gaussian bump of
    standard deviation `blur_px` pixels centred at its own centre moved by a
    smooth random displacement of about `shift_px` pixels, cut to a square
    window of half-width `radius_px` and renormalised to mass M_i. ν is the sum
    of these bumps, so Σ_i ν_i = ν and ‖ν_i‖ = ‖μ_i‖ hold by construction.

    Returns (nu_image, row_ptr int64, col int32, val float64) with one row per
    basic cell in natural (row-major) order and each row sorted by pixel index.
    """
    n = mu.shape[0]
    nb = n // b
    rng = _rng(seed)
    # smooth displacement field from a few random Fourier modes
    modes = []
    for _ in range(3):
        k1, k2 = rng.integers(1, 3, size=2)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        amp = rng.uniform(-1.0, 1.0, size=2)
        modes.append((k1, k2, ph, amp))
    M = mu.reshape(nb, b, nb, b).sum(axis=(1, 3))
    rows_c, rows_v = [], []
    offs = np.arange(-radius_px, radius_px + 1)
    for r in range(nb):
        for s in range(nb):
            ci, cj = (r + 0.5) * b, (s + 0.5) * b        # cell centre in pixels
            u, v = ci / n, cj / n
            di = sum(a[0] * math.sin(2 * math.pi * (k1 * u + k2 * v) + p[0]) for k1, k2, p, a in modes)
            dj = sum(a[1] * math.sin(2 * math.pi * (k2 * u + k1 * v) + p[1]) for k1, k2, p, a in modes)
            ti = min(max(ci + shift_px * di / 3.0, 0.0), n - 1e-9)
            tj = min(max(cj + shift_px * dj / 3.0, 0.0), n - 1e-9)
            pi0, pj0 = int(ti), int(tj)
            ii = pi0 + offs
            jj = pj0 + offs
            ii = ii[(ii >= 0) & (ii < n)]
            jj = jj[(jj >= 0) & (jj < n)]
            wi = np.exp(-0.5 * ((ii + 0.5 - ti) / blur_px) ** 2)
            wj = np.exp(-0.5 * ((jj + 0.5 - tj) / blur_px) ** 2)
            w = np.outer(wi, wj)
            w *= M[r, s] / w.sum()
            cols = (ii[:, None] * n + jj[None, :]).ravel()
            rows_c.append(cols.astype(np.int32))
            rows_v.append(w.ravel())
    nu = np.zeros(n * n)
    for c, v in zip(rows_c, rows_v):
        nu[c] += v
    row_ptr = np.zeros(nb * nb + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in rows_c])
    return nu.reshape(n, n), row_ptr, np.concatenate(rows_c), np.concatenate(rows_v)


# sizes of the warm-start network: 1089 inputs (64 μ values, a 32×32 ν
# histogram, log ε), two hidden layers of 256, 64 outputs
MLP_LAYERS = ((256, 1089), (256, 256), (64, 256))


def mlp_init(seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded initial parameters of the warm-start network as one FP32 vector:
    for each layer (out × in) the weights row-major, drawn uniformly in
    ±scale·√(6/in), then `out` zero biases."""
    rng = _rng(seed)
    parts = []
    for o, i in MLP_LAYERS:
        lim = scale * math.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)
