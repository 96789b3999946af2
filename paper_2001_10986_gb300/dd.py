"""Python binding of the C ABI in include/dd.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards
its arguments; all computation runs in libddot.so. Importing this module
raises if the library has not been built (see paper_2001_10986_gb300.build).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

(DD_OK, DD_ERR_ARG, DD_ERR_CUDA, DD_ERR_OOM, DD_ERR_CAPACITY, DD_ERR_NUMERIC, DD_ERR_STATE,
 DD_ERR_NOT_CONVERGED) = range(8)
_STATUS = {0: "DD_OK", 1: "DD_ERR_ARG", 2: "DD_ERR_CUDA", 3: "DD_ERR_OOM", 4: "DD_ERR_CAPACITY",
           5: "DD_ERR_NUMERIC", 6: "DD_ERR_STATE", 7: "DD_ERR_NOT_CONVERGED"}


class dd_grid(C.Structure):
    _fields_ = [("n", C.c_int32), ("levels", C.c_int32)]


class dd_eps_step(C.Structure):
    _fields_ = [("eps", C.c_double), ("sweeps", C.c_int32), ("level", C.c_int32)]


class dd_options(C.Structure):
    _fields_ = [("err_tol", C.c_double), ("trunc", C.c_double), ("max_iter", C.c_int32),
                ("threads_per_cell", C.c_int32), ("max_cluster_cells", C.c_int32), ("x_newton", C.c_int32),
                ("warm", C.c_int32), ("dual_refine", C.c_int32), ("mode", C.c_int32), ("stream", C.c_void_p),
                ("debug_flags", C.c_uint64), ("safeguard", C.c_int32)]


class dd_sweep_stats(C.Structure):
    _fields_ = [("level", C.c_int32), ("partition", C.c_int32), ("eps", C.c_double), ("nnz", C.c_int64),
                ("max_iters", C.c_int32), ("mean_iters", C.c_double), ("cells_not_converged", C.c_int32),
                ("sweeps_done", C.c_int64), ("cells_rescued", C.c_int32), ("cells_escalated", C.c_int32)]


class dd_profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("half_sweeps", C.c_int64), ("solve_launches", C.c_int64),
                ("solve_ms", C.c_double), ("gather_launches", C.c_int64), ("gather_ms", C.c_double),
                ("cluster_ms", C.c_double), ("kernel_evals", C.c_double), ("sinkhorn_iters", C.c_double), ("cells", C.c_int64),
                ("newton_steps", C.c_int64), ("hessian_fma", C.c_double), ("learned_cells", C.c_int64),
                ("compared_cells", C.c_int64), ("rescued_cells", C.c_int64), ("graph_reruns", C.c_int64),
                ("peak_nnz", C.c_int64), ("peak_state_bytes", C.c_int64), ("peak_work_bytes", C.c_int64),
                ("escalated_cells", C.c_int64)]


class DDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class DDNotConverged(DDError):
    """Cell solves stayed at max_iter after the safeguard. The call completed
    its sweeps and the state is feasible; `stats` holds the call's statistics
    (None for dd_half_sweep)."""

    def __init__(self, msg, stats=None):
        super().__init__(DD_ERR_NOT_CONVERGED, msg)
        self.stats = stats


if not os.path.exists(LIB):
    raise ImportError(f"{LIB} is missing: build it with paper_2001_10986_gb300.build.build()")
_lib = C.CDLL(LIB)

_P = C.c_void_p
_pd = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_pi64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_pi32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")

_lib.dd_options_default.argtypes = [C.POINTER(dd_options)]
_lib.dd_options_default.restype = None
_lib.dd_create.argtypes = [_pd, _pd, C.POINTER(dd_grid), C.c_int32, C.POINTER(dd_eps_step), C.c_int32,
                           C.POINTER(dd_options), C.POINTER(_P)]
_lib.dd_set_state.argtypes = [_P, _pi64, _pi32, _pd, _P, _P]
_lib.dd_half_sweep.argtypes = [_P, C.c_int32, C.c_double]
_lib.dd_refine.argtypes = [_P]
_lib.dd_save.argtypes = [_P, C.c_char_p]
_lib.dd_load.argtypes = [C.c_char_p, C.POINTER(dd_options), C.POINTER(_P)]
_lib.dd_sweep.argtypes = [_P, C.c_int32, C.POINTER(dd_sweep_stats)]
_lib.dd_run_schedule.argtypes = [_P, C.POINTER(dd_sweep_stats)]
_lib.dd_cost.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.dd_get_basic_marginals.argtypes = [_P, C.POINTER(C.c_int64), _P, _P, _P, C.c_int64]
_lib.dd_get_plan.argtypes = [_P, C.c_double, C.POINTER(C.c_int64), _P, _P, _P, C.c_int64]
_lib.dd_get_duals.argtypes = [_P, C.c_int32, _pd]
_lib.dd_glue_potential.argtypes = [C.c_int32, C.c_int64, _P, _P, _P, C.c_double, C.c_int32, _P,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_double)]
_lib.dd_glue_duals_host.argtypes = [C.c_int32, C.c_int32, _P, _P, _P, C.c_double, _P, _P]
_lib.dd_interpolate_dual_host.argtypes = [C.c_int32, _P, _P]
_lib.dd_relative_pd_gap_host.argtypes = [C.c_int32, _P, _P, C.c_double, _P, _P, _P, _P,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.dd_coupling_image_host.argtypes = [C.c_int32, C.c_int32, _P, _P, _P, _P, _P]
_lib.dd_coupling_image.argtypes = [_P, _P, _P]
_lib.dd_objective.argtypes = [_P, C.c_int32, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_double)]
_lib.dd_glue_duals.argtypes = [_P, _P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
_lib.dd_relative_pd_gap.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.dd_get_info.argtypes = [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                             C.POINTER(C.c_double), C.POINTER(C.c_int64)]
_lib.dd_solve_cell_noalloc.argtypes = [_P, C.c_int32, C.c_double, C.c_int32, _P, _P, _P, C.c_double,
                                       C.c_double, C.c_int32, C.c_double, _P, _P, _P]
_lib.dd_solve_cell_noalloc.restype = C.c_int
_lib.dd_get_cell_stats.argtypes = [_P, _P, _P, _P, _P, _P, _P, C.c_int32, C.POINTER(C.c_int32)]
_lib.dd_get_profile.argtypes = [_P, C.POINTER(dd_profile)]
_lib.dd_reset_profile.argtypes = [_P]
_lib.dd_destroy.argtypes = [_P]
_lib.dd_destroy.restype = None
_lib.dd_last_error.argtypes = [_P]
_lib.dd_last_error.restype = C.c_char_p
_lib.dd_mlp_num_params.argtypes = []
_lib.dd_mlp_num_params.restype = C.c_int64
_lib.dd_mlp_create.argtypes = [np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS"), C.POINTER(_P)]
_lib.dd_mlp_destroy.argtypes = [_P]
_lib.dd_mlp_destroy.restype = None
_lib.dd_mlp_get_params.argtypes = [_P, np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")]
_lib.dd_mlp_set_params.argtypes = [_P, np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")]
_lib.dd_mlp_forward.argtypes = [_P, _P, C.c_int64, _P, _P]
_lib.dd_mlp_loss_grad.argtypes = [_P, _P, _P, C.c_int64, C.POINTER(C.c_double), _P, _P]
_lib.dd_mlp_train_step.argtypes = [_P, _P, _P, C.c_int64, C.c_float, C.POINTER(C.c_double), _P]
_lib.dd_attach_mlp.argtypes = [_P, _P]
_lib.dd_autotune.argtypes = [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.dd_cell_training_pairs.argtypes = [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]
for _f in ("dd_create", "dd_set_state", "dd_half_sweep", "dd_refine", "dd_save", "dd_load", "dd_sweep", "dd_run_schedule", "dd_cost",
           "dd_get_basic_marginals", "dd_get_plan", "dd_get_duals", "dd_get_info", "dd_get_profile",
           "dd_reset_profile", "dd_get_cell_stats", "dd_mlp_create", "dd_mlp_get_params", "dd_mlp_set_params",
           "dd_mlp_forward", "dd_mlp_loss_grad", "dd_mlp_train_step", "dd_attach_mlp", "dd_cell_training_pairs",
           "dd_autotune", "dd_objective", "dd_glue_potential", "dd_glue_duals_host",
           "dd_interpolate_dual_host", "dd_relative_pd_gap_host", "dd_coupling_image_host", "dd_coupling_image",
           "dd_glue_duals", "dd_relative_pd_gap"):
    getattr(_lib, _f).restype = C.c_int

EXPORTED = ("dd_options_default", "dd_create", "dd_set_state", "dd_half_sweep", "dd_refine", "dd_save", "dd_load", "dd_sweep",
            "dd_run_schedule", "dd_cost", "dd_get_basic_marginals", "dd_get_plan", "dd_get_duals",
            "dd_get_info", "dd_get_cell_stats", "dd_get_profile", "dd_reset_profile", "dd_destroy",
            "dd_last_error", "dd_solve_cell_noalloc", "dd_mlp_num_params", "dd_mlp_create", "dd_mlp_destroy",
            "dd_mlp_get_params", "dd_mlp_set_params", "dd_mlp_forward", "dd_mlp_loss_grad", "dd_mlp_train_step",
            "dd_attach_mlp", "dd_cell_training_pairs", "dd_autotune", "dd_objective", "dd_glue_potential",
            "dd_glue_duals_host", "dd_interpolate_dual_host", "dd_relative_pd_gap_host",
            "dd_coupling_image_host", "dd_coupling_image", "dd_glue_duals", "dd_relative_pd_gap")


def _check(ctx, st, stats=None):
    if st == DD_ERR_NOT_CONVERGED and ctx is not None:
        raise DDNotConverged((_lib.dd_last_error(ctx) or b"").decode(), stats)
    if st != DD_OK:
        raise DDError(st, (_lib.dd_last_error(ctx) or b"").decode())


class DDConvergenceWarning(UserWarning):
    """Issued by DD.sweep / run_schedule / half_sweep when cell solves stayed
    at max_iter after the safeguard (the C call returned DD_ERR_NOT_CONVERGED
    after completing its sweeps)."""


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)      # torch.cuda.Stream


def dd_options_default(**overrides) -> dd_options:
    o = dd_options()
    _lib.dd_options_default(C.byref(o))
    names = {f[0] for f in dd_options._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"unknown dd_options field {k!r}")
        if k == "stream":
            v = _stream_ptr(v)
        setattr(o, k, v)
    return o


def dd_create(mu, nu, n, levels, b, schedule, opt: dd_options | None = None):
    """schedule: iterable of (eps, sweeps, level). Returns an opaque handle."""
    mu = np.ascontiguousarray(mu, dtype=np.float64).ravel()
    nu = np.ascontiguousarray(nu, dtype=np.float64).ravel()
    steps = list(schedule)
    arr = (dd_eps_step * len(steps))(*[dd_eps_step(float(e), int(s), int(l)) for e, s, l in steps])
    g = dd_grid(int(n), int(levels))
    out = _P()
    st = _lib.dd_create(mu, nu, C.byref(g), int(b), arr, len(steps),
                        C.byref(opt) if opt is not None else None, C.byref(out))
    _check(None, st)
    return out


def dd_set_state(ctx, row_ptr, col, val, alpha_A=None, alpha_B=None):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    vl = np.ascontiguousarray(val, dtype=np.float64)
    aA = None if alpha_A is None else np.ascontiguousarray(alpha_A, dtype=np.float64).ravel()
    aB = None if alpha_B is None else np.ascontiguousarray(alpha_B, dtype=np.float64).ravel()
    _check(ctx, _lib.dd_set_state(ctx, rp, cl, vl, None if aA is None else aA.ctypes.data,
                                  None if aB is None else aB.ctypes.data))


def dd_half_sweep(ctx, partition, eps):
    _check(ctx, _lib.dd_half_sweep(ctx, int(partition), float(eps)))


def dd_refine(ctx):
    _check(ctx, _lib.dd_refine(ctx))


def dd_save(ctx, path):
    _check(ctx, _lib.dd_save(ctx, os.fsencode(path)))


def dd_load(path, opt: dd_options | None = None):
    h = _P()
    _check(None, _lib.dd_load(os.fsencode(path), C.byref(opt) if opt is not None else None, C.byref(h)))
    return h


def dd_sweep(ctx, n_sweeps=1) -> dd_sweep_stats:
    st = dd_sweep_stats()
    _check(ctx, _lib.dd_sweep(ctx, int(n_sweeps), C.byref(st)), st)
    return st


def dd_run_schedule(ctx) -> dd_sweep_stats:
    st = dd_sweep_stats()
    _check(ctx, _lib.dd_run_schedule(ctx, C.byref(st)), st)
    return st


def dd_cost(ctx, with_y=True):
    c, ex, ey = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, _lib.dd_cost(ctx, C.byref(c), C.byref(ex), C.byref(ey) if with_y else None))
    return c.value, ex.value, (ey.value if with_y else None)


def dd_get_info(ctx):
    """Returns (level, n_level, n_basic, eps, nnz)."""
    lv, nl, nbs, e, nz = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double(), C.c_int64()
    _check(ctx, _lib.dd_get_info(ctx, C.byref(lv), C.byref(nl), C.byref(nbs), C.byref(e), C.byref(nz)))
    return lv.value, nl.value, nbs.value, e.value, nz.value


def dd_get_basic_marginals(ctx):
    """Returns (row_ptr int64, col int32, val float64), natural order of basic cells."""
    _, _, nrows, _, _ = dd_get_info(ctx)
    nnz = C.c_int64()
    _check(ctx, _lib.dd_get_basic_marginals(ctx, C.byref(nnz), None, None, None, 0))
    rp = np.zeros(nrows + 1, dtype=np.int64)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1), dtype=np.float64)
    _check(ctx, _lib.dd_get_basic_marginals(ctx, C.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                            val.ctypes.data, col.size))
    return rp, col[:nnz.value], val[:nnz.value]


def dd_get_plan(ctx, trunc=0.0):
    """Returns (row_ptr over X pixels, col, val) of the coupling of the last partition."""
    _, nl, _, _, _ = dd_get_info(ctx)
    nnz = C.c_int64()
    _check(ctx, _lib.dd_get_plan(ctx, float(trunc), C.byref(nnz), None, None, None, 0))
    rp = np.zeros(nl * nl + 1, dtype=np.int64)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1), dtype=np.float64)
    _check(ctx, _lib.dd_get_plan(ctx, float(trunc), C.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                 val.ctypes.data, col.size))
    return rp, col[:nnz.value], val[:nnz.value]


def dd_objective(ctx, partition=-1, eps=0.0):
    """(primal, gap, gap_abs): KL(π|K) − ‖K‖ summed over the composite cells,
    and the sum and absolute sum of the cell problems' primal-dual gaps, for
    the last partition's coupling (partition -1) or for partition 0/1 at ε."""
    p, g, ga = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, _lib.dd_objective(ctx, int(partition), float(eps), C.byref(p), C.byref(g), C.byref(ga)))
    return p.value, g.value, ga.value


def dd_glue_duals(ctx):
    """Glued X-dual of §6.3 of the context's current level, on the GPU.
    Returns (alpha_hat (n_l² FP64), V ((n_l/2b)² FP64), CG iterations,
    relative residual)."""
    _, nl, nbasic, _, _ = dd_get_info(ctx)
    na = int(round(nbasic ** 0.5)) // 2
    a = np.zeros(nl * nl, dtype=np.float64)
    V = np.zeros(na * na, dtype=np.float64)
    it, rr = C.c_int32(), C.c_double()
    _check(ctx, _lib.dd_glue_duals(ctx, a.ctypes.data, V.ctypes.data, C.byref(it), C.byref(rr)))
    return a, V, it.value, rr.value


def dd_relative_pd_gap(ctx):
    """eq. RelPDGap of the last partition's coupling with the glued duals, on
    the GPU. Returns (rel, gap, primal)."""
    r, g, p = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, _lib.dd_relative_pd_gap(ctx, C.byref(r), C.byref(g), C.byref(p)))
    return r.value, g.value, p.value


def dd_glue_potential(n_nodes, j1, j2, logq, tol=1e-12, max_iter=100000):
    """Least-squares potential V of the dual gluing on a graph of n_nodes
    vertices and edges (j1, j2) with values logq (host solve, no GPU).
    Returns (V, iterations, relative residual)."""
    a = np.ascontiguousarray(j1, dtype=np.int32)
    b = np.ascontiguousarray(j2, dtype=np.int32)
    q = np.ascontiguousarray(logq, dtype=np.float64)
    if not (a.shape == b.shape == q.shape and a.ndim == 1):
        raise DDError(DD_ERR_ARG, "j1, j2 and logq must be 1-D arrays of one length")
    V = np.zeros(int(n_nodes), dtype=np.float64)
    it, res = C.c_int32(), C.c_double()
    st = _lib.dd_glue_potential(int(n_nodes), a.size, a.ctypes.data, b.ctypes.data, q.ctypes.data, float(tol),
                                int(max_iter), V.ctypes.data, C.byref(it), C.byref(res))
    if st != DD_OK:
        raise DDError(st, _STATUS.get(st, "unknown status"))
    return V, it.value, res.value


def dd_glue_duals_host(mu, alpha_A, alpha_B, b, eps):
    """Glued X-dual α̂ (n×n, FP64) and the A-cell potentials V from the duals
    of both partitions (host solve, no GPU)."""
    m = np.ascontiguousarray(mu, dtype=np.float64)
    n = m.shape[0]
    if m.shape != (n, n):
        raise DDError(DD_ERR_ARG, "mu must be n×n")
    a = np.ascontiguousarray(alpha_A, dtype=np.float64).reshape(n, n)
    bb = np.ascontiguousarray(alpha_B, dtype=np.float64).reshape(n, n)
    out = np.zeros((n, n), dtype=np.float64)
    na = max(n // max(int(b), 1) // 2, 1)
    V = np.zeros(na * na, dtype=np.float64)
    st = _lib.dd_glue_duals_host(n, int(b), m.ctypes.data, a.ctypes.data, bb.ctypes.data, float(eps),
                                 out.ctypes.data, V.ctypes.data)
    if st != DD_OK:
        raise DDError(st, _STATUS.get(st, "unknown status"))
    return out, V


def dd_interpolate_dual_host(alpha_c):
    """α on the level twice as fine from an n_c×n_c glued α (host, no GPU)."""
    a = np.ascontiguousarray(alpha_c, dtype=np.float64)
    nc = a.shape[0]
    if a.shape != (nc, nc):
        raise DDError(DD_ERR_ARG, "alpha_c must be n×n")
    out = np.zeros((2 * nc, 2 * nc), dtype=np.float64)
    st = _lib.dd_interpolate_dual_host(nc, a.ctypes.data, out.ctypes.data)
    if st != DD_OK:
        raise DDError(st, _STATUS.get(st, "unknown status"))
    return out


def dd_relative_pd_gap_host(mu, nu, eps, plan, alpha_hat):
    """(rel, gap, primal) of eq. RelPDGap for plan = (row_ptr, col, val) as
    dd_get_plan returns it and a glued X-dual (host, no GPU)."""
    m = np.ascontiguousarray(mu, dtype=np.float64)
    n = m.shape[0]
    v = np.ascontiguousarray(nu, dtype=np.float64).reshape(n, n)
    rp = np.ascontiguousarray(plan[0], dtype=np.int64)
    cl = np.ascontiguousarray(plan[1], dtype=np.int32)
    vl = np.ascontiguousarray(plan[2], dtype=np.float64)
    a = np.ascontiguousarray(alpha_hat, dtype=np.float64).reshape(n, n)
    if m.shape != (n, n) or rp.size != n * n + 1 or cl.size != vl.size or cl.size < rp[-1]:
        raise DDError(DD_ERR_ARG, "inconsistent sizes")
    r, g, p = C.c_double(), C.c_double(), C.c_double()
    st = _lib.dd_relative_pd_gap_host(n, m.ctypes.data, v.ctypes.data, float(eps), rp.ctypes.data,
                                      cl.ctypes.data if cl.size else None, vl.ctypes.data if vl.size else None,
                                      a.ctypes.data, C.byref(r), C.byref(g), C.byref(p))
    if st != DD_OK:
        raise DDError(st, _STATUS.get(st, "unknown status"))
    return r.value, g.value, p.value


def checkerboard_colours(n_basic_side, a=(0.95, 0.55, 0.1), b=(0.1, 0.35, 0.9)):
    """Colours of the basic cells in a checkerboard of two colours (§7.2)."""
    i, j = np.divmod(np.arange(n_basic_side * n_basic_side), n_basic_side)
    return np.where(((i + j) % 2 == 0)[:, None], np.array(a, np.float32), np.array(b, np.float32))


def dd_coupling_image_host(n, basic_marginals, colours):
    """n×n×3 float image Σ_i col_i·ν_i/ν of basic marginals (row_ptr, col, val)."""
    rp = np.ascontiguousarray(basic_marginals[0], dtype=np.int64)
    cl = np.ascontiguousarray(basic_marginals[1], dtype=np.int32)
    vl = np.ascontiguousarray(basic_marginals[2], dtype=np.float64)
    cs = np.ascontiguousarray(colours, dtype=np.float32)
    nb = rp.size - 1
    if cs.shape != (nb, 3) or cl.size != vl.size or cl.size < rp[-1]:
        raise DDError(DD_ERR_ARG, "inconsistent sizes")
    out = np.zeros((int(n), int(n), 3), dtype=np.float32)
    st = _lib.dd_coupling_image_host(int(n), nb, rp.ctypes.data, cl.ctypes.data if cl.size else None,
                                     vl.ctypes.data if vl.size else None, cs.ctypes.data, out.ctypes.data)
    if st != DD_OK:
        raise DDError(st, _STATUS.get(st, "unknown status"))
    return out


def dd_coupling_image(ctx, colours):
    """§7.2 image of the current basic marginals, computed on the GPU;
    colours: n_basic × 3. Returns n_l × n_l × 3 float32."""
    _, nl, nbasic, _, _ = dd_get_info(ctx)
    cl = np.ascontiguousarray(colours, dtype=np.float32).reshape(-1)
    if cl.size != 3 * nbasic:
        raise DDError(DD_ERR_ARG, "colours must hold 3 values per basic cell")
    out = np.empty(3 * nl * nl, dtype=np.float32)
    _check(ctx, _lib.dd_coupling_image(ctx, cl.ctypes.data, out.ctypes.data))
    return out.reshape(nl, nl, 3)


def write_ppm(path, rgb):
    """Write an n×m×3 image with values in [0, 1] as a binary PPM file."""
    img = (np.clip(np.asarray(rgb, dtype=np.float64), 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())


def dd_get_duals(ctx, partition):
    _, nl, _, _, _ = dd_get_info(ctx)
    out = np.zeros(nl * nl, dtype=np.float64)
    _check(ctx, _lib.dd_get_duals(ctx, int(partition), out))
    return out


def dd_get_cell_stats(ctx):
    """Returns dict of per-cell arrays (iters, err_x, n_y, status, cost,
    cluster) of the last half-sweep."""
    nc = C.c_int32()
    _check(ctx, _lib.dd_get_cell_stats(ctx, None, None, None, None, None, None, 0, C.byref(nc)))
    it = np.zeros(nc.value, np.int32)
    ex = np.zeros(nc.value, np.float64)
    ny = np.zeros(nc.value, np.int32)
    st = np.zeros(nc.value, np.int32)
    co = np.zeros(nc.value, np.float64)
    cl = np.zeros(nc.value, np.int32)
    _check(ctx, _lib.dd_get_cell_stats(ctx, it.ctypes.data, ex.ctypes.data, ny.ctypes.data, st.ctypes.data,
                                       co.ctypes.data, cl.ctypes.data, nc.value, C.byref(nc)))
    return {"iters": it, "err_x": ex, "n_y": ny, "status": st, "cost": co, "cluster": cl}


def dd_solve_cell_noalloc(mu, b, spacing, n_y, y_row, y_col, nu, eps, err_tol, max_iter, trunc,
                          alpha, nu_basic, stream=None):
    """All array arguments are device addresses (ints, e.g. tensor.data_ptr())."""
    _check(None, _lib.dd_solve_cell_noalloc(mu, int(b), float(spacing), int(n_y), y_row, y_col, nu,
                                            float(eps), float(err_tol), int(max_iter), float(trunc),
                                            alpha, nu_basic, _stream_ptr(stream)))


def dd_mlp_num_params() -> int:
    return int(_lib.dd_mlp_num_params())


def dd_mlp_create(params):
    """params: host FP32 vector of dd_mlp_num_params() floats. Returns a handle."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != dd_mlp_num_params():
        raise DDError(DD_ERR_ARG, f"expected {dd_mlp_num_params()} parameters, got {p.size}")
    h = _P()
    _check(None, _lib.dd_mlp_create(p, C.byref(h)))
    return h


def dd_mlp_destroy(mlp):
    _lib.dd_mlp_destroy(mlp)


def dd_mlp_get_params(mlp):
    out = np.empty(dd_mlp_num_params(), dtype=np.float32)
    _check(None, _lib.dd_mlp_get_params(mlp, out))
    return out


def dd_mlp_set_params(mlp, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != dd_mlp_num_params():
        raise DDError(DD_ERR_ARG, "wrong number of parameters")
    _check(None, _lib.dd_mlp_set_params(mlp, p))


def dd_mlp_forward(mlp, x_ptr, n, y_ptr, stream=None):
    """x_ptr, y_ptr: device addresses (n·1089 and n·64 floats)."""
    _check(None, _lib.dd_mlp_forward(mlp, x_ptr, int(n), y_ptr, _stream_ptr(stream)))


def dd_mlp_loss_grad(mlp, x_ptr, t_ptr, n, stream=None):
    """Returns (loss, gradient as a host FP32 vector)."""
    g = np.empty(dd_mlp_num_params(), dtype=np.float32)
    loss = C.c_double()
    _check(None, _lib.dd_mlp_loss_grad(mlp, x_ptr, t_ptr, int(n), C.byref(loss), g.ctypes.data, _stream_ptr(stream)))
    return loss.value, g


def dd_mlp_train_step(mlp, x_ptr, t_ptr, n, lr, stream=None):
    loss = C.c_double()
    _check(None, _lib.dd_mlp_train_step(mlp, x_ptr, t_ptr, int(n), float(lr), C.byref(loss), _stream_ptr(stream)))
    return loss.value


def dd_autotune(ctx, rounds=2):
    """Returns the chosen (threads_per_cell, max_cluster_cells)."""
    t, cl = C.c_int32(), C.c_int32()
    _check(ctx, _lib.dd_autotune(ctx, int(rounds), C.byref(t), C.byref(cl)))
    return t.value, cl.value


def dd_attach_mlp(ctx, mlp):
    _check(ctx, _lib.dd_attach_mlp(ctx, mlp))


def dd_cell_training_pairs(ctx, feat_ptr, tgt_ptr, ok_ptr, cap):
    n = C.c_int64()
    _check(ctx, _lib.dd_cell_training_pairs(ctx, feat_ptr, tgt_ptr, ok_ptr, int(cap), C.byref(n)))
    return n.value


def dd_get_profile(ctx) -> dd_profile:
    p = dd_profile()
    _check(ctx, _lib.dd_get_profile(ctx, C.byref(p)))
    return p


def dd_reset_profile(ctx):
    _check(ctx, _lib.dd_reset_profile(ctx))


def dd_destroy(ctx):
    _lib.dd_destroy(ctx)


def dd_last_error(ctx=None) -> str:
    return (_lib.dd_last_error(ctx) or b"").decode()


class DD:
    """Owner of one context; methods forward to the functions above."""

    def __init__(self, mu, nu, b, levels, schedule, **opts):
        mu = np.asarray(mu)
        self.n = mu.shape[0]
        self.b = b
        self.levels = levels
        self.opt = dd_options_default(**opts)
        self.ctx = dd_create(mu, nu, self.n, levels, b, schedule, self.opt)

    def set_state(self, row_ptr, col, val, alpha_A=None, alpha_B=None):
        dd_set_state(self.ctx, row_ptr, col, val, alpha_A, alpha_B)

    def _sweeps(self, fn, *args, strict=False):
        # a DD_ERR_NOT_CONVERGED call has completed its sweeps: by default it
        # is reported as a warning and its statistics are returned
        try:
            return fn(self.ctx, *args)
        except DDNotConverged as e:
            if strict:
                raise
            import warnings
            warnings.warn(str(e), DDConvergenceWarning, stacklevel=3)
            return e.stats

    def half_sweep(self, partition, eps, strict=False):
        self._sweeps(dd_half_sweep, partition, eps, strict=strict)

    def refine(self):
        dd_refine(self.ctx)

    def save(self, path):
        dd_save(self.ctx, path)

    @classmethod
    def load(cls, path, b=None, **opts):
        """A context resumed from a dd_save file; with keyword options the
        saved options are replaced by dd_options_default(**opts)."""
        self = cls.__new__(cls)
        self.opt = dd_options_default(**opts) if opts else None
        self.ctx = dd_load(path, self.opt)
        _, nl, nbasic, _, _ = dd_get_info(self.ctx)
        self.b = b if b is not None else nl // int(round(nbasic ** 0.5))
        self.n = None
        self.levels = None
        return self

    def sweep(self, n=1, strict=False):
        return self._sweeps(dd_sweep, n, strict=strict)

    def run_schedule(self, strict=False):
        return self._sweeps(dd_run_schedule, strict=strict)

    def cost(self, with_y=True):
        return dd_cost(self.ctx, with_y)

    def info(self):
        return dd_get_info(self.ctx)

    def basic_marginals(self):
        return dd_get_basic_marginals(self.ctx)

    def plan(self, trunc=0.0):
        return dd_get_plan(self.ctx, trunc)

    def duals(self, partition):
        return dd_get_duals(self.ctx, partition)

    def objective(self, partition=-1, eps=0.0):
        return dd_objective(self.ctx, partition, eps)

    def coupling_image(self, colours=None, device=True):
        """§7.2 colour image (n_l×n_l×3) of the current basic marginals, on
        the GPU (device=True) or on the host from the downloaded marginals;
        the default colours are a checkerboard over the basic cells."""
        _, nl, nbasic, _, _ = dd_get_info(self.ctx)
        if colours is None:
            colours = checkerboard_colours(int(round(nbasic ** 0.5)))
        if device:
            return dd_coupling_image(self.ctx, colours)
        return dd_coupling_image_host(nl, self.basic_marginals(), colours)

    def glue_duals(self):
        """(alpha_hat, V, CG iterations, relative residual): the glued X-dual
        of §6.3 of the current level, computed on the GPU."""
        return dd_glue_duals(self.ctx)

    def relative_pd_gap(self, mu=None, nu=None, device=True):
        """eq. RelPDGap of the current state (§6.3): (rel, gap, primal) for the
        coupling of the last partition and the glued duals of both
        partitions. device=True: all on the GPU. device=False: gluing and
        gap on the host from the downloaded duals and coupling; mu, nu are
        then the images at the current level."""
        if device:
            return dd_relative_pd_gap(self.ctx)
        _, nl, _, eps, _ = dd_get_info(self.ctx)
        a_hat, _ = dd_glue_duals_host(mu, self.duals(0), self.duals(1), self.b, eps)
        return dd_relative_pd_gap_host(mu, nu, eps, self.plan(0.0), a_hat)

    def cell_stats(self):
        return dd_get_cell_stats(self.ctx)

    def profile(self):
        return dd_get_profile(self.ctx)

    def reset_profile(self):
        dd_reset_profile(self.ctx)

    def autotune(self, rounds=2):
        return dd_autotune(self.ctx, rounds)

    def attach_mlp(self, mlp):
        """Attach an MLP (or None); its handle must outlive the attachment."""
        self._mlp = mlp
        dd_attach_mlp(self.ctx, mlp.handle if mlp is not None else None)

    def training_pairs(self):
        """(features, targets) of the 8×8 cells of the last half-sweep as CUDA
        tensors (n × 1089, n × 64); torch provides the device memory."""
        import torch
        nb = self.info()[2]
        cap = (int(round(nb ** 0.5)) // 2 + 1) ** 2
        dev = torch.device("cuda", torch.cuda.current_device())
        feat = torch.empty((cap, 1089), dtype=torch.float32, device=dev)
        tgt = torch.empty((cap, 64), dtype=torch.float32, device=dev)
        ok = torch.zeros(cap, dtype=torch.int32, device=dev)
        n = dd_cell_training_pairs(self.ctx, feat.data_ptr(), tgt.data_ptr(), ok.data_ptr(), cap)
        sel = ok[:n] != 0
        return feat[:n][sel].contiguous(), tgt[:n][sel].contiguous()

    def close(self):
        if self.ctx:
            dd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f32_cuda(t, cols):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2 or t.shape[1] != cols:
        raise DDError(DD_ERR_ARG, f"expected a CUDA float32 tensor of shape (n, {cols})")
    return t.contiguous()


class MLP:
    """Owner of one warm-start network; tensors are CUDA float32 (torch only
    holds the memory)."""

    def __init__(self, params):
        self.handle = dd_mlp_create(params)

    @property
    def params(self):
        return dd_mlp_get_params(self.handle)

    @params.setter
    def params(self, p):
        dd_mlp_set_params(self.handle, p)

    def forward(self, x, stream=None):
        import torch
        x = _f32_cuda(x, 1089)
        y = torch.empty((x.shape[0], 64), dtype=torch.float32, device=x.device)
        dd_mlp_forward(self.handle, x.data_ptr(), x.shape[0], y.data_ptr(), stream)
        return y

    def loss_grad(self, x, t, stream=None):
        x, t = _f32_cuda(x, 1089), _f32_cuda(t, 64)
        return dd_mlp_loss_grad(self.handle, x.data_ptr(), t.data_ptr(), x.shape[0], stream)

    def train_step(self, x, t, lr, stream=None):
        x, t = _f32_cuda(x, 1089), _f32_cuda(t, 64)
        return dd_mlp_train_step(self.handle, x.data_ptr(), t.data_ptr(), x.shape[0], lr, stream)

    def close(self):
        if self.handle:
            dd_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
