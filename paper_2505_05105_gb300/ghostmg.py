"""ctypes binding of libghostmg.so (declared in include/ghostmg.h).

Argument marshalling only: every step runs in the CUDA library.  Array
arguments may be CUDA torch tensors (float64, contiguous; used on the handle's
stream), NumPy float64 C-contiguous host arrays, or raw integer addresses.
Importing this module does not build anything; loading fails loudly when the
library has not been built (``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

# GHOSTMG_CHECKED=1 loads the bounds-checked debug variant (build(checked=True))
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libghostmg_checked.so" if os.environ.get("GHOSTMG_CHECKED") == "1"
                        else "libghostmg.so")

MG_OK = 0
MG_ERR_INVALID_ARG = 1
MG_ERR_CUDA = 2
MG_ERR_NOT_CONVERGED = 3
MG_ERR_DIVERGED = 4
MG_ERR_NOT_SPD = 5
MG_ERR_TIMEOUT = 6
MG_ERR_UNIMPLEMENTED = 7
MG_ERR_INTERNAL = 8
MG_ERR_OUT_OF_MEMORY = 9
MG_BC_DIRICHLET = 0
MG_BC_MIXED = 1
MG_LAMBDA_LOCAL = 0
MG_LAMBDA_GLOBAL = 1
MG_FP64 = 0
MG_MIXED = 1
MG_COARSE_GALERKIN = 0
MG_COARSE_REDISCRETISE = 1


class mg_grid(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("h", ctypes.c_double), ("coarsest_cells", ctypes.c_int)]


class mg_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("neumann_mask", ctypes.c_void_p),
                ("box_sides", ctypes.c_int)]


class mg_stab(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("eta", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("lambda_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("inner", ctypes.c_int), ("cycle", ctypes.c_int),
                ("coarse_op", ctypes.c_int), ("c_global", ctypes.c_double),
                ("fuse_max_tiles", ctypes.c_int)]


class mg_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("res_hist", ctypes.c_double * 64), ("n_dof", ctypes.c_int),
                ("n_cut", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("setup_ms", ctypes.c_float), ("solve_ms", ctypes.c_float),
                ("checks", ctypes.c_int)]

    def history(self):
        return [self.res_hist[k] for k in range(min(self.checks + 1, 64))]


class mg1d_problem(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("theta1", ctypes.c_double),
                ("theta2", ctypes.c_double), ("lambda_", ctypes.c_double)]


MG1D_MAX_CELLS = 2048


class mg_batch_shape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("first_group", ctypes.c_int),
                ("cluster", ctypes.c_int), ("coop_min_dof", ctypes.c_int)]

    def astuple(self):
        return (self.threads, self.first_group, self.cluster, self.coop_min_dof)


class mg_batch_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int), ("checks", ctypes.c_int),
                ("n_dof", ctypes.c_int), ("rel_res", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); the order of declaration in include/ghostmg.h
SIGNATURES = {
    "mg_default_stab": (_I, [ctypes.POINTER(mg_stab)]),
    "mg_setup": (_I, [ctypes.POINTER(_P), _P, ctypes.POINTER(mg_grid), ctypes.POINTER(mg_bc),
                      ctypes.POINTER(mg_stab), _P]),
    "mg_solve": (_I, [_P, _P, _P, _P, _D, ctypes.POINTER(mg_info)]),
    "mg_solve_bc": (_I, [_P, _P, _P, _P, _P, _D, ctypes.POINTER(mg_info)]),
    "mg_adjoint": (_I, [_P, _P, _P, _P]),
    "mg_adjoint_bc": (_I, [_P, _P, _P, _P, _P]),
    "mg_destroy": (None, [_P]),
    "mg_strerror": (ctypes.c_char_p, [_I]),
    "mg_get_c_global": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mg_set_wait_limit": (_I, [_P, ctypes.c_longlong]),
    "mg_get_counts": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                           ctypes.POINTER(_I)]),
    "mg_level_cells": (_I, [_P, _I]),
    "mg_level_dofs": (_I, [_P, _I]),
    "mg_export_stencil": (_I, [_P, _I, _P]),
    "mg_export_cut_cells": (_I, [_P, _I, _P, _P, ctypes.POINTER(_I)]),
    "mg_rhs": (_I, [_P, _P, _P, _P]),
    "mg_rhs_bc": (_I, [_P, _P, _P, _P, _P]),
    "mg_cycles": (_I, [_P, _P, _P, _I, _I]),
    "mg_cycles_transposed": (_I, [_P, _P, _P, _I]),
    "mg_residual": (_I, [_P, _P, _P, _P, _P]),
    "mg_residual_static": (_I, [_P, _P, _P, _P, _P]),
    "mg_set_profiling": (_I, [_P, _I]),
    "mg_get_profile": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), _P, _P]),
    "mg_batch_setup": (_I, [ctypes.POINTER(_P), _I, _P, _P, ctypes.POINTER(mg_bc),
                            ctypes.POINTER(mg_stab), _P]),
    "mg_batch_buffers": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "mg_batch_solve": (_I, [_P, _P, _P, _P, _D, _P]),
    "mg_batch_solve_bc": (_I, [_P, _P, _P, _P, _P, _D, _P]),
    "mg_batch_set_shape": (_I, [_P, ctypes.POINTER(mg_batch_shape)]),
    "mg_batch_get_shape": (_I, [_P, ctypes.POINTER(mg_batch_shape)]),
    "mg_batch_tune": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(mg_batch_shape),
                           ctypes.POINTER(ctypes.c_float)]),
    "mg_batch_timing": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "mg_batch_destroy": (None, [_P]),
    "mg1d_cycles": (_I, [_I, _P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "mg_bounds_check": (_I, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint), _I]),
}

PROF_SLOTS = ("sweep", "band", "restrict", "prolong", "residual", "update", "coarse", "io",
              "levels", "fused", "tail", "levels_band", "levels_restrict")

_lib = None


def load() -> ctypes.CDLL:
    """Load libghostmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GhostMGError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load().mg_strerror(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")


def _check(code: int, where: str, ok=(MG_OK,)):
    if code not in ok:
        raise GhostMGError(code, where)
    return code


def _addr(x, writable=False):
    """Address of an array argument (torch tensor, NumPy array or int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if x.dtype not in (np.float64, np.int32) or not x.flags.c_contiguous:
            raise TypeError("NumPy arrays must be C-contiguous float64 (int32 for cell lists)")
        if writable and not x.flags.writeable:
            raise TypeError("output array is read-only")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise TypeError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


# --- same-name wrappers of the C entry points ------------------------------------

def mg_default_stab() -> mg_stab:
    s = mg_stab()
    _check(load().mg_default_stab(ctypes.byref(s)), "mg_default_stab")
    return s


def mg_setup(levelset, grid: mg_grid, bc: Optional[mg_bc] = None, stab: Optional[mg_stab] = None,
             stream: int = 0) -> int:
    h = _P()
    _check(load().mg_setup(ctypes.byref(h), _addr(levelset), ctypes.byref(grid),
                           ctypes.byref(bc) if bc is not None else None,
                           ctypes.byref(stab) if stab is not None else None,
                           _P(stream) if stream else None), "mg_setup")
    return h.value


def mg_solve(handle: int, f, g, u, tol: float, info: Optional[mg_info] = None,
             ok=(MG_OK,)) -> int:
    return _check(load().mg_solve(handle, _addr(f), _addr(g), _addr(u, True), tol,
                                  ctypes.byref(info) if info is not None else None),
                  "mg_solve", ok)


def mg_solve_bc(handle: int, f, gD, gN, u, tol: float, info: Optional[mg_info] = None,
                ok=(MG_OK,)) -> int:
    return _check(load().mg_solve_bc(handle, _addr(f), _addr(gD), _addr(gN), _addr(u, True),
                                     tol, ctypes.byref(info) if info is not None else None),
                  "mg_solve_bc", ok)


def mg_rhs_bc(handle: int, f, gD, gN, F) -> int:
    return _check(load().mg_rhs_bc(handle, _addr(f), _addr(gD), _addr(gN), _addr(F, True)),
                  "mg_rhs_bc")


def mg_adjoint(handle: int, dLdu, dLdf=None, dLdg=None, ok=(MG_OK,)) -> int:
    return _check(load().mg_adjoint(handle, _addr(dLdu), _addr(dLdf, True), _addr(dLdg, True)),
                  "mg_adjoint", ok)


def mg_adjoint_bc(handle: int, dLdu, dLdf=None, dLdg=None, dLdgN=None, ok=(MG_OK,)) -> int:
    return _check(load().mg_adjoint_bc(handle, _addr(dLdu), _addr(dLdf, True), _addr(dLdg, True),
                                       _addr(dLdgN, True)), "mg_adjoint_bc", ok)


def mg_destroy(handle: int) -> None:
    if handle:
        load().mg_destroy(handle)


def mg_strerror(code: int) -> str:
    return load().mg_strerror(code).decode()


def mg_get_c_global(handle: int):
    """(c_global, Lanczos steps, CG iterations) of the handle (see the header)."""
    c, st, it = _D(), _I(), _I()
    _check(load().mg_get_c_global(handle, ctypes.byref(c), ctypes.byref(st), ctypes.byref(it)),
           "mg_get_c_global")
    return c.value, st.value, it.value


def mg_bounds_check(reset: bool = False):
    """(enabled, hits) of the bounds-checked build; (False, 0) in the normal one."""
    en, hits = ctypes.c_int(), ctypes.c_uint()
    _check(load().mg_bounds_check(ctypes.byref(en), ctypes.byref(hits), int(reset)),
           "mg_bounds_check")
    return bool(en.value), int(hits.value)


def mg_set_wait_limit(handle: int, polls: int) -> int:
    """Poll budget of the handle's bounded device waits (< 0: default)."""
    return _check(load().mg_set_wait_limit(handle, int(polls)), "mg_set_wait_limit")


def mg_get_counts(handle: int):
    vals = [_I() for _ in range(4)]
    _check(load().mg_get_counts(handle, *[ctypes.byref(v) for v in vals]), "mg_get_counts")
    return tuple(v.value for v in vals)


def mg_level_cells(handle: int, level: int) -> int:
    return load().mg_level_cells(handle, level)


def mg_level_dofs(handle: int, level: int) -> int:
    return load().mg_level_dofs(handle, level)


def mg_export_stencil(handle: int, level: int, out) -> int:
    return _check(load().mg_export_stencil(handle, level, _addr(out, True)), "mg_export_stencil")


def mg_export_cut_cells(handle: int, max_cells: int, cells, data) -> int:
    n = _I()
    _check(load().mg_export_cut_cells(handle, max_cells, _addr(cells, True), _addr(data, True),
                                      ctypes.byref(n)), "mg_export_cut_cells")
    return n.value


def mg_rhs(handle: int, f, g, F) -> int:
    return _check(load().mg_rhs(handle, _addr(f), _addr(g), _addr(F, True)), "mg_rhs")


def mg_cycles(handle: int, F, u, k: int, precision: int = MG_FP64) -> int:
    return _check(load().mg_cycles(handle, _addr(F), _addr(u, True), k, precision), "mg_cycles")


def mg_cycles_transposed(handle: int, F, u, k: int) -> int:
    return _check(load().mg_cycles_transposed(handle, _addr(F), _addr(u, True), k),
                  "mg_cycles_transposed")


def mg_residual(handle: int, F, u, r=None):
    norms = np.zeros(2)
    _check(load().mg_residual(handle, _addr(F), _addr(u), _addr(r, True), norms.ctypes.data),
           "mg_residual")
    return float(norms[0]), float(norms[1])


def mg_residual_static(handle: int, F, u, r=None):
    """Allocation-free fine-level residual (device F, u, r); returns
    (||r||_inf, ||r||_2).  See include/ghostmg.h."""
    norms = np.zeros(2)
    _check(load().mg_residual_static(handle, _addr(F), _addr(u), _addr(r, True),
                                     norms.ctypes.data), "mg_residual_static")
    return float(norms[0]), float(norms[1])


def mg1d_cycles(problems, u, F=None, cycle: str = "two-grid", nu1: int = 2, nu2: int = 1,
                cycles: int = 50, stream: int = 0):
    """The 1D model of Sec. 4 (include/ghostmg.h, mg1d_cycles).
    problems: list of (n_cells, theta1, theta2, lambda); u: device float64
    tensor holding the packed first iterates (updated in place); F: packed
    device right-hand sides or None (F = 0).  cycle: "two-grid", "V" or "W".
    Returns the residual norms, one list of cycles + 1 values per problem."""
    total = sum(int(n) + 1 for (n, *_) in problems)
    for x in (u, F):
        if x is None or isinstance(x, int):
            continue
        size = x.numel() if hasattr(x, "numel") else x.size
        if size < total:
            raise ValueError(f"packed arrays need {total} values")
    arr = (mg1d_problem * len(problems))(*[mg1d_problem(int(n), t1, t2, lam)
                                           for (n, t1, t2, lam) in problems])
    res = np.zeros(len(problems) * (cycles + 1))
    code = {"two-grid": 0, "V": 1, "W": 2}[cycle]
    _check(load().mg1d_cycles(len(problems), ctypes.addressof(arr), code, nu1, nu2, cycles,
                              _addr(F), _addr(u, True), res.ctypes.data, stream),
           "mg1d_cycles")
    return res.reshape(len(problems), cycles + 1)


def mg_set_profiling(handle: int, enable: bool) -> int:
    return _check(load().mg_set_profiling(handle, int(bool(enable))), "mg_set_profiling")


def mg_get_profile(handle: int):
    """(total launches, {slot: (launch groups, device ms)})."""
    n = ctypes.c_longlong()
    counts = np.zeros(len(PROF_SLOTS), dtype=np.int64)
    ms = np.zeros(len(PROF_SLOTS))
    _check(load().mg_get_profile(handle, ctypes.byref(n), counts.ctypes.data, ms.ctypes.data),
           "mg_get_profile")
    return n.value, {k: (int(counts[i]), float(ms[i])) for i, k in enumerate(PROF_SLOTS)}


def mg_batch_setup(grids, levelsets, bc: Optional[mg_bc] = None,
                   stab: Optional[mg_stab] = None, stream: int = 0) -> int:
    """grids: sequence of mg_grid; levelsets: packed array of all members'
    nodal psi (host or device)."""
    arr = (mg_grid * len(grids))(*grids)
    h = _P()
    _check(load().mg_batch_setup(ctypes.byref(h), len(grids), ctypes.addressof(arr),
                                 _addr(levelsets), ctypes.byref(bc) if bc is not None else None,
                                 ctypes.byref(stab) if stab is not None else None,
                                 _P(stream) if stream else None), "mg_batch_setup")
    return h.value


def mg_batch_buffers(batch: int):
    """(total_nodes, f, g, u): the batch's own device packed arrays (addresses)."""
    n = ctypes.c_longlong()
    f, g, u = _P(), _P(), _P()
    _check(load().mg_batch_buffers(batch, ctypes.byref(n), ctypes.byref(f), ctypes.byref(g),
                                   ctypes.byref(u)), "mg_batch_buffers")
    return n.value, f.value, g.value, u.value


def mg_batch_solve(batch: int, f, g, u, tol: float, info=None, ok=(MG_OK,)) -> int:
    return _check(load().mg_batch_solve(batch, _addr(f), _addr(g), _addr(u, True), tol,
                                        ctypes.addressof(info) if info is not None else None),
                  "mg_batch_solve", ok)


def mg_batch_tune(batch: int, f, g, tol: float, reps: int = 3):
    """(mg_batch_shape, ms) of the fastest launch shape (see the header)."""
    best, ms = mg_batch_shape(), ctypes.c_float()
    _check(load().mg_batch_tune(batch, _addr(f), _addr(g), tol, reps, ctypes.byref(best),
                                ctypes.byref(ms)), "mg_batch_tune")
    return best, ms.value


def mg_batch_set_shape(batch: int, shape: mg_batch_shape) -> int:
    return _check(load().mg_batch_set_shape(batch, ctypes.byref(shape)), "mg_batch_set_shape")


def mg_batch_get_shape(batch: int) -> mg_batch_shape:
    s = mg_batch_shape()
    _check(load().mg_batch_get_shape(batch, ctypes.byref(s)), "mg_batch_get_shape")
    return s


def mg_batch_timing(batch: int):
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().mg_batch_timing(batch, ctypes.byref(a), ctypes.byref(b)), "mg_batch_timing")
    return a.value, b.value


def mg_batch_destroy(batch: int) -> None:
    if batch:
        load().mg_batch_destroy(batch)


# --- convenience object ------------------------------------------------------------

class Solver:
    """Owns one handle.  ``psi`` is the (N+1)^2 nodal level set (host or
    device); arrays passed to the methods may live on host or device."""

    def __init__(self, psi, n_cells: int, x0: float, y0: float, h: float, *,
                 coarsest: int = 8, gamma: float = 2.0, alpha: float = 1.75, eta: int = 4,
                 nu1: int = 2, nu2: int = 1, precision: str = "fp64", max_cycles: int = 100,
                 inner: int = 0, stream: int = 0, neumann_mask=None, cycle: str = "V",
                 coarse: str = "galerkin", box_sides: bool = False, c_global=None,
                 fuse_max_tiles: int = 0):
        """neumann_mask: (n_cells, n_cells) uint8 cells [jc, ic] (host array,
        or a device tensor), nonzero where a cut cell's boundary piece is
        Neumann (MG_BC_MIXED); None: all Dirichlet.
        c_global: the global constant C of Sec. 5.2 (MG_LAMBDA_GLOBAL:
        lambda = gamma c_global on every cut cell); 0: computed by mg_setup
        on the GPU; None: local lambda_K.
        fuse_max_tiles: mg_stab.fuse_max_tiles (0 default, -1 never fused)."""
        self.N = n_cells
        stab = mg_default_stab()
        stab.gamma, stab.alpha, stab.eta = gamma, alpha, eta
        stab.nu1, stab.nu2, stab.max_cycles, stab.inner = nu1, nu2, max_cycles, inner
        stab.fuse_max_tiles = fuse_max_tiles
        stab.precision = {"fp64": MG_FP64, "mixed": MG_MIXED}[precision]
        stab.cycle = {"V": 1, "W": 2, "two-grid": 0}[cycle]
        stab.coarse_op = {"galerkin": MG_COARSE_GALERKIN,
                          "rediscretise": MG_COARSE_REDISCRETISE}[coarse]
        if c_global is not None:
            stab.lambda_mode, stab.c_global = MG_LAMBDA_GLOBAL, float(c_global)
        grid = mg_grid(n_cells, x0, y0, h, coarsest)
        if neumann_mask is None:
            bc = mg_bc(MG_BC_DIRICHLET, None, int(box_sides))
        else:
            if isinstance(neumann_mask, np.ndarray):
                neumann_mask = np.ascontiguousarray(neumann_mask, dtype=np.uint8)
                if neumann_mask.size != n_cells * n_cells:
                    raise ValueError("neumann_mask must have n_cells^2 entries")
                ptr = neumann_mask.ctypes.data
            else:
                ptr = neumann_mask.data_ptr()
            bc = mg_bc(MG_BC_MIXED, ptr, int(box_sides))
        self.handle = mg_setup(psi, grid, bc, stab, stream)

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(np.ascontiguousarray(prob.psi, dtype=np.float64).ravel(), prob.N, prob.x0,
                   prob.y0, prob.h, **kw)

    def counts(self):
        return mg_get_counts(self.handle)

    def solve(self, f, g, u, tol: float = 1e-10, allow_not_converged: bool = False,
              gN=None) -> mg_info:
        """g: Dirichlet data; gN: nodal Neumann data (mixed boundary
        conditions; None = 0)."""
        info = mg_info()
        ok = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        if gN is None:
            mg_solve(self.handle, f, g, u, tol, info, ok)
        else:
            mg_solve_bc(self.handle, f, g, gN, u, tol, info, ok)
        return info

    def rhs(self, f, g, F, gN=None):
        if gN is None:
            mg_rhs(self.handle, f, g, F)
        else:
            mg_rhs_bc(self.handle, f, g, gN, F)
        return F

    def cycles(self, F, u, k: int, precision: str = "fp64"):
        mg_cycles(self.handle, F, u, k, {"fp64": MG_FP64, "mixed": MG_MIXED}[precision])
        return u

    def cycles_transposed(self, F, u, k: int):
        mg_cycles_transposed(self.handle, F, u, k)
        return u

    def residual(self, F, u, r=None):
        return mg_residual(self.handle, F, u, r)

    def adjoint(self, dLdu, dLdf=None, dLdg=None, allow_not_converged: bool = False,
                dLdgN=None):
        """dL/df, dL/dg (and dL/dg_N with mixed conditions) of a loss of the
        last solve's u (outputs may be None): solves A w = dL/du to the last
        solve's tolerance."""
        ok = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        if dLdgN is None:
            mg_adjoint(self.handle, dLdu, dLdf, dLdg, ok)
            return dLdf, dLdg
        mg_adjoint_bc(self.handle, dLdu, dLdf, dLdg, dLdgN, ok)
        return dLdf, dLdg, dLdgN

    def stencil(self, level: int) -> np.ndarray:
        n = mg_level_cells(self.handle, level)
        out = np.zeros((n + 1) * (n + 1) * 9)
        mg_export_stencil(self.handle, level, out)
        return out.reshape(-1, 9)

    def cut_cells(self):
        total = mg_export_cut_cells(self.handle, 0, None, None)
        cells = np.zeros(total, dtype=np.int32)
        data = np.zeros(total * 52)
        mg_export_cut_cells(self.handle, total, cells, data)
        return cells, data.reshape(-1, 52)

    def close(self):
        if getattr(self, "handle", None):
            mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _DeviceArray:
    """A raw device allocation seen through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None}


class BatchSolver:
    """Owns one batch of independent problems (see mg_batch_setup).
    ``problems``: objects with psi, N, x0, y0, h (workloads.Problem).  Packed
    arrays put member p's (N_p+1)^2 nodes at offsets()[p]."""

    def __init__(self, problems, *, gamma: float = 2.0, alpha: float = 1.75, eta: int = 4,
                 nu1: int = 2, nu2: int = 1, max_cycles: int = 100, inner: int = 0,
                 stream: int = 0, box_sides: bool = False):
        """Members with a ``neumann_mask`` attribute make a MG_BC_MIXED batch
        (members without one get an all-zero mask); box_sides applies to all
        members."""
        stab = mg_default_stab()
        stab.gamma, stab.alpha, stab.eta = gamma, alpha, eta
        stab.nu1, stab.nu2, stab.max_cycles, stab.inner = nu1, nu2, max_cycles, inner
        stab.precision = MG_MIXED
        self.sizes = [int(p.N) for p in problems]
        grids = [mg_grid(p.N, p.x0, p.y0, p.h, 8) for p in problems]
        psi = self.pack([p.psi for p in problems])
        masks = [getattr(p, "neumann_mask", None) for p in problems]
        if any(m is not None for m in masks):
            self._mask = np.concatenate([
                (np.zeros(p.N * p.N, np.uint8) if m is None
                 else np.ascontiguousarray(m, dtype=np.uint8).ravel())
                for p, m in zip(problems, masks)])
            bc = mg_bc(MG_BC_MIXED, self._mask.ctypes.data, int(box_sides))
        else:
            bc = mg_bc(MG_BC_DIRICHLET, None, int(box_sides))
        self.handle = mg_batch_setup(grids, psi, bc, stab, stream)
        self.count = len(problems)
        self.total, self._f, self._g, self._u = mg_batch_buffers(self.handle)

    def offsets(self):
        off = np.zeros(len(self.sizes) + 1, dtype=np.int64)
        off[1:] = np.cumsum([(n + 1) ** 2 for n in self.sizes])
        return off

    def pack(self, arrays) -> np.ndarray:
        return np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays])

    def unpack(self, packed):
        off = self.offsets()
        return [packed[off[p]:off[p + 1]] for p in range(len(self.sizes))]

    def buffers(self):
        """(f, g, u): torch views of the batch's own device packed arrays;
        solving from them skips every copy."""
        import torch
        return tuple(torch.as_tensor(_DeviceArray(ptr, self.total), device="cuda")
                     for ptr in (self._f, self._g, self._u))

    def solve(self, f, g, u, tol: float = 1e-10, allow_not_converged: bool = False, gN=None):
        info = (mg_batch_info * self.count)()
        ok = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        if gN is None:
            mg_batch_solve(self.handle, f, g, u, tol, info, ok)
        else:
            _check(load().mg_batch_solve_bc(self.handle, _addr(f), _addr(g), _addr(gN),
                                            _addr(u, True), tol, ctypes.addressof(info)),
                   "mg_batch_solve_bc", ok)
        return list(info)

    def solve_status(self, f, g, u, tol: float = 1e-10):
        """(return code, per-member info) without raising on member failures."""
        info = (mg_batch_info * self.count)()
        code = load().mg_batch_solve(self.handle, _addr(f), _addr(g), _addr(u, True), tol,
                                     ctypes.addressof(info))
        return code, list(info)

    def tune(self, f, g, tol: float = 1e-10, reps: int = 3):
        """Autotunes the launch shape; returns (shape tuple, ms per solve)."""
        best, ms = mg_batch_tune(self.handle, f, g, tol, reps)
        return best.astuple(), ms

    def set_shape(self, threads: int = 512, first_group: int = 4, cluster: int = 1,
                  coop_min_dof: int = 0):
        mg_batch_set_shape(self.handle, mg_batch_shape(threads, first_group, cluster,
                                                       coop_min_dof))

    def shape(self):
        return mg_batch_get_shape(self.handle).astuple()

    def timing(self):
        return mg_batch_timing(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            mg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# --- differentiation --------------------------------------------------------

def solve_diff(solver: "Solver", f, g, tol: float = 1e-10):
    """u = solve(f, g) as a differentiable torch operation: the backward pass
    runs mg_adjoint (dL/df = M^T w, dL/dg = G^T w with A w = dL/du).  f and g
    are (N+1)^2 float64 CUDA tensors; u has the same shape."""
    import torch

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, f_, g_):
            u = torch.zeros_like(f_)
            solver.solve(f_.detach().contiguous(), g_.detach().contiguous(), u, tol=tol)
            return u

        @staticmethod
        def backward(ctx, dLdu):
            need_f, need_g = ctx.needs_input_grad
            if not (need_f or need_g):
                return None, None
            dLdf = torch.zeros_like(dLdu) if need_f else None
            dLdg = torch.zeros_like(dLdu) if need_g else None
            solver.adjoint(dLdu.detach().contiguous(), dLdf, dLdg)
            return dLdf, dLdg

    return _Solve.apply(f, g)
