"""Oracle (test infrastructure and CPU baseline only): ctypes binding of
oracle/vcycle.c, the plain-C OpenMP restatement of oracle.multigrid's
4-colour V(nu1, nu2)-cycle, used to time the method on the host cores.

``build()`` compiles it with gcc (-O3 -fopenmp, no machine-specific flags);
``CVCycle(levels)`` copies a hierarchy from oracle.multigrid.build_hierarchy
(operators, DOF and cut-node masks, P and P^T of every level) into C.
Pinned against oracle.multigrid.mg_cycle in tests/test_oracle_cvcycle.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vcycle.c")
LIB = os.path.join(HERE, "libvcycle.so")

_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        cmd = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c99", SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed on {SRC}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.vc_create.restype = P
        lib.vc_create.argtypes = [I]
        lib.vc_destroy.restype = None
        lib.vc_destroy.argtypes = [P]
        lib.vc_set_level.restype = I
        lib.vc_set_level.argtypes = [P, I, I] + [P] * 11 + [I]
        lib.vc_cycles.restype = I
        lib.vc_cycles.argtypes = [P, P, P, I, I, I, I, I]
        lib.vc_solve.restype = I
        lib.vc_solve.argtypes = [P, P, P, D, I, I, I, I, I, P]
        lib.vc_threads.restype = I
        lib.vc_threads.argtypes = [I]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class CVCycle:
    """The hierarchy of oracle.multigrid.build_hierarchy, copied into C."""

    def __init__(self, levels):
        lib = load()
        self._h = lib.vc_create(len(levels))
        if not self._h:
            raise MemoryError("vc_create")
        self.m = (levels[0].n + 1) ** 2
        for l, L in enumerate(levels):
            A = sp.csr_matrix(L.A)
            A.sort_indices()
            Ap, Ai = A.indptr.astype(np.int32), A.indices.astype(np.int32)
            Ax = A.data.astype(np.float64)
            dof = np.ascontiguousarray(L.dof, dtype=np.uint8)
            cut = np.ascontiguousarray(L.cut_nodes & L.dof, dtype=np.uint8)
            arrs = [None] * 6
            mc = 0
            if l + 1 < len(levels):
                P = sp.csr_matrix(L.P)
                T = sp.csr_matrix(P.T)
                arrs = [P.indptr.astype(np.int32), P.indices.astype(np.int32),
                        P.data.astype(np.float64), T.indptr.astype(np.int32),
                        T.indices.astype(np.int32), T.data.astype(np.float64)]
                mc = (levels[l + 1].n + 1) ** 2
            keep = [Ap, Ai, Ax, dof, cut] + arrs
            rc = lib.vc_set_level(self._h, l, L.n, *[_ptr(a) for a in keep], mc)
            if rc != 0:
                raise RuntimeError(f"vc_set_level({l}) failed: {rc}")

    def cycles(self, F, u, k=1, nu1=2, nu2=1, eta=4, threads=0):
        F = np.ascontiguousarray(F, dtype=np.float64)
        assert u.dtype == np.float64 and u.flags.c_contiguous and u.size == self.m
        load().vc_cycles(self._h, _ptr(F), _ptr(u), k, nu1, nu2, eta, threads)
        return u

    def solve(self, F, u=None, tol=1e-10, max_cycles=100, nu1=2, nu2=1, eta=4, threads=0):
        """(u, history of relative residuals, cycles); cycles -1 if tol
        was not reached."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        u = np.zeros(self.m) if u is None else np.ascontiguousarray(u, dtype=np.float64).copy()
        hist = np.zeros(max_cycles + 1)
        k = load().vc_solve(self._h, _ptr(F), _ptr(u), tol, max_cycles, nu1, nu2, eta, threads,
                            _ptr(hist))
        n = k if k >= 0 else max_cycles
        return u, hist[:n + 1].tolist(), k

    @staticmethod
    def threads(requested=0):
        return load().vc_threads(requested)

    def close(self):
        if getattr(self, "_h", None):
            load().vc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
