"""FP64 CPU oracle of the domain-wall multigrid solve.

TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The library's
product path never imports, links or runs it, and it shares no code with
the GPU path (it reads the same seeded inputs, nothing else).

Contents
  dwf_oracle.c : the fine Shamir operator D, D^+ = Gamma D Gamma and the
                 single hopping terms, plain loops in FP64 (Sec. 2, Sec. 4 of
                 Cohen-Brower-Clark-Osborn, "Multigrid Algorithms for
                 Domain-Wall Fermions").
  mg.py        : blocking, block Gram-Schmidt, restrictor/prolongator, the
                 Galerkin coarse operator R D P and the squared operator's
                 P^+ D^+ D P (brute force and by stencil), GCR / CGNR,
                 the V-cycle and the adaptive setup, in numpy FP64.
  net.py       : the learned near-null proposal's network, loss and gradient.
  eig.py       : the low-mode diagnostic (dense eigenpairs of D^+ D, coarse
                 overlaps).
  dwf2d.py     : the 2D U(1) domain-wall operator of the toy model (Sec. 3).
Parity status of every function is listed in each module's header.
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "libdwforacle.so"
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the oracle's C code (gcc, OpenMP) into oracle/libdwforacle.so."""
    src = _HERE / "dwf_oracle.c"
    if force or not _SO.exists() or _SO.stat().st_mtime < src.stat().st_mtime:
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", str(src), "-o",
               str(_SO) + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(str(_SO) + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_SO))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        ci, cd = ctypes.c_int, ctypes.c_double
        L.orc_gamma.argtypes = [ci, dp]
        L.orc_apply_D.argtypes = [dp, dp, dp, ip, ci, cd, cd, ci]
        L.orc_apply_Ddag.argtypes = [dp, dp, dp, ip, ci, cd, cd, ci]
        L.orc_apply_D_sites.argtypes = [dp, dp, dp, ip, ci, cd, cd, ci,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]
        L.orc_hop.argtypes = [dp, dp, dp, ip, ci, ci, ci, ci]
        _lib = L
    return _lib


def _dp(a):
    assert a.flags.c_contiguous and a.dtype == np.complex128
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gamma(mu: int) -> np.ndarray:
    """The 4x4 gamma matrix the oracle uses for direction mu (0..3 = x,y,z,t)."""
    g = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(mu, _dp(g))
    return g


class DWF:
    """Fine Shamir domain-wall operator on one lattice (FP64).

    dims = (X, Y, Z, T); links U shape (T, Z, Y, X, 4, 3, 3); fermion fields
    shape (Ls, T, Z, Y, X, 4, 3).
    """

    def __init__(self, U, dims, Ls, M5, mf, antiperiodic_t=True):
        self.U = np.ascontiguousarray(U, dtype=np.complex128)
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.M5 = float(M5)
        self.mf = float(mf)
        self.ap = 1 if antiperiodic_t else 0
        X, Y, Z, T = self.dims
        self.shape = (self.Ls, T, Z, Y, X, 4, 3)
        self._cd = (ctypes.c_int * 4)(*self.dims)

    def _prep(self, f):
        f = np.ascontiguousarray(f, dtype=np.complex128)
        assert f.shape == self.shape, (f.shape, self.shape)
        return f

    def D(self, f):
        f = self._prep(f)
        out = np.empty_like(f)
        lib().orc_apply_D(_dp(out), _dp(f), _dp(self.U), self._cd, self.Ls, self.M5, self.mf, self.ap)
        return out

    def Ddag(self, f):
        f = self._prep(f)
        out = np.empty_like(f)
        lib().orc_apply_Ddag(_dp(out), _dp(f), _dp(self.U), self._cd, self.Ls, self.M5, self.mf, self.ap)
        return out

    def D_sites(self, f, idx5):
        """(D f) at 5D sites idx5 = s*V + site4; returns shape (n, 4, 3)."""
        f = self._prep(f)
        idx = np.ascontiguousarray(idx5, dtype=np.int64)
        out = np.empty((idx.size, 4, 3), dtype=np.complex128)
        lib().orc_apply_D_sites(_dp(out), _dp(f), _dp(self.U), self._cd, self.Ls, self.M5, self.mf,
                                self.ap, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), idx.size)
        return out

    def hop(self, f, mu, d):
        """-1/2 (1 - d gamma_mu) U^(d) f(x + d mu): one of the 8 hopping terms of D."""
        f = self._prep(f)
        out = np.empty_like(f)
        lib().orc_hop(_dp(out), _dp(f), _dp(self.U), self._cd, self.Ls, mu, d, self.ap)
        return out
