"""ctypes wrapper of the plain-C matrix-free oracle ``mf.c`` (test infrastructure)."""
import ctypes
import os
import subprocess

import numpy as np

from .bie import janus_slip, self_correction
from .quadrature import surface_nodes

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmf_oracle.so")
_lib = None


def build_library(force: bool = False) -> str:
    """Compile mf.c with gcc/OpenMP into oracle/libmf_oracle.so."""
    src = os.path.join(_HERE, "mf.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build_library()
        _lib = ctypes.CDLL(_SO)
        D = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        _lib.mf_apply.argtypes = [i, i, D, D, D, D, D, D, D]
        _lib.mf_rigid_coeffs.argtypes = [i, i, D, D, D, D, D]
        _lib.mf_stokeslet_rhs.argtypes = [i, i, D, D, D, ctypes.c_double, D]
        _lib.mf_gmres.argtypes = [i, i, D, D, D, D, D, D, D, ctypes.c_double, i, i]
        _lib.mf_gmres.restype = i
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class MatrixFreeMobility:
    """Mobility of one configuration by matrix-free GMRES (same operator as DenseMobility,
    including its optional accurate self-interaction)."""

    def __init__(self, centers, n_theta, n_phi, a=1.0, mu=1.0, tol=1e-12, restart=60, maxit=500,
                 self_quadrature=False):
        self.lib = _load()
        self.centers = np.ascontiguousarray(centers, dtype=np.float64)
        self.M = self.centers.shape[0]
        self.ns = n_theta * n_phi
        self.mu, self.tol, self.restart, self.maxit = mu, tol, restart, maxit
        x, n, w, body = surface_nodes(self.centers, n_theta, n_phi, a)
        self.x = np.ascontiguousarray(x)
        self.n = np.ascontiguousarray(n)
        self.w = np.ascontiguousarray(w)
        self.body = body
        self.last_iterations = 0
        self.cself = np.ascontiguousarray(self_correction(n_theta, n_phi, a)) if self_quadrature else None

    def _c(self):
        return _p(self.cself) if self.cself is not None else None

    def apply_operator(self, phi):
        out = np.empty(3 * self.M * self.ns)
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        self.lib.mf_apply(self.M, self.ns, _p(self.x), _p(self.n), _p(self.w), _p(self.centers), self._c(),
                          _p(phi), _p(out))
        return out

    def rhs(self, FT, axes=None):
        out = np.empty(3 * self.M * self.ns)
        FT = np.ascontiguousarray(FT, dtype=np.float64).reshape(-1)
        self.lib.mf_stokeslet_rhs(self.M, self.ns, _p(self.x), _p(self.centers), _p(FT), self.mu, _p(out))
        if axes is not None:
            out += janus_slip(self.n, self.body, np.asarray(axes, float)).reshape(-1)
        return out

    def solve_density(self, rhs):
        phi = np.empty(3 * self.M * self.ns)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
        it = self.lib.mf_gmres(self.M, self.ns, _p(self.x), _p(self.n), _p(self.w), _p(self.centers), self._c(),
                               _p(rhs), _p(phi), self.tol, self.restart, self.maxit)
        self.last_iterations = it
        if it < 0:
            raise RuntimeError("matrix-free GMRES did not converge")
        return phi

    def velocities(self, phi):
        coeff = np.empty(6 * self.M)
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        self.lib.mf_rigid_coeffs(self.M, self.ns, _p(self.x), _p(self.w), _p(self.centers), _p(phi), _p(coeff))
        return -coeff

    def apply(self, FT, axes=None):
        """U = M FT (+ slip-driven velocity when Janus axes are given); [6M]."""
        return self.velocities(self.solve_density(self.rhs(FT, axes)))
