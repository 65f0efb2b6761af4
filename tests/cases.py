"""Shared test helpers: oracle data for a workload instance (CPU, FP64)."""
from __future__ import annotations

import functools

import numpy as np

from oracle.bie import DenseMobility, janus_slip, stokeslet_rotlet_rhs
from oracle.contacts import contact_matrix, detect_contacts
from oracle.lcp import lcp_data, pgs
from oracle.rpy import rpy_matrix
from workloads import make_instance


# The library's default operator takes each sphere's self-interaction with the high-order rule
# (cfg.self_quadrature = 1): oracles compared with default contexts do the same.
SELF_QUADRATURE = True


@functools.lru_cache(maxsize=8)
def dense_case(name: str, index: int):
    """Instance plus its dense oracle: mobility, D, U_nc, A, b, A_hat, LCP solution."""
    inst = make_instance(name, index)
    mob = DenseMobility(inst.centers, inst.n_theta, inst.n_phi, a=inst.radius, mu=inst.viscosity,
                        self_quadrature=SELF_QUADRATURE)
    pairs, normals, gaps = detect_contacts(inst.centers, inst.contact_radius, inst.delta)
    D = contact_matrix(inst.n_bodies, pairs, normals)
    U_nc = mob.apply(np.zeros(6 * inst.n_bodies), axes=inst.axes)
    Mob = mob.matrix()
    A, b = lcp_data(D, Mob, U_nc, gaps, inst.dt)
    Ahat = D.T @ rpy_matrix(inst.centers, a=inst.radius, mu=inst.viscosity) @ D
    xs = pgs(A, b)
    return dict(inst=inst, mob=mob, pairs=pairs, normals=normals, gaps=gaps, D=D, U_nc=U_nc, Mob=Mob,
                A=A, b=b, Ahat=Ahat, x=xs)


def active_set(x, g, scale=1.0):
    """Indices with x_l > 1e-9 max(1, ||x||_inf); ambiguous ones (both tiny) excluded."""
    thr = 1e-9 * max(1.0, np.abs(x).max() if x.size else 1.0) * scale
    act = set(np.nonzero(x > thr)[0].tolist())
    amb = set(np.nonzero((np.abs(x) <= thr) & (np.abs(g) <= thr))[0].tolist())
    return act, amb


def rhs_oracle(mob: DenseMobility, FT, axes=None):
    r = stokeslet_rotlet_rhs(mob.x, mob.centers, np.asarray(FT, float), mob.mu)
    if axes is not None:
        r = r + janus_slip(mob.n, mob.body, np.asarray(axes, float))
    return r.reshape(-1)


# Relative accuracy of one GPU mobility solve inside an MVP: GMRES (or its
# refinement) stops at a relative residual of 1e-12 on (K + P), whose condition
# number is 2-3 on these packings; 1e-11 leaves a margin of more than 3.
MVP_SOLVE_REL = 1e-11

# Bound on the measured gap ||A_oracle x + b_oracle - (A_gpu x + b_gpu)||_2 at a
# solution, relative to ||b||_2: both sides solve the same discrete mobility
# problem to a relative residual of 1e-12.
MISMATCH_REL = 1e-10


def kkt_bound(tol, x, g_oracle, g_gpu, b, hi_mvps):
    """Tolerance for ||min(x, A_oracle x + b)||_2 at a GPU solution x.

    The GPU stops when ||min(x, g_int)||_2 <= tol for its incrementally updated
    gradient g_int.  min(x, .) is 1-Lipschitz, so the oracle's KKT error is at
    most tol + ||g_oracle - g_int||_2, and
      ||g_oracle - g_int|| <= ||g_oracle - g_gpu|| + ||g_gpu - g_int||,
    with g_gpu = A_gpu x + b_gpu one fresh GPU MVP at x (the measured operator
    and b mismatch) and the second term the drift of g_int: each of the
    hi_mvps + 1 MVPs that built it carries a solve error of at most
    MVP_SOLVE_REL times its increment, and every increment eta A p is below
    ||b|| on these packings (measured <= 2.3 %).  Returns (eps_op, mismatch).
    tol is the solve tolerance the bound is added to (kept for the call's
    readability; eps_op does not depend on it)."""
    mismatch = float(np.linalg.norm(np.asarray(g_oracle) - np.asarray(g_gpu)))
    drift = MVP_SOLVE_REL * (hi_mvps + 1) * float(np.linalg.norm(b))
    return mismatch + drift, mismatch
