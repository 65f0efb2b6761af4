"""LCP definitions and reference solvers (test infrastructure).

Sec. 3, Eqs. (LCP) and (defAandb): find x with 0 <= x  perp  A x + b >= 0,
A = D^T M D and b = (Phi + dt D^T U_nc) / dt.  Sec. 3.1, Eq. (qp): this is the
KKT system of min_{x >= 0} 1/2 x^T A x + x^T b.  Sec. 6, Eq. (kkt-error): the
absolute KKT error is ||min(x, A x + b)||.

The solvers here are independent of the paper's methods: projected
Gauss-Seidel on the dense matrix, followed by an exact solve on the detected
active set, and brute-force enumeration of all 2^n active sets for small n.
"""
import itertools

import numpy as np


def lcp_data(D: np.ndarray, Mob: np.ndarray, U_nc: np.ndarray, gaps: np.ndarray, dt: float):
    """A = D^T M D and b = gaps / dt + D^T U_nc (Eq. defAandb)."""
    return D.T @ Mob @ D, gaps / dt + D.T @ U_nc


def kkt_abs(x: np.ndarray, g: np.ndarray, ord=2) -> float:
    """||min(x, g)|| with g = A x + b (Eq. kkt-error)."""
    return float(np.linalg.norm(np.minimum(x, g), ord=ord)) if x.size else 0.0


def objective(A, b, x) -> float:
    """1/2 x^T A x + x^T b (Eq. qp)."""
    return float(0.5 * x @ (A @ x) + b @ x)


def polish(A, b, active) -> np.ndarray:
    """Solve A_SS x_S = -b_S on a given active set S, zero elsewhere."""
    x = np.zeros(b.shape[0])
    S = np.nonzero(active)[0]
    if S.size:
        x[S] = np.linalg.solve(A[np.ix_(S, S)], -b[S])
    return x


def pgs(A, b, tol=1e-13, max_sweeps=200000, x0=None) -> np.ndarray:
    """Projected Gauss-Seidel, then an exact solve on the active set it finds."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.maximum(np.array(x0, float), 0.0)
    for _ in range(max_sweeps):
        for l in range(n):
            r = b[l] + A[l] @ x
            x[l] = max(0.0, x[l] - r / A[l, l])
        if kkt_abs(x, A @ x + b, ord=np.inf) <= tol:
            break
    xp = polish(A, b, x > 0.0)
    if (xp >= 0).all() and kkt_abs(xp, A @ xp + b, ord=np.inf) <= kkt_abs(x, A @ x + b, ord=np.inf):
        return xp
    return x


def brute_force(A, b) -> np.ndarray:
    """Enumerate all active sets (n <= 12); return the unique LCP solution."""
    n = b.shape[0]
    assert n <= 12
    best = None
    for k in range(n + 1):
        for S in itertools.combinations(range(n), k):
            act = np.zeros(n, dtype=bool)
            act[list(S)] = True
            x = polish(A, b, act)
            if (x[act] >= -1e-12).all():
                g = A @ x + b
                if (g[~act] >= -1e-12).all():
                    best = x
                    return np.maximum(best, 0.0)
    raise RuntimeError("no LCP solution found")
