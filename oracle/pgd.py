"""BB-PGD: proximal gradient descent with the Barzilai-Borwein step (test infrastructure).

Sec. 6, Eq. (spectralStepSize) and Table 1: x_{k+1} = (x_k - tau_k g_k)_+ with
over-relaxation 1 and tau_bb = ||x_k - x_{k-1}||^2 / ((x_k - x_{k-1})^T (A x_k - A x_{k-1})),
one MVP per iteration.  The paper gives no first step; the reading used here
is tau_0 = 3 pi mu a, the inverse of the normal self-mobility 2 / (6 pi mu a)
of a contact between two free spheres.
"""
import numpy as np


def bb_pgd(mvp, b, x0, tau0, tol=1e-8, kmax=500):
    """Returns (x, g, iterations, mvps, converged)."""
    b = np.asarray(b, float)
    x = np.maximum(np.asarray(x0, float), 0.0)
    g = mvp(x) + b
    mvps = 1
    tau = tau0
    for k in range(kmax):
        if np.linalg.norm(np.minimum(x, g)) <= tol:
            return x, g, k, mvps, True
        p = np.maximum(x - tau * g, 0.0) - x
        Ap = mvp(p)
        mvps += 1
        x = x + p
        g = g + Ap
        pAp = float(p @ Ap)
        tau = float(p @ p) / pAp if pAp > 0.0 else tau0
    return x, g, kmax, mvps, bool(np.linalg.norm(np.minimum(x, g)) <= tol)
