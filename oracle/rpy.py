"""Rotne-Prager-Yamakawa mobility (test infrastructure).

The low-fidelity operator of Bi-PQN (Sec. 5) is left open by the paper; the
stand-in is the RPY pairwise mobility for equal non-overlapping spheres of
radius a (centre distance r >= 2a), r_vec = c_i - c_j, rhat = r_vec / r:

  self:  tt = I / (6 pi mu a),  rr = I / (8 pi mu a^3),  tr = rt = 0
  pair:  tt = [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) rhat rhat^T] / (8 pi mu r)
         rr = (3 rhat rhat^T - I) / (16 pi mu r^3)
         tr:  U_i from T_j = (T_j x r_vec) / (8 pi mu r^3)   (rotlet)
         rt:  Omega_i from F_j = (F_j x r_vec) / (8 pi mu r^3) (half the Stokeslet vorticity)
"""
import numpy as np


def _cross_matrix(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rpy_matrix(centers: np.ndarray, a: float = 1.0, mu: float = 1.0) -> np.ndarray:
    """Dense 6M x 6M RPY mobility with per-body rows (U, Omega), columns (F, T)."""
    M = centers.shape[0]
    out = np.zeros((6 * M, 6 * M))
    I3 = np.eye(3)
    for i in range(M):
        out[6 * i:6 * i + 3, 6 * i:6 * i + 3] = I3 / (6 * np.pi * mu * a)
        out[6 * i + 3:6 * i + 6, 6 * i + 3:6 * i + 6] = I3 / (8 * np.pi * mu * a ** 3)
        for j in range(M):
            if j == i:
                continue
            rv = centers[i] - centers[j]
            r = float(np.sqrt(rv @ rv))
            rh = rv / r
            P = np.outer(rh, rh)
            tt = ((1 + 2 * a * a / (3 * r * r)) * I3 + (1 - 2 * a * a / (r * r)) * P) / (8 * np.pi * mu * r)
            rr = (3 * P - I3) / (16 * np.pi * mu * r ** 3)
            # (T x r) = -[r]_x T ;  (F x r) = -[r]_x F
            tr = -_cross_matrix(rv) / (8 * np.pi * mu * r ** 3)
            out[6 * i:6 * i + 3, 6 * j:6 * j + 3] = tt
            out[6 * i + 3:6 * i + 6, 6 * j + 3:6 * j + 6] = rr
            out[6 * i:6 * i + 3, 6 * j + 3:6 * j + 6] = tr
            out[6 * i + 3:6 * i + 6, 6 * j:6 * j + 3] = tr
    return out
