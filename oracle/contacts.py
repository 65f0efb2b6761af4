"""Collisional set and contact matrix (test infrastructure).

Sec. 3, Eq. (collisional-set): a pair (i, j) enters the LCP when its gap
Phi = |c_j - c_i| - 2a is at most the threshold delta.  For spheres, column l
of D (Sec. 3, after Eq. DVI) holds the force of a unit repulsive normal
contact force: -n on body i and +n on body j with n = (c_j - c_i)/|c_j - c_i|,
and zero torques (6 non-zeros).  Hence (D^T U)_l = n . (U_j - U_i), the rate of
change of the gap.
"""
import numpy as np


def detect_contacts(centers: np.ndarray, a: float, delta: float):
    """All pairs i < j with gap <= delta, in lexicographic (i, j) order.

    Returns (pairs [n,2] int, normals [n,3], gaps [n]).
    """
    M = centers.shape[0]
    pairs, normals, gaps = [], [], []
    for i in range(M):
        for j in range(i + 1, M):
            d = centers[j] - centers[i]
            r = float(np.sqrt(d @ d))
            gap = r - 2.0 * a
            if gap <= delta:
                pairs.append((i, j))
                normals.append(d / r)
                gaps.append(gap)
    return (np.array(pairs, dtype=np.int64).reshape(-1, 2),
            np.array(normals).reshape(-1, 3), np.array(gaps))


def contact_matrix(M: int, pairs: np.ndarray, normals: np.ndarray) -> np.ndarray:
    """Dense D in R^{6M x n}; rows per body are (Fx, Fy, Fz, Tx, Ty, Tz)."""
    n = pairs.shape[0]
    D = np.zeros((6 * M, n))
    for l in range(n):
        i, j = pairs[l]
        D[6 * i:6 * i + 3, l] = -normals[l]
        D[6 * j:6 * j + 3, l] = normals[l]
    return D
