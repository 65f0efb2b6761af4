"""Dense boundary-integral mobility (test infrastructure).

Sec. 2 of the paper writes the mobility as M ~ P M_stk P^T (Fig. 1) and cites
a second-kind boundary-integral formulation without fixing its details.  The
concrete stand-in used here (and by the GPU library) is the completed
double-layer representation of exterior Stokes flow past M rigid spheres:

    u(x) = D[phi](x) + sum_j [ G(x - c_j) F_j + R(x - c_j) T_j ]

with the stresslet double layer D, the Stokeslet G(r) = (I/|r| + r r^T/|r|^3)
/ (8 pi mu) and the rotlet R(r) T = (T x r) / (8 pi mu |r|^3).  On the surfaces
u = U_i + Omega_i x (x - c_i) + s(x) (Eq. stokes-bc, plus an active slip s).
The exterior limit of D annihilates piecewise-rigid densities, so the rigid
part of the density is pinned with the weighted orthogonal projector P onto
the rigid modes of each body:

    (K + P) phi = s - S[F, T]|_Gamma,      (U_i, Omega_i) = -(rigid coefficients of P phi on body i)

K is the exterior limit of D after global singularity subtraction on the
product quadrature (valid because the double layer of a constant density is
zero outside the body and the identity inside):

    (K phi)_p = sum_{q != p} w_q T(x_p - x_q, n_q) (phi_q - phi_p),
    T(r, n) v = -(3 / (4 pi)) r (r . n)(r . v) / |r|^5.

Everything here is dense FP64 and solved by LU (SciPy/LAPACK).
"""
import numpy as np
import scipy.linalg as sla

from .quadrature import surface_nodes


def stresslet_matrix(x: np.ndarray, n: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Dense 3N x 3N matrix of K (global singularity subtraction)."""
    N = x.shape[0]
    K = np.zeros((3 * N, 3 * N))
    c = -3.0 / (4.0 * np.pi)
    for p in range(N):
        r = x[p] - x                      # r_pq = x_p - x_q for every q
        r2 = np.einsum("ij,ij->i", r, r)
        r2[p] = 1.0
        rn = np.einsum("ij,ij->i", r, n)
        coef = c * w * rn / r2 ** 2.5
        coef[p] = 0.0
        blocks = coef[:, None, None] * r[:, :, None] * r[:, None, :]   # [N,3,3]
        K[3 * p:3 * p + 3, :] = blocks.transpose(1, 0, 2).reshape(3, 3 * N)
        K[3 * p:3 * p + 3, 3 * p:3 * p + 3] -= blocks.sum(axis=0)
    return K


def rigid_basis(xi: np.ndarray) -> np.ndarray:
    """Rigid modes on one body: columns e_k (translation) and e_k x xi (rotation)."""
    ns = xi.shape[0]
    Psi = np.zeros((3 * ns, 6))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        Psi[:, k] = np.tile(e, ns)
        Psi[:, 3 + k] = np.cross(e, xi).reshape(-1)
    return Psi


def rigid_projector(centers, x, w, body) -> tuple[np.ndarray, list]:
    """Block-diagonal weighted orthogonal projector P and per-body (Psi, G)."""
    N = x.shape[0]
    P = np.zeros((3 * N, 3 * N))
    parts = []
    for i in range(centers.shape[0]):
        idx = np.nonzero(body == i)[0]
        Psi = rigid_basis(x[idx] - centers[i])
        W = np.repeat(w[idx], 3)
        G = Psi.T @ (W[:, None] * Psi)
        rows = (3 * idx[:, None] + np.arange(3)).reshape(-1)
        P[np.ix_(rows, rows)] = Psi @ np.linalg.solve(G, Psi.T * W[None, :])
        parts.append((rows, Psi, W, G))
    return P, parts


def rigid_velocities(phi: np.ndarray, parts) -> np.ndarray:
    """(U_i, Omega_i) = -(rigid coefficients of P phi) for every body; [6M]."""
    out = []
    for rows, Psi, W, G in parts:
        coeff = np.linalg.solve(G, Psi.T @ (W * phi[rows]))
        out.append(-coeff)
    return np.concatenate(out)


def stokeslet_rotlet_rhs(x: np.ndarray, centers: np.ndarray, FT: np.ndarray,
                         mu: float) -> np.ndarray:
    """-S[F, T] at every node: minus the Stokeslet and rotlet fields of all bodies."""
    out = np.zeros_like(x)
    FT = FT.reshape(-1, 6)
    for j in range(centers.shape[0]):
        r = x - centers[j]
        rr = np.sqrt(np.einsum("ij,ij->i", r, r))
        F = FT[j, :3]
        T = FT[j, 3:]
        u = (F[None, :] / rr[:, None] + r * (r @ F)[:, None] / rr[:, None] ** 3) / (8 * np.pi * mu)
        u += np.cross(T[None, :], r) / (8 * np.pi * mu * rr[:, None] ** 3)
        out -= u
    return out


def janus_slip(n: np.ndarray, body: np.ndarray, axes: np.ndarray) -> np.ndarray:
    """Tangential slip -(I - n n^T) e on the hemisphere n . e >= 0, zero elsewhere."""
    e = axes[body]
    ne = np.einsum("ij,ij->i", n, e)
    s = -(e - ne[:, None] * n)
    s[ne < 0.0] = 0.0
    return s


class DenseMobility:
    """Dense LU of (K + P) for one configuration; applies the mobility M."""

    def __init__(self, centers, n_theta, n_phi, a=1.0, mu=1.0):
        self.centers = np.asarray(centers, dtype=np.float64)
        self.a, self.mu = a, mu
        self.x, self.n, self.w, self.body = surface_nodes(self.centers, n_theta, n_phi, a)
        self.K = stresslet_matrix(self.x, self.n, self.w)
        self.P, self.parts = rigid_projector(self.centers, self.x, self.w, self.body)
        self.lu = sla.lu_factor(self.K + self.P)

    def solve_density(self, rhs: np.ndarray) -> np.ndarray:
        return sla.lu_solve(self.lu, rhs.reshape(-1))

    def apply(self, FT: np.ndarray, axes=None) -> np.ndarray:
        """U = M FT (+ the slip-driven velocity when Janus axes are given); [6M]."""
        rhs = stokeslet_rotlet_rhs(self.x, self.centers, np.asarray(FT, float), self.mu)
        if axes is not None:
            rhs = rhs + janus_slip(self.n, self.body, np.asarray(axes, float))
        return rigid_velocities(self.solve_density(rhs), self.parts)

    def matrix(self) -> np.ndarray:
        """Dense 6M x 6M mobility, one column per unit force/torque."""
        M6 = 6 * self.centers.shape[0]
        cols = [self.apply(np.eye(M6)[:, k]) for k in range(M6)]
        return np.stack(cols, axis=1)
