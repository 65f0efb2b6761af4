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

Optionally (``self_quadrature``) each body's self-interaction is taken by a
high-order rule instead of the product rule: ``self_correction`` below.
"""
import functools

import numpy as np
import scipy.linalg as sla

from .quadrature import sphere_template, surface_nodes


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


def _real_harmonics(u: np.ndarray, L: int) -> np.ndarray:
    """Orthonormal real spherical harmonics of degree <= L at unit vectors u: [len(u), (L+1)^2]."""
    from scipy.special import sph_harm_y
    th = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    ph = np.arctan2(u[:, 1], u[:, 0])
    cols = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            y = sph_harm_y(l, abs(m), th, ph)
            if m < 0:
                cols.append(np.sqrt(2.0) * y.imag)
            elif m == 0:
                cols.append(y.real)
            else:
                cols.append(np.sqrt(2.0) * y.real)
    return np.stack(cols, axis=1)


def self_correction(n_theta: int, n_phi: int, a: float = 1.0, n_polar=None, n_azim=None) -> np.ndarray:
    """Cached wrapper of _self_correction (a fresh copy per call)."""
    return _self_correction(int(n_theta), int(n_phi), float(a), n_polar, n_azim).copy()


@functools.lru_cache(maxsize=8)
def _self_correction(n_theta: int, n_phi: int, a: float = 1.0, n_polar=None, n_azim=None) -> np.ndarray:
    """Accurate minus product-rule self-interaction block of one sphere template [3ns, 3ns].

    The exact self part of (K phi)_p is the integral over the sphere of
    T(x_p - y, n(y)) (phi(y) - phi_p).  Around each node p it is taken on a polar
    grid with its pole at x_p: Gauss-Legendre in the polar angle on (0, pi) and the
    uniform rule in the azimuth.  On a sphere (x - y).n(y) = -|x - y|^2/(2a), so the
    kernel is O(1/|x - y|) and the area element a^2 sin(theta) removes the
    singularity.  phi(y) is the projection of the nodal values on the real spherical
    harmonics of degree <= n_theta - 1 (coefficients by the template's own
    quadrature).  The product-rule block is the one stresslet_matrix takes for a
    single sphere.  (A refinement of the stand-in operator above, not the paper's.)
    """
    xi, nrm, w = sphere_template(n_theta, n_phi, a)
    ns = xi.shape[0]
    L = n_theta - 1
    n_polar = n_polar or 3 * n_theta
    n_azim = n_azim or 6 * n_theta
    coef_of = (_real_harmonics(nrm, L) * (w / a ** 2)[:, None]).T          # nodal values -> coefficients
    tg, wg = np.polynomial.legendre.leggauss(n_polar)
    th = 0.5 * np.pi * (tg + 1.0)
    wth = 0.5 * np.pi * wg
    ph = 2.0 * np.pi * np.arange(n_azim) / n_azim
    c = -3.0 / (4.0 * np.pi)
    S = np.zeros((3 * ns, 3 * ns))
    for p in range(ns):
        e = nrm[p]
        helper = np.array([1.0, 0.0, 0.0]) if abs(e[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        t1 = np.cross(e, helper)
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(e, t1)
        u = (np.cos(th)[:, None, None] * e
             + np.sin(th)[:, None, None] * (np.cos(ph)[None, :, None] * t1 + np.sin(ph)[None, :, None] * t2))
        u = u.reshape(-1, 3)
        W = (a * a * (np.sin(th) * wth)[:, None] * (2.0 * np.pi / n_azim) * np.ones(n_azim)[None, :]).reshape(-1)
        r = xi[p] - a * u
        r2 = np.einsum("ij,ij->i", r, r)
        rn = np.einsum("ij,ij->i", r, u)
        blocks = (c * W * rn / r2 ** 2.5)[:, None, None] * r[:, :, None] * r[:, None, :]
        interp = _real_harmonics(u, L) @ coef_of                            # [points, ns]
        S[3 * p:3 * p + 3, :] = np.einsum("kab,kq->aqb", blocks, interp).reshape(3, 3 * ns)
        S[3 * p:3 * p + 3, 3 * p:3 * p + 3] -= blocks.sum(axis=0)
    return S - stresslet_matrix(xi, nrm, w)


class DenseMobility:
    """Dense LU of (K + P) for one configuration; applies the mobility M."""

    def __init__(self, centers, n_theta, n_phi, a=1.0, mu=1.0, self_quadrature=False):
        self.centers = np.asarray(centers, dtype=np.float64)
        self.a, self.mu = a, mu
        self.x, self.n, self.w, self.body = surface_nodes(self.centers, n_theta, n_phi, a)
        self.K = stresslet_matrix(self.x, self.n, self.w)
        if self_quadrature:   # the accurate self-interaction on every body
            C = self_correction(n_theta, n_phi, a)
            b = C.shape[0]
            for i in range(self.centers.shape[0]):
                self.K[i * b:(i + 1) * b, i * b:(i + 1) * b] += C
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
