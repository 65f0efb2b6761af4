"""Sphere surface quadrature (test infrastructure; see ``oracle/__init__``).

The paper discretises each particle surface with order-p spherical-harmonic
bases (Sec. 5.1, "Coarseness of discretization").  The stand-in operator uses
the matching product rule: Gauss-Legendre in t = cos(theta) (n_theta nodes)
times the uniform rule in the azimuth (n_phi nodes).  Node order inside a
sphere is polar-major: q = j * n_phi + k with t_j ascending and
phi_k = 2 pi k / n_phi.
"""
import numpy as np


def sphere_template(n_theta: int, n_phi: int, a: float = 1.0):
    """Return (xi [n,3], normal [n,3], weight [n]) for one sphere of radius a.

    xi is the node position relative to the sphere centre, the normal points
    out of the particle into the fluid, and the weights integrate functions
    on the sphere surface (sum = 4 pi a^2).
    """
    t, wt = np.polynomial.legendre.leggauss(n_theta)
    phis = 2.0 * np.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - t * t)
    nrm = np.empty((n_theta * n_phi, 3))
    w = np.empty(n_theta * n_phi)
    for j in range(n_theta):
        for k in range(n_phi):
            q = j * n_phi + k
            nrm[q] = (st[j] * np.cos(phis[k]), st[j] * np.sin(phis[k]), t[j])
            w[q] = a * a * wt[j] * 2.0 * np.pi / n_phi
    return a * nrm, nrm, w


def surface_nodes(centers: np.ndarray, n_theta: int, n_phi: int, a: float = 1.0):
    """All nodes, body-major: node (i, q) has global index i * n_s + q."""
    xi, nrm, w = sphere_template(n_theta, n_phi, a)
    M = centers.shape[0]
    x = (centers[:, None, :] + xi[None, :, :]).reshape(M * xi.shape[0], 3)
    n = np.tile(nrm, (M, 1))
    ww = np.tile(w, M)
    body = np.repeat(np.arange(M), xi.shape[0])
    return x, n, ww, body
