"""Mono-PQN and Bi-PQN in FP64, in the paper's order (test infrastructure).

* Algorithm 1 (Mono-PQN): proximal quasi-Newton with H^(0) = I, the weighted
  prox of Eq. (prox-pqn) and the over-relaxation of Algorithm 2.
* Algorithm 2: the exact minimiser of f(x + eta p) over the feasible eta.
* Proposition 1 / Appendix A.2 (Algorithm 3): the weighted prox under
  B = D + U U^T - V V^T by semi-smooth Newton on the 2r-dimensional root.
* Sec. 4 / Appendix D.1: BFGS stored unrolled, u = y / sqrt(y^T s),
  v = B s / sqrt(s^T B s), so B_{k+1} = B_k + u u^T - v v^T; H g by the
  two-loop recursion over the same pairs with H_0 = D^{-1}.
* Algorithm 4 (Bi-PQN) with the low-fidelity initialisation (Sec. 5.2), the
  subproblem of Eq. (pqnSubproblem), the cached A_hat s of Appendix D.2 and
  the secant carry-over of Sec. 5.2.

Readings taken where the paper is silent or garbled (listed in the design
notes): x_tilde = x - H g with tau = 1 (Alg. 1 vs Eq. prox-pqn and Fig. 2);
stop when ||min(x, g)||_2 <= tol (Sec. 6); the root function of Prop. 1 is
[alpha; alpha_tilde] + L(alpha, alpha_tilde), as its Jacobian (+I) shows;
the carried secant matrix is Y_hat + (u u^T - v v^T) S_hat, which makes
B^(k+1) S = Y hold exactly; a direction with p^T g >= 0 resets the memory and
falls back to the projected-gradient direction.

Memory: Sec. 6 keeps every secant pair (full memory), which is the default
here (r_max=None).  A finite r_max models a storage bound: once more than
r_max pairs are held, the oldest quarter is dropped at once and the unrolled
factors are rebuilt from the pairs that remain (the GPU library's limit is 32
pairs; runs that stay below it do not depend on the rule).
"""
from __future__ import annotations

import dataclasses

import numpy as np


# ----------------------------------------------------------------- Algorithm 2
def step_size(x, p, g, Ap):
    """Optimal over-relaxation eta* = min(eta', min_{p_l < 0} -x_l / p_l).

    Returns (eta, blocking index or -1).
    """
    pAp = float(p @ Ap)
    eta = -float(p @ g) / pAp
    blocking = -1
    for l in range(x.shape[0]):
        if p[l] < 0.0:
            eh = -x[l] / p[l]
            if eh < eta:
                eta, blocking = eh, l
    return eta, blocking


# --------------------------------------------------- quasi-Newton model (BFGS)
class QNModel:
    """B = diag(d) + U U^T - V V^T built from secant pairs (s, y) in order."""

    def __init__(self, d, r_max=None):
        self.d = np.asarray(d, dtype=np.float64)
        self.r_max = r_max
        self.S, self.Y, self.B0S = [], [], []
        self.U, self.V = [], []

    @property
    def r(self):
        return len(self.U)

    def _Umat(self):
        n = self.d.shape[0]
        return (np.array(self.U).T if self.U else np.zeros((n, 0)),
                np.array(self.V).T if self.V else np.zeros((n, 0)))

    def low_rank(self, z):
        U, V = self._Umat()
        return U @ (U.T @ z) - V @ (V.T @ z)

    def B(self, z):
        return self.d * z + self.low_rank(z)

    def H(self, g):
        """Two-loop recursion (Nocedal-Wright Alg. 7.4) with H_0 = diag(1/d)."""
        q = np.array(g, dtype=np.float64)
        alphas = []
        for s, y in zip(reversed(self.S), reversed(self.Y)):
            rho = 1.0 / float(y @ s)
            a = rho * float(s @ q)
            q -= a * y
            alphas.append(a)
        q = q / self.d
        for (s, y), a in zip(zip(self.S, self.Y), reversed(alphas)):
            rho = 1.0 / float(y @ s)
            beta = rho * float(y @ q)
            q += s * (a - beta)
        return q

    def _append_uv(self, s, y, b0s):
        Bs = b0s + self.low_rank(s)
        ys = float(y @ s)
        sBs = float(s @ Bs)
        self.U.append(y / np.sqrt(ys))
        self.V.append(Bs / np.sqrt(sBs))

    def accepts(self, s, y, b0s):
        ys = float(y @ s)
        sBs = float(s @ (b0s + self.low_rank(s)))
        return ys > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y) and sBs > 0.0

    def update(self, s, y, b0s=None):
        """BFGS update with the pair (s, y); b0s = B_0 s (d * s by default)."""
        s = np.asarray(s, float)
        y = np.asarray(y, float)
        b0s = self.d * s if b0s is None else np.asarray(b0s, float)
        if not self.accepts(s, y, b0s):
            return False
        self.S.append(s)
        self.Y.append(y)
        self.B0S.append(b0s)
        if self.r_max is not None and len(self.S) > self.r_max:
            # memory full: the oldest quarter of the pairs is dropped at once
            drop = max(1, self.r_max // 4)
            del self.S[:drop], self.Y[:drop], self.B0S[:drop]
            self.U, self.V = [], []
            for s_, y_, b_ in zip(self.S, self.Y, self.B0S):
                self._append_uv(s_, y_, b_)
        else:
            self._append_uv(s, y, b0s)
        return True

    def reset(self):
        self.S, self.Y, self.B0S, self.U, self.V = [], [], [], [], []


# ------------------------------------------------ Proposition 1 / Algorithm 3
def prox_ssn(d, U, V, xt, jmax=50, tol=1e-13):
    """prox^B_{x>=0}(xt) for B = diag(d) + U U^T - V V^T.

    Root of G(a, at) = [a + U^T(xt + C^-1 V at - z); at + V^T(xt - z)],
    z = (xt + C^-1 V at - D^-1 U a)_+, C = D + U U^T, by semi-smooth Newton
    with the generalised Jacobian of Appendix A.2 and backtracking on ||G||.
    Returns (z, newton_iterations, converged).
    """
    n = xt.shape[0]
    r = U.shape[1]
    if r == 0:
        return np.maximum(xt, 0.0), 0, True
    DU = U / d[:, None]
    small = np.eye(r) + U.T @ DU
    CV = V / d[:, None] - DU @ np.linalg.solve(small, DU.T @ V)

    def resid(a, at):
        y = xt + CV @ at - DU @ a
        z = np.maximum(y, 0.0)
        G = np.concatenate([a + U.T @ (xt + CV @ at - z), at + V.T @ (xt - z)])
        return G, y, z

    a = np.zeros(r)
    at = np.zeros(r)
    G, y, z = resid(a, at)
    scale = 1.0 + np.linalg.norm(xt)
    for j in range(jmax):
        gn = np.linalg.norm(G)
        if gn <= tol * scale:
            return z, j, True
        lam = (y > 0.0).astype(np.float64)
        J = np.block([[U.T @ (lam[:, None] * DU), U.T @ ((1.0 - lam)[:, None] * CV)],
                      [V.T @ (lam[:, None] * DU), -V.T @ (lam[:, None] * CV)]]) + np.eye(2 * r)
        delta = np.linalg.solve(J, G)
        t = 1.0
        for _ in range(30):
            a1, at1 = a - t * delta[:r], at - t * delta[r:]
            G1, y1, z1 = resid(a1, at1)
            if np.linalg.norm(G1) <= (1.0 - 1e-4 * t) * gn or t < 1e-8:
                break
            t *= 0.5
        a, at, G, y, z = a1, at1, G1, y1, z1
    return z, jmax, bool(np.linalg.norm(G) <= 1e-9 * scale)


def prox_dense(Bmat, xt, sweeps=100000, tol=1e-14):
    """Fallback: projected Gauss-Seidel on min_{z>=0} 1/2 (z - xt)^T B (z - xt)."""
    z = np.maximum(xt, 0.0)
    c = -Bmat @ xt
    for _ in range(sweeps):
        for l in range(z.shape[0]):
            z[l] = max(0.0, z[l] - (Bmat[l] @ z + c[l]) / Bmat[l, l])
        g = Bmat @ z + c
        if np.linalg.norm(np.minimum(z, g), np.inf) <= tol * (1 + np.abs(xt).max()):
            break
    return z


def weighted_prox(model: QNModel, xt):
    U, V = model._Umat()
    z, it, ok = prox_ssn(model.d, U, V, xt)
    if not ok:
        Bmat = np.diag(model.d) + U @ U.T - V @ V.T
        z = prox_dense(Bmat, xt)
    return z, it, ok


# -------------------------------------------------------------- Algorithm 1
@dataclasses.dataclass
class PQNResult:
    x: np.ndarray
    g: np.ndarray
    iterations: int
    mvps: int
    kkt: float
    converged: bool
    model: QNModel
    history: list
    extra: np.ndarray | None = None
    resets: int = 0
    prox_fallbacks: int = 0


def mono_pqn(mvp, b, x0, tol=1e-8, kmax=100, d=None, pairs=(), r_max=None,
             g0=None, extra_mvp=None, scale0=False, tol_rel=0.0):
    """Algorithm 1 (Mono-PQN).

    mvp(v) returns A[v].  With g0 given the initial gradient is taken as is
    (no MVP).  pairs = [(s, y), ...] seeds the quasi-Newton memory.  If
    extra_mvp is given, mvp(v) returns (A[v], E[v]) and E[x - x0] is
    accumulated with the same MVP reuse as the gradient (Appendix D.2).
    Stops at ||min(x, g)|| <= max(tol, tol_rel * ||min(x0, g0)||).
    """
    b = np.asarray(b, float)
    n = b.shape[0]
    x = np.maximum(np.asarray(x0, float), 0.0)
    model = QNModel(np.ones(n) if d is None else d, r_max)
    for s, y in pairs:
        model.update(s, y)
    mvps = 0
    extra = np.zeros(n) if extra_mvp else None
    if g0 is None:
        out = mvp(x)
        mvps += 1
        g = (out[0] if extra_mvp else out) + b
    else:
        g = np.array(g0, float)
    hist = []
    resets = fallbacks = 0
    for k in range(kmax):
        kkt = float(np.linalg.norm(np.minimum(x, g)))
        hist.append(kkt)
        if k == 0:
            tol = max(tol, tol_rel * kkt)
        if kkt <= tol:
            return PQNResult(x, g, k, mvps, kkt, True, model, hist, extra, resets, fallbacks)
        xt = x - model.H(g)
        xh, _, ok = weighted_prox(model, xt)
        fallbacks += 0 if ok else 1
        p = xh - x
        if float(p @ g) >= 0.0:
            model.reset()
            resets += 1
            p = np.maximum(x - g, 0.0) - x
        if not np.any(p):
            return PQNResult(x, g, k, mvps, kkt, kkt <= tol, model, hist, extra, resets, fallbacks)
        out = mvp(p)
        mvps += 1
        Ap = out[0] if extra_mvp else out
        eta, blk = step_size(x, p, g, Ap)
        x = np.maximum(x + eta * p, 0.0)
        if blk >= 0:
            x[blk] = 0.0
        g = g + eta * Ap
        if extra_mvp:
            extra = extra + eta * out[1]
        if scale0 and model.r == 0 and not getattr(model, "scaled", False):
            sv, yv = eta * p, eta * Ap
            model.d = np.full(n, float(yv @ sv) / float(sv @ sv))
            model.scaled = True
        model.update(eta * p, eta * Ap)
    kkt = float(np.linalg.norm(np.minimum(x, g)))
    hist.append(kkt)
    return PQNResult(x, g, kmax, mvps, kkt, kkt <= tol, model, hist, extra, resets, fallbacks)


# -------------------------------------------------------------- Algorithm 4
@dataclasses.dataclass
class BiPQNResult:
    x: np.ndarray
    g: np.ndarray
    outer_iterations: int
    hi_mvps: int
    lo_mvps: int
    kkt: float
    converged: bool
    history: list
    resets: int = 0
    prox_fallbacks: int = 0


def bi_pqn(mvp_hi, mvp_lo, b, x_init, tol=1e-8, kmax=50, kmax_inner=100,
           forcing=1e-3, r_max=None, scale0=False, init_forcing=0.0):
    """Algorithm 4 (Bi-PQN) with B^(0) = A_hat.

    The subproblem min_{z>=0} 1/2 z^T B z + (g - B x)^T z (Eq. pqnSubproblem)
    is solved by Algorithm 1 started at x with gradient g, using only
    low-fidelity MVPs B[v] = A_hat[v] + U_h U_h^T v - V_h V_h^T v.  Its
    tolerance is max(0.1 tol, forcing * ||min(x, g)||).  The low-fidelity
    initialisation (Sec. 5.2, solved "approximately") stops at
    max(tol, init_forcing * its initial KKT error); init_forcing = 0 solves it
    to tol.
    """
    b = np.asarray(b, float)
    n = b.shape[0]
    # low-fidelity initialisation (Sec. 5.2)
    init = mono_pqn(mvp_lo, b, x_init, tol=tol, kmax=kmax_inner, r_max=r_max, scale0=scale0,
                    tol_rel=init_forcing)
    d_inner = init.model.d
    lo = init.mvps
    resets, fallbacks = init.resets, init.prox_fallbacks
    S_low = list(init.model.S)
    Y_low = list(init.model.Y)
    x = init.x
    Uh, Vh = [], []

    def lowrank(v):
        out = np.zeros(n)
        for u_, v_ in zip(Uh, Vh):
            out += u_ * (u_ @ v) - v_ * (v_ @ v)
        return out

    def sub_mvp(v):
        ahv = mvp_lo(v)
        return ahv + lowrank(v), ahv

    g = mvp_hi(x) + b
    hi = 1
    hist = []
    for k in range(kmax):
        kkt = float(np.linalg.norm(np.minimum(x, g)))
        hist.append(kkt)
        if kkt <= tol:
            return BiPQNResult(x, g, k, hi, lo, kkt, True, hist, resets, fallbacks)
        sub = mono_pqn(sub_mvp, b, x, tol=max(0.1 * tol, forcing * kkt), kmax=kmax_inner, d=d_inner,
                       pairs=list(zip(S_low, Y_low)), r_max=r_max, g0=g, extra_mvp=True)
        lo += sub.mvps
        resets += sub.resets
        fallbacks += sub.prox_fallbacks
        p = sub.x - x
        if float(p @ g) >= 0.0 or not np.any(p):
            p = np.maximum(x - g, 0.0) - x
            if not np.any(p):
                return BiPQNResult(x, g, k, hi, lo, kkt, kkt <= tol, hist, resets, fallbacks)
            ahp = mvp_lo(p)
            lo += 1
            a_lo_s_over_eta = ahp
        else:
            a_lo_s_over_eta = sub.extra
        Ap = mvp_hi(p)
        hi += 1
        eta, blk = step_size(x, p, g, Ap)
        x = np.maximum(x + eta * p, 0.0)
        if blk >= 0:
            x[blk] = 0.0
        g = g + eta * Ap
        s = eta * p
        y = eta * Ap
        Bs = eta * a_lo_s_over_eta + lowrank(s)          # Appendix D.2
        ys, sBs = float(y @ s), float(s @ Bs)
        S_hat, Y_hat = list(sub.model.S), list(sub.model.Y)
        if ys > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y) and sBs > 0.0:
            u = y / np.sqrt(ys)
            v = Bs / np.sqrt(sBs)
            Uh.append(u)
            Vh.append(v)
            Y_hat = [yy + u * (u @ ss) - v * (v @ ss) for ss, yy in zip(S_hat, Y_hat)]
        S_low, Y_low = S_hat, Y_hat
    kkt = float(np.linalg.norm(np.minimum(x, g)))
    hist.append(kkt)
    return BiPQNResult(x, g, kmax, hi, lo, kkt, kkt <= tol, hist, resets, fallbacks)
