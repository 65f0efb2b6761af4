"""Python binding of the C ABI (include/lcp_gb300.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Host arrays are
NumPy FP64; ``*_dev`` functions take CUDA tensors (or raw device pointers) and
run on the context's stream.  No computation happens here: a missing or
failing library raises, there is no fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (LCP_BB_PGD, LCP_BI_PQN, LCP_ERR_CUDA, LCP_ERR_INVALID_ARG, LCP_ERR_NOT_CONVERGED,  # noqa: F401
                   LCP_ERR_NUMERICAL, LCP_ERR_OOM, LCP_ERR_REJECTED, LCP_ERR_TIMEOUT, LCP_DF64, LCP_FP64, LCP_HIGH,
                   LCP_LOW_BIE, LCP_LOW_RPY, LCP_MIXED, LCP_MONO_PQN, LCP_OK, LCP_WARM_FORCES, LCP_WARM_NO_INIT,
                   LCP_WARM_SLIP,
                   STATUS_NAMES)


class LcpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _lib():
    return _abi.load()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        out = out.reshape(shape)
    return out


def _devptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("device buffers must be contiguous CUDA float64 tensors")
    return t.data_ptr()


def _check(status: int, ctx=None, allow=(LCP_OK,)):
    if status not in allow:
        msg = _lib().lcp_last_error(ctx)
        raise LcpError(status, msg.decode() if msg else "")
    return status


def lcp_default_config(**overrides) -> _abi.lcp_config:
    cfg = _abi.lcp_config()
    _lib().lcp_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _contacts(contacts):
    if contacts is None:
        return None, 0
    nc = len(contacts)
    cont = (_abi.lcp_contact * max(nc, 1))()
    for l, (i, j, nrm, gap) in enumerate(contacts):
        cont[l].i, cont[l].j, cont[l].gap = int(i), int(j), float(gap)
        for d in range(3):
            cont[l].normal[d] = float(nrm[d])
    return cont, nc


def lcp_setup(cfg: _abi.lcp_config, centers, axes=None, contacts=None):
    """Returns the opaque context handle (an int)."""
    c = _f64(centers, (-1, 3))
    M = c.shape[0]
    a = None if axes is None else _f64(axes, (M, 3))
    cont, nc = _contacts(contacts)
    out = ctypes.c_void_p()
    st = _lib().lcp_setup(ctypes.byref(cfg), M, _dptr(c), None if a is None else _dptr(a), nc, cont,
                          ctypes.byref(out))
    _check(st, None)
    return out.value


def lcp_update(ctx, centers, axes=None, contacts=None) -> None:
    M, _, _ = lcp_sizes(ctx)
    c = _f64(centers, (M, 3))
    a = None if axes is None else _f64(axes, (M, 3))
    cont, nc = _contacts(contacts)
    _check(_lib().lcp_update(ctx, _dptr(c), None if a is None else _dptr(a), nc, cont), ctx)


def lcp_update_dev(ctx, centers, axes=None) -> None:
    _check(_lib().lcp_update_dev(ctx, _devptr(centers), _devptr(axes)), ctx)


def lcp_step(ctx, dt: float):
    """Advance the configuration by one time step; returns the new (centers, axes)."""
    M, _, _ = lcp_sizes(ctx)
    c = np.empty(3 * M)
    a = np.empty(3 * M)
    _check(_lib().lcp_step(ctx, float(dt), _dptr(c), _dptr(a)), ctx)
    return c.reshape(M, 3), a.reshape(M, 3)


def lcp_profile(ctx, enable: bool) -> None:
    _check(_lib().lcp_profile(ctx, int(enable)), ctx)


def lcp_launch_count(ctx) -> int:
    c = ctypes.c_ulonglong()
    _check(_lib().lcp_launch_count(ctx, ctypes.byref(c)), ctx)
    return c.value


def lcp_self_correction(n_theta: int, n_phi: int, radius: float = 1.0) -> np.ndarray:
    """The 3 ns x 3 ns self-interaction correction of one sphere template (host computation)."""
    n = 3 * n_theta * n_phi
    C = np.empty((n, n))
    _check(_lib().lcp_self_correction(int(n_theta), int(n_phi), float(radius), _dptr(C)))
    return C


def lcp_solve_counters(ctx, fidelity: int = 0):
    """(mobility solves, their GMRES iterations, projected starts) of one grid since set-up."""
    a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib().lcp_solve_counters(ctx, fidelity, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), ctx)
    return a.value, b.value, c.value


def lcp_profile_read(ctx, kind: int):
    """(launch count, total milliseconds) of kind 0 = FP32 pair sum, 1 = FP64 pair sum."""
    c, t = ctypes.c_int(), ctypes.c_double()
    _check(_lib().lcp_profile_read(ctx, int(kind), ctypes.byref(c), ctypes.byref(t)), ctx)
    return c.value, t.value


def lcp_destroy(ctx) -> None:
    if ctx:
        _lib().lcp_destroy(ctx)


def lcp_last_error(ctx) -> str:
    m = _lib().lcp_last_error(ctx)
    return m.decode() if m else ""


def lcp_sizes(ctx):
    M, N, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib().lcp_sizes(ctx, ctypes.byref(M), ctypes.byref(N), ctypes.byref(n)), ctx)
    return M.value, N.value, n.value


def lcp_get_contacts(ctx):
    """Returns (pairs [n,2] int, normals [n,3], gaps [n])."""
    _, _, n = lcp_sizes(ctx)
    buf = (_abi.lcp_contact * max(n, 1))()
    _check(_lib().lcp_get_contacts(ctx, buf), ctx)
    pairs = np.array([(buf[l].i, buf[l].j) for l in range(n)], dtype=np.int64).reshape(-1, 2)
    normals = np.array([list(buf[l].normal) for l in range(n)]).reshape(-1, 3)
    gaps = np.array([buf[l].gap for l in range(n)])
    return pairs, normals, gaps


def lcp_get_b(ctx) -> np.ndarray:
    _, _, n = lcp_sizes(ctx)
    out = np.empty(n)
    _check(_lib().lcp_get_b(ctx, _dptr(out)), ctx)
    return out


def lcp_get_unc(ctx) -> np.ndarray:
    M, _, _ = lcp_sizes(ctx)
    out = np.empty(6 * M)
    _check(_lib().lcp_get_unc(ctx, _dptr(out)), ctx)
    return out


def mobility_apply(ctx, FT, include_slip: bool = False, fidelity: int = LCP_HIGH) -> np.ndarray:
    M, _, _ = lcp_sizes(ctx)
    f = _f64(FT, (6 * M,))
    out = np.empty(6 * M)
    _check(_lib().mobility_apply(ctx, _dptr(f), _dptr(out), int(include_slip), int(fidelity)), ctx)
    return out


def mobility_apply_dev(ctx, FT, UO, include_slip: bool = False, fidelity: int = LCP_HIGH) -> None:
    _check(_lib().mobility_apply_dev(ctx, _devptr(FT), _devptr(UO), int(include_slip), int(fidelity)), ctx)


def lcp_apply_A(ctx, x, fidelity: int = LCP_HIGH) -> np.ndarray:
    _, _, n = lcp_sizes(ctx)
    xv = _f64(x, (n,))
    out = np.empty(n)
    _check(_lib().lcp_apply_A(ctx, _dptr(xv), _dptr(out), int(fidelity)), ctx)
    return out


def lcp_solve(ctx, method: int, tol: float, x0=None, allow_not_converged: bool = False):
    """Returns (x, stats dict, status)."""
    _, _, n = lcp_sizes(ctx)
    x = np.empty(n)
    st = _abi.lcp_stats()
    x0v = None if x0 is None else _f64(x0, (n,))
    status = _lib().lcp_solve(ctx, int(method), float(tol), None if x0v is None else _dptr(x0v), _dptr(x),
                              ctypes.byref(st))
    allow = (LCP_OK, LCP_ERR_NOT_CONVERGED) if allow_not_converged else (LCP_OK,)
    _check(status, ctx, allow)
    return x, st.as_dict(), status


def lcp_solve_dev(ctx, method: int, tol: float, x0, x, allow_not_converged: bool = False):
    """x0 (or None) and x are CUDA float64 tensors [n]; returns (stats dict, status)."""
    st = _abi.lcp_stats()
    status = _lib().lcp_solve_dev(ctx, int(method), float(tol), _devptr(x0), _devptr(x), ctypes.byref(st))
    allow = (LCP_OK, LCP_ERR_NOT_CONVERGED) if allow_not_converged else (LCP_OK,)
    _check(status, ctx, allow)
    return st.as_dict(), status


def lcp_stokes_apply_dev(ctx, phi, out, precision: int = LCP_FP64) -> None:
    _check(_lib().lcp_stokes_apply_dev(ctx, _devptr(phi), _devptr(out), int(precision)), ctx)


def lcp_stokes_rhs_dev(ctx, FT, include_slip: bool, rhs) -> None:
    _check(_lib().lcp_stokes_rhs_dev(ctx, _devptr(FT), int(include_slip), _devptr(rhs)), ctx)


def lcp_rigid_velocity_dev(ctx, phi, UO) -> None:
    _check(_lib().lcp_rigid_velocity_dev(ctx, _devptr(phi), _devptr(UO)), ctx)


def lcp_stokes_apply_noalloc(n_bodies, n_theta, n_phi, radius, centers, phi, out,
                             precision: int = LCP_FP64, stream=None) -> None:
    """Allocation-free (K + P) phi (no context); centers, phi, out are CUDA float64 tensors."""
    _check(_lib().lcp_stokes_apply_noalloc(int(n_bodies), int(n_theta), int(n_phi), float(radius),
                                           _devptr(centers), _devptr(phi), _devptr(out), int(precision),
                                           stream), None)


def lcp_footprint(ctx) -> int:
    b = ctypes.c_size_t()
    _check(_lib().lcp_footprint(ctx, ctypes.byref(b)), ctx)
    return b.value


def lcp_footprint_estimate(cfg, n_bodies: int, n_contacts: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib().lcp_footprint_estimate(ctypes.byref(cfg), int(n_bodies), int(n_contacts), ctypes.byref(b)), None)
    return b.value


def lcp_kernel_variant(ctx) -> str:
    return _lib().lcp_kernel_variant(ctx).decode()


def lcp_select_kernel_variant(ctx, name: str) -> None:
    """Forces the FP32 pair-kernel variant (a name lcp_kernel_variant can return)."""
    _check(_lib().lcp_select_kernel_variant(ctx, name.encode()), ctx)


def lcp_batch_solve(ctxs, method: int, tol: float, xs=None, workers: int = 8):
    """Solve contexts concurrently; xs: optional CUDA tensors.  Returns (statuses, stats dicts)."""
    n = len(ctxs)
    carr = (ctypes.c_void_p * max(n, 1))(*ctxs)
    xarr = None
    if xs is not None:
        xarr = (ctypes.c_void_p * max(n, 1))(*[_devptr(x) for x in xs])
    st = (_abi.lcp_stats * max(n, 1))()
    sts = (ctypes.c_int * max(n, 1))()
    _lib().lcp_batch_solve(carr, n, int(method), float(tol), xarr, st, sts, int(workers))
    return [sts[i] for i in range(n)], [st[i].as_dict() for i in range(n)]


def lcp_server_create(workers: int, hbm_budget_bytes: int):
    out = ctypes.c_void_p()
    _check(_lib().lcp_server_create(int(workers), int(hbm_budget_bytes), ctypes.byref(out)), None)
    return out.value


def lcp_server_destroy(srv) -> None:
    if srv:
        _lib().lcp_server_destroy(srv)


def lcp_server_admit(srv, ctx) -> int:
    """Returns LCP_OK or LCP_ERR_REJECTED (memory budget)."""
    return _lib().lcp_server_admit(srv, ctx)


def lcp_server_release(srv, ctx) -> None:
    _check(_lib().lcp_server_release(srv, ctx), None)


def lcp_server_submit(srv, ctx, method: int, tol: float) -> int:
    t = ctypes.c_uint64()
    _check(_lib().lcp_server_submit(srv, ctx, int(method), float(tol), ctypes.byref(t)), None)
    return t.value


def lcp_server_poll(srv, ticket: int, n: int, timeout_us: int):
    """Returns (status, x, stats dict); status LCP_ERR_TIMEOUT if not ready."""
    x = np.empty(max(n, 1))
    st = _abi.lcp_stats()
    status = _lib().lcp_server_poll(srv, ctypes.c_uint64(ticket), _dptr(x), max(n, 1), ctypes.byref(st),
                                    int(timeout_us))
    return status, x[:n], st.as_dict()


def lcp_server_open(srv, cfg: _abi.lcp_config, centers, axes=None) -> int:
    """Registers a server-owned simulation; returns its id."""
    c = _f64(centers).reshape(-1, 3)
    a = None if axes is None else _f64(axes, c.shape)
    sim = ctypes.c_uint64()
    _check(_lib().lcp_server_open(srv, ctypes.byref(cfg), c.shape[0], _dptr(c), None if a is None else _dptr(a),
                                  ctypes.byref(sim)), None)
    return sim.value


def lcp_server_request(srv, sim: int, method: int, tol: float, step_dt: float = 0.0) -> int:
    """Queues (or holds until the budget admits it) a solve of the simulation; returns the ticket."""
    t = ctypes.c_uint64()
    _check(_lib().lcp_server_request(srv, ctypes.c_uint64(sim), int(method), float(tol), float(step_dt),
                                     ctypes.byref(t)), None)
    return t.value


def lcp_server_close(srv, sim: int) -> None:
    _check(_lib().lcp_server_close(srv, ctypes.c_uint64(sim)), None)


def lcp_server_stats(srv):
    b, q, f = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    _check(_lib().lcp_server_stats(srv, ctypes.byref(b), ctypes.byref(q), ctypes.byref(f)), None)
    return b.value, q.value, f.value


def config_for(instance, precision: int = LCP_FP64, **overrides) -> _abi.lcp_config:
    """Config of a workload instance (grid, radii, dt, delta) with overrides."""
    cfg = lcp_default_config(n_theta=instance.n_theta, n_phi=instance.n_phi, radius=instance.radius,
                             contact_radius=instance.contact_radius, viscosity=instance.viscosity,
                             dt=instance.dt, delta=instance.delta, precision=precision)
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg
