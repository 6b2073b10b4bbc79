"""CPU FP64 oracle for the demag-extrapolated explicit LLG integrator
(arXiv 2107.06729).  TEST INFRASTRUCTURE ONLY: only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  It shares no code with the CUDA
library; see ``mmx_oracle.c`` for the definitions it follows and the readings
it takes where the paper is silent.

Arrays are numpy float64, magnetisation as unit vectors m = M/Ms in SoA
layout ``[3, nz, ny, nx]``; fields in A/m.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force, the
published prism demag factor and order conditions).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

METHODS = {"RK4": 0, "HEUN12": 1, "RK23": 2, "RKF45": 3, "RKCK45": 4, "RKDP54": 5, "RKF56": 6, "ABM2": 7}
MU0 = 4e-7 * np.pi


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("Ms", ctypes.c_double), ("A", ctypes.c_double), ("K", ctypes.c_double),
                ("ku", ctypes.c_double * 3), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("H0", ctypes.c_double * 3), ("pulse", ctypes.c_double * 3),
                ("t_on", ctypes.c_double), ("t_off", ctypes.c_double)]


class _Integrator(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("extrap_order", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("h", ctypes.c_double), ("tol", ctypes.c_double), ("hmin", ctypes.c_double),
                ("hmax", ctypes.c_double), ("cmin", ctypes.c_double), ("cmax", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double),
                ("accepted", ctypes.c_long), ("rejected", ctypes.c_long),
                ("exact_evals", ctypes.c_long), ("extrap_evals", ctypes.c_long),
                ("forced", ctypes.c_long), ("last_err", ctypes.c_double)]


class Tableau(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("order", ctypes.c_int), ("adaptive", ctypes.c_int),
                ("fsal", ctypes.c_int), ("a", ctypes.c_double * 8), ("b", (ctypes.c_double * 8) * 8),
                ("c", ctypes.c_double * 8), ("chat", ctypes.c_double * 8)]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.om_newell_entry.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_D]
        L.om_newell_octant.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_D]
        L.om_demag_direct.argtypes = [ctypes.c_int] * 3 + [_D, ctypes.c_double, _D, _D]
        L.om_demag_fft.argtypes = [ctypes.c_int] * 3 + [_D, ctypes.c_double, _D, _D]
        L.om_applied_field.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, _D]
        L.om_exchange_anisotropy.argtypes = [ctypes.POINTER(_Problem), _D, _D]
        L.om_llg_rhs.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        L.om_get_tableau.argtypes = [ctypes.c_int, ctypes.POINTER(Tableau)]
        L.om_lagrange_weights.argtypes = [ctypes.c_int, _D, ctypes.c_double, _D]
        L.om_controller_factor.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double]
        L.om_controller_factor.restype = ctypes.c_double
        L.om_epsilon.argtypes = [ctypes.c_long, _D, _D]
        L.om_epsilon.restype = ctypes.c_double
        L.om_sim_create.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Integrator), _D, _D]
        L.om_sim_create.restype = ctypes.c_void_p
        L.om_sim_destroy.argtypes = [ctypes.c_void_p]
        L.om_sim_get_m.argtypes = [ctypes.c_void_p, _D]
        L.om_sim_set_time.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.om_sim_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Stats)]
        L.om_sim_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_long]
        L.om_sim_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def newell_entry(X, Y, Z, dx, dy, dz):
    """Newell tensor {Nxx, Nyy, Nzz, Nxy, Nxz, Nyz} at cell offset (X, Y, Z)."""
    out = np.zeros(6)
    lib().om_newell_entry(int(X), int(Y), int(Z), dx, dy, dz, _p(out))
    return out


def newell_octant(nx, ny, nz, dx, dy, dz):
    """Tensor at all offsets 0 <= X < nx, ...; shape [6, nz, ny, nx]."""
    out = np.zeros((6, nz, ny, nx))
    lib().om_newell_octant(nx, ny, nz, dx, dy, dz, _p(out))
    return out


def demag_direct(N6, Ms, m):
    """Eq. 2 as the literal O(N^2) sum; returns H [3, nz, ny, nx] in A/m."""
    m = _f64(m)
    N6 = _f64(N6)
    nz, ny, nx = m.shape[1:]
    H = np.zeros_like(m)
    lib().om_demag_direct(nx, ny, nz, _p(N6), Ms, _p(m), _p(H))
    return H


def demag_fft(N6, Ms, m):
    """Eq. 2 through a zero-padded textbook radix-2 FFT convolution."""
    m = _f64(m)
    N6 = _f64(N6)
    nz, ny, nx = m.shape[1:]
    H = np.zeros_like(m)
    lib().om_demag_fft(nx, ny, nz, _p(N6), Ms, _p(m), _p(H))
    return H


def _problem(mesh, material, field):
    P = _Problem()
    P.nx, P.ny, P.nz = mesh["n"]
    P.dx, P.dy, P.dz = mesh["d"]
    P.Ms = material["Ms"]
    P.A = material.get("A", 0.0)
    P.K = material.get("K", 0.0)
    for i, v in enumerate(material.get("ku", (1.0, 0.0, 0.0))):
        P.ku[i] = v
    P.alpha = material["alpha"]
    P.gamma = material["gamma"]
    for i in range(3):
        P.H0[i] = field.get("H0", (0, 0, 0))[i]
        P.pulse[i] = field.get("pulse", (0, 0, 0))[i]
    P.t_on = field.get("t_on", 0.0)
    P.t_off = field.get("t_off", 0.0)
    return P


def applied_field(mesh, material, field, t):
    out = np.zeros(3)
    P = _problem(mesh, material, field)
    lib().om_applied_field(ctypes.byref(P), t, _p(out))
    return out


def exchange_anisotropy(mesh, material, m):
    m = _f64(m)
    H = np.zeros_like(m)
    P = _problem(mesh, material, {})
    lib().om_exchange_anisotropy(ctypes.byref(P), _p(m), _p(H))
    return H


def llg_rhs(gamma, alpha, m, H):
    m = _f64(m)
    H = _f64(H)
    F = np.zeros_like(m)
    n = m.size // 3
    lib().om_llg_rhs(n, gamma, alpha, _p(m), _p(H), _p(F))
    return F


def tableau(method):
    T = Tableau()
    if lib().om_get_tableau(METHODS[method], ctypes.byref(T)) != 0:
        raise ValueError(method)
    s = T.s
    return {"s": s, "order": T.order, "adaptive": bool(T.adaptive), "fsal": bool(T.fsal),
            "a": np.array(T.a[:s]), "b": np.array([[T.b[i][j] for j in range(s)] for i in range(s)]),
            "c": np.array(T.c[:s]), "chat": np.array(T.chat[:s])}


def lagrange_weights(tau_nodes, tau):
    tau_nodes = _f64(tau_nodes)
    w = np.zeros(len(tau_nodes))
    lib().om_lagrange_weights(len(tau_nodes) - 1, _p(tau_nodes), tau, _p(w))
    return w


def controller_factor(e, e_max, order, cmin=0.01, cmax=2.0):
    return lib().om_controller_factor(e, e_max, order, cmin, cmax)


def epsilon(m, mref):
    """Eq. 7 over cells (epsilon_space): m, mref arrays [3, ...]."""
    m = _f64(m)
    mref = _f64(mref)
    return lib().om_epsilon(m.size // 3, _p(m), _p(mref))


def epsilon_time(mbar, mbar_ref):
    """Eq. 7 with its N points taken as time samples of the mean
    magnetisation (the reading for the paper's error-versus-time curves,
    Sec. III): mbar, mbar_ref arrays [3, S] of <m> at the same S times."""
    mbar = _f64(mbar).reshape(3, -1)
    mbar_ref = _f64(mbar_ref).reshape(3, -1)
    if mbar.shape != mbar_ref.shape:
        raise ValueError("sample counts differ")
    return lib().om_epsilon(mbar.shape[1], _p(mbar), _p(mbar_ref))


class Simulation:
    """Oracle integrator (Eq. 3-6) over a whole mesh.

    integrator: dict(method, extrap_order (-1 = full demag), adaptive, h, tol,
    hmin, hmax, cmin, cmax)."""

    def __init__(self, mesh, material, field, integrator, m0, N6=None):
        nx, ny, nz = mesh["n"]
        if N6 is None:
            N6 = newell_octant(nx, ny, nz, *mesh["d"])
        self.N6 = _f64(N6)
        self._P = _problem(mesh, material, field)
        I = _Integrator()
        I.method = METHODS[integrator["method"]]
        I.extrap_order = integrator.get("extrap_order", -1)
        I.adaptive = int(integrator.get("adaptive", False))
        I.h = integrator["h"]
        I.tol = integrator.get("tol", 1e-5)
        I.hmin = integrator.get("hmin", 1e-15)
        I.hmax = integrator.get("hmax", 3e-12)
        I.cmin = integrator.get("cmin", 0.01)
        I.cmax = integrator.get("cmax", 2.0)
        self._I = I
        self.shape = (3, nz, ny, nx)
        m0 = _f64(m0).reshape(self.shape)
        self._h = lib().om_sim_create(ctypes.byref(self._P), ctypes.byref(I), _p(self.N6), _p(m0))
        if not self._h:
            raise ValueError("oracle: bad integrator settings")

    def run(self, t_end, max_attempts=0):
        rc = lib().om_sim_run(self._h, float(t_end), int(max_attempts))
        if rc < 0:
            raise FloatingPointError("oracle: non-finite error estimate")
        return rc

    def m(self):
        out = np.zeros(self.shape)
        lib().om_sim_get_m(self._h, _p(out))
        return out

    def stats(self):
        s = _Stats()
        lib().om_sim_get_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def close(self):
        if self._h:
            lib().om_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
