"""ctypes wrapper around the plain FP64 C oracle (test infrastructure only).

Loads ``oracle/_build/liboracle.so`` (built by ``oracle/build.py``).  Arrays
follow the public state layout: ``u`` of shape ``(N + K, V)`` float64,
phase-major, x fastest.  Nothing here is imported by the product library.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None
_libs = {}
_openmp = False


def set_openmp(flag):
    """Use the OpenMP build of the oracle (RHS loop shared among the host
    cores; identical results) from now on: only for timing the all-core CPU
    baseline."""
    global _openmp, _lib
    _openmp = bool(flag)
    _lib = None

FEULER, SSP2, SSP104, RKL1, RKL2 = 0, 1, 2, 3, 4
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_ubp = C.POINTER(C.c_ubyte)


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("N", C.c_int), ("ptype", _ip), ("gamma", _dp),
                ("mob", _dp), ("W", C.c_double), ("Lover", _dp), ("K", C.c_int),
                ("k", C.c_double * 2), ("c0", C.c_double * 2), ("D", C.c_double * 2),
                ("bc_phi", C.c_int * 6), ("bc_c", C.c_int * 6), ("cdir", C.c_double * 6),
                ("simplex", C.c_int), ("n_slots", C.c_int)]


class _Tol(C.Structure):
    _fields_ = [("r_phi", C.c_double), ("a_phi", C.c_double), ("r_c", C.c_double), ("a_c", C.c_double)]


class _Ctrl(C.Structure):
    _fields_ = [("b", C.c_double), ("E1", C.c_double), ("E2", C.c_double),
                ("dt1", C.c_double), ("dt2", C.c_double), ("nhist", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("rhs_evals", C.c_long), ("accepted", C.c_long), ("rejected", C.c_long),
                ("dt_last", C.c_double), ("err_last", C.c_double), ("dt_next", C.c_double)]


_RHSFN = C.CFUNCTYPE(None, C.c_void_p, _dp, _dp)
_PROJFN = C.CFUNCTYPE(C.c_int, C.c_void_p, _dp, _ubp)


class _Sys(C.Structure):
    _fields_ = [("n", C.c_long), ("N", C.c_int), ("K", C.c_int), ("V", C.c_long),
                ("ctx", C.c_void_p), ("rhs", _RHSFN), ("proj", _PROJFN), ("keep_rhs", C.c_void_p)]


def lib():
    global _lib
    if _lib is None and _openmp in _libs:
        _lib = _libs[_openmp]
    if _lib is None:
        path = _build.build(openmp=_openmp)
        L = C.CDLL(path)
        L.or_rhs.argtypes = [C.POINTER(_Params), _dp, _dp, _ubp]
        L.or_project.argtypes = [C.POINTER(_Params), _dp, _ubp]
        L.or_project_cell_mobility.argtypes = [C.c_int, _dp, _dp]
        L.or_project_cell_mobility.restype = C.c_int
        L.or_evict_cell.argtypes = [C.c_int, C.c_int, _dp]
        L.or_evict_cell.restype = C.c_int
        L.or_keep_rhs_cell.argtypes = [C.c_int, C.c_int, _dp]
        L.or_keep_rhs_cell.restype = C.c_int
        L.or_dt_e.argtypes = [C.POINTER(_Params)]
        L.or_dt_e.restype = C.c_double
        L.or_reduce.argtypes = [C.POINTER(_Params), _dp, _dp, _dp, _ip]
        L.or_energy.argtypes = [C.POINTER(_Params), _dp]
        L.or_energy.restype = C.c_double
        L.or_coeffs.argtypes = [C.POINTER(_Params), _dp, _dp, _dp]
        L.or_sys_pde.argtypes = [C.POINTER(_Sys), C.POINTER(_Params)]
        L.or_sys_dahlquist.argtypes = [C.POINTER(_Sys), _dp]
        L.or_step.argtypes = [C.POINTER(_Sys), C.c_int, C.c_double, C.c_int, _dp, _dp, _dp, _dp]
        L.or_step.restype = C.c_long
        L.or_sts_stages.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_sts_stages.restype = C.c_int
        L.or_err_sts.argtypes = [C.POINTER(_Sys), C.POINTER(_Tol), C.c_double, _dp, _dp, _dp, _dp,
                                 C.POINTER(C.c_long)]
        L.or_err_sts.restype = C.c_double
        L.or_err_embedded.argtypes = [C.POINTER(_Sys), C.POINTER(_Tol), _dp, _dp, _dp,
                                      C.POINTER(C.c_long)]
        L.or_err_embedded.restype = C.c_double
        L.or_ssp104_embedded_weights.argtypes = [_dp]
        L.or_ctrl_init.argtypes = [C.POINTER(_Ctrl)]
        L.or_ctrl_update.argtypes = [C.POINTER(_Ctrl), C.c_double, C.c_double, C.c_int, _ip]
        L.or_ctrl_update.restype = C.c_double
        L.or_order.argtypes = [C.c_int]
        L.or_order.restype = C.c_int
        L.or_run.argtypes = [C.POINTER(_Params), C.c_int, C.c_double, C.POINTER(_Tol),
                             C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp,
                             C.POINTER(_Ctrl), C.POINTER(_Stats), C.c_int, _dp, _ip, _dp, _ip, _ip,
                             C.c_int, _dp, _ip, _ip]
        L.or_run.restype = C.c_int
        L.or_drive.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _dp, _dp,
                               _dp, C.POINTER(_Ctrl), _dp, C.c_int, _dp, _ip, _ip]
        L.or_drive.restype = C.c_int
        _libs[_openmp] = L
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


class Oracle:
    """Oracle bound to one Problem (see paper_2601_16522_gb300.inputs.Problem)."""

    def __init__(self, prob):
        self.prob = prob
        N = prob.n_phases
        self._ptype = np.ascontiguousarray(prob.phase_type, dtype=np.int32)
        self._gamma = np.ascontiguousarray(prob.gamma, dtype=np.float64).reshape(N * N)
        self._mob = np.ascontiguousarray(prob.mobility, dtype=np.float64).reshape(N * N)
        self._L = (None if prob.L_override is None else
                   np.ascontiguousarray(prob.L_override, dtype=np.float64).reshape(N * N))
        p = _Params()
        p.dim, p.nx, p.ny, p.nz = prob.dim, prob.nx, prob.ny, prob.nz
        p.dx = prob.dx
        p.N = N
        p.ptype = self._ptype.ctypes.data_as(_ip)
        p.gamma = _d(self._gamma)
        p.mob = _d(self._mob)
        p.W = prob.W
        p.Lover = _d(self._L) if self._L is not None else _dp()
        p.K = prob.has_conc
        for t in range(2):
            p.k[t], p.c0[t], p.D[t] = prob.k[t], prob.c0[t], prob.D[t]
        for f in range(6):
            p.bc_phi[f], p.bc_c[f], p.cdir[f] = prob.bc_phi[f], prob.bc_c[f], prob.c_dirichlet[f]
        p.simplex = int(getattr(prob, "simplex", 0))
        p.n_slots = int(getattr(prob, "n_slots", 0))
        self.p = p
        self.sys = _Sys()
        lib().or_sys_pde(C.byref(self.sys), C.byref(self.p))
        self.ctrl = _Ctrl()
        lib().or_ctrl_init(C.byref(self.ctrl))
        self.stats = _Stats()

    # -- model --------------------------------------------------------------
    def coeffs(self):
        N = self.prob.n_phases
        A, B, L = (np.zeros(N * N) for _ in range(3))
        lib().or_coeffs(C.byref(self.p), _d(A), _d(B), _d(L))
        return A.reshape(N, N), B.reshape(N, N), L.reshape(N, N)

    def _u(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (self.prob.nfields, self.prob.V), u.shape
        return u

    def rhs(self, u):
        u = self._u(u)
        r = np.zeros_like(u)
        nz = np.zeros(self.prob.V, np.uint8)
        lib().or_rhs(C.byref(self.p), _d(u), _d(r), nz.ctypes.data_as(_ubp))
        return r, nz

    def project(self, u):
        u = self._u(u).copy()
        acted = np.zeros(self.prob.V, np.uint8)
        st = lib().or_project(C.byref(self.p), _d(u), acted.ctypes.data_as(_ubp))
        return u, acted, st

    def dt_e(self):
        return lib().or_dt_e(C.byref(self.p))

    def energy(self, u):
        return lib().or_energy(C.byref(self.p), _d(self._u(u)))

    def reduce(self, u):
        u = self._u(u)
        mass = C.c_double()
        vol = np.zeros(self.prob.n_phases)
        alive = C.c_int()
        lib().or_reduce(C.byref(self.p), _d(u), C.byref(mass), _d(vol), C.byref(alive))
        return mass.value, vol, alive.value

    # -- one step with given dt and stages --------------------------------
    def step(self, integ, dt, s, u):
        """Returns (u_new, rn_effective, z_embedded or None, n_rhs)."""
        u = self._u(u)
        un = np.zeros_like(u)
        rn = np.zeros_like(u)
        z = np.zeros_like(u) if integ == SSP104 else None
        ev = lib().or_step(C.byref(self.sys), integ, dt, s, _d(u), _d(un), _d(rn),
                           _d(z) if z is not None else _dp())
        if ev < 0:
            raise RuntimeError("or_step failed (%d)" % ev)
        return un, rn, z, ev

    def err_sts(self, tol, dt, un, unew, rn, rn1):
        t = _Tol(*tol)
        nd = C.c_long()
        e = lib().or_err_sts(C.byref(self.sys), C.byref(t), dt, _d(self._u(un)), _d(self._u(unew)),
                             _d(self._u(rn)), _d(self._u(rn1)), C.byref(nd))
        return e, nd.value

    def err_embedded(self, tol, un, unew, z):
        t = _Tol(*tol)
        nd = C.c_long()
        e = lib().or_err_embedded(C.byref(self.sys), C.byref(t), _d(self._u(un)), _d(self._u(unew)),
                                  _d(self._u(z)), C.byref(nd))
        return e, nd.value

    def step_error(self, integ, dt, s, u, tol):
        """One step plus its local error norm (Sec. 3.3) -> (u_new, err, ndof)."""
        un, rn, z, _ = self.step(integ, dt, s, u)
        if integ in (RKL1, RKL2):
            rn1, _ = self.rhs(un)
            e, nd = self.err_sts(tol, dt, u, un, rn, rn1)
        elif integ == SSP104:
            e, nd = self.err_embedded(tol, u, un, z)
        else:
            e, nd = 0.0, 0
        return un, e, nd

    # -- run ----------------------------------------------------------------
    def run(self, integ, u, t0, t_end, tol=(1e-4, 1e-4, 1e-4, 1e-4), dt_mult=0.0, dt0=0.0,
            ssp_stages=5, max_stages=1001, trace_cap=0, replay=None):
        u = self._u(u).copy()
        t = C.c_double(t0)
        t_ = _Tol(*tol)
        cap = trace_cap
        tr_dt = np.zeros(max(cap, 1))
        tr_s = np.zeros(max(cap, 1), np.int32)
        tr_err = np.zeros(max(cap, 1))
        tr_acc = np.zeros(max(cap, 1), np.int32)
        tr_len = C.c_int()
        if replay is not None:
            rdt = np.ascontiguousarray(replay[0], np.float64)
            rs = np.ascontiguousarray(replay[1], np.int32)
            racc = np.ascontiguousarray(replay[2], np.int32)
            rn = len(rdt)
        else:
            rdt = np.zeros(1); rs = np.zeros(1, np.int32); racc = np.zeros(1, np.int32); rn = 0
        st = lib().or_run(C.byref(self.p), integ, t_end, C.byref(t_), dt_mult, dt0, ssp_stages,
                          max_stages, _d(u), C.byref(t), C.byref(self.ctrl), C.byref(self.stats),
                          cap, _d(tr_dt), tr_s.ctypes.data_as(_ip), _d(tr_err),
                          tr_acc.ctypes.data_as(_ip), C.byref(tr_len), rn, _d(rdt),
                          rs.ctypes.data_as(_ip), racc.ctypes.data_as(_ip))
        n = tr_len.value
        trace = dict(dt=tr_dt[:n].copy(), s=tr_s[:n].copy(), err=tr_err[:n].copy(), acc=tr_acc[:n].copy())
        return st, u, t.value, trace


# -- scalar helpers for the integrator pins --------------------------------

def dahlquist_step(integ, z, s=1, dt=1.0):
    """One step of u' = lam u from u = 1 with lam*dt = z (complex): returns R(z)."""
    lam = np.array([z.real / dt, z.imag / dt], dtype=np.float64)
    sysd = _Sys()
    lib().or_sys_dahlquist(C.byref(sysd), _d(lam))
    u0 = np.array([1.0, 0.0])
    u1 = np.zeros(2)
    rn = np.zeros(2)
    zz = np.zeros(2)
    ev = lib().or_step(C.byref(sysd), integ, dt, s, _d(u0), _d(u1), _d(rn), _d(zz))
    if ev < 0:
        raise RuntimeError("or_step failed")
    return complex(u1[0], u1[1]), complex(zz[0], zz[1])


def dahlquist_solve(integ, lam, t_end, nsteps, s=1):
    """Integrate u' = lam u, u(0)=1 over nsteps equal steps."""
    lamv = np.array([lam.real, lam.imag], dtype=np.float64)
    sysd = _Sys()
    lib().or_sys_dahlquist(C.byref(sysd), _d(lamv))
    u = np.array([1.0, 0.0])
    un = np.zeros(2)
    rn = np.zeros(2)
    zz = np.zeros(2)
    dt = t_end / nsteps
    for _ in range(nsteps):
        lib().or_step(C.byref(sysd), integ, dt, s, _d(u), _d(un), _d(rn), _d(zz))
        u, un = un, u
    return complex(u[0], u[1])


def project_cell_mobility(L, y):
    """or_project_cell_mobility: the mobility-weighted projection of one
    cell's values y (length N) with phase-field mobilities L (N x N).
    Returns (x, code), code 1 if a value changed, -1 if none is positive."""
    y = np.array(y, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(-1)
    r = lib().or_project_cell_mobility(len(y), _d(L), _d(y))
    return y, r


def evict_cell(y, n_slots):
    """or_evict_cell: the per-cell slot rule on one cell's values y."""
    y = np.array(y, dtype=np.float64)
    r = lib().or_evict_cell(len(y), int(n_slots), _d(y))
    return y, r


def keep_rhs_cell(r, n_slots):
    """or_keep_rhs_cell: the slot rule for one cell's stored RHS r."""
    r = np.array(r, dtype=np.float64)
    code = lib().or_keep_rhs_cell(len(r), int(n_slots), _d(r))
    return r, code


def sts_stages(integ, dt, dte):
    return lib().or_sts_stages(integ, dt, dte)


def ssp104_embedded_weights():
    bh = np.zeros(10)
    lib().or_ssp104_embedded_weights(_d(bh))
    return bh


class Drive:
    """Controller-only run (Sec. 3.2-3.3, ``or_drive``): the attempt sizes,
    stage counts and accept flags the oracle's adaptive loop takes when the
    error norms come from elsewhere (e.g. the GPU's trace).  The controller
    state and the proposal for the next step carry over between calls, as
    they do between pf_step calls."""

    def __init__(self, integ, dte, dt0=0.0, max_stages=1001, t=0.0):
        self.integ, self.dte, self.dt0, self.max_stages = integ, dte, dt0, max_stages
        self.t = t
        self.ctrl = _Ctrl()
        lib().or_ctrl_init(C.byref(self.ctrl))
        self.dt_next = 0.0

    def run(self, t_end, errs, given=None):
        """Attempts to t_end for the error norms errs.  given: the step sizes
        actually taken (continue from those; see or_drive)."""
        errs = np.ascontiguousarray(errs, np.float64)
        n = len(errs)
        hg = None if given is None else np.ascontiguousarray(given, np.float64)
        assert hg is None or len(hg) == n
        dt = np.zeros(max(n, 1))
        s = np.zeros(max(n, 1), np.int32)
        acc = np.zeros(max(n, 1), np.int32)
        t = C.c_double(self.t)
        dn = C.c_double(self.dt_next)
        k = lib().or_drive(self.integ, self.dte, t_end, self.dt0, self.max_stages, n, _d(errs),
                           _d(hg) if hg is not None else _dp(),
                           C.byref(t), C.byref(self.ctrl), C.byref(dn), n, _d(dt),
                           s.ctypes.data_as(_ip), acc.ctypes.data_as(_ip))
        self.t, self.dt_next = t.value, dn.value
        return dict(dt=dt[:k].copy(), s=s[:k].copy(), acc=acc[:k].copy())


def ctrl_sequence(errs, dts, P):
    """Feed errors/step sizes through a fresh controller: list of (dt_next, acc, b)."""
    c = _Ctrl()
    lib().or_ctrl_init(C.byref(c))
    out = []
    for e, h in zip(errs, dts):
        acc = C.c_int()
        nxt = lib().or_ctrl_update(C.byref(c), e, h, P, C.byref(acc))
        out.append((nxt, acc.value, c.b))
    return out
