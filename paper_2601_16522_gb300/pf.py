"""ctypes binding of libpf (include/pf.h): argument marshalling only.

Every step of the path runs in the CUDA library; this module converts a
``Problem`` (paper_2601_16522_gb300.inputs) into ``pf_params``, moves numpy
arrays or torch tensors across the ABI and raises on non-zero status.  If the
compiled library is missing it raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpf.so")

FEULER, SSP2, SSP104, RKL1, RKL2 = 0, 1, 2, 3, 4
PASS_KINDS = ["euler", "ssp", "sts_first", "rkl1", "rkl2", "sts_err", "rhs", "other"]
PF_OK, PF_EINVAL, PF_ENOMEM, PF_EUNSTABLE, PF_ETIMEOUT, PF_EDEVICE, PF_ESTATE = range(7)

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_ubp = C.POINTER(C.c_ubyte)


class PfError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (what, _lib().pf_strerror(status).decode(), status))


class pf_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("n_phases", C.c_int), ("phase_type", _ip),
                ("gamma", _dp), ("mobility", _dp), ("W", C.c_double), ("L_override", _dp),
                ("has_conc", C.c_int), ("k", C.c_double * 2), ("c0", C.c_double * 2),
                ("D", C.c_double * 2), ("bc_phi", C.c_int * 6), ("bc_c", C.c_int * 6),
                ("c_dirichlet", C.c_double * 6), ("precision", C.c_int), ("options", C.c_int),
                ("c_ref", C.c_double)]


class pf_controller(C.Structure):
    _fields_ = [("b", C.c_double), ("E1", C.c_double), ("E2", C.c_double), ("dt1", C.c_double),
                ("dt2", C.c_double), ("dt_next", C.c_double), ("nhist", C.c_int)]


class pf_tol(C.Structure):
    _fields_ = [("r_phi", C.c_double), ("a_phi", C.c_double), ("r_c", C.c_double), ("a_c", C.c_double)]


class pf_step_opts(C.Structure):
    _fields_ = [("ssp_stages", C.c_int), ("dt_mult", C.c_double), ("dt0", C.c_double),
                ("max_stages", C.c_int), ("max_attempts", C.c_int), ("trace_cap", C.c_int),
                ("trace_dt", _dp), ("trace_s", _ip), ("trace_err", _dp), ("trace_acc", _ip),
                ("trace_len", _ip), ("flags", C.c_int)]


class pf_stats(C.Structure):
    _fields_ = [("rhs_evals", C.c_longlong), ("steps_accepted", C.c_longlong),
                ("steps_rejected", C.c_longlong), ("t", C.c_double), ("dt_last", C.c_double),
                ("err_last", C.c_double), ("dt_e", C.c_double), ("dt_next", C.c_double),
                ("kernel_launches", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpf.so not built (run paper_2601_16522_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        H = C.c_void_p
        L.pf_create.argtypes = [C.POINTER(pf_params), C.c_void_p, C.POINTER(H)]
        L.pf_set_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_double, C.c_int]
        L.pf_rhs.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.pf_step.argtypes = [H, C.c_int, C.c_double, C.POINTER(pf_tol), C.POINTER(pf_step_opts),
                              C.POINTER(pf_stats)]
        L.pf_get_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, _dp, C.c_int]
        L.pf_set_state_slots.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_int]
        L.pf_get_state_slots.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, _dp, C.c_int]
        L.pf_reduce.argtypes = [H, _dp, _dp, _ip]
        L.pf_energy.argtypes = [H, _dp]
        L.pf_dt_e.argtypes = [H, _dp]
        L.pf_selftest_wait.argtypes = [C.c_void_p, C.c_uint]
        L.pf_get_controller.argtypes = [H, C.POINTER(pf_controller)]
        L.pf_set_controller.argtypes = [H, C.POINTER(pf_controller)]
        L.pf_destroy.argtypes = [H]
        L.pf_profile.argtypes = [H, C.c_int, _dp, C.POINTER(C.c_longlong)]
        L.pf_footprint.argtypes = [C.POINTER(pf_params), C.POINTER(C.c_longlong)]
        L.pf_autotune.argtypes = [H, _ip, _dp]
        L.pf_launch_count.argtypes = [H]
        L.pf_launch_count.restype = C.c_longlong
        L.pf_strerror.argtypes = [C.c_int]
        L.pf_strerror.restype = C.c_char_p
        L.pf_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, C.c_void_p]
        L.pf_batch_create.argtypes = [C.c_longlong, C.c_void_p, C.POINTER(C.c_void_p)]
        L.pf_batch_admit.argtypes = [C.c_void_p, H, C.c_int, C.c_double, C.POINTER(pf_tol),
                                     C.POINTER(pf_step_opts), _ip]
        L.pf_batch_run.argtypes = [C.c_void_p, C.c_int, _ip]
        L.pf_batch_result.argtypes = [C.c_void_p, C.c_int, _ip, _ip, C.POINTER(pf_stats)]
        L.pf_batch_destroy.argtypes = [C.c_void_p]
        _LIB = L
    return _LIB


def lib():
    """The loaded libpf (ctypes CDLL)."""
    return _lib()


def _check(st, what):
    if st != PF_OK:
        raise PfError(st, what)


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_dev(a):
    """True for a CUDA tensor, False for numpy arrays and (pinned) CPU tensors."""
    if isinstance(a, np.ndarray):
        return False
    return bool(getattr(a, "is_cuda", False))


def make_params(prob, precision=64, options=0):
    """pf_params for a Problem; returns (params, keep-alive arrays)."""
    N = prob.n_phases
    keep = [np.ascontiguousarray(prob.phase_type, np.int32),
            np.ascontiguousarray(prob.gamma, np.float64).reshape(-1),
            np.ascontiguousarray(prob.mobility, np.float64).reshape(-1)]
    p = pf_params()
    p.dim, p.nx, p.ny, p.nz, p.dx = prob.dim, prob.nx, prob.ny, prob.nz, prob.dx
    p.n_phases = N
    p.phase_type = keep[0].ctypes.data_as(_ip)
    p.gamma = keep[1].ctypes.data_as(_dp)
    p.mobility = keep[2].ctypes.data_as(_dp)
    p.W = prob.W
    if prob.L_override is not None:
        Lm = np.ascontiguousarray(prob.L_override, np.float64).reshape(-1)
        keep.append(Lm)
        p.L_override = Lm.ctypes.data_as(_dp)
    p.has_conc = prob.has_conc
    for t in range(2):
        p.k[t], p.c0[t], p.D[t] = prob.k[t], prob.c0[t], prob.D[t]
    for f in range(6):
        p.bc_phi[f], p.bc_c[f], p.c_dirichlet[f] = prob.bc_phi[f], prob.bc_c[f], prob.c_dirichlet[f]
    p.precision = precision
    if getattr(prob, "simplex", 0) == 1:
        options |= Simulation.OPT_MOBILITY_SIMPLEX
    if getattr(prob, "n_slots", 0):
        if prob.n_slots != Simulation.N_SLOTS:
            raise ValueError("slot storage holds %d phases per cell" % Simulation.N_SLOTS)
        options |= Simulation.OPT_SLOTS
    p.options = options
    p.c_ref = float(getattr(prob, "c_ref", 0.0) or 0.0)
    return p, keep


def selftest_wait(polls=1 << 16, stream=None):
    """Bounded-wait self-test (pf_selftest_wait): returns the status, which is
    PF_ETIMEOUT (4) when the device wait gave up as designed."""
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    return _lib().pf_selftest_wait(s, polls)


def footprint(prob, precision=64, options=0):
    """Device bytes a Simulation of this problem holds (pf_footprint)."""
    p, keep = make_params(prob, precision, options)
    b = C.c_longlong()
    _check(_lib().pf_footprint(C.byref(p), C.byref(b)), "pf_footprint")
    return b.value


class Simulation:
    """One simulation handle (pf_create .. pf_destroy)."""

    OPT_TMA = 1
    OPT_MASKED = 2
    OPT_ONE_CELL = 4
    OPT_MOBILITY_SIMPLEX = 8
    OPT_SLOTS = 16
    N_SLOTS = 12
    KVAR_TWO_CELL, KVAR_ONE_CELL, KVAR_TMA = 0, 1, 2

    def __init__(self, prob, precision=64, stream=None, options=0):
        self.prob = prob
        N = prob.n_phases
        p, self._keep = make_params(prob, precision, options)
        self.params = p
        self.precision = precision
        self._stream = stream
        sptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
        h = C.c_void_p()
        _check(_lib().pf_create(C.byref(p), sptr, C.byref(h)), "pf_create")
        self.h = h
        self.V = prob.V
        self.N = N
        self.K = prob.has_conc

    def close(self):
        if getattr(self, "h", None):
            _lib().pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------------
    def dt_e(self):
        d = C.c_double()
        _check(_lib().pf_dt_e(self.h, C.byref(d)), "pf_dt_e")
        return d.value

    def _wait_for_torch(self, t):
        """Order the simulation's stream after the work torch has queued on
        its current stream (which may still be writing the tensor t)."""
        import torch
        cur = torch.cuda.current_stream(t.device)
        if self._stream is not None:
            self._stream.wait_stream(cur)
        else:
            cur.synchronize()

    def _torch_waits(self, t):
        """Order torch's current stream after the simulation's stream (which
        is writing the tensor t)."""
        import torch
        cur = torch.cuda.current_stream(t.device)
        cur.wait_stream(self._stream if self._stream is not None else torch.cuda.default_stream(t.device))

    def set_state(self, u, t=0.0):
        """u: (N+K, V) float64 numpy array (host) or torch CUDA tensor (device).
        A CUDA tensor is read on the simulation's stream after the work torch
        has queued on its current stream."""
        dev = _is_dev(u)
        if not dev:
            u = np.ascontiguousarray(u, np.float64)
        assert tuple(u.shape) == (self.N + self.K, self.V), tuple(u.shape)
        if dev:
            self._wait_for_torch(u)
        phi = _ptr(u)
        c = phi + 8 * self.N * self.V if self.K else None
        _check(_lib().pf_set_state(self.h, phi, c, float(t), int(dev)), "pf_set_state")
        self._last_in = u

    def get_state(self, out=None, with_nz=False):
        """Returns (u, t[, nz]); out may be a preallocated numpy array or CUDA tensor.
        Into a CUDA tensor the copy runs on the simulation's stream, and
        torch's current stream is made to wait for it."""
        if out is None:
            out = np.zeros((self.N + self.K, self.V))
        dev = _is_dev(out)
        phi = _ptr(out)
        c = phi + 8 * self.N * self.V if self.K else None
        nz = None
        if with_nz:
            nz = np.zeros(self.V, np.uint8) if not dev else None
            if dev:
                import torch
                nz = torch.zeros(self.V, dtype=torch.uint8, device=out.device)
        t = C.c_double()
        if dev:
            self._wait_for_torch(out)
        _check(_lib().pf_get_state(self.h, phi, c, _ptr(nz), C.byref(t), int(dev)), "pf_get_state")
        if dev:
            self._torch_waits(out)
        return (out, t.value, nz) if with_nz else (out, t.value)

    def set_state_slots(self, vals, ids, c=None, t=0.0):
        """Slot form (slot storage): vals (n_in, V) float64 and ids (n_in, V)
        int32 (-1: empty), c (V,) float64 when K = 1; numpy arrays or CUDA
        tensors (all of one kind)."""
        dev = _is_dev(vals)
        if not dev:
            vals = np.ascontiguousarray(vals, np.float64)
            ids = np.ascontiguousarray(ids, np.int32)
            c = None if c is None else np.ascontiguousarray(c, np.float64)
        assert vals.shape == ids.shape and vals.shape[1] == self.V, (vals.shape, ids.shape)
        if dev:
            self._wait_for_torch(vals)
        _check(_lib().pf_set_state_slots(self.h, _ptr(vals), _ptr(ids), int(vals.shape[0]),
                                         _ptr(c) if c is not None else None, float(t), int(dev)),
               "pf_set_state_slots")
        self._last_in = (vals, ids, c)

    def get_state_slots(self, device=None):
        """Returns (vals (12, V) float64, ids (12, V) int32, c or None, t):
        numpy arrays, or CUDA tensors on `device`."""
        n = self.N_SLOTS
        if device is None:
            vals = np.zeros((n, self.V))
            ids = np.zeros((n, self.V), np.int32)
            c = np.zeros(self.V) if self.K else None
        else:
            import torch
            vals = torch.empty((n, self.V), dtype=torch.float64, device=device)
            ids = torch.empty((n, self.V), dtype=torch.int32, device=device)
            c = torch.empty(self.V, dtype=torch.float64, device=device) if self.K else None
            self._wait_for_torch(vals)
        t = C.c_double()
        _check(_lib().pf_get_state_slots(self.h, _ptr(vals), _ptr(ids), _ptr(c) if c is not None else None,
                                         C.byref(t), int(device is not None)), "pf_get_state_slots")
        if device is not None:
            self._torch_waits(vals)
        return vals, ids, c, t.value

    def rhs(self):
        """RHS of the current state -> ((N+K, V) float64, nz uint8) on the host."""
        r = np.zeros((self.N + self.K, self.V))
        nz = np.zeros(self.V, np.uint8)
        phi = r.ctypes.data
        c = phi + 8 * self.N * self.V if self.K else None
        _check(_lib().pf_rhs(self.h, phi, c, nz.ctypes.data, 0), "pf_rhs")
        return r, nz

    STEP_NO_GRAPH = 1
    STEP_REUSE_RHS = 2
    STEP_DEVICE_LOOP = 4

    def step(self, integ, t_end, tol=None, dt_mult=0.0, ssp_stages=5, dt0=0.0, max_stages=0,
             max_attempts=0, trace_cap=0, flags=0):
        o = pf_step_opts()
        o.ssp_stages, o.dt_mult, o.dt0, o.max_stages, o.max_attempts = ssp_stages, dt_mult, dt0, max_stages, max_attempts
        o.flags = flags
        tr = None
        if trace_cap:
            tr = dict(dt=np.zeros(trace_cap), s=np.zeros(trace_cap, np.int32), err=np.zeros(trace_cap),
                      acc=np.zeros(trace_cap, np.int32), n=C.c_int())
            o.trace_cap = trace_cap
            o.trace_dt = tr["dt"].ctypes.data_as(_dp)
            o.trace_s = tr["s"].ctypes.data_as(_ip)
            o.trace_err = tr["err"].ctypes.data_as(_dp)
            o.trace_acc = tr["acc"].ctypes.data_as(_ip)
            o.trace_len = C.pointer(tr["n"])
        tl = pf_tol(*tol) if tol is not None else None
        st = pf_stats()
        s = _lib().pf_step(self.h, int(integ), float(t_end), C.byref(tl) if tl is not None else None,
                           C.byref(o), C.byref(st))
        _check(s, "pf_step")
        out = st.as_dict()
        if tr is not None:
            n = tr["n"].value
            out["trace"] = dict(dt=tr["dt"][:n].copy(), s=tr["s"][:n].copy(),
                                err=tr["err"][:n].copy(), acc=tr["acc"][:n].copy())
        return out

    def profile(self, enable):
        """Read per-pass event timings accumulated so far, then (enable=1)
        restart or (enable=0) stop recording; enable=-1 only reads.
        Returns {kind: (ms, launches)}."""
        ms = (C.c_double * 8)()
        n = (C.c_longlong * 8)()
        _check(_lib().pf_profile(self.h, int(enable), ms, n), "pf_profile")
        return {k: (ms[i], n[i]) for i, k in enumerate(PASS_KINDS)}

    def autotune(self):
        """pf_autotune: returns (choice, {variant: ms}) with choice one of
        KVAR_TWO_CELL, KVAR_ONE_CELL, KVAR_TMA; variants that do not apply are
        left out of the dict."""
        c = C.c_int()
        ms = (C.c_double * 3)()
        _check(_lib().pf_autotune(self.h, C.byref(c), ms), "pf_autotune")
        return c.value, {k: ms[k] for k in range(3) if ms[k] >= 0.0}

    def launch_count(self):
        return _lib().pf_launch_count(self.h)

    def get_controller(self):
        """Adaptive controller state (bias, error/step history, next step) as a dict."""
        c = pf_controller()
        _check(_lib().pf_get_controller(self.h, C.byref(c)), "pf_get_controller")
        return {k: getattr(c, k) for k, _ in pf_controller._fields_}

    def set_controller(self, state):
        """Restore a state from get_controller (after set_state)."""
        c = pf_controller(**{k: state[k] for k, _ in pf_controller._fields_})
        _check(_lib().pf_set_controller(self.h, C.byref(c)), "pf_set_controller")

    def reduce(self):
        m = C.c_double()
        vol = np.zeros(self.N)
        alive = C.c_int()
        _check(_lib().pf_reduce(self.h, C.byref(m), vol.ctypes.data_as(_dp), C.byref(alive)), "pf_reduce")
        return m.value, vol, alive.value

    def energy(self):
        """Energy functional F of the current state (Eq. energy), FP64."""
        F = C.c_double()
        _check(_lib().pf_energy(self.h, C.byref(F)), "pf_energy")
        return F.value


# ---------------------------------------------------------------------------
# Device memory from torch's caching allocator (pf_set_allocator)
# ---------------------------------------------------------------------------
_HOOK = None


def use_torch_allocator(enable=True):
    """Route the device buffers of handles created from now on through
    torch's caching allocator (torch.cuda.caching_allocator_alloc / _delete on
    the handle's stream), so simulations and torch share one memory pool;
    enable=False restores CUDA's stream-ordered allocator."""
    global _HOOK
    L = _lib()
    if not enable:
        _check(L.pf_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "pf_set_allocator")
        return
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream(dev)
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
        except Exception:
            return None

    def free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    _HOOK = (_ALLOC_FN(alloc), _FREE_FN(free))      # kept alive while set
    _check(L.pf_set_allocator(_HOOK[0], _HOOK[1], None), "pf_set_allocator")


# ---------------------------------------------------------------------------
# Batched stepping (pf_batch_*)
# ---------------------------------------------------------------------------
class Batch:
    """Continuous batching of Simulations on one stream (pf_batch_*): admit
    requests as memory allows, run rounds, collect finished results."""

    def __init__(self, max_bytes, stream=None):
        self._stream = stream
        b = C.c_void_p()
        sptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(_lib().pf_batch_create(int(max_bytes), sptr, C.byref(b)), "pf_batch_create")
        self.b = b
        self._sims = {}

    def admit(self, sim, integ, t_end, tol=None, dt_mult=0.0, ssp_stages=5, dt0=0.0, max_stages=0):
        """Returns the slot, or None when the request does not fit the budget now."""
        o = pf_step_opts()
        o.ssp_stages, o.dt_mult, o.dt0, o.max_stages = ssp_stages, dt_mult, dt0, max_stages
        tl = pf_tol(*tol) if tol is not None else None
        slot = C.c_int()
        st = _lib().pf_batch_admit(self.b, sim.h, int(integ), float(t_end),
                                   C.byref(tl) if tl is not None else None, C.byref(o), C.byref(slot))
        if st == PF_ENOMEM:
            return None
        _check(st, "pf_batch_admit")
        self._sims[slot.value] = sim
        return slot.value

    def run(self, rounds=1):
        """Runs up to `rounds` rounds; returns the number of running requests."""
        n = C.c_int()
        _check(_lib().pf_batch_run(self.b, int(rounds), C.byref(n)), "pf_batch_run")
        return n.value

    def result(self, slot):
        """None while running; else (status, stats dict), releasing the slot."""
        done, status, st = C.c_int(), C.c_int(), pf_stats()
        _check(_lib().pf_batch_result(self.b, int(slot), C.byref(done), C.byref(status), C.byref(st)),
               "pf_batch_result")
        if not done.value:
            return None
        self._sims.pop(slot, None)
        return status.value, st.as_dict()

    def close(self):
        if getattr(self, "b", None):
            _lib().pf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
