"""Thin ctypes binding of libscale.so (include/scale.h): same names, argument marshalling
only. Every step of the computation runs in the CUDA library; there is no fallback.

Tensors are torch CUDA tensors (device memory and streams come from PyTorch); the binding
checks dtype / device / contiguity / shape and passes raw pointers.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import inputs as I

_lock = threading.Lock()
_lib = None
MAX_LAYERS = 32

OK, EINVAL, ENOMEM, EBUDGET, ECUDA, ETIMEOUT, EUNSUPPORTED, ECANCELED = range(8)
PATH_LOWRANK, PATH_FULL = 0, 1
SAMPLE_BAD_COUNT, SAMPLE_DOUBLE_OCC, SAMPLE_SINGULAR, SAMPLE_DRIFT = 1, 2, 4, 8

EXPORTED = [
    "scale_param_count", "scale_footprint_bytes", "scale_create", "scale_set_params", "scale_load",
    "scale_log_psi", "scale_get_occ", "scale_ratios", "scale_local_energy", "scale_commit",
    "scale_refresh", "scale_grad_logpsi", "scale_get_stats", "scale_last_error", "scale_destroy",
    "scale_sweep", "scale_log_psi_sym", "scale_test_inject",
]


class ScaleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"scale status {status}: {msg}")
        self.status = status


class scale_system(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("pbc_x", ctypes.c_int32),
                ("pbc_y", ctypes.c_int32), ("n_up", ctypes.c_int32), ("n_dn", ctypes.c_int32),
                ("model", ctypes.c_int32), ("t", ctypes.c_double), ("tp", ctypes.c_double),
                ("U", ctypes.c_double), ("J", ctypes.c_double)]


class scale_arch(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("h", ctypes.c_int32), ("act", ctypes.c_int32),
                ("per_site_embed", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refresh_every", ctypes.c_int32), ("drift_tol", ctypes.c_double),
                ("ksize", ctypes.c_int32 * MAX_LAYERS), ("residual", ctypes.c_int32 * MAX_LAYERS),
                ("family", ctypes.c_int32), ("n_conv", ctypes.c_int32), ("h_mlp", ctypes.c_int32),
                ("ln_eps", ctypes.c_double), ("stencil", ctypes.c_int32), ("lowrank_kernel", ctypes.c_int32)]


class scale_stats(ctypes.Structure):
    _fields_ = [("n_eloc", ctypes.c_int64), ("n_eloc_full", ctypes.c_int64),
                ("n_commits", ctypes.c_int64), ("n_refresh", ctypes.c_int64),
                ("n_drift_refresh", ctypes.c_int64), ("drift_max", ctypes.c_double),
                ("batch", ctypes.c_int32), ("max_moves", ctypes.c_int32), ("full_chunk", ctypes.c_int32),
                ("wait_timeouts", ctypes.c_int32)]


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libscale.so")


def load_library(build: bool = True):
    """Load libscale.so (building it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                from .build import build as _build
                _build()
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libscale.so missing at {path}; run paper_2604_25775_gb300.build")
            lib = ctypes.CDLL(path)
            P, V = ctypes.POINTER, ctypes.c_void_p
            lib.scale_param_count.restype = ctypes.c_int64
            lib.scale_param_count.argtypes = [P(scale_system), P(scale_arch)]
            lib.scale_footprint_bytes.restype = ctypes.c_size_t
            lib.scale_footprint_bytes.argtypes = [P(scale_system), P(scale_arch), ctypes.c_int32]
            lib.scale_create.restype = ctypes.c_int
            lib.scale_create.argtypes = [P(scale_system), P(scale_arch), ctypes.c_int32, ctypes.c_size_t, V,
                                         P(V)]
            for name, args in (("scale_set_params", [V, V, V]), ("scale_load", [V, V, ctypes.c_int32, V]),
                               ("scale_log_psi", [V, V, V]), ("scale_get_occ", [V, V]),
                               ("scale_ratios", [V, V, ctypes.c_int32, V]),
                               ("scale_local_energy", [V, ctypes.c_int32, V]), ("scale_commit", [V, V]),
                               ("scale_refresh", [V, ctypes.c_int32]),
                               ("scale_grad_logpsi", [V, V, ctypes.c_int32]),
                               ("scale_get_stats", [V, P(scale_stats)]),
                               ("scale_sweep", [V, ctypes.c_int32, V, V, V, V]),
                               ("scale_log_psi_sym", [V, ctypes.c_int32, V, V, V, V]),
                               ("scale_test_inject", [V, ctypes.c_int32])):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = args
            lib.scale_last_error.restype = ctypes.c_char_p
            lib.scale_last_error.argtypes = [V]
            lib.scale_destroy.restype = None
            lib.scale_destroy.argtypes = [V]
            _lib = lib
    return _lib


def make_descriptors(pb: I.Problem):
    s = scale_system(pb.Lx, pb.Ly, pb.pbc_x, pb.pbc_y, pb.n_up, pb.n_dn, pb.model, pb.t, pb.tp, pb.U, pb.J)
    a = scale_arch()
    a.n_layers, a.h, a.act, a.per_site_embed = pb.n_layers, pb.h, pb.act, pb.per_site_embed
    a.precision, a.refresh_every, a.drift_tol = pb.precision, pb.refresh_every, pb.drift_tol
    for l in range(pb.n_layers):
        a.ksize[l] = int(pb.ksize[l])
        a.residual[l] = int(pb.residual[l])
    a.family, a.n_conv, a.h_mlp, a.ln_eps = pb.family, pb.n_conv, pb.h_mlp, pb.ln_eps
    a.stencil = pb.stencil
    a.lowrank_kernel = pb.lowrank_kernel
    return s, a


def scale_param_count(pb: I.Problem) -> int:
    s, a = make_descriptors(pb)
    return int(load_library().scale_param_count(ctypes.byref(s), ctypes.byref(a)))


def scale_footprint_bytes(pb: I.Problem, max_batch: int) -> int:
    s, a = make_descriptors(pb)
    return int(load_library().scale_footprint_bytes(ctypes.byref(s), ctypes.byref(a), max_batch))


def _ptr(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """Owns a scale_ctx. Methods mirror the C entry points (scale_<name>)."""

    def __init__(self, pb: I.Problem, max_batch: int, hbm_budget_bytes: int = 0, stream=None):
        import torch
        self.lib = load_library()
        self.pb = pb
        self.N, self.Ne = pb.N, pb.Ne
        self.max_batch = max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        s, a = make_descriptors(pb)
        self._s, self._a = s, a
        h = ctypes.c_void_p()
        st = self.lib.scale_create(ctypes.byref(s), ctypes.byref(a), max_batch, hbm_budget_bytes,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise ScaleError(st, "scale_create failed")
        self.h = h
        self.P = int(self.lib.scale_param_count(ctypes.byref(s), ctypes.byref(a)))
        self.B = 0
        self._keep = []

    def _check(self, st):
        if st != OK:
            raise ScaleError(st, self.lib.scale_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.scale_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -------------------------------------------------------------------
    def scale_set_params(self, params, M0):
        import torch
        self._check(self.lib.scale_set_params(self.h, _ptr(params, torch.float64, (self.P,), "params"),
                                              _ptr(M0, torch.float64, (2 * self.N, self.Ne), "M0")))
        self._keep = [params, M0]

    def scale_load(self, occ, sample_status=None):
        import torch
        B = occ.shape[0]
        p_st = None if sample_status is None else _ptr(sample_status, torch.int32, (B,), "sample_status")
        self._check(self.lib.scale_load(self.h, _ptr(occ, torch.int8, (B, self.N), "occ"), B, p_st))
        self.B = B

    def scale_log_psi(self, logabs=None, sign=None):
        import torch
        la = None if logabs is None else _ptr(logabs, torch.float64, (self.B,), "logabs")
        sg = None if sign is None else _ptr(sign, torch.int32, (self.B,), "sign")
        self._check(self.lib.scale_log_psi(self.h, la, sg))

    def scale_get_occ(self, occ):
        import torch
        self._check(self.lib.scale_get_occ(self.h, _ptr(occ, torch.int8, (self.B, self.N), "occ")))

    def scale_ratios(self, moves, ratio):
        import torch
        M = moves.shape[1]
        self._check(self.lib.scale_ratios(self.h, _ptr(moves, torch.int32, (self.B, M, 4), "moves"), M,
                                          _ptr(ratio, torch.float64, (self.B, M), "ratio")))

    def scale_local_energy(self, eloc, path=PATH_LOWRANK):
        import torch
        self._check(self.lib.scale_local_energy(self.h, path, _ptr(eloc, torch.float64, (self.B,), "eloc")))

    def scale_commit(self, moves):
        import torch
        self._check(self.lib.scale_commit(self.h, _ptr(moves, torch.int32, (self.B, 4), "moves")))

    def scale_sweep(self, pick, direction, u, accepted):
        """Metropolis steps: pick, direction int32 [S][B], u float64 [S][B], accepted int32 [B]."""
        import torch
        S = int(u.shape[0]) if u.dim() == 2 else 0
        self._check(self.lib.scale_sweep(self.h, S, _ptr(pick, torch.int32, (S, self.B), "pick"),
                                         _ptr(direction, torch.int32, (S, self.B), "direction"),
                                         _ptr(u, torch.float64, (S, self.B), "u"),
                                         _ptr(accepted, torch.int32, (self.B,), "accepted")))

    def scale_log_psi_sym(self, perms, chi, logabs, sign):
        """perms int32 [G][2N], chi float64 [G], logabs float64 [B], sign int32 [B]."""
        import torch
        G = int(perms.shape[0])
        self._check(self.lib.scale_log_psi_sym(self.h, G, _ptr(perms, torch.int32, (G, 2 * self.N), "perms"),
                                               _ptr(chi, torch.float64, (G,), "chi"),
                                               _ptr(logabs, torch.float64, (self.B,), "logabs"),
                                               _ptr(sign, torch.int32, (self.B,), "sign")))

    def log_psi_sym(self, perms, chi):
        import torch
        la = torch.empty(self.B, dtype=torch.float64, device="cuda")
        sg = torch.empty(self.B, dtype=torch.int32, device="cuda")
        self.scale_log_psi_sym(perms, chi, la, sg)
        return la, sg

    def scale_test_inject(self, what=1):
        self._check(self.lib.scale_test_inject(self.h, what))

    def scale_refresh(self, force_all=True):
        self._check(self.lib.scale_refresh(self.h, 1 if force_all else 0))

    def scale_grad_logpsi(self, grad, recompute=False):
        import torch
        self._check(self.lib.scale_grad_logpsi(self.h, _ptr(grad, torch.float64, (self.B, self.P), "grad"),
                                               1 if recompute else 0))

    def scale_get_stats(self) -> dict:
        st = scale_stats()
        self._check(self.lib.scale_get_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in scale_stats._fields_}

    # -- conveniences (allocate outputs with torch, then call the entry points) ---------
    def log_psi(self):
        import torch
        la = torch.empty(self.B, dtype=torch.float64, device="cuda")
        sg = torch.empty(self.B, dtype=torch.int32, device="cuda")
        self.scale_log_psi(la, sg)
        return la, sg

    def sweep(self, pick, direction, u):
        """Run the Metropolis steps; returns the number of accepted steps per sample."""
        import torch
        acc = torch.empty(self.B, dtype=torch.int32, device="cuda")
        self.scale_sweep(pick, direction, u, acc)
        return acc

    def local_energy(self, path=PATH_LOWRANK):
        import torch
        e = torch.empty(self.B, dtype=torch.float64, device="cuda")
        self.scale_local_energy(e, path)
        return e

    def ratios(self, moves):
        import torch
        r = torch.empty(moves.shape[:2], dtype=torch.float64, device="cuda")
        self.scale_ratios(moves, r)
        return r

    def grad_logpsi(self, recompute=False):
        import torch
        g = torch.empty((self.B, self.P), dtype=torch.float64, device="cuda")
        self.scale_grad_logpsi(g, recompute)
        return g

    def get_occ(self):
        import torch
        o = torch.empty((self.B, self.N), dtype=torch.int8, device="cuda")
        self.scale_get_occ(o)
        return o


def make_context(pb: I.Problem, params: np.ndarray, M0: np.ndarray, max_batch: int, **kw) -> Context:
    """Context with parameters uploaded (float64 device copies kept alive by the context)."""
    import torch
    ctx = Context(pb, max_batch, **kw)
    ctx.scale_set_params(torch.from_numpy(np.ascontiguousarray(params, dtype=np.float64)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(M0, dtype=np.float64)).cuda())
    return ctx


# ---------------------------------------------------------------------------------------
# Serving (scale_server_*): continuous batching over device-resident chains.
# ---------------------------------------------------------------------------------------
def scale_log_psi_noalloc(pb, params, M0, occ, logabs, sign, stream=None):
    """scale_log_psi_noalloc: log|psi| / sign of occ without a context or a device
    allocation (all tensors are the caller's CUDA tensors)."""
    import torch
    lib = load_library()
    if not getattr(lib, "_na_ready", False):
        V = ctypes.c_void_p
        lib.scale_log_psi_noalloc.restype = ctypes.c_int
        lib.scale_log_psi_noalloc.argtypes = [ctypes.POINTER(scale_system), ctypes.POINTER(scale_arch), V, V, V,
                                              ctypes.c_int32, V, V, V]
        lib._na_ready = True
    s, a = make_descriptors(pb)
    B = occ.shape[0]
    st = stream if stream is not None else torch.cuda.current_stream()
    status = lib.scale_log_psi_noalloc(
        ctypes.byref(s), ctypes.byref(a), _ptr(params, torch.float64, (I.param_count(pb),), "params"),
        _ptr(M0, torch.float64, (2 * pb.N, pb.Ne), "M0"), _ptr(occ, torch.int8, (B, pb.N), "occ"), B,
        _ptr(logabs, torch.float64, (B,), "logabs"), _ptr(sign, torch.int32, (B,), "sign"),
        ctypes.c_void_p(st.cuda_stream))
    if status != OK:
        raise ScaleError(status, "scale_log_psi_noalloc failed")


EXPORTED += ["scale_log_psi_noalloc"]

SRV_OPEN, SRV_ELOC, SRV_STEP, SRV_LOGPSI, SRV_CLOSE = range(5)
EXPORTED += ["scale_server_create", "scale_server_submit", "scale_server_poll", "scale_server_stats",
             "scale_server_destroy", "scale_server_cancel"]


class scale_server_cfg(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("sys", ctypes.POINTER(scale_system)),
                ("arch", ctypes.POINTER(scale_arch)), ("params", ctypes.POINTER(ctypes.c_void_p)),
                ("M0", ctypes.POINTER(ctypes.c_void_p)), ("slots", ctypes.POINTER(ctypes.c_int32)),
                ("hbm_budget_bytes", ctypes.c_size_t)]


class scale_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("cls", ctypes.c_int32), ("n_walkers", ctypes.c_int32),
                ("chain", ctypes.c_uint64), ("occ_host", ctypes.c_void_p), ("moves_host", ctypes.c_void_p),
                ("out_host", ctypes.c_void_p)]


class scale_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("latency_us", ctypes.c_double), ("chain", ctypes.c_uint64)]


class scale_server_stats_t(ctypes.Structure):
    _fields_ = [("resident_bytes", ctypes.c_size_t), ("resident_max_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("n_batches", ctypes.c_int64),
                ("n_requests", ctypes.c_int64), ("open_chains", ctypes.c_int64)]


def _server_lib():
    lib = load_library()
    if not getattr(lib, "_srv_ready", False):
        P, V = ctypes.POINTER, ctypes.c_void_p
        lib.scale_server_create.restype = ctypes.c_int
        lib.scale_server_create.argtypes = [P(scale_server_cfg), P(V)]
        lib.scale_server_submit.restype = ctypes.c_int
        lib.scale_server_submit.argtypes = [V, P(scale_request), P(ctypes.c_uint64)]
        lib.scale_server_poll.restype = ctypes.c_int
        lib.scale_server_poll.argtypes = [V, ctypes.c_uint64, P(scale_result), ctypes.c_int32]
        lib.scale_server_cancel.restype = ctypes.c_int
        lib.scale_server_cancel.argtypes = [V, ctypes.c_uint64]
        lib.scale_server_stats.restype = ctypes.c_int
        lib.scale_server_stats.argtypes = [V, P(scale_server_stats_t)]
        lib.scale_server_destroy.restype = None
        lib.scale_server_destroy.argtypes = [V]
        lib._srv_ready = True
    return lib


class Server:
    """scale_server_* wrapper. classes: list of (Problem, params, M0, slots)."""

    def __init__(self, classes, hbm_budget_bytes: int = 0):
        import torch
        self.lib = _server_lib()
        n = len(classes)
        self.problems = [c[0] for c in classes]
        descs = [make_descriptors(c[0]) for c in classes]
        self._sys = (scale_system * n)(*[d[0] for d in descs])
        self._arch = (scale_arch * n)(*[d[1] for d in descs])
        self._dev = [(torch.from_numpy(np.ascontiguousarray(c[1], dtype=np.float64)).cuda(),
                      torch.from_numpy(np.ascontiguousarray(c[2], dtype=np.float64)).cuda()) for c in classes]
        self._params = (ctypes.c_void_p * n)(*[p.data_ptr() for p, _ in self._dev])
        self._M0 = (ctypes.c_void_p * n)(*[m.data_ptr() for _, m in self._dev])
        self._slots = (ctypes.c_int32 * n)(*[int(c[3]) for c in classes])
        cfg = scale_server_cfg(n, self._sys, self._arch, self._params, self._M0, self._slots, hbm_budget_bytes)
        torch.cuda.synchronize()
        h = ctypes.c_void_p()
        st = self.lib.scale_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise ScaleError(st, "scale_server_create failed")
        self.h = h
        self._keep = {}
        self._n = {}

    def _submit(self, req, keep=()):
        t = ctypes.c_uint64()
        st = self.lib.scale_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != OK:
            raise ScaleError(st, "scale_server_submit failed")
        self._keep[t.value] = keep
        return t.value

    def open(self, cls: int, occ: np.ndarray) -> int:
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        req = scale_request(SRV_OPEN, cls, occ.shape[0], 0, occ.ctypes.data, None, None)
        t = self._submit(req, (occ,))
        self._n[t] = occ.shape[0]
        return t

    def eloc(self, chain: int, out: np.ndarray) -> int:
        req = scale_request(SRV_ELOC, 0, 0, chain, None, None, out.ctypes.data)
        return self._submit(req, (out,))

    def step(self, chain: int, moves: np.ndarray, out: np.ndarray) -> int:
        moves = np.ascontiguousarray(moves, dtype=np.int32)
        req = scale_request(SRV_STEP, 0, 0, chain, None, moves.ctypes.data, out.ctypes.data)
        return self._submit(req, (moves, out))

    def logpsi(self, chain: int, out: np.ndarray) -> int:
        req = scale_request(SRV_LOGPSI, 0, 0, chain, None, None, out.ctypes.data)
        return self._submit(req, (out,))

    def close(self, chain: int) -> int:
        return self._submit(scale_request(SRV_CLOSE, 0, 0, chain, None, None, None))

    def poll(self, ticket: int, timeout_us: int = 10_000_000):
        """(status, latency_us) when done, None on timeout."""
        r = scale_result()
        st = self.lib.scale_server_poll(self.h, ticket, ctypes.byref(r), timeout_us)
        if st == ETIMEOUT:
            return None
        if st != OK:
            raise ScaleError(st, "scale_server_poll failed")
        self._keep.pop(ticket, None)
        return r.status, r.latency_us

    def cancel(self, ticket: int) -> bool:
        """scale_server_cancel: True when the request was still queued and is now cancelled
        (poll it to release it: status ECANCELED), False when it had started or finished."""
        st = self.lib.scale_server_cancel(self.h, ticket)
        if st not in (OK, EINVAL):
            raise ScaleError(st, "scale_server_cancel failed")
        return st == OK

    def stats(self) -> dict:
        s = scale_server_stats_t()
        self.lib.scale_server_stats(self.h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in scale_server_stats_t._fields_}

    def destroy(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.scale_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
