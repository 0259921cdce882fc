"""ctypes front of the FP64 C oracle (oracle.c) plus whole-Hilbert-space enumeration.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the bench's CPU-baseline
leg, never by the product path. Problems are passed as plain mappings (or any object with
an ``as_dict()``), so this module imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_LAYERS = 32


class _Model(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("pbc_x", ctypes.c_int32),
        ("pbc_y", ctypes.c_int32), ("n_up", ctypes.c_int32), ("n_dn", ctypes.c_int32),
        ("model", ctypes.c_int32),
        ("t", ctypes.c_double), ("tp", ctypes.c_double), ("U", ctypes.c_double),
        ("J", ctypes.c_double),
        ("n_layers", ctypes.c_int32), ("h", ctypes.c_int32), ("act", ctypes.c_int32),
        ("per_site_embed", ctypes.c_int32),
        ("ksize", ctypes.c_int32 * MAX_LAYERS), ("residual", ctypes.c_int32 * MAX_LAYERS),
        ("family", ctypes.c_int32), ("n_conv", ctypes.c_int32), ("h_mlp", ctypes.c_int32),
        ("ln_eps", ctypes.c_double), ("stencil", ctypes.c_int32),
        ("params", ctypes.POINTER(ctypes.c_double)), ("M0", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            lib.ora_param_count.restype = ctypes.c_int64
            lib.ora_param_count.argtypes = [P(_Model)]
            lib.ora_bonds.restype = ctypes.c_int
            lib.ora_bonds.argtypes = [P(_Model), ctypes.c_int, ctypes.c_void_p]
            lib.ora_slogdet.restype = ctypes.c_double
            lib.ora_slogdet.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            for name in ("ora_log_psi", "ora_orbitals", "ora_local_energy", "ora_ratio",
                         "ora_grad_logpsi"):
                getattr(lib, name).restype = ctypes.c_int
            lib.ora_log_psi.argtypes = [P(_Model), ctypes.c_int] + [ctypes.c_void_p] * 3
            lib.ora_orbitals.argtypes = [P(_Model), ctypes.c_int] + [ctypes.c_void_p] * 3
            lib.ora_local_energy.argtypes = [P(_Model), ctypes.c_int] + [ctypes.c_void_p] * 3
            lib.ora_ratio.argtypes = [P(_Model), ctypes.c_int] + [ctypes.c_void_p] * 3
            lib.ora_grad_logpsi.argtypes = [P(_Model), ctypes.c_int] + [ctypes.c_void_p] * 2
            lib.ora_features.restype = ctypes.c_int
            lib.ora_features.argtypes = [P(_Model), ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_connected.restype = ctypes.c_int
            lib.ora_connected.argtypes = [P(_Model), ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_diag.restype = ctypes.c_double
            lib.ora_diag.argtypes = [P(_Model), ctypes.c_void_p]
            lib.ora_num_threads.restype = ctypes.c_int
            lib.ora_metropolis.restype = ctypes.c_int
            lib.ora_log_psi_sym.restype = ctypes.c_int
            lib.ora_log_psi_sym.argtypes = [P(_Model), ctypes.c_int, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4
            lib.ora_metropolis.argtypes = [P(_Model), ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 5
            _lib = lib
    return _lib


def _as_dict(pb):
    return pb.as_dict() if hasattr(pb, "as_dict") else dict(pb)


class Model:
    """A problem bound to its parameters and reference orbitals (kept alive here)."""

    def __init__(self, problem, params: np.ndarray, M0: np.ndarray):
        d = _as_dict(problem)
        self.d = d
        self.N = d["Lx"] * d["Ly"]
        self.Ne = d["n_up"] + d["n_dn"]
        self.h = d["h"]
        self.L = d["n_layers"]
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self.M0 = np.ascontiguousarray(M0, dtype=np.float64)
        assert self.M0.shape == (2 * self.N, self.Ne)
        s = _Model()
        for k in ("Lx", "Ly", "pbc_x", "pbc_y", "n_up", "n_dn", "model", "n_layers", "h",
                  "act", "per_site_embed"):
            setattr(s, k, int(d[k]))
        for k in ("t", "tp", "U", "J"):
            setattr(s, k, float(d[k]))
        for l in range(self.L):
            s.ksize[l] = int(d["ksize"][l])
            s.residual[l] = int(d["residual"][l])
        s.family = int(d.get("family", 0))
        s.n_conv = int(d.get("n_conv", 0))
        s.h_mlp = int(d.get("h_mlp", 0)) or self.h
        s.ln_eps = float(d.get("ln_eps", 1e-5))
        s.stencil = int(d.get("stencil", 0))
        ace = s.family != 0 and self.L > s.n_conv
        self.h_last = s.h_mlp if ace else self.h
        self.h_max = max(self.h, self.h_last)
        s.params = self.params.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.M0 = self.M0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.s = s
        lib = _load()
        self.P = int(lib.ora_param_count(ctypes.byref(s)))
        assert self.params.size == self.P, (self.params.size, self.P)

    # -- thin wrappers -------------------------------------------------------------------
    def bonds(self, which: int) -> np.ndarray:
        lib = _load()
        buf = np.zeros((4 * self.N, 2), dtype=np.int32)
        n = lib.ora_bonds(ctypes.byref(self.s), which, buf.ctypes.data)
        return buf[:n].copy()

    def log_psi(self, occ: np.ndarray):
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        B = occ.shape[0]
        la = np.zeros(B)
        sg = np.zeros(B, dtype=np.int32)
        _load().ora_log_psi(ctypes.byref(self.s), B, occ.ctypes.data, la.ctypes.data, sg.ctypes.data)
        return la, sg

    def orbitals(self, occ: np.ndarray):
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        B = occ.shape[0]
        HL = np.zeros((B, self.N, self.h_last))
        M = np.zeros((B, 2 * self.N, self.Ne))
        _load().ora_orbitals(ctypes.byref(self.s), B, occ.ctypes.data, HL.ctypes.data, M.ctypes.data)
        return HL, M

    def features(self, occ1: np.ndarray) -> np.ndarray:
        occ1 = np.ascontiguousarray(occ1, dtype=np.int8)
        H = np.zeros((self.L + 1, self.N, self.h_max))
        _load().ora_features(ctypes.byref(self.s), occ1.ctypes.data, H.ctypes.data)
        return H

    def local_energy(self, occ: np.ndarray):
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        B = occ.shape[0]
        e = np.zeros(B)
        st = np.zeros(B, dtype=np.int32)
        _load().ora_local_energy(ctypes.byref(self.s), B, occ.ctypes.data, e.ctypes.data, st.ctypes.data)
        return e, st

    def ratio(self, occ: np.ndarray, moves: np.ndarray) -> np.ndarray:
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        moves = np.ascontiguousarray(moves, dtype=np.int32)
        B = occ.shape[0]
        r = np.zeros(B)
        _load().ora_ratio(ctypes.byref(self.s), B, occ.ctypes.data, moves.ctypes.data, r.ctypes.data)
        return r

    def grad_logpsi(self, occ: np.ndarray) -> np.ndarray:
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        B = occ.shape[0]
        g = np.zeros((B, self.P))
        if _load().ora_grad_logpsi(ctypes.byref(self.s), B, occ.ctypes.data, g.ctypes.data) != 0:
            raise NotImplementedError("the oracle's backward pass covers the SCALE family")
        return g

    def connected(self, occ1: np.ndarray):
        occ1 = np.ascontiguousarray(occ1, dtype=np.int8)
        cap = 12 * self.N + 8
        xp = np.zeros((cap, self.N), dtype=np.int8)
        cf = np.zeros(cap)
        n = _load().ora_connected(ctypes.byref(self.s), occ1.ctypes.data, cap, xp.ctypes.data, cf.ctypes.data)
        return xp[:n].copy(), cf[:n].copy()

    def diag(self, occ1: np.ndarray) -> float:
        occ1 = np.ascontiguousarray(occ1, dtype=np.int8)
        return float(_load().ora_diag(ctypes.byref(self.s), occ1.ctypes.data))

    def log_psi_sym(self, occ: np.ndarray, perms: np.ndarray, chi: np.ndarray):
        """log|psi_sym| and sign of sum_g Pi(n, g) chi_g psi(g n); perms [G][2N] orbital
        permutations, chi [G] real characters."""
        occ = np.ascontiguousarray(occ, dtype=np.int8)
        perms = np.ascontiguousarray(perms, dtype=np.int32)
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        B, G = occ.shape[0], perms.shape[0]
        assert perms.shape == (G, 2 * self.N) and chi.shape == (G,)
        la = np.zeros(B)
        sg = np.zeros(B, dtype=np.int32)
        _load().ora_log_psi_sym(ctypes.byref(self.s), B, occ.ctypes.data, G, perms.ctypes.data, chi.ctypes.data,
                                la.ctypes.data, sg.ctypes.data)
        return la, sg

    def metropolis(self, occ: np.ndarray, pick: np.ndarray, direction: np.ndarray, u: np.ndarray):
        """Metropolis steps (hop proposals, acceptance min(1, |psi'/psi|^2)); pick, direction
        and u are [S][B]. Returns (final occ [B][N], accepted [B])."""
        x = np.array(occ, dtype=np.int8, order="C", copy=True)
        pick = np.ascontiguousarray(pick, dtype=np.int32)
        direction = np.ascontiguousarray(direction, dtype=np.int32)
        u = np.ascontiguousarray(u, dtype=np.float64)
        S, B = u.shape
        assert x.shape[0] == B and pick.shape == (S, B) and direction.shape == (S, B)
        acc = np.zeros(B, dtype=np.int32)
        _load().ora_metropolis(ctypes.byref(self.s), B, S, x.ctypes.data, pick.ctypes.data,
                               direction.ctypes.data, u.ctypes.data, acc.ctypes.data)
        return x, acc

    def with_params(self, params: np.ndarray) -> "Model":
        return Model(self.d, params, self.M0)


def slogdet(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    sg = np.zeros(1, dtype=np.int32)
    la = _load().ora_slogdet(n, A.ctypes.data, sg.ctypes.data)
    return int(sg[0]), float(la)


def num_threads() -> int:
    return int(_load().ora_num_threads())


def all_configurations(problem) -> np.ndarray:
    """Every configuration with the problem's particle numbers (t-J: no double occupancy)."""
    d = _as_dict(problem)
    N = d["Lx"] * d["Ly"]
    out = []
    for up in itertools.combinations(range(N), d["n_up"]):
        for dn in itertools.combinations(range(N), d["n_dn"]):
            if d["model"] == 1 and set(up) & set(dn):
                continue
            x = np.zeros(N, dtype=np.int8)
            x[list(up)] |= 1
            x[list(dn)] |= 2
            out.append(x)
    return np.array(out, dtype=np.int8)


def enumerate_energy(model: Model):
    """<H> = sum_n psi(n)^2 E_loc(n) / sum_n psi(n)^2 over the whole space (tiny lattices),
    with E_loc from the oracle's full-recompute local energy (Sec. II.A)."""
    xs = all_configurations(model.d)
    la, sg = model.log_psi(xs)
    e, st = model.local_energy(xs)
    ok = sg != 0
    w = np.exp(2.0 * (la[ok] - la[ok].max()))
    return float(np.sum(w * e[ok]) / np.sum(w)), xs, la, sg
