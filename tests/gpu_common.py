"""Shared set-up for the GPU parity tests: the same seeded inputs go to the CUDA library
(through the C ABI) and to the FP64 oracle."""
import numpy as np

from oracle import oracle as O
from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I


def rel_err(gpu, ora):
    """|E_gpu - E_ora| / max(|E_ora|, 1) elementwise."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ora = np.asarray(ora, dtype=np.float64)
    return np.abs(gpu - ora) / np.maximum(np.abs(ora), 1.0)


def setup(pb, B, pseed=11, cseed=21, scale=0.05, params=None, occ=None):
    import torch
    if params is None:
        params = I.random_params(pb, pseed, scale)
    M0 = I.plane_wave_M0(pb)
    if occ is None:
        occ = I.random_configs(pb, B, cseed)
    ctx = Bd.make_context(pb, params, M0, max_batch=occ.shape[0])
    occ_d = torch.from_numpy(occ).cuda()
    st = torch.zeros(occ.shape[0], dtype=torch.int32, device="cuda")
    ctx.scale_load(occ_d, st)
    ora = O.Model(pb, params, M0)
    return ctx, ora, occ, st.cpu().numpy()


def conditioning(ora, occ):
    """2-norm condition number of Phi(n) per sample (oracle orbitals)."""
    _, M = ora.orbitals(occ)
    N = ora.N
    out = np.zeros(occ.shape[0])
    for b in range(occ.shape[0]):
        orbs = [s * N + i for s in range(2) for i in range(N) if (occ[b, i] >> s) & 1]
        if len(orbs) != ora.Ne:
            out[b] = np.inf
            continue
        out[b] = np.linalg.cond(M[b][orbs])
    return out


def eloc_term_scale(ora, occ):
    """|diag| + sum over connected n' of |<n|H|n'> psi(n')/psi(n)| per sample (oracle): the
    scale of the absolute error of E_loc when every ratio carries the same relative error,
    |dE| <= delta * scale. Where E_loc is a cancelling sum this exceeds |E_loc| by far."""
    la, sg = ora.log_psi(occ)
    out = np.zeros(occ.shape[0])
    for b in range(occ.shape[0]):
        xp, cf = ora.connected(occ[b])
        s = abs(ora.diag(occ[b]))
        if len(cf):
            la2, sg2 = ora.log_psi(xp)
            s += float(np.sum(np.abs(cf) * np.exp(la2 - la[b]) * (sg2 != 0)))
        out[b] = s
    return out
