"""GPU Metropolis sweep (scale_sweep): hop proposals, the rank-r ratio against the cached
inverse, acceptance u < |psi'/psi|^2 and the Woodbury commit of accepted moves, checked
against the oracle's Metropolis step on the same random numbers (Sec. II.A: configurations
sampled from |psi|^2 by local updates)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, rel_err, setup

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("name", ["hubbard8x8", "tj8x8"])
def test_sweep_trajectory_matches_oracle_fp64(name):
    """FP64: the acceptance decisions are taken in FP64 on both sides, so every chain must
    end in the same configuration with the same number of accepted steps."""
    pb = I.workload(name).replace(precision=I.PREC_FP64, refresh_every=16, drift_tol=1e-8)
    B, S = 64, 48
    ctx, ora, occ, st = setup(pb, B, 7, 8, scale=0.1)
    pick, direction, u = I.metropolis_randoms(pb, B, S, 31)
    acc = ctx.sweep(*_dev(pick, direction, u)).cpu().numpy()
    occ_gpu = ctx.get_occ().cpu().numpy()
    occ_ora, acc_ora = ora.metropolis(occ, pick, direction, u)
    print(f"{name}: acceptance {acc.mean() / S:.3f}")
    assert np.array_equal(acc, acc_ora)
    assert np.array_equal(occ_gpu, occ_ora)
    assert acc.sum() > 0 and (acc < S).any()
    cond = conditioning(ora, occ_gpu)
    good = cond < 1e6
    la, sg = ctx.log_psi()
    la_o, sg_o = ora.log_psi(occ_gpu)
    assert (sg.cpu().numpy()[good] == sg_o[good]).all()
    assert rel_err(la.cpu().numpy()[good], la_o[good]).max() <= 1e-9
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(occ_gpu)
    tight = cond < 1e4
    err = rel_err(e, e_o)
    print(f"{name}: E_loc after the sweep, max err (cond < 1e4) {err[tight].max():.3e}")
    assert err[tight].max() <= 1e-9
    assert (err[good] <= np.maximum(1e-9, S * cond[good] * 2.0 ** -52)).all()


def test_sweep_mixed_single_step_decisions():
    """Mixed precision: det R in FP32, so decisions are compared where they are not within
    the FP32 ratio error of the threshold; the rest must still be valid moves."""
    pb = I.workload("hubbard8x8")
    B = 512
    ctx, ora, occ, st = setup(pb, B, 7, 9, scale=0.1)
    pick, direction, u = I.metropolis_randoms(pb, B, 1, 41)
    acc = ctx.sweep(*_dev(pick, direction, u)).cpu().numpy()
    occ_gpu = ctx.get_occ().cpu().numpy()
    occ_ora, acc_ora = ora.metropolis(occ, pick, direction, u)
    # the oracle's |psi'/psi|^2 of each proposal, to tell ambiguous decisions apart
    occ_prop, acc_all = ora.metropolis(occ, pick, direction, np.zeros_like(u))
    la0, _ = ora.log_psi(occ)
    la1, _ = ora.log_psi(occ_prop)
    rho2 = np.exp(2 * (la1 - la0))
    cond = conditioning(ora, occ)
    clear = (np.abs(u[0] - rho2) > 1e-3 * np.maximum(rho2, u[0])) & (cond < 1e3)
    print(f"mixed: {clear.sum()} of {B} decisions away from the threshold")
    assert clear.sum() > B // 4
    assert np.array_equal(acc[clear], acc_ora[clear])
    assert np.array_equal(occ_gpu[clear], occ_ora[clear])
    # every chain ends either where it started or at its proposal
    same = (occ_gpu == occ).all(1)
    moved = (occ_gpu == occ_prop).all(1) & (acc_all == 1)
    assert (same | moved).all()
    assert np.array_equal(acc == 1, moved & ~same)


def test_sweep_stationary_distribution_tiny_torus():
    """End to end on a 3x3 torus (1 up + 1 down, 81 states): the chains' histogram is
    |psi|^2 from complete enumeration by the oracle, and is far from |psi|."""
    ks, rs = I.scale_layout(2)
    pb = I.Problem(3, 3, 1, 1, 1, 1, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 4, ks, rs, I.ACT_TANH, 1,
                   I.PREC_FP64, 64, 1e-8)
    xs = O.all_configurations(pb)
    B = 8192
    rng = np.random.default_rng(3)
    occ0 = xs[rng.integers(len(xs), size=B)]
    ctx, ora, occ, st = setup(pb, B, 5, 0, scale=0.8, occ=occ0)
    la, sg = ora.log_psi(xs)
    assert (sg != 0).all()
    p2 = np.exp(2 * (la - la.max()))
    p2 /= p2.sum()
    p1 = np.exp(la - la.max())
    p1 /= p1.sum()
    assert 0.5 * np.abs(p2 - p1).sum() > 0.1
    key = {x.tobytes(): n for n, x in enumerate(xs)}
    counts = np.zeros(len(xs))
    for c in range(12):
        pick, direction, u = I.metropolis_randoms(pb, B, 16, 500 + c)
        ctx.sweep(*_dev(pick, direction, u))
        if c >= 2:
            for x in ctx.get_occ().cpu().numpy():
                counts[key[x.tobytes()]] += 1
    emp = counts / counts.sum()
    tvd = 0.5 * np.abs(emp - p2).sum()
    tvd1 = 0.5 * np.abs(emp - p1).sum()
    print(f"tiny torus: TVD(empirical, |psi|^2) = {tvd:.4f}, TVD(empirical, |psi|) = {tvd1:.4f}")
    assert tvd < 0.03
    assert tvd1 > 2 * tvd
