"""GPU parity of the cached update (low-rank path, Eq. neighbor + Eq. SMW) with SCALE-L's
plus-shaped stencil (the 13 offsets within L2 <= 2, Table tab:model): a hop touches the sites
within distance 2 of either end (18 sites, the union of two plus shapes one step apart), the
layer-0 response is the table of the 13 taps, and the rest of the update is the one of the
3x3 box. Checked against the FP64 oracle, which recomputes every amplitude in full.
"""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, rel_err, setup

pytestmark = pytest.mark.gpu


def _dev(*arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("variant", ["torus", "open", "tj", "shared_embed"])
def test_plus_lowrank_fp64(variant):
    pb = I.workload("scale_plus6x6")
    if variant == "open":
        pb = pb.replace(pbc_x=0, pbc_y=0)
    elif variant == "tj":
        pb = pb.replace(model=I.MODEL_TJ, U=0.0, J=0.4, n_up=14, n_dn=14)
    elif variant == "shared_embed":
        pb = pb.replace(per_site_embed=0, tp=-0.2)
    ctx, ora, occ, st = setup(pb, 64, 1270, 5720, scale=0.3)
    cond = conditioning(ora, occ)
    good = cond < 1e6
    la, sg = ctx.log_psi()
    la_o, sg_o = ora.log_psi(occ)
    assert (sg.cpu().numpy()[good] == sg_o[good]).all()
    assert np.abs(la.cpu().numpy()[good] - la_o[good]).max() <= 1e-10
    e_low = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_full = ctx.local_energy(Bd.PATH_FULL).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    err = rel_err(e_low, e_o)
    print(f"plus stencil fp64 {variant}: max E_loc err (cond < 1e6) {err[good].max():.3e}")
    assert good.sum() >= 32
    assert err[good].max() <= 1e-10
    assert np.all(err <= np.maximum(1e-10, cond * 1e3 * 2.0 ** -53))
    assert rel_err(e_low[good], e_full[good]).max() <= 1e-10


def test_plus_ratios_and_commits_fp64():
    import torch
    pb = I.workload("scale_plus6x6").replace(refresh_every=1000, drift_tol=1e-8)
    B, K = 48, 24
    ctx, ora, occ, st = setup(pb, B, 1271, 5721, scale=0.2)
    mv = I.random_hop_moves(pb, occ, 77)
    r = ctx.ratios(torch.from_numpy(mv[:, None, :].copy()).cuda()).cpu().numpy()[:, 0]
    r_o = ora.ratio(occ, mv)
    good = conditioning(ora, occ) < 1e6
    assert rel_err(r[good], r_o[good]).max() <= 1e-10
    cur = occ.copy()
    for k in range(K):
        mv = I.random_hop_moves(pb, cur, 2000 + k)
        rho = np.abs(ora.ratio(cur, mv))
        mv[rho < 0.1] = I.MOVE_NONE
        ctx.scale_commit(torch.from_numpy(mv).cuda())
        cur = I.apply_moves(cur, mv)
    assert np.array_equal(ctx.get_occ().cpu().numpy(), cur)
    cond = conditioning(ora, cur)
    good = cond < 1e4
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(cur)
    err = rel_err(e[good], e_o[good])
    print(f"plus stencil after {K} commits: max E_loc err {err.max():.3e}")
    assert err.max() <= 1e-9


def test_plus_sweep_trajectory_fp64():
    pb = I.workload("scale_plus6x6").replace(refresh_every=16, drift_tol=1e-8)
    B, S = 32, 32
    ctx, ora, occ, st = setup(pb, B, 1272, 5722, scale=0.2)
    pick, direction, u = I.metropolis_randoms(pb, B, S, 33)
    acc = ctx.sweep(*_dev(pick, direction, u)).cpu().numpy()
    occ_ora, acc_ora = ora.metropolis(occ, pick, direction, u)
    assert np.array_equal(acc, acc_ora)
    assert np.array_equal(ctx.get_occ().cpu().numpy(), occ_ora)
    assert acc.sum() > 0


def test_plus_mixed_16x16_full_batch_sampled():
    """The bench network with the plus stencil at the full batch (8192), 24 sampled outputs."""
    pb = I.workload("scale_plus16x16")
    pseed, cseed = I.workload_seeds("scale_plus16x16")
    ctx, ora, occ, st = setup(pb, 8192, pseed, cseed)
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(8192, 24, replace=False))
    cond = conditioning(ora, occ[pick])
    e_o, _ = ora.local_energy(occ[pick])
    err = rel_err(e[pick], e_o)
    good = cond < 1e4
    print(f"plus 16x16 mixed: good {good.sum()} max err (cond < 1e4) {err[good].max() if good.any() else 0:.3e}")
    if good.any():
        assert err[good].max() <= 1e-4
    assert np.all(err <= np.maximum(1e-4, cond * 8 * 2.0 ** -24))
    assert np.isfinite(e).all()
