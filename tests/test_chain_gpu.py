"""GPU chain path: Woodbury commits (Eq. SMW, second line), FP64 refresh and drift check,
checked against the oracle recomputing every amplitude from the final configurations."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, rel_err, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol,refresh", [(I.PREC_FP64, 1e-9, 1000), (I.PREC_FP64, 1e-9, 7),
                                               (I.PREC_MIXED, 1e-4, 16), (I.PREC_MIXED_FP16, 1e-4, 16),
                                               (I.PREC_MIXED_BF16, 5e-4, 16)])
def test_commits_match_oracle(prec, tol, refresh):
    import torch
    pb = I.workload("hubbard8x8").replace(precision=prec, refresh_every=refresh, tp=-0.2,
                                          drift_tol=1e-8 if prec == I.PREC_FP64 else 1e-3)
    B, K = 64, 40
    ctx, ora, occ, st = setup(pb, B, 5, 6, scale=0.1)
    cur = occ.copy()
    min_ratio = np.inf
    for k in range(K):
        mv = I.random_hop_moves(pb, cur, 1000 + k)
        # commit the moves a Metropolis chain plausibly accepts (|psi'/psi| >= 0.1, acceptance
        # >= 1%): a Woodbury step through a near-singular capacitance matrix loses about
        # log10(1/|det R|) digits, which is the conditioning of that step, not of the update
        rho = np.abs(ora.ratio(cur, mv))
        mv[rho < 0.1] = I.MOVE_NONE
        min_ratio = min(min_ratio, rho[mv[:, 0] >= 0].min(initial=np.inf))
        ctx.scale_commit(torch.from_numpy(mv).cuda())
        cur = I.apply_moves(cur, mv)
    occ_gpu = ctx.get_occ().cpu().numpy()
    assert np.array_equal(occ_gpu, cur)
    assert min_ratio >= 0.1
    cond = conditioning(ora, cur)
    good = cond < (1e6 if prec == I.PREC_FP64 else 1e3)
    la, sg = ctx.log_psi()
    la_o, sg_o = ora.log_psi(cur)
    assert (sg.cpu().numpy()[good] == sg_o[good]).all()
    # Forward error of K rank-r Woodbury steps grows like K cond(Phi) u (u the unit roundoff of
    # the update precision): FP64 samples with cond < 1e4 meet the flat tolerance, every sample
    # kept meets max(tol, K cond u). Mixed mode keeps the flat band of the other mixed tests.
    if prec == I.PREC_FP64:
        bound = np.maximum(tol, K * cond[good] * 2.0 ** -52)
        tight = cond[good] < 1e4
    else:
        bound = np.full(int(good.sum()), tol)
        tight = np.ones(int(good.sum()), dtype=bool)
    la_err = rel_err(la.cpu().numpy()[good], la_o[good])
    print(f"prec={prec} refresh={refresh}: max log|psi| rel err after {K} commits = {la_err.max():.3e}")
    assert (la_err <= bound).all() and la_err[tight].max() <= tol
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(cur)
    err = rel_err(e[good], e_o[good])
    print(f"prec={prec} refresh={refresh}: max E_loc err after {K} commits = {err.max():.3e} "
          f"(cond < 1e4: {err[tight].max():.3e})")
    assert (err <= bound).all() and err[tight].max() <= tol
    stats = ctx.scale_get_stats()
    assert stats["n_commits"] > 0
    if refresh < K:
        assert stats["n_refresh"] >= B * (K // refresh) // 2


def test_exchange_commits_tj():
    import torch
    pb = I.workload("tj8x8").replace(precision=I.PREC_FP64, refresh_every=1000)
    B = 16
    ctx, ora, occ, st = setup(pb, B, 8, 9, scale=0.1)
    cur = occ.copy()
    rng = np.random.default_rng(4)
    for k in range(10):
        mv = np.full((B, 4), -1, dtype=np.int32)
        for b in range(B):
            for _ in range(200):
                i = int(rng.integers(pb.N))
                x, y = i % pb.Lx, i // pb.Lx
                j = y * pb.Lx + (x + 1) % pb.Lx
                if {int(cur[b, i]), int(cur[b, j])} == {1, 2}:
                    mv[b] = (I.MOVE_EXCHANGE, i, j, 0)
                    break
        ctx.scale_commit(torch.from_numpy(mv).cuda())
        cur = I.apply_moves(cur, mv)
    assert np.array_equal(ctx.get_occ().cpu().numpy(), cur)
    cond = conditioning(ora, cur)
    good = cond < 1e6
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(cur)
    assert rel_err(e[good], e_o[good]).max() <= 1e-9


def test_drift_check_forces_refresh():
    """A drift threshold below FP32 rounding makes every commit trigger an FP64 refresh."""
    import torch
    pb = I.workload("hubbard8x8").replace(refresh_every=10 ** 6, drift_tol=1e-12)
    B = 32
    ctx, ora, occ, st = setup(pb, B, 5, 6, scale=0.1)
    mv = I.random_hop_moves(pb, occ, 3)
    ctx.scale_commit(torch.from_numpy(mv).cuda())
    stats = ctx.scale_get_stats()
    n_moved = int((mv[:, 0] >= 0).sum())
    assert stats["n_drift_refresh"] >= n_moved // 2
    assert stats["drift_max"] > 1e-12
