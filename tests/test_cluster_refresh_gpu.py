"""The FP64 refresh of matrices above 448 rows runs on an 8-CTA thread-block cluster per
matrix (dense_inverse.cu, k_gj_cluster); loading runs one CTA per matrix (k_gj). Both apply
the same operations to every element in the same order, so a forced refresh right after a
load must reproduce the load's log|psi|, sign and low-rank ratios bit for bit; log|psi| is
also checked against the oracle (Sec. II.C: one LU gives the determinant and the inverse)."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, rel_err, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_MIXED])
def test_cluster_refresh_reproduces_single_cta_load(prec):
    import torch
    ks, rs = I.scale_layout(2)
    pb = I.Problem(24, 24, 1, 1, 230, 230, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 8, ks, rs,
                   I.ACT_TANH, 1, prec, 64, 1e-4)
    assert pb.Ne > 448
    B = 4
    ctx, ora, occ, st = setup(pb, B, 3, 4, scale=0.05)  # load: one CTA per matrix
    la1, sg1 = ctx.log_psi()
    mv = np.ascontiguousarray(np.stack([I.random_hop_moves(pb, occ, 50 + k) for k in range(3)], axis=1))
    mv_d = torch.from_numpy(mv).cuda()
    r1 = ctx.ratios(mv_d)
    ctx.scale_refresh(True)  # listed refresh of every sample: the cluster kernel
    la2, sg2 = ctx.log_psi()
    r2 = ctx.ratios(mv_d)
    assert torch.equal(sg1, sg2)
    assert torch.equal(la1, la2)
    assert torch.equal(r1, r2)
    la_o, sg_o = ora.log_psi(occ)
    cond = conditioning(ora, occ)
    good = cond < 1e8
    assert good.any()
    assert (sg2.cpu().numpy()[good] == sg_o[good]).all()
    err = rel_err(la2.cpu().numpy()[good], la_o[good]).max()
    print(f"n={pb.Ne}: log|psi| rel err {err:.3e}, cond max {cond.max():.2e}")
    # FP64: the LU in FP64 on an FP64 Phi; mixed: Phi itself comes from the FP32 network
    assert err <= (1e-10 * max(1.0, cond[good].max() / 1e4) if prec == I.PREC_FP64 else 1e-4)
