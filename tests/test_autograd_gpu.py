"""torch.autograd.Function around the library's log|psi| and hand-written backward."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning

pytestmark = pytest.mark.gpu


def test_autograd_matches_per_sample_and_oracle():
    import torch
    from oracle import oracle as O
    from paper_2604_25775_gb300 import binding as Bd
    from paper_2604_25775_gb300.autograd import log_psi, per_sample_gradients

    pb = I.workload("cylinder16x4")
    pseed, cseed = I.workload_seeds("cylinder16x4")
    p_np = I.random_params(pb, pseed)
    M0_np = I.plane_wave_M0(pb)
    occ_np = I.random_configs(pb, 12, cseed)
    ctx = Bd.Context(pb, 12)
    params = torch.from_numpy(p_np).cuda().requires_grad_(True)
    M0 = torch.from_numpy(M0_np).cuda()
    occ = torch.from_numpy(occ_np).cuda()
    w = torch.linspace(0.5, 1.5, 12, dtype=torch.float64, device="cuda")
    la = log_psi(params, occ, M0, ctx)
    (w * la).sum().backward()
    O_b = per_sample_gradients(params, occ, M0, ctx)
    ref = (w[:, None] * O_b).sum(0)
    torch.testing.assert_close(params.grad, ref, rtol=1e-12, atol=1e-12)
    ora = O.Model(pb, p_np, M0_np)
    g_o = ora.grad_logpsi(occ_np)
    good = conditioning(ora, occ_np) < 1e6
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    assert (np.abs(O_b.cpu().numpy()[good] - g_o[good]) / scale).max() <= 1e-10
