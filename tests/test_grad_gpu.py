"""GPU per-sample gradients d log|psi| / d theta against the FP64 oracle's backward pass and
against central finite differences of the GPU's own log|psi| (16x4 cylinder, 12 residual
3x3 layers, t' = -0.2)."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, setup

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recompute", [False, True])
def test_grad_matches_oracle_fp64(recompute):
    pb = I.workload("cylinder16x4")
    pseed, cseed = I.workload_seeds("cylinder16x4")
    ctx, ora, occ, st = setup(pb, 32, pseed, cseed)
    g = ctx.grad_logpsi(recompute=recompute).cpu().numpy()
    g_o = ora.grad_logpsi(occ)
    cond = conditioning(ora, occ)
    good = cond < 1e6
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    err = np.abs(g[good] - g_o[good]) / scale
    print(f"grad recompute={recompute}: max rel err {err.max():.3e}")
    assert err.max() <= 1e-10


def test_grad_mixed_8x8():
    """Mixed mode (FP32 network and inverse): gradients within 1e-4 of the FP64 oracle,
    relative to the largest gradient entry of the sample, for cond(Phi) <= 1e3."""
    pb = I.workload("hubbard8x8")
    ctx, ora, occ, st = setup(pb, 32, 3, 4)
    g = ctx.grad_logpsi().cpu().numpy()
    g_o = ora.grad_logpsi(occ)
    cond = conditioning(ora, occ)
    good = cond < 1e3
    assert good.sum() >= 4
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    err = (np.abs(g[good] - g_o[good]) / scale).max()
    print(f"grad mixed 8x8: max rel err {err:.3e}")
    assert err <= 1e-4


@pytest.mark.parametrize("recompute", [False, True])
def test_grad_mixed_cylinder(recompute):
    """Mixed mode on the gradient workload (16x4 cylinder, 12 residual 3x3 layers, t' = -0.2):
    within 1e-4 of the FP64 oracle relative to the sample's largest entry for cond(Phi) <= 1e3.
    The output is filled with NaN first: every entry must be written by the call."""
    import torch
    pb = I.workload("cylinder16x4").replace(precision=I.PREC_MIXED)
    pseed, cseed = I.workload_seeds("cylinder16x4")
    ctx, ora, occ, st = setup(pb, 32, pseed, cseed)
    g_d = torch.full((ctx.B, ctx.P), float("nan"), dtype=torch.float64, device="cuda")
    ctx.scale_grad_logpsi(g_d, recompute)
    g = g_d.cpu().numpy()
    ok = st == 0
    assert np.isfinite(g[ok]).all()
    g_o = ora.grad_logpsi(occ)
    cond = conditioning(ora, occ)
    good = ok & (cond < 1e3)
    assert good.sum() >= 4
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    err = (np.abs(g[good] - g_o[good]) / scale).max()
    print(f"grad mixed cylinder recompute={recompute}: max rel err {err:.3e} ({good.sum()} samples)")
    assert err <= 1e-4


def test_grad_width_not_multiple_of_four_fp64():
    """h = 6: the per-element kernels (the tiled ones need h % 4 == 0), FP64, against the oracle;
    NaN-filled output as above."""
    import torch
    pb = I.workload("hubbard4x4").replace(h=6)
    ctx, ora, occ, st = setup(pb, 16, 11, 12)
    g_d = torch.full((ctx.B, ctx.P), float("nan"), dtype=torch.float64, device="cuda")
    ctx.scale_grad_logpsi(g_d, False)
    g = g_d.cpu().numpy()
    g_o = ora.grad_logpsi(occ)
    cond = conditioning(ora, occ)
    good = (st == 0) & (cond < 1e6)
    assert good.sum() >= 4
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    err = (np.abs(g[good] - g_o[good]) / scale).max()
    print(f"grad h=6 fp64: max rel err {err:.3e}")
    assert err <= 1e-10


def test_grad_central_differences_gpu():
    """Central differences (h = 1e-6, FP64) of the GPU log|psi| on 20 random parameters."""
    import torch
    from paper_2604_25775_gb300 import binding as Bd
    pb = I.workload("cylinder16x4")
    pseed, cseed = I.workload_seeds("cylinder16x4")
    params = I.random_params(pb, pseed)
    occ = I.random_configs(pb, 16, cseed)
    ctx, ora, _, _ = setup(pb, 16, params=params, occ=occ)
    g = ctx.grad_logpsi().cpu().numpy()
    M0 = I.plane_wave_M0(pb)
    occ_d = torch.from_numpy(occ).cuda()
    rng = np.random.default_rng(7)
    idx = rng.choice(params.size, 20, replace=False)
    h = 1e-6
    for q in idx:
        vals = []
        for sgn in (1, -1):
            p2 = params.copy()
            p2[q] += sgn * h
            c2 = Bd.make_context(pb, p2, M0, 16)
            c2.scale_load(occ_d)
            vals.append(c2.log_psi()[0].cpu().numpy())
            c2.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        np.testing.assert_allclose(g[:, q], fd, rtol=2e-5, atol=2e-7)


@pytest.mark.parametrize("variant", ["torus_fp64", "open_fp64", "mixed"])
def test_grad_plus_stencil(variant):
    """SCALE-L's 13-site plus stencil in layer 0 (weights per tap): gradients against the
    oracle's backward pass, FP64 within 1e-10 and mixed within 1e-4 of each sample's largest
    entry."""
    pb = I.workload("scale_plus6x6")
    if variant == "open_fp64":
        pb = pb.replace(pbc_x=0, tp=-0.2)
    elif variant == "mixed":
        pb = pb.replace(precision=I.PREC_MIXED)
    ctx, ora, occ, st = setup(pb, 24, 1273, 5723, scale=0.3)
    g = ctx.grad_logpsi().cpu().numpy()
    g_o = ora.grad_logpsi(occ)
    cond = conditioning(ora, occ)
    tol, cond_ok = (1e-4, 1e3) if variant == "mixed" else (1e-10, 1e6)
    good = cond < cond_ok
    assert good.sum() >= 4
    scale = np.maximum(np.abs(g_o[good]).max(axis=1, keepdims=True), 1.0)
    err = (np.abs(g[good] - g_o[good]) / scale).max()
    print(f"grad plus stencil {variant}: max rel err {err:.3e}")
    assert err <= tol

