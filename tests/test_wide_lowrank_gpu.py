"""GPU parity of the cached update (low-rank local energies) at the wide SCALE shapes of Table
tab:model -- SCALE-L's 13-site plus stencil or the 3x3 box as layer 0, site-wise layers up to
512 channels -- against the FP64 oracle (full recompute) and against the library's own
full-recompute path, through the C ABI.

Tolerances as for the narrow shapes: FP64 <= 1e-10 relative (cond(Phi) < 1e6); mixed <= 1e-4
of the local energy's term scale on samples with cond < 1e3, every sample within cond * c * u.
"""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, eloc_term_scale, rel_err, setup

pytestmark = pytest.mark.gpu


def _check(name, gpu, ref, cond, tol, cond_ok, min_good=1):
    err = rel_err(gpu, ref)
    good = cond < cond_ok
    unit, c = (2.0 ** -24, 8.0) if tol > 1e-8 else (2.0 ** -53, 1e3)
    print(f"{name}: n={len(err)} good={good.sum()} max_err(good)={err[good].max() if good.any() else 0:.3e} "
          f"max_err={err.max():.3e}")
    assert good.sum() >= min_good
    if good.any():
        assert err[good].max() <= tol
    assert np.all(err <= np.maximum(tol, cond * c * unit))


@pytest.mark.parametrize("variant", ["torus", "open_tj", "box_stencil_tp", "no_residual"])
def test_wide_lowrank_fp64(variant):
    """FP64, small widths (conv 6, site-wise 10): every layer on the FP64 kernels."""
    pb = I.workload("scale_l5x5")
    if variant == "open_tj":
        pb = pb.replace(pbc_y=0, model=I.MODEL_TJ, U=0.0, J=0.4, n_up=7, n_dn=7)
    elif variant == "box_stencil_tp":
        pb = pb.replace(stencil=I.STENCIL_BOX, ksize=[3, 1, 1], tp=-0.2)
    elif variant == "no_residual":
        pb = pb.replace(residual=[0, 0, 0])
    ctx, ora, occ, st = setup(pb, 48, 1270, 5720, scale=0.3)
    cond = conditioning(ora, occ)
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    _check(f"wide low-rank fp64 {variant}", e, e_o, cond, 1e-10, 1e6, min_good=24)
    e_f = ctx.local_energy(Bd.PATH_FULL).cpu().numpy()
    _check(f"wide low-rank vs full fp64 {variant}", e, e_f, cond, 1e-10, 1e6, min_good=24)


def test_wide_lowrank_mixed_8x8():
    """Mixed, plus stencil at width 96 (FP32 conv table), site-wise 128 on mma.sync TF32x3."""
    pb = I.workload("scale_l8x8")
    ctx, ora, occ, st = setup(pb, 16, 1271, 5721, scale=0.05)
    cond = conditioning(ora, occ)
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    scale = np.maximum(eloc_term_scale(ora, occ), 1.0)
    _check("scale_l8x8 low-rank E_loc / term scale", e / scale, e_o / scale, cond, 1e-4, 1e3)


def test_wide_lowrank_table_widths_8x8():
    """Table tab:model SCALE-L widths (conv 384 with the plus stencil, 4 site-wise layers of 512
    on tcgen05) on an 8x8 torus, against the oracle."""
    pb = I.workload("scale_l16x16").replace(Lx=8, Ly=8, n_up=28, n_dn=28)
    ctx, ora, occ, st = setup(pb, 4, 1272, 5722, scale=0.02)
    cond = conditioning(ora, occ)
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    scale = np.maximum(eloc_term_scale(ora, occ), 1.0)
    _check("SCALE-L widths 8x8 low-rank E_loc / term scale", e / scale, e_o / scale, cond, 1e-4, 1e3)


def test_wide_lowrank_table_widths_16x16_vs_full():
    """SCALE-L on the 16x16 torus (Table tab:model), 16 walkers: about 8,000 moves, more than one
    chunk of the row buffers holds (6,101 moves), so a chunk boundary falls inside a walker. The
    cached update against the full-recompute path of the same context (FP64 determinants; that
    path is checked against the oracle in tests/test_wide_gpu.py), relative to max(|E_loc|, 1)."""
    pb = I.workload("scale_l16x16")
    ctx, ora, occ, st = setup(pb, 16, 1273, 5723, scale=0.02)
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_f = ctx.local_energy(Bd.PATH_FULL).cpu().numpy()
    cond = conditioning(ora, occ)
    scale = np.maximum(np.abs(e_f), 1.0)
    err = np.abs(e - e_f) / scale
    print(f"SCALE-L 16x16 low-rank vs full: cond median {np.median(cond):.2e}; err median {np.median(err):.2e} "
          f"max {err.max():.2e}")
    assert np.isfinite(e).all()
    good = cond < 1e4
    assert good.sum() >= 1
    assert err[good].max() <= 1e-4
    assert np.all(err <= np.maximum(1e-4, cond * 8 * 2.0 ** -24 * 10))
