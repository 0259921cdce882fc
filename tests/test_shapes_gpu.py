"""GPU parity at the edges of the supported shapes: the widest network (h = 64, tensor-core
layers in mixed precision), a width off the tensor-core tiles (h = 12), a width whose rows
are not whole 16-byte chunks (h = 3), a single layer (no site-wise layers), a 1x1 first layer
(the affected set is the two touched sites), a lattice open on both axes, one-walker and
empty batches, and the degenerate sectors: a completely filled lattice (no move exists,
E_loc = U N exactly) and a fully polarised one (no down electrons)."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, eloc_term_scale, rel_err, setup

pytestmark = pytest.mark.gpu


def _pb(name):
    base = I.Problem(6, 5, 1, 1, 9, 8, I.MODEL_HUBBARD, 1.0, 0.0, 6.0, 0.0, 3, 8, [3, 1, 1], [1, 0, 0])
    return {
        "h64_fp64": base.replace(h=64),
        "h64_mixed": base.replace(h=64, precision=I.PREC_MIXED),
        "h12_mixed": base.replace(h=12, precision=I.PREC_MIXED),
        "h3_fp64": base.replace(h=3),
        "one_layer": base.replace(n_layers=1, ksize=[3], residual=[1]),
        "one_layer_mixed": base.replace(n_layers=1, ksize=[3], residual=[1], precision=I.PREC_MIXED),
        "k1_first_layer": base.replace(ksize=[1, 1, 1]),
        "open_3x3": base.replace(Lx=3, Ly=3, pbc_x=0, pbc_y=0, n_up=3, n_dn=2, tp=-0.3),
    }[name]


@pytest.mark.parametrize("name", ["h64_fp64", "h64_mixed", "h12_mixed", "h3_fp64", "one_layer",
                                  "one_layer_mixed", "k1_first_layer", "open_3x3"])
def test_local_energy_at_shape_edges(name):
    pb = _pb(name)
    mixed = pb.precision != I.PREC_FP64
    ctx, ora, occ, st = setup(pb, 40, 21, 22, scale=0.15)
    cond = conditioning(ora, occ)
    e1 = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e2 = ctx.local_energy(Bd.PATH_FULL).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    good = cond < (1e3 if mixed else 1e6)
    tol = 1e-4 if mixed else 1e-10
    assert good.sum() >= 5
    err1, err2 = rel_err(e1, e_o), rel_err(e2, e_o)
    print(f"{name}: lowrank {err1[good].max():.3e}, full {err2[good].max():.3e} ({good.sum()} of {len(good)})")
    assert err1[good].max() <= tol and err2[good].max() <= tol
    la, sg = ctx.log_psi()
    la_o, sg_o = ora.log_psi(occ)
    assert (sg.cpu().numpy()[good] == sg_o[good]).all()
    assert rel_err(la.cpu().numpy()[good], la_o[good]).max() <= tol


def test_one_walker_and_empty_batch():
    import torch
    pb = I.workload("hubbard8x8").replace(precision=I.PREC_FP64)
    ctx, ora, occ, st = setup(pb, 1, 3, 4, scale=0.1)
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    assert rel_err(e, e_o).max() <= 1e-9
    with pytest.raises(Bd.ScaleError):
        ctx.scale_load(torch.zeros((0, pb.N), dtype=torch.int8, device="cuda"))
    with pytest.raises(Bd.ScaleError):
        ctx.scale_load(torch.from_numpy(np.repeat(occ, 2, axis=0)).cuda())  # more than max_batch


def test_filled_lattice_has_no_moves():
    """Every orbital occupied: no hop exists and E_loc = U N, psi = det of the full M."""
    ks, rs = I.scale_layout(2)
    pb = I.Problem(3, 3, 1, 1, 9, 9, I.MODEL_HUBBARD, 1.0, 0.0, 5.0, 0.0, 2, 8, ks, rs)
    ctx, ora, occ, st = setup(pb, 2, 3, 4, scale=0.1)
    assert (occ == 3).all()
    e = ctx.local_energy().cpu().numpy()
    np.testing.assert_allclose(e, 5.0 * 9, rtol=0, atol=1e-12)
    la, sg = ctx.log_psi()
    la_o, sg_o = ora.log_psi(occ)
    assert rel_err(la.cpu().numpy(), la_o).max() <= 1e-10


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_MIXED])
def test_fully_polarised_sector(prec):
    pb = I.Problem(6, 5, 1, 1, 11, 0, I.MODEL_HUBBARD, 1.0, -0.2, 6.0, 0.0, 3, 16, [3, 1, 1], [1, 0, 0],
                   precision=prec)
    ctx, ora, occ, st = setup(pb, 40, 5, 6, scale=0.15)
    cond = conditioning(ora, occ)
    good = cond < (1e6 if prec == I.PREC_FP64 else 1e3)
    e = ctx.local_energy().cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    assert good.sum() >= 5
    tol = 1e-10 if prec == I.PREC_FP64 else 1e-4
    # Some configurations here give E_loc as a strongly cancelling sum (sum |terms| up to
    # 100 |E_loc|); the error of each ratio then scales with the terms, not with E_loc.
    scale = eloc_term_scale(ora, occ)
    amp = scale / np.maximum(np.abs(e_o), 1.0)
    err_terms = np.abs(e - e_o) / np.maximum(scale, 1.0)
    err_e = rel_err(e, e_o)
    print(f"polarised prec={prec}: max err / sum|terms| {err_terms[good].max():.3e}; "
          f"max rel err (amplification <= 10) {err_e[good & (amp <= 10)].max():.3e}")
    assert err_terms[good].max() <= tol
    assert err_e[good & (amp <= 10)].max() <= tol
