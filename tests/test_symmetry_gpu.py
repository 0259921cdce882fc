"""GPU parity of the symmetry-projected amplitude psi_sym(n) = sum_g Pi(n, g) chi_g psi(g n)
(App. "Symmetry Projection") against the FP64 oracle, through the C ABI.

psi_sym is a signed sum of |G| amplitudes and can cancel, so the error is measured against
the sum of the magnitudes of its terms, S(n) = sum_g |psi(g n)| (oracle):
    |psi_sym_gpu - psi_sym_ora| / S  <=  1e-10 (FP64) or 1e-4 (mixed)
on samples whose terms' magnitude-weighted cond(Phi(g n)) is below 1e6 (FP64) / 1e3 (mixed),
and below cond * c * u for the rest (u = 2^-53 with c = 1e3, or 2^-24 with c = 8, as for
log psi).
"""
import numpy as np
import pytest

from paper_2604_25775_gb300 import inputs as I
from tests.gpu_common import conditioning, setup

pytestmark = pytest.mark.gpu


def _images(pb, occ, perm):
    """g n of every sample for one orbital map (orbital o goes to perm[o]). A sample whose
    occupied orbitals are not sent one-to-one into [0, 2N) gets the empty configuration,
    which lies outside every particle-number sector (no term)."""
    N = pb.N
    on = np.concatenate([(occ >> 0) & 1, (occ >> 1) & 1], axis=1).astype(bool)  # [B][2N]
    out = np.zeros((occ.shape[0], 2 * N), dtype=np.int64)
    for b in range(occ.shape[0]):
        img = perm[on[b]]
        if img.min() < 0 or img.max() >= 2 * N or len(set(img.tolist())) != len(img):
            continue
        out[b, img] = 1
    return (out[:, :N] + 2 * out[:, N:]).astype(np.int8)


def _term_scale(pb, ora, occ, perms):
    """log S(n) and the magnitude-weighted condition number of the terms,
    sum_g |psi(g n)| cond(Phi(g n)) / S(n): each term carries a relative error of about
    cond * u, so the error of the sum relative to S is about this weighted cond times u."""
    la = np.stack([ora.log_psi(_images(pb, occ, p))[0] for p in perms])  # [G][B]
    cond = np.stack([conditioning(ora, _images(pb, occ, p)) for p in perms])
    cond[~np.isfinite(la)] = 1.0  # images outside the space: no term
    m = np.max(la, axis=0)
    w = np.exp(la - m)
    logS = m + np.log(np.sum(w, axis=0))
    return logS, np.sum(w * cond, axis=0) / np.sum(w, axis=0)


def _compare(name, pb, ctx, ora, occ, perms, chi, tol, cond_ok, min_good=None):
    import torch
    la, sg = ctx.log_psi_sym(torch.from_numpy(perms).cuda(), torch.from_numpy(chi).cuda())
    la, sg = la.cpu().numpy(), sg.cpu().numpy()
    la_o, sg_o = ora.log_psi_sym(occ, perms, chi)
    logS, cond = _term_scale(pb, ora, occ, perms)
    err = np.abs(sg * np.exp(la - logS) - sg_o * np.exp(la_o - logS))
    mixed = tol > 1e-8
    unit, c = (2.0 ** -24, 8.0) if mixed else (2.0 ** -53, 1e3)
    good = cond < cond_ok
    print(f"{name}: G={len(perms)} n={len(err)} good={good.sum()} max_err/S={err.max():.3e} "
          f"weighted cond max={cond.max():.2e} cancel(|psi_sym|/S) min={np.exp(la_o - logS).min():.2e}")
    assert good.sum() >= (min_good if min_good is not None else max(1, len(err) // 4))
    assert err[good].max() <= tol
    assert np.all(err <= np.maximum(tol, cond * c * unit))
    # the sign is decided where the sum is not lost to rounding
    clear = good & (np.exp(la_o - logS) > 100 * tol)
    assert (sg[clear] == sg_o[clear]).all()
    return la, sg


def _momentum_pi(pb, perms):
    """Characters of the (pi, pi) representation of the translations: (-1)^(tx + ty), read
    from where each translation sends site 0."""
    return np.array([(-1.0) ** ((int(p[0]) % pb.Lx) + (int(p[0]) // pb.Lx)) for p in perms])


@pytest.mark.parametrize("momentum", [False, True])
def test_sym_fp64_4x4_full_group(momentum):
    pb = I.workload("hubbard4x4")  # 7+7: spin inversion maps the sector onto itself
    ctx, ora, occ, _ = setup(pb, 64, 1240, 5690)
    perms = I.symmetry_group(pb, translations=True, reflections=not momentum, spin_inversion=not momentum)
    chi = _momentum_pi(pb, perms) if momentum else np.ones(len(perms))
    _compare("fp64 4x4", pb, ctx, ora, occ, perms, chi, 1e-10, 1e6)


def test_sym_trivial_group_is_log_psi():
    pb = I.workload("hubbard4x4")
    ctx, ora, occ, _ = setup(pb, 64, 1241, 5691)
    ident = I.symmetry_group(pb, translations=False)
    la, sg = _compare("fp64 identity", pb, ctx, ora, occ, ident, np.ones(1), 1e-10, 1e6)
    la0, sg0 = ctx.log_psi()
    la0, sg0 = la0.cpu().numpy(), sg0.cpu().numpy()
    ok = np.isfinite(la0)
    assert (sg[ok] == sg0[ok]).all()
    assert np.abs(la[ok] - la0[ok]).max() <= 1e-10


def test_sym_leaves_the_cache():
    """The projection evaluates fresh configurations in scratch: local energies of the
    loaded samples afterwards still match the oracle."""
    import torch
    pb = I.workload("hubbard4x4")
    ctx, ora, occ, _ = setup(pb, 32, 1242, 5692)
    perms = I.symmetry_group(pb, reflections=True)
    ctx.log_psi_sym(torch.from_numpy(perms).cuda(), torch.ones(len(perms), dtype=torch.float64, device="cuda"))
    from paper_2604_25775_gb300 import binding as Bd
    e = ctx.local_energy(Bd.PATH_LOWRANK).cpu().numpy()
    e_o, _ = ora.local_energy(occ)
    assert np.max(np.abs(e - e_o) / np.maximum(np.abs(e_o), 1.0)) <= 1e-10


def test_sym_images_outside_the_space():
    """Spin inversion with n_up != n_dn leaves the sector: those terms vanish on both sides."""
    pb = I.workload("hubbard_ph8x8")  # 28 + 36
    ctx, ora, occ, _ = setup(pb, 16, 1243, 5693)
    perms = I.symmetry_group(pb, translations=True, spin_inversion=True)
    _compare("ph8x8 + spin inversion", pb, ctx, ora, occ, perms, np.ones(len(perms)), 1e-4, 1e3)


def test_sym_maps_that_are_not_permutations():
    """A map sending two occupied orbitals onto one, or an occupied orbital past 2N, gives
    no term for that sample; where the offending entries meet only empty orbitals the map
    still relabels the electrons and its term counts."""
    pb = I.workload("hubbard4x4")
    ctx, ora, occ, _ = setup(pb, 64, 1246, 5696)
    N = pb.N
    ident = np.arange(2 * N, dtype=np.int32)
    merge, past, shift = ident.copy(), ident.copy(), I.symmetry_group(pb)[5]
    merge[1] = 0
    past[5] = 2 * N + 3
    perms = np.stack([ident, merge, past, shift]).astype(np.int32)
    chi = np.array([1.0, -0.5, 2.0, 1.0])
    _compare("fp64 non-permutations", pb, ctx, ora, occ, perms, chi, 1e-10, 1e6)


@pytest.mark.parametrize("name,reflections", [("tj8x8", True), ("hubbard8x8", False)])
def test_sym_mixed_8x8(name, reflections):
    pb = I.workload(name)
    ctx, ora, occ, _ = setup(pb, 24, 1244, 5694)
    perms = I.symmetry_group(pb, translations=True, reflections=reflections, spin_inversion=True)
    _compare(f"mixed {name}", pb, ctx, ora, occ, perms, np.ones(len(perms)), 1e-4, 1e3)


def test_sym_mixed_16x16_translations():
    pb = I.workload("hubbard16x16")
    ctx, ora, occ, _ = setup(pb, 6, 1245, 5695)
    perms = I.symmetry_group(pb, translations=True)
    # uniformly random 16x16 configurations have cond(Phi) >= 1e3: the strict band is 1e4 here
    _compare("mixed 16x16", pb, ctx, ora, occ, perms, _momentum_pi(pb, perms), 1e-4, 1e4, min_good=2)


def test_sym_single_walker_and_single_element():
    """One walker, and a group of one translation (no identity): psi_sym = Pi psi(t n)."""
    pb = I.workload("hubbard4x4")
    ctx, ora, occ, _ = setup(pb, 1, 1247, 5697)
    perms = I.symmetry_group(pb)[3:4].copy()
    _compare("fp64 single", pb, ctx, ora, occ, perms, np.array([-1.0]), 1e-10, 1e6, min_good=0)
