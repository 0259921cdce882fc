"""CPU pins of the oracle's symmetry-projected amplitude (App. "Symmetry Projection"):
psi_sym(n) = sum_g Pi(n, g) chi_g psi(g n), with Pi the fermionic sign of relabelling the
occupied orbitals. Pins: the trivial group gives psi itself; the projection identity
psi_sym(h n) Pi(n, h) = chi_h psi_sym(n) for every group element h (it holds for any psi
exactly when the signs compose as fermion operators do, Pi(n, g h) = Pi(h n, g) Pi(n, h),
so a wrong sign convention or a wrong direction of the group action breaks it); and the
group generator's closure."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I

_KS, _RS = I.scale_layout(2)
TORUS = I.Problem(4, 4, 1, 1, 3, 3, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 4, _KS, _RS)


def _model(pb, seed=7, scale=0.4):
    M0 = np.random.default_rng(seed).normal(size=(2 * pb.N, pb.Ne))
    return O.Model(pb, I.random_params(pb, seed, scale), M0)


def _act(pb, perm, x):
    """(g n, Pi(n, g)) written out directly: the image of every occupied orbital, and the
    parity of the inversions of the images listed in ascending order of the originals."""
    N = pb.N
    orbs = [o for o in range(2 * N) if (x[o % N] >> (o // N)) & 1]
    img = [int(perm[o]) for o in orbs]
    y = np.zeros(N, dtype=np.int8)
    for o in img:
        y[o % N] |= np.int8(1 << (o // N))
    inv = sum(1 for a in range(len(img)) for b in range(a + 1, len(img)) if img[a] > img[b])
    return y, (-1 if inv % 2 else 1)


def test_trivial_group_is_psi():
    m = _model(TORUS)
    occ = I.random_configs(TORUS, 20, 3)
    ident = I.symmetry_group(TORUS, translations=False)
    assert ident.shape[0] == 1 and (ident[0] == np.arange(2 * TORUS.N)).all()
    la, sg = m.log_psi_sym(occ, ident, np.ones(1))
    la0, sg0 = m.log_psi(occ)
    assert (sg == sg0).all()
    np.testing.assert_allclose(la, la0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("reflections,spin,momentum", [(False, False, False), (False, False, True),
                                                       (True, True, False)])
def test_projection_identity(reflections, spin, momentum):
    pb = TORUS
    m = _model(pb)
    perms = I.symmetry_group(pb, translations=True, reflections=reflections, spin_inversion=spin)
    G = perms.shape[0]
    if momentum:  # the (pi, pi) representation of the translations: chi = (-1)^(tx + ty)
        # translation by (tx, ty) sends site 0 to tx + Lx ty
        chi = np.array([(-1.0) ** ((int(p[0]) % pb.Lx) + (int(p[0]) // pb.Lx)) for p in perms])
    else:
        chi = np.ones(G)
    occ = I.random_configs(pb, 6, 11)
    la, sg = m.log_psi_sym(occ, perms, chi)
    for b in range(occ.shape[0]):
        # term scale of the orbit (the same set of configurations for n and every h n)
        imgs = np.array([_act(pb, p, occ[b])[0] for p in perms])
        lt, st = m.log_psi(imgs)
        ref = lt[st != 0].max()
        scale = np.exp(lt[st != 0] - ref).sum()
        v = sg[b] * np.exp(la[b] - ref)
        for h in range(G):
            y, pi = _act(pb, perms[h], occ[b])
            la_h, sg_h = m.log_psi_sym(y[None], perms, chi)
            v_h = sg_h[0] * np.exp(la_h[0] - ref)
            assert abs(v_h * pi - chi[h] * v) <= 1e-10 * scale, (b, h, v_h * pi, chi[h] * v)


def test_group_generator_closure():
    pb = TORUS
    perms = I.symmetry_group(pb, translations=True, reflections=True, spin_inversion=True)
    assert perms.shape[0] == 16 * 4 * 2
    keys = {p.tobytes() for p in perms}
    assert len(keys) == perms.shape[0]
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = perms[rng.integers(len(perms))], perms[rng.integers(len(perms))]
        assert a[b].astype(np.int32).tobytes() in keys  # composition stays in the group
    for p in perms:
        assert sorted(p.tolist()) == list(range(2 * pb.N))
