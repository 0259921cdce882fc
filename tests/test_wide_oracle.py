"""CPU pins of the oracle's wide SCALE shapes of Table tab:model: the SCALE layout (one residual
conv, then site-wise layers, Sec. II.B) with per-layer widths (conv h, site-wise h_mlp) and
SCALE-L's plus-shaped stencil (the offsets within L2 distance 2, 13 sites, in place of the
3x3 box of L2 <= sqrt 2).

Pins, each against something other than the oracle's own loops:
  * the conv with the plus stencil and the Hamiltonian's boundary conditions against torch
    conv2d with the 13 taps placed in an otherwise zero 5x5 kernel; the site-wise layers of
    different widths against matmul; log|psi| against torch slogdet;
  * the receptive field of the plus stencil: one changed site moves exactly the 13 sites
    within L2 <= 2 (a box stencil would move 25);
  * the local energy against a dense Hamiltonian written independently;
  * the parameter counts of Table tab:model SCALE-L (16x16) and SCALE-XL (32x32).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I
from tests.dense_hamiltonian import dense_h, state_to_occ


def _wide(Lx, Ly, pbc_x=1, pbc_y=1, n_up=4, n_dn=4, h=6, h_mlp=10, n_mlp=2, k=5, stencil=I.STENCIL_DISK,
          model=I.MODEL_HUBBARD, per_site=1):
    L = 1 + n_mlp
    return I.Problem(Lx, Ly, pbc_x, pbc_y, n_up, n_dn, model, 1.0, 0.0, 4.0, 0.0, L, h, [k] + [1] * n_mlp,
                     [1] + [0] * n_mlp, I.ACT_SILU, per_site, I.PREC_FP64, 64, 1e-10, I.FAMILY_WIDE, 1, h_mlp,
                     1e-5, stencil)


def _model(pb, seed=4, scale=0.3):
    return O.Model(pb, I.random_params(pb, seed, scale), I.plane_wave_M0(pb))


def _tensor(m, pb, name):
    o, s = I.param_offsets(pb)[name]
    return m.params[o:o + int(np.prod(s))].reshape(s)


def test_stencil_taps():
    assert len(I.stencil_taps(3, I.STENCIL_BOX)) == 9
    assert len(I.stencil_taps(5, I.STENCIL_DISK)) == 13
    assert (2, 1) not in I.stencil_taps(5, I.STENCIL_DISK) and (2, 0) in I.stencil_taps(5, I.STENCIL_DISK)


@pytest.mark.parametrize("pbc", [(1, 1), (1, 0), (0, 0)])
def test_plus_stencil_forward_matches_torch(pbc):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    pb = _wide(6, 5, *pbc)
    m = _model(pb)
    occ = I.random_configs(pb, 3, 8)
    la, sg = m.log_psi(occ)
    taps = I.stencil_taps(5, I.STENCIL_DISK)
    K = _tensor(m, pb, "kernel0")  # [13][h][h]
    W5 = np.zeros((5, 5, pb.h, pb.h))
    for t, (dx, dy) in enumerate(taps):
        W5[dy + 2, dx + 2] = K[t]
    w = torch.tensor(W5).permute(3, 2, 0, 1).contiguous()
    for b in range(occ.shape[0]):
        H = m.features(occ[b])
        img = torch.tensor(H[0][:, :pb.h]).reshape(pb.Ly, pb.Lx, pb.h).permute(2, 0, 1)[None]
        pad = F.pad(img, (2, 2, 0, 0), mode="circular") if pb.pbc_x else F.pad(img, (2, 2, 0, 0))
        pad = F.pad(pad, (0, 0, 2, 2), mode="circular") if pb.pbc_y else F.pad(pad, (0, 0, 2, 2))
        z = F.conv2d(pad, w) + torch.tensor(_tensor(m, pb, "bias0"))[None, :, None, None]
        ref = (img + F.silu(z))[0].permute(1, 2, 0).reshape(pb.N, pb.h)
        np.testing.assert_allclose(H[1][:, :pb.h], ref.numpy(), rtol=0, atol=1e-12)
        x = ref
        for l in range(1, pb.n_layers):
            Kl = _tensor(m, pb, f"kernel{l}")
            Wl = torch.tensor(Kl.reshape(Kl.shape[-2], Kl.shape[-1]))
            x = F.silu(x @ Wl + torch.tensor(_tensor(m, pb, f"bias{l}")))
            np.testing.assert_allclose(H[l + 1][:, :Wl.shape[1]], x.numpy(), rtol=0, atol=1e-12)
        P = x @ torch.tensor(_tensor(m, pb, "proj_w")) + torch.tensor(_tensor(m, pb, "proj_b"))
        M = torch.tensor(m.M0).clone()
        M[:pb.N] += P[:, :pb.Ne]
        M[pb.N:] += P[:, pb.Ne:]
        rows = [s * pb.N + i for s in range(2) for i in range(pb.N) if (occ[b, i] >> s) & 1]
        s2, la2 = torch.linalg.slogdet(M[rows])
        assert int(s2) == sg[b] and abs(float(la2) - la[b]) <= 1e-11


@pytest.mark.parametrize("stencil,n_moved", [(I.STENCIL_DISK, 13), (I.STENCIL_BOX, 25)])
def test_receptive_field_of_the_stencil(stencil, n_moved):
    pb = _wide(9, 9, 0, 0, stencil=stencil)
    m = _model(pb, seed=5, scale=0.5)
    x = I.random_configs(pb, 1, 2)[0]
    c = 4 * 9 + 4
    x2 = x.copy()
    x2[c] = (x[c] + 1) % 4
    H, H2 = m.features(x), m.features(x2)
    moved = np.abs(H[-1] - H2[-1]).max(axis=1) > 0
    assert moved.sum() == n_moved
    dist2 = np.array([(i % 9 - 4) ** 2 + (i // 9 - 4) ** 2 for i in range(pb.N)])
    if stencil == I.STENCIL_DISK:
        assert (moved == (dist2 <= 4)).all()


@pytest.mark.parametrize("model", [I.MODEL_HUBBARD, I.MODEL_TJ])
def test_wide_enumeration_matches_dense_hamiltonian(model):
    pb = _wide(3, 3, 1, 1, 2, 2, h=4, h_mlp=6, n_mlp=1, model=model)
    if model == I.MODEL_TJ:
        pb = pb.replace(U=0.0, J=0.4)
    m = _model(pb, seed=6, scale=0.4)
    E, xs, la, sg = O.enumerate_energy(m)
    H, states = dense_h(pb.as_dict())
    occ = np.array([state_to_occ(s, pb.N) for s in states])
    la2, sg2 = m.log_psi(occ)
    psi = sg2 * np.exp(la2 - la2.max())
    E_dense = psi @ H @ psi / (psi @ psi)
    assert abs(E - E_dense) <= 1e-10 * max(1.0, abs(E_dense))


@pytest.mark.parametrize("name,N,taps,h,hm,Ne", [("scale_l16x16", 256, 13, 384, 512, 224),
                                                 ("scale_xl32x32", 1024, 9, 640, 1280, 896)])
def test_table_parameter_counts(name, N, taps, h, hm, Ne):
    pb = I.workload(name)
    want = N * 4 * h + (taps * h * h + h) + (h * hm + hm) + 3 * (hm * hm + hm) + hm * 2 * Ne + 2 * Ne
    assert I.param_count(pb) == want
    assert O.Model(pb, np.zeros(want), I.plane_wave_M0(pb)).P == want
