"""CPU pins of the oracle's ACE network (Sec. II "ACE", Eq. ACE): a stack of residual 3x3
conv blocks, each followed by a layer normalisation of every site's channel vector, then
the site-wise layers of Eq. MLP at width h_mlp and the orbital projection.

Pins, each against something other than the oracle's own loops:
  * the whole forward, the projection and log|psi| against torch's conv2d (circular or
    zero padding), layer_norm, silu, matmul and slogdet, layer by layer;
  * the moments a layer normalisation fixes (eps = 0, unit gain, zero shift: every site's
    channels have mean 0 and variance 1);
  * translation equivariance of the features on a torus with a shared embedding;
  * the receptive field: after l blocks a change at one site reaches exactly the sites
    within Chebyshev distance l (a normalisation over sites instead of channels, or an extra
    or missing block, breaks it);
  * the local energy against a dense Hamiltonian written independently, on a tiny lattice.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I
from tests.dense_hamiltonian import dense_h, state_to_occ


def _ace(Lx, Ly, pbc_x=1, pbc_y=1, n_up=3, n_dn=3, n_conv=3, n_mlp=2, h=6, h_mlp=10, per_site=1, eps=1e-5,
         model=I.MODEL_HUBBARD):
    ks, rs = I.ace_layout(n_conv, n_mlp)
    return I.Problem(Lx, Ly, pbc_x, pbc_y, n_up, n_dn, model, 1.0, 0.0, 4.0, 0.0, n_conv + n_mlp, h, ks, rs,
                     I.ACT_SILU, per_site, I.PREC_FP64, 64, 1e-10, I.FAMILY_ACE, n_conv, h_mlp, eps)


def _model(pb, seed=3, scale=0.3):
    return O.Model(pb, I.random_params(pb, seed, scale), I.plane_wave_M0(pb))


def _tensor(m, pb, name):
    o, s = I.param_offsets(pb)[name]
    return m.params[o:o + int(np.prod(s))].reshape(s)


@pytest.mark.parametrize("pbc", [(1, 1), (1, 0), (0, 0)])
def test_ace_forward_matches_torch(pbc):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    pb = _ace(5, 4, *pbc)
    m = _model(pb)
    occ = I.random_configs(pb, 3, 4)
    la, sg = m.log_psi(occ)
    for b in range(occ.shape[0]):
        H = m.features(occ[b])
        emb = _tensor(m, pb, "embed")  # [N][4][h]
        x = torch.tensor(np.stack([emb[i, occ[b, i]] for i in range(pb.N)]))  # [N][h]
        np.testing.assert_allclose(H[0][:, :pb.h], x.numpy(), rtol=0, atol=0)
        img = x.reshape(pb.Ly, pb.Lx, pb.h).permute(2, 0, 1)[None]
        for l in range(pb.n_conv):
            w = torch.tensor(_tensor(m, pb, f"kernel{l}")).permute(3, 2, 0, 1).contiguous()
            pad = img
            # circular padding on periodic axes, zeros on open ones (Hamiltonian boundaries)
            pad = F.pad(pad, (1, 1, 0, 0), mode="circular") if pb.pbc_x else F.pad(pad, (1, 1, 0, 0))
            pad = F.pad(pad, (0, 0, 1, 1), mode="circular") if pb.pbc_y else F.pad(pad, (0, 0, 1, 1))
            z = F.conv2d(pad, w) + torch.tensor(_tensor(m, pb, f"bias{l}"))[None, :, None, None]
            u = (img + F.silu(z))[0].permute(1, 2, 0)  # [Ly][Lx][h]
            y = F.layer_norm(u, (pb.h,), torch.tensor(_tensor(m, pb, f"ln_gamma{l}")),
                             torch.tensor(_tensor(m, pb, f"ln_beta{l}")), pb.ln_eps)
            ref = y.reshape(pb.N, pb.h)
            np.testing.assert_allclose(H[l + 1][:, :pb.h], ref.numpy(), rtol=0, atol=1e-12)
            img = torch.tensor(H[l + 1][:, :pb.h]).reshape(pb.Ly, pb.Lx, pb.h).permute(2, 0, 1)[None]
        x = torch.tensor(H[pb.n_conv][:, :pb.h])
        for l in range(pb.n_conv, pb.n_layers):
            W = torch.tensor(_tensor(m, pb, f"kernel{l}")[0, 0])
            x = F.silu(x @ W + torch.tensor(_tensor(m, pb, f"bias{l}")))
            np.testing.assert_allclose(H[l + 1][:, :W.shape[1]], x.numpy(), rtol=0, atol=1e-12)
        Wp = torch.tensor(_tensor(m, pb, "proj_w"))
        bp = torch.tensor(_tensor(m, pb, "proj_b"))
        P = x @ Wp + bp  # [N][2Ne]
        M = torch.tensor(m.M0).clone()
        M[:pb.N] += P[:, :pb.Ne]
        M[pb.N:] += P[:, pb.Ne:]
        rows = [s * pb.N + i for s in range(2) for i in range(pb.N) if (occ[b, i] >> s) & 1]
        s2, la2 = torch.linalg.slogdet(M[rows])
        assert int(s2) == sg[b]
        assert abs(float(la2) - la[b]) <= 1e-11


def test_layer_norm_moments():
    pb = _ace(4, 4, eps=0.0)
    p = I.random_params(pb, 8, 0.3)
    off = I.param_offsets(pb)
    for l in range(pb.n_conv):
        o, s = off[f"ln_gamma{l}"]
        p[o:o + s[0]] = 1.0
        o, s = off[f"ln_beta{l}"]
        p[o:o + s[0]] = 0.0
    m = O.Model(pb, p, I.plane_wave_M0(pb))
    for x in I.random_configs(pb, 4, 2):
        H = m.features(x)
        for l in range(1, pb.n_conv + 1):
            f = H[l][:, :pb.h]
            np.testing.assert_allclose(f.mean(axis=1), 0.0, atol=1e-14)
            np.testing.assert_allclose((f * f).mean(axis=1), 1.0, atol=1e-13)


def test_translation_equivariance():
    pb = _ace(5, 4, per_site=0)
    m = _model(pb)
    x = I.random_configs(pb, 1, 6)[0]
    H = m.features(x)
    for tx, ty in ((1, 0), (0, 1), (2, 3)):
        src = np.array([((i // pb.Lx + ty) % pb.Ly) * pb.Lx + (i % pb.Lx + tx) % pb.Lx for i in range(pb.N)])
        xt = np.zeros_like(x)
        xt[src] = x  # site i moves to src[i]
        Ht = m.features(xt)
        for l in range(pb.n_layers + 1):
            np.testing.assert_allclose(Ht[l][src], H[l], rtol=0, atol=1e-12)


def test_receptive_field_grows_one_site_per_block():
    pb = _ace(9, 9, 0, 0, n_conv=3, n_mlp=1)
    m = _model(pb, seed=12, scale=0.5)
    x = I.random_configs(pb, 1, 7)[0]
    c = 4 * pb.Lx + 4  # centre site
    x2 = x.copy()
    x2[c] = (x[c] + 1) % 4  # a local change (particle numbers are irrelevant to the features)
    H, H2 = m.features(x), m.features(x2)
    cheb = np.array([max(abs(i % pb.Lx - 4), abs(i // pb.Lx - 4)) for i in range(pb.N)])
    for l in range(pb.n_conv + 1):
        diff = np.abs(H[l] - H2[l]).max(axis=1)
        assert (diff[cheb > l] == 0).all(), l
        assert (diff[cheb <= l] > 1e-9).all(), l
    last = np.abs(H[-1] - H2[-1]).max(axis=1)
    assert (last[cheb > pb.n_conv] == 0).all() and (last[cheb <= pb.n_conv] > 0).all()


@pytest.mark.parametrize("model", [I.MODEL_HUBBARD, I.MODEL_TJ])
def test_ace_enumeration_matches_dense_hamiltonian(model):
    """sum_n psi^2 E_loc / sum psi^2 (oracle, ACE amplitudes) == psi^T H psi / psi^T psi with
    H built independently."""
    pb = _ace(3, 2, 0, 0, 2, 2, n_conv=2, n_mlp=1, h=4, h_mlp=6, model=model)
    if model == I.MODEL_TJ:
        pb = pb.replace(U=0.0, J=0.4)
    m = _model(pb, seed=9, scale=0.4)
    E, xs, la, sg = O.enumerate_energy(m)
    H, states = dense_h(pb.as_dict())
    occ = np.array([state_to_occ(s, pb.N) for s in states])
    la2, sg2 = m.log_psi(occ)
    psi = sg2 * np.exp(la2 - la2.max())
    E_dense = psi @ H @ psi / (psi @ psi)
    assert abs(E - E_dense) <= 1e-10 * max(1.0, abs(E_dense))
    assert E >= np.linalg.eigvalsh(H)[0] - 1e-10


def test_ace_parameter_count():
    """Table tab:model ACE at 16x16 (h = 144, h_mlp = 256, 16 blocks, 2 site-wise layers)."""
    pb = I.workload("ace16x16")
    N, h, hm, Ne = 256, 144, 256, 224
    want = N * 4 * h + 16 * (9 * h * h + 3 * h) + (h * hm + hm) + (hm * hm + hm) + hm * 2 * Ne + 2 * Ne
    assert I.param_count(pb) == want
    m = O.Model(pb, np.zeros(want), I.plane_wave_M0(pb))
    assert m.P == want
