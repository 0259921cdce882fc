"""CPU pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets one way the oracle could be wrong (a dropped term, a wrong sign or
index, a transposed operand) and checks it against something other than the oracle:
closed forms, library routines, an independently written dense Hamiltonian, finite
differences and the receptive-field geometry of Eq. neighbor.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I
from tests.dense_hamiltonian import dense_h, state_to_occ

GOLD = os.path.join(os.path.dirname(__file__), "golden", "u0_energies.json")


def _model(pb, seed=11, scale=0.05, zero=False):
    p = I.random_params(pb, seed, scale)
    if zero:
        p = np.zeros_like(p)
    return O.Model(pb, p, I.plane_wave_M0(pb))


def _cond_ok(m, occ, limit=1e8):
    _, M = m.orbitals(occ)
    N = m.N
    ok = []
    for b in range(occ.shape[0]):
        orbs = [s * N + i for s in range(2) for i in range(N) if (occ[b, i] >> s) & 1]
        ok.append(np.linalg.cond(M[b][orbs]) < limit)
    return np.array(ok)


# -- library pins ---------------------------------------------------------------------

def test_slogdet_matches_numpy():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 14, 56, 97):
        A = rng.normal(size=(n, n))
        s, la = O.slogdet(A)
        s2, la2 = np.linalg.slogdet(A)
        assert s == int(s2)
        assert abs(la - la2) <= 1e-12 * max(1.0, abs(la2))
    assert O.slogdet(np.zeros((3, 3)))[0] == 0


@pytest.mark.parametrize("pbc", [1, 0])
@pytest.mark.parametrize("act", [I.ACT_TANH, I.ACT_SILU])
def test_conv_layer_matches_torch(pbc, act):
    """Eq. conv with the Hamiltonian's boundary conditions vs torch conv2d (FP64)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    pb = I.Problem(5, 4, pbc, pbc, 3, 2, n_layers=2, h=6, ksize=[3, 1], residual=[1, 0], act=act)
    m = _model(pb, seed=3, scale=0.3)
    occ = I.random_configs(pb, 1, 9)[0]
    H = m.features(occ)
    off = I.param_offsets(pb)
    o, s = off["kernel0"]
    K = torch.tensor(m.params[o:o + np.prod(s)].reshape(s))  # [ky][kx][ci][co]
    o, s = off["bias0"]
    b = torch.tensor(m.params[o:o + np.prod(s)])
    x = torch.tensor(H[0].reshape(pb.Ly, pb.Lx, pb.h)).permute(2, 0, 1)[None]
    w = K.permute(3, 2, 0, 1).contiguous()
    if pbc:
        z = F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), w)
    else:
        z = F.conv2d(x, w, padding=1)
    z = z + b[None, :, None, None]
    a = torch.tanh(z) if act == I.ACT_TANH else F.silu(z)
    ref = (x + a)[0].permute(1, 2, 0).reshape(pb.N, pb.h).numpy()
    np.testing.assert_allclose(H[1], ref, rtol=0, atol=1e-13)
    # the site-wise layer (Eq. MLP, no residual) against a plain matmul
    o, s = off["kernel1"]
    W1 = m.params[o:o + np.prod(s)].reshape(pb.h, pb.h)
    o, s = off["bias1"]
    b1 = m.params[o:o + np.prod(s)]
    z1 = H[1] @ W1 + b1
    ref1 = np.tanh(z1) if act == I.ACT_TANH else z1 / (1 + np.exp(-z1))
    np.testing.assert_allclose(H[2], ref1, rtol=0, atol=1e-13)


def test_projection_matches_matmul():
    pb = I.workload("hubbard4x4")
    m = _model(pb)
    occ = I.random_configs(pb, 2, 1)
    HL, M = m.orbitals(occ)
    off = I.param_offsets(pb)
    o, s = off["proj_w"]
    W = m.params[o:o + np.prod(s)].reshape(s)
    o, s = off["proj_b"]
    bp = m.params[o:o + np.prod(s)]
    Ne, N = pb.Ne, pb.N
    for b in range(2):
        ref = m.M0.copy()
        ref[:N] += HL[b] @ W[:, :Ne] + bp[:Ne]
        ref[N:] += HL[b] @ W[:, Ne:] + bp[Ne:]
        np.testing.assert_allclose(M[b], ref, atol=1e-14)


# -- lattice and reference orbitals ----------------------------------------------------

@pytest.mark.parametrize("Lx,Ly,px,py,nn,nnn", [
    (4, 4, 1, 1, 32, 32), (16, 4, 1, 0, 112, 96), (5, 3, 0, 0, 22, 16), (3, 3, 1, 1, 18, 18)])
def test_bond_counts(Lx, Ly, px, py, nn, nnn):
    pb = I.Problem(Lx, Ly, px, py, 1, 1, n_layers=1, h=2, ksize=[1], residual=[0])
    m = _model(pb)
    b0, b1 = m.bonds(0), m.bonds(1)
    assert len(b0) == nn and len(b1) == nnn
    assert len({tuple(sorted(p)) for p in b0.tolist()}) == nn  # each unordered pair once


@pytest.mark.parametrize("name", ["hubbard4x4", "hubbard8x8", "cylinder16x4"])
def test_plane_waves_are_hopping_eigenvectors(name):
    pb = I.workload(name)
    from tests.dense_hamiltonian import bonds
    N = pb.N
    T = np.zeros((N, N))
    for i, j in bonds(pb.Lx, pb.Ly, pb.pbc_x, pb.pbc_y):
        T[i, j] = T[j, i] = -pb.t
    for i, j in bonds(pb.Lx, pb.Ly, pb.pbc_x, pb.pbc_y, True):
        T[i, j] = T[j, i] = -pb.tp
    eps, V = I.plane_wave_orbitals(pb)
    np.testing.assert_allclose(T @ V, V * eps, atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(N), atol=1e-12)
    np.testing.assert_allclose(eps, np.sort(np.linalg.eigvalsh(T)), atol=1e-12)


# -- zero-variance closed form ---------------------------------------------------------

@pytest.mark.parametrize("name", ["hubbard4x4", "hubbard8x8", "cylinder16x4", "open6x4_tp"])
def test_zero_backflow_local_energy_is_closed_form(name):
    """All network weights zero: psi is a Slater determinant of hopping eigenvectors, so
    E_loc(n) = E0 + U * (#doubly occupied sites) exactly for every n with psi(n) != 0."""
    gold = json.load(open(GOLD))["cases"][name]
    if name == "open6x4_tp":
        pb = I.Problem(6, 4, 0, 0, 9, 8, tp=0.3, U=5.0, n_layers=2, h=4, ksize=[3, 1], residual=[1, 0])
    else:
        pb = I.workload(name)
    m = _model(pb, zero=True)
    occ = I.random_configs(pb, 64, 77)
    ok = _cond_ok(m, occ)
    assert ok.sum() >= 5
    e, st = m.local_energy(occ[ok])
    D = (occ[ok] == 3).sum(1)
    ref = gold["E0"] + pb.U * D
    np.testing.assert_allclose(e, ref, rtol=1e-9, atol=1e-9)


# -- whole-space enumeration against an independent dense Hamiltonian -----------------

TINY = [
    I.Problem(3, 3, 1, 1, 2, 2, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 4, [3, 1], [1, 0]),
    I.Problem(3, 2, 1, 0, 2, 1, I.MODEL_HUBBARD, 1.0, -0.3, 6.0, 0.0, 2, 3, [3, 1], [1, 0], I.ACT_SILU),
    I.Problem(3, 3, 1, 1, 2, 2, I.MODEL_TJ, 1.0, 0.0, 0.0, 0.4, 2, 4, [3, 1], [1, 0]),
    I.Problem(4, 2, 0, 0, 2, 2, I.MODEL_TJ, 1.0, 0.2, 0.0, 1.0 / 3.0, 3, 3, [3, 3, 1], [1, 1, 0]),
    I.Problem(3, 2, 0, 0, 2, 4, I.MODEL_HUBBARD_PH, 1.0, 0.0, -4.0, 0.0, 2, 4, [3, 1], [1, 0]),
]


@pytest.mark.parametrize("k", range(len(TINY)))
def test_enumeration_matches_dense_hamiltonian(k):
    """sum_n psi^2 E_loc / sum psi^2 (oracle) == psi^T H psi / psi^T psi with H built
    independently; H symmetric; variational bound <H> >= E_ground."""
    pb = TINY[k]
    m = _model(pb, seed=5 + k, scale=0.3)
    E, xs, la, sg = O.enumerate_energy(m)
    H, states = dense_h(pb.as_dict())
    np.testing.assert_allclose(H, H.T, atol=0)
    occ = np.array([state_to_occ(s, pb.N) for s in states])
    la2, sg2 = m.log_psi(occ)
    psi = sg2 * np.exp(la2 - la2.max())
    E_dense = psi @ H @ psi / (psi @ psi)
    assert abs(E - E_dense) <= 1e-10 * max(1.0, abs(E_dense))
    assert E >= np.linalg.eigvalsh(H)[0] - 1e-10


@pytest.mark.parametrize("Lx,Ly,n_up,n_dn", [(3, 2, 2, 2), (4, 2, 2, 3), (4, 2, 3, 3)])
def test_particle_hole_transformation_spectrum(Lx, Ly, n_up, n_dn):
    """App. "particle-hole transformation": c_dn -> (-1)^i c_dn^+ maps the attractive Hubbard
    model with (n_up, n_dn) onto -t sum hops + U sum n_up (1 - n_dn) with (n_up, N - n_dn) on a
    bipartite lattice, a unitary map: the two dense Hamiltonians (the PH diagonal written
    independently in the dense builder) have the same spectrum."""
    U = -4.0
    base = dict(Lx=Lx, Ly=Ly, pbc_x=0, pbc_y=0, t=1.0, tp=0.0, U=U, J=0.0)
    H_attr, _ = dense_h(dict(base, n_up=n_up, n_dn=n_dn, model=I.MODEL_HUBBARD))
    H_ph, _ = dense_h(dict(base, n_up=n_up, n_dn=Lx * Ly - n_dn, model=I.MODEL_HUBBARD_PH))
    assert H_attr.shape == H_ph.shape
    np.testing.assert_allclose(np.linalg.eigvalsh(H_ph), np.linalg.eigvalsh(H_attr), atol=1e-10)
    # and the transformed model is not trivially the repulsive one
    H_rep, _ = dense_h(dict(base, n_up=n_up, n_dn=Lx * Ly - n_dn, model=I.MODEL_HUBBARD))
    assert abs(np.linalg.eigvalsh(H_rep)[0] - np.linalg.eigvalsh(H_ph)[0]) > 0.1


def test_dense_builder_two_site_closed_form():
    """Two-site Hubbard dimer, one up + one down: E_ground = U/2 - sqrt(U^2/4 + 4 t^2)."""
    for U in (0.0, 4.0, 8.0):
        d = I.Problem(2, 1, 0, 0, 1, 1, U=U, n_layers=1, h=1, ksize=[1], residual=[0]).as_dict()
        H, _ = dense_h(d)
        e = np.linalg.eigvalsh(H)[0]
        assert abs(e - (U / 2 - np.sqrt(U * U / 4 + 4))) < 1e-12


def test_dense_builder_free_fermions():
    """U = 0 on a 3x3 torus: dense ground energy equals the closed-form free-fermion sum."""
    pb = I.Problem(3, 3, 1, 1, 2, 3, U=0.0, tp=-0.25, n_layers=1, h=1, ksize=[1], residual=[0])
    H, _ = dense_h(pb.as_dict())
    eps, _ = I.plane_wave_orbitals(pb)
    assert abs(np.linalg.eigvalsh(H)[0] - (eps[:2].sum() + eps[:3].sum())) < 1e-10


# -- ratio properties -----------------------------------------------------------------

@pytest.mark.parametrize("name", ["hubbard8x8", "tj8x8"])
def test_hermiticity_and_reciprocity(name):
    pb = I.workload(name).replace(tp=-0.2 if name == "hubbard8x8" else 0.0)
    m = _model(pb, scale=0.2)
    x = I.random_configs(pb, 1, 3)[0]
    xs, cf = m.connected(x)
    assert len(xs) > 0
    for x2, c in zip(xs[:40], cf[:40]):
        back, cb = m.connected(x2)
        k = [i for i in range(len(back)) if np.array_equal(back[i], x)]
        assert len(k) == 1 and cb[k[0]] == c
        la, sg = m.log_psi(np.stack([x, x2]))
        r12 = sg[0] * sg[1] * np.exp(la[1] - la[0])
        r21 = sg[0] * sg[1] * np.exp(la[0] - la[1])
        assert abs(r12 * r21 - 1) < 1e-12


def _hop(occ, src, dst, spin):
    x = occ.copy()
    x[src] &= ~(1 << spin)
    x[dst] |= 1 << spin
    return x


def test_lowrank_identity_and_jordan_wigner_sign():
    """Eq. SMW: det(Phi')/det(Phi) = det(I_r + V^T Phi^-1 U) with the changed rows in
    place (slot order), and the ascending-order ratio of the oracle differs from it by
    (-1)^(occupied orbitals strictly between source and destination)."""
    pb = I.workload("hubbard8x8")
    m = _model(pb, scale=0.2)
    occ = I.random_configs(pb, 6, 21)
    moves = I.random_hop_moves(pb, occ, 4)
    N, Ne = pb.N, pb.Ne
    r_ora = m.ratio(occ, moves)
    for b in range(occ.shape[0]):
        kind, src, dst, spin = moves[b]
        if kind < 0:
            continue
        x2 = _hop(occ[b], src, dst, spin)
        _, M = m.orbitals(np.stack([occ[b], x2]))
        orbs = [s * N + i for s in range(2) for i in range(N) if (occ[b, i] >> s) & 1]
        Phi = M[0][orbs]
        # slot order: the moved electron keeps its row, every row takes x2's orbitals
        orbs2 = [spin * N + dst if o == spin * N + src else o for o in orbs]
        Phi2 = M[1][orbs2]
        rows = [a for a in range(Ne) if not np.array_equal(Phi2[a], Phi[a])]
        Uc = np.zeros((Ne, len(rows)))
        for c, a in enumerate(rows):
            Uc[a, c] = 1.0
        V = (Phi2[rows] - Phi[rows]).T
        A = np.eye(len(rows)) + V.T @ np.linalg.inv(Phi) @ Uc
        r_slot = np.linalg.det(A)
        assert abs(r_slot - np.linalg.det(Phi2) / np.linalg.det(Phi)) < 1e-9 * max(1, abs(r_slot))
        lo, hi = sorted((spin * N + src, spin * N + dst))
        between = sum(1 for o in orbs if lo < o < hi)
        assert abs(r_ora[b] - (-1) ** between * r_slot) < 1e-9 * max(1.0, abs(r_slot))


def test_locality_of_features():
    """Eq. neighbor: after a hop, last-layer features change only within Chebyshev
    distance sum_l (k_l - 1)/2 of the two touched sites."""
    pb = I.Problem(8, 7, 1, 1, 10, 9, n_layers=4, h=6, ksize=[3, 1, 3, 1], residual=[1, 0, 1, 0])
    m = _model(pb, scale=0.3)
    occ = I.random_configs(pb, 4, 2)
    moves = I.random_hop_moves(pb, occ, 8)
    R = 2
    for b in range(4):
        kind, src, dst, spin = moves[b]
        if kind < 0:
            continue
        H1 = m.features(occ[b])[-1]
        H2 = m.features(_hop(occ[b], src, dst, spin))[-1]
        changed = np.where(np.abs(H1 - H2).max(1) > 0)[0]

        def cheb(i, j):
            dx = abs(i % pb.Lx - j % pb.Lx)
            dy = abs(i // pb.Lx - j // pb.Lx)
            return max(min(dx, pb.Lx - dx), min(dy, pb.Ly - dy))
        allowed = {i for i in range(pb.N) if min(cheb(i, src), cheb(i, dst)) <= R}
        assert set(changed.tolist()) <= allowed
        assert len(changed) > 0


# -- gradient ------------------------------------------------------------------------

def test_gradient_matches_central_differences():
    """d log|psi| / d theta vs central differences (h = 1e-6, FP64) on 20 random
    parameters of the deep residual stack on the 16x4 cylinder."""
    pb = I.workload("cylinder16x4")
    m = _model(pb, seed=1237)
    occ = I.random_configs(pb, 3, 5681)
    g = m.grad_logpsi(occ)
    rng = np.random.default_rng(99)
    idx = rng.choice(m.P, 20, replace=False)
    # make sure every tensor kind is probed
    off = I.param_offsets(pb)
    extra = [off["embed"][0] + 4 * pb.h * 5 + int(occ[0, 5]) * pb.h + 1,
             off["proj_b"][0] + 3, off["proj_w"][0] + 7, off["bias11"][0] + 2]
    idx = np.concatenate([idx, extra])
    h = 1e-6
    for q in idx:
        p1 = m.params.copy(); p1[q] += h
        p2 = m.params.copy(); p2[q] -= h
        l1, _ = m.with_params(p1).log_psi(occ)
        l2, _ = m.with_params(p2).log_psi(occ)
        fd = (l1 - l2) / (2 * h)
        np.testing.assert_allclose(g[:, q], fd, rtol=2e-5, atol=2e-7)


@pytest.mark.parametrize("pbc", [(1, 1), (0, 1)])
def test_gradient_plus_stencil_central_differences(pbc):
    """The backward pass with SCALE-L's 13-site plus stencil (weights stored for the taps
    only, row-major over the 5x5 box) vs central differences: every tap of the first
    kernel (the four arms' tips included), the site-wise layer, bias, embedding and
    projection, on the torus and on a cylinder with open x edges."""
    pb = I.workload("scale_plus6x6").replace(pbc_x=pbc[0], pbc_y=pbc[1], n_layers=3, ksize=[5, 1, 1],
                                             residual=[1, 0, 0])
    m = _model(pb, seed=1238, scale=0.3)
    occ = I.random_configs(pb, 2, 5682)
    g = m.grad_logpsi(occ)
    off = I.param_offsets(pb)
    h = pb.h
    k0 = off["kernel0"][0]
    idx = [k0 + d * h * h + (d % h) * h + (3 * d) % h for d in range(13)]
    idx += [off["kernel1"][0] + 5, off["kernel2"][0] + h * h - 1, off["bias0"][0] + 1, off["bias2"][0] + 3,
            off["embed"][0] + 4 * h * 7 + int(occ[0, 7]) * h + 2, off["proj_b"][0] + 5, off["proj_w"][0] + 11]
    eps = 1e-6
    for q in idx:
        p1 = m.params.copy(); p1[q] += eps
        p2 = m.params.copy(); p2[q] -= eps
        l1, _ = m.with_params(p1).log_psi(occ)
        l2, _ = m.with_params(p2).log_psi(occ)
        fd = (l1 - l2) / (2 * eps)
        np.testing.assert_allclose(g[:, q], fd, rtol=2e-5, atol=2e-7)
    # a weight of a tap a box stencil would have (dx = 2, dy = 1) does not exist: 13 taps
    assert off["bias0"][0] - k0 == 13 * h * h


def test_projection_bias_gradient_closed_form():
    """d log|det Phi| / d proj_b[s*Ne+k] = sum over spin-s rows a of (Phi^-1)[k][a]."""
    pb = I.workload("hubbard4x4")
    m = _model(pb, scale=0.2)
    occ = I.random_configs(pb, 3, 8)
    g = m.grad_logpsi(occ)
    _, M = m.orbitals(occ)
    off = I.param_offsets(pb)["proj_b"][0]
    N, Ne = pb.N, pb.Ne
    for b in range(3):
        orbs = [s * N + i for s in range(2) for i in range(N) if (occ[b, i] >> s) & 1]
        Pinv = np.linalg.inv(M[b][orbs])
        for s in range(2):
            rows = [a for a, o in enumerate(orbs) if o // N == s]
            ref = Pinv[:, rows].sum(1)
            np.testing.assert_allclose(g[b, off + s * Ne: off + (s + 1) * Ne], ref, atol=1e-10)


# -- model-space rules ---------------------------------------------------------------

def test_tj_double_occupancy_has_zero_amplitude():
    pb = I.workload("tj8x8")
    m = _model(pb)
    occ = I.random_configs(pb, 2, 1)
    occ[0, np.where(occ[0] == 1)[0][0]] = 3
    occ[0, np.where(occ[0] == 2)[0][0]] = 0
    la, sg = m.log_psi(occ)
    assert sg[0] == 0 and np.isneginf(la[0]) and sg[1] != 0
    e, st = m.local_energy(occ)
    assert st[0] == 1 and np.isnan(e[0]) and st[1] == 0


def test_wrong_particle_number_rejected():
    pb = I.workload("hubbard4x4")
    m = _model(pb)
    occ = I.random_configs(pb, 1, 1)
    occ[0, np.where((occ[0] & 1) == 1)[0][0]] &= ~1
    la, sg = m.log_psi(occ)
    assert sg[0] == 0
