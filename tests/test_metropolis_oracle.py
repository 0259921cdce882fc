"""CPU pins of the oracle's Metropolis step: configurations are drawn from
P(n) ~ |psi(n)|^2 by local updates (Sec. II.A; 2.5 N steps per sample in the optimisation
settings). The proposal is the symmetric single-electron hop (the pick-th occupied orbital
in ascending order, one of four nearest-neighbour directions); the acceptance is
min(1, |psi(n')/psi(n)|^2).

The pins: the proposal and the acceptance rule against a brute-force construction and
amplitudes from the oracle's own log|psi| on every (state, pick, direction) of a tiny
lattice, and the stationary distribution of the chain against |psi|^2 from complete
enumeration (a test that also tells |psi|^2 apart from |psi|).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_25775_gb300 import inputs as I

_KS, _RS = I.scale_layout(2)
TINY = I.Problem(3, 2, 0, 0, 2, 1, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 4, _KS, _RS,
                 I.ACT_TANH, 1, I.PREC_FP64, 64, 1e-10)
TINY_TJ = TINY.replace(model=I.MODEL_TJ, U=0.0, J=0.4)
TINY_PBC = I.Problem(3, 3, 1, 1, 2, 1, I.MODEL_HUBBARD, 1.0, 0.0, 4.0, 0.0, 2, 4, _KS, _RS,
                     I.ACT_TANH, 1, I.PREC_FP64, 64, 1e-10)


def _model(pb, seed=3, scale=0.6):
    M0 = np.random.default_rng(seed).normal(size=(2 * pb.N, pb.Ne))
    return O.Model(pb, I.random_params(pb, seed, scale), M0)


def _brute_move(pb, x, pick, d):
    """Configuration after hopping the pick-th occupied orbital (ascending o = s*N + i) one
    site along direction d, or None when the proposal is rejected outright."""
    N = pb.N
    orbs = [o for o in range(2 * N) if (x[o % N] >> (o // N)) & 1]
    s, i = divmod(orbs[pick], N)
    xx = i % pb.Lx + (1, -1, 0, 0)[d]
    yy = i // pb.Lx + (0, 0, 1, -1)[d]
    if not 0 <= xx < pb.Lx:
        if not pb.pbc_x:
            return None
        xx %= pb.Lx
    if not 0 <= yy < pb.Ly:
        if not pb.pbc_y:
            return None
        yy %= pb.Ly
    j = yy * pb.Lx + xx
    if (x[j] != 0) if pb.model == I.MODEL_TJ else ((x[j] >> s) & 1):
        return None
    x2 = x.copy()
    x2[i] &= ~np.int8(1 << s)
    x2[j] |= np.int8(1 << s)
    return x2


@pytest.mark.parametrize("pb", [TINY, TINY_TJ, TINY_PBC], ids=["open", "tj", "torus"])
def test_proposal_and_acceptance_rule(pb):
    m = _model(pb)
    xs = O.all_configurations(pb)
    la, sg = m.log_psi(xs)
    assert (sg != 0).all()
    rows, expect_lo, expect_hi, x_new = [], [], [], []
    for n, x in enumerate(xs):
        for pick in range(pb.Ne):
            for d in range(4):
                x2 = _brute_move(pb, x, pick, d)
                rows.append((n, pick, d))
                if x2 is None:
                    x_new.append(x)
                    expect_lo.append(None)
                    expect_hi.append(None)
                    continue
                la2, sg2 = m.log_psi(x2[None])
                rho = np.exp(2.0 * (la2[0] - la[n]))
                x_new.append(x2)
                # u just below min(rho, 1) accepts; u just above rho rejects (when rho < 1)
                expect_lo.append(min(rho, 1.0) * (1 - 1e-7))
                expect_hi.append(rho * (1 + 1e-7) if rho < 0.999 else None)
    idx = np.array([r[0] for r in rows])
    pick = np.array([[r[1] for r in rows]], dtype=np.int32)
    dirs = np.array([[r[2] for r in rows]], dtype=np.int32)
    valid = np.array([e is not None for e in expect_lo])
    x_new = np.array(x_new, dtype=np.int8)
    # below the threshold: every valid proposal is accepted
    u = np.array([[e if e is not None else 0.0 for e in expect_lo]])
    out, acc = m.metropolis(xs[idx], pick, dirs, u)
    assert (acc == valid).all()
    assert np.array_equal(out, x_new)
    # above the threshold: rejected, configuration unchanged
    has_hi = np.array([e is not None for e in expect_hi])
    u = np.array([[e if e is not None else 0.5 for e in expect_hi]])
    out, acc = m.metropolis(xs[idx[has_hi]], pick[:, has_hi], dirs[:, has_hi], u[:, has_hi])
    assert (acc == 0).all()
    assert np.array_equal(out, xs[idx[has_hi]])
    # invalid proposals never move, whatever u
    inv = ~valid
    out, acc = m.metropolis(xs[idx[inv]], pick[:, inv], dirs[:, inv], np.zeros((1, int(inv.sum()))))
    assert (acc == 0).all() and np.array_equal(out, xs[idx[inv]])


@pytest.mark.parametrize("pb", [TINY, TINY_TJ], ids=["hubbard", "tj"])
def test_stationary_distribution_is_psi_squared(pb):
    m = _model(pb, seed=5, scale=0.8)
    xs = O.all_configurations(pb)
    la, sg = m.log_psi(xs)
    p2 = np.exp(2 * (la - la.max()))
    p2 /= p2.sum()
    p1 = np.exp(la - la.max())
    p1 /= p1.sum()
    tvd_12 = 0.5 * np.abs(p2 - p1).sum()
    assert tvd_12 > 0.12, "test cannot tell |psi|^2 from |psi| with these weights"
    key = {x.tobytes(): n for n, x in enumerate(xs)}
    B, S, calls, burn = 512, 8, 160, 10
    rng = np.random.default_rng(9)
    x = xs[rng.integers(len(xs), size=B)]
    counts = np.zeros(len(xs))
    for c in range(calls):
        pick, d, u = I.metropolis_randoms(pb, B, S, 100 + c)
        x, _ = m.metropolis(x, pick, d, u)
        assert (np.array([(xi & 1).sum() for xi in x]) == pb.n_up).all()
        assert (np.array([(xi >> 1).sum() for xi in x]) == pb.n_dn).all()
        if pb.model == I.MODEL_TJ:
            assert not (x == 3).any()
        if c >= burn:
            for xi in x:
                counts[key[xi.tobytes()]] += 1
    emp = counts / counts.sum()
    tvd = 0.5 * np.abs(emp - p2).sum()
    print(f"TVD(empirical, |psi|^2) = {tvd:.4f}, TVD(|psi|^2, |psi|) = {tvd_12:.4f}")
    assert tvd < 0.04
    assert 0.5 * np.abs(emp - p1).sum() > 2 * tvd
