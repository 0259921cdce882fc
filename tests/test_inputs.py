"""Seeded input generators: validity and determinism (no method arithmetic here)."""
import numpy as np

from paper_2604_25775_gb300 import inputs as I


def test_configs_valid_and_deterministic():
    for name in ("hubbard4x4", "hubbard16x16", "tj8x8", "cylinder16x4"):
        pb = I.workload(name)
        occ = I.random_configs(pb, 16, 5)
        assert occ.dtype == np.int8 and occ.shape == (16, pb.N)
        assert ((occ & 1).sum(1) == pb.n_up).all()
        assert (((occ >> 1) & 1).sum(1) == pb.n_dn).all()
        if pb.model == I.MODEL_TJ:
            assert not (occ == 3).any()
        assert np.array_equal(occ, I.random_configs(pb, 16, 5))


def test_param_count_and_distribution():
    pb = I.workload("hubbard16x16")
    p = I.random_params(pb, 1236)
    n = pb.N * 4 * pb.h + (9 * pb.h * pb.h + pb.h) + 5 * (pb.h * pb.h + pb.h) + pb.h * 2 * pb.Ne + 2 * pb.Ne
    assert p.size == I.param_count(pb) == n
    assert abs(p.std() - 0.05) < 0.002 and abs(p.mean()) < 0.002


def test_moves_are_allowed():
    pb = I.workload("tj8x8")
    occ = I.random_configs(pb, 32, 1)
    mv = I.random_hop_moves(pb, occ, 2)
    after = I.apply_moves(occ, mv)
    assert ((after & 1).sum(1) == pb.n_up).all()
    assert not (after == 3).any()
    assert (mv[:, 0] == I.MOVE_HOP).sum() >= 28


def test_tanh_series_and_identity_bound():
    """The FP32 tanh of the tensor-core layers uses the odd Taylor series through z^15 for
    |z| < 0.5 and (1 - e^{-2|z|})/(1 + e^{-2|z|}) above; in exact arithmetic the series'
    truncation error is below 1e-8 relative (FP32 rounding is checked by the GPU parity)."""
    import numpy as np
    c = [1.0, -1 / 3, 2 / 15, -17 / 315, 62 / 2835, -1382 / 155925, 21844 / 6081075, -929569 / 638512875]
    z = np.linspace(-0.5, 0.5, 20001)
    series = sum(ck * z ** (2 * k + 1) for k, ck in enumerate(c))
    assert np.max(np.abs(series - np.tanh(z)) / np.maximum(np.abs(np.tanh(z)), 1e-300)) < 1e-8
    z2 = np.linspace(0.5, 20, 20001)
    e = np.exp(-2 * z2)
    assert np.max(np.abs((1 - e) / (1 + e) - np.tanh(z2))) < 1e-15
