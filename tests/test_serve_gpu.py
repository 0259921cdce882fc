"""Serving on the GPU: continuous batching over device-resident chains of different
lattices and models. Each chain's results are the same alone and in the mix; admission
never exceeds the HBM budget; latencies are reported."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _classes():
    out = []
    for k, name in enumerate(["hubbard8x8", "tj8x8", "hubbard16x16"]):
        pb = I.workload(name)
        out.append((pb, I.random_params(pb, 50 + k), I.plane_wave_M0(pb), 512))
    return out


def _chains(classes, n_per_class, rng):
    chains = []
    for ci, (pb, _, _, _) in enumerate(classes):
        for j in range(n_per_class):
            n = int(rng.integers(16, 96))
            occ = I.random_configs(pb, n, 1000 * ci + j)
            moves = [I.random_hop_moves(pb, occ, 7 * j + s) for s in range(1)]
            chains.append((ci, occ, moves))
    return chains


def _run(server, chains, steps):
    """Per chain, all submitted at once without waiting: OPEN, ELOC, STEP, ELOC, LOGPSI,
    CLOSE. Chains beyond the budget wait for admission until earlier ones close.
    Returns per-chain results and request latencies."""
    results, lat, opens, tickets = {}, [], [], []
    for ci, occ, mv in chains:
        chain = server.open(ci, occ)
        n = occ.shape[0]
        e0, e1, e2, lp = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
        tickets += [server.eloc(chain, e0), server.step(chain, mv[0], e1), server.eloc(chain, e2),
                    server.logpsi(chain, lp)]
        results[chain] = (e0, e1, e2, lp)
        opens.append(chain)
        tickets.append(server.close(chain))
    for chain in opens:
        r = server.poll(chain, 120_000_000)
        assert r is not None and r[0] == 0
    for t in tickets:
        r = server.poll(t, 120_000_000)
        assert r is not None and r[0] == 0
        lat.append(r[1])
    return [results[c] for c in opens], np.array(lat)


def test_alone_equals_mix_and_budget():
    rng = np.random.default_rng(3)
    classes = _classes()
    chains = _chains(classes, 3, rng)
    # mix: everything submitted at once, budget for about half of the chains
    per = [Bd.scale_footprint_bytes(pb, slots) // slots for pb, _, _, slots in classes]
    need = sum(per[ci] * occ.shape[0] for ci, occ, _ in chains)
    budget = need // 2 + max(per) * 96
    srv = Bd.Server(classes, hbm_budget_bytes=budget)
    mixed, lat = _run(srv, chains, 1)
    st = srv.stats()
    assert st["resident_max_bytes"] <= budget
    assert st["n_batches"] < st["n_requests"]  # requests were merged into batches
    srv.destroy()
    print(f"mix: {len(lat)} requests, p50 {np.percentile(lat, 50) / 1e3:.2f} ms, "
          f"p99 {np.percentile(lat, 99) / 1e3:.2f} ms, batches {st['n_batches']}")
    # alone: one chain per server
    for k, (ci, occ, mv) in enumerate(chains[::3]):
        srv1 = Bd.Server(classes)
        alone, _ = _run(srv1, [(ci, occ, mv)], 1)
        srv1.destroy()
        for a, b in zip(alone[0], mixed[3 * k]):
            np.testing.assert_array_equal(a, b)


def test_results_match_direct_context():
    """A served chain's local energies equal those of a plain context on the same walkers."""
    import torch
    classes = _classes()[:1]
    pb, params, M0, _ = classes[0]
    occ = I.random_configs(pb, 40, 9)
    srv = Bd.Server(classes)
    chain = srv.open(0, occ)
    e = np.zeros(40)
    t = srv.eloc(chain, e)
    assert srv.poll(chain)[0] == 0 and srv.poll(t)[0] == 0
    srv.destroy()
    ctx = Bd.make_context(pb, params, M0, 40)
    ctx.scale_load(torch.from_numpy(occ).cuda())
    np.testing.assert_array_equal(ctx.local_energy().cpu().numpy(), e)


def test_oversized_open_rejected():
    classes = _classes()[:1]
    srv = Bd.Server(classes, hbm_budget_bytes=1 << 20)
    with pytest.raises(Bd.ScaleError) as ex:
        srv.open(0, I.random_configs(classes[0][0], 64, 1))
    assert ex.value.status == Bd.EBUDGET
    srv.destroy()


def test_poll_timeout_then_completion_and_cancel():
    """A poll whose bound runs out returns SCALE_ETIMEOUT while the request keeps running, and a
    later poll collects it; its local energies equal a plain context's. A request still waiting
    behind its chain's running request is cancelled: the ticket completes with SCALE_ECANCELED
    and its output is left untouched, the chain's next request runs normally, and a finished
    (released) ticket cannot be cancelled."""
    import torch
    pb = I.workload("hubbard16x16")
    params, M0 = I.random_params(pb, 52), I.plane_wave_M0(pb)
    B = 2048
    occ = I.random_configs(pb, B, 17)
    srv = Bd.Server([(pb, params, M0, B)])
    chain = srv.open(0, occ)
    assert srv.poll(chain, 600_000_000)[0] == Bd.OK
    e1, e2, e3 = np.zeros(B), np.full(B, 7.0), np.zeros(B)
    t1 = srv.eloc(chain, e1)  # milliseconds on the GPU
    t2 = srv.eloc(chain, e2)  # one request per chain per batch: waits behind t1
    assert srv.poll(t1, 1) is None  # a one-microsecond bound runs out; t1 keeps running
    assert srv.cancel(t2)
    r2 = srv.poll(t2, 1_000_000)
    assert r2 is not None and r2[0] == Bd.ECANCELED
    r1 = srv.poll(t1, 600_000_000)
    assert r1 is not None and r1[0] == Bd.OK
    assert not srv.cancel(t1)  # released by its poll
    assert (e2 == 7.0).all()
    t3 = srv.eloc(chain, e3)
    assert srv.poll(t3, 600_000_000)[0] == Bd.OK
    np.testing.assert_array_equal(e1, e3)
    srv.destroy()
    ctx = Bd.make_context(pb, params, M0, B)
    ctx.scale_load(torch.from_numpy(occ).cuda())
    np.testing.assert_array_equal(ctx.local_energy().cpu().numpy(), e1)
