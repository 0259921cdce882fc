"""Serving measurement: a Poisson stream of sweep-step requests (local energies of a chain's
walkers, then one Woodbury commit per walker) over open chains of mixed lattices, models
and sizes, submitted open-loop to the continuous-batching server. Reports p50/p99 latency
(submission to completion) and throughput. Used by bench.py; callable on its own:
    python -m paper_2604_25775_gb300.serve_bench
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import binding as Bd
from . import inputs as I

CLASSES = ["hubbard8x8", "tj8x8", "hubbard16x16", "tj16x16", "hubbard32x32"]
SLOTS = {"hubbard8x8": 4096, "tj8x8": 4096, "hubbard16x16": 4096, "tj16x16": 4096, "hubbard32x32": 256}


def _open_chains(srv, problems, rng, n_chains, max_walkers):
    """Chains spread round-robin over the classes; walkers per chain log-uniform in
    [64, cap] with cap chosen so that every class's chains fit its slot pool at once."""
    per_class = [len(range(ci, n_chains, len(problems))) for ci in range(len(problems))]
    chains, lat = [], []
    for k in range(n_chains):
        ci = k % len(problems)
        cap = max(64, min(max_walkers, SLOTS[CLASSES[ci]] // per_class[ci]))
        n = int(np.exp(rng.uniform(np.log(64), np.log(cap)))) if cap > 64 else 64
        occ = I.random_configs(problems[ci], n, 4000 + k)
        chains.append({"cls": ci, "occ": occ, "id": srv.open(ci, occ), "n": n})
    for ch in chains:
        r = srv.poll(ch["id"], 600_000_000)
        assert r is not None and r[0] == 0, r
        lat.append(r[1])
    return chains, np.array(lat)


def _stream(srv, problems, chains, rate_hz, duration_s, rng):
    """Open-loop Poisson submissions; returns (latencies_us, walkers_done, wall_s)."""
    t_next = time.perf_counter()
    t_end = t_next + duration_s
    pending, lat = [], []
    walkers = 0
    lock = threading.Lock()
    done_flag = {"stop": False}

    def poller():
        while True:
            with lock:
                item = pending.pop(0) if pending else None
            if item is None:
                if done_flag["stop"]:
                    return
                time.sleep(1e-4)
                continue
            t, n = item
            r = srv.poll(t, 600_000_000)
            assert r is not None and r[0] == 0
            lat.append(r[1])

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    k = 0
    while True:
        now = time.perf_counter()
        if now >= t_end:
            break
        if now < t_next:
            time.sleep(min(t_next - now, 1e-3))
            continue
        ch = chains[int(rng.integers(len(chains)))]
        pb = problems[ch["cls"]]
        mv = I.random_hop_moves(pb, ch["occ"], 9000 + k)
        ch["occ"] = I.apply_moves(ch["occ"], mv)
        out = np.zeros(ch["n"])
        t = srv.step(ch["id"], mv, out)
        with lock:
            pending.append((t, ch["n"]))
        walkers += ch["n"]
        k += 1
        t_next += rng.exponential(1.0 / rate_hz)
    done_flag["stop"] = True
    th.join()
    return np.array(lat), walkers, time.perf_counter() - t0


def run(duration_s=8.0, n_chains=20, max_walkers=1024, load=0.6, seed=0):
    rng = np.random.default_rng(seed)
    problems = [I.workload(n) for n in CLASSES]
    classes = [(pb, I.random_params(pb, 300 + i), I.plane_wave_M0(pb), SLOTS[CLASSES[i]])
               for i, pb in enumerate(problems)]
    srv = Bd.Server(classes)
    t_open = time.perf_counter()
    chains, open_lat = _open_chains(srv, problems, rng, n_chains, max_walkers)
    t_open = time.perf_counter() - t_open
    # capacity: closed loop, every chain keeps one request in flight for a few rounds
    t0 = time.perf_counter()
    walkers = 0
    for rnd in range(3):
        ts = []
        for ch in chains:
            mv = I.random_hop_moves(problems[ch["cls"]], ch["occ"], 7000 + rnd)
            ch["occ"] = I.apply_moves(ch["occ"], mv)
            ts.append(srv.step(ch["id"], mv, np.zeros(ch["n"])))
            walkers += ch["n"]
        for t in ts:
            srv.poll(t, 600_000_000)
    cap_walkers_per_s = walkers / (time.perf_counter() - t0)
    mean_walkers = np.mean([c["n"] for c in chains])
    rate = load * cap_walkers_per_s / mean_walkers
    lat, done, wall = _stream(srv, problems, chains, rate, duration_s, rng)
    st = srv.stats()
    srv.destroy()
    return {"classes": CLASSES, "chains": n_chains, "walkers_per_chain": "log-uniform [64, %d]" % max_walkers,
            "open_s": t_open, "open_p50_ms": float(np.percentile(open_lat, 50) / 1e3),
            "open_p99_ms": float(np.percentile(open_lat, 99) / 1e3),
            "capacity_eloc_per_s": cap_walkers_per_s, "offered_load": load,
            "arrival_rate_hz": rate, "requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) / 1e3),
            "p99_ms": float(np.percentile(lat, 99) / 1e3), "throughput_eloc_per_s": done / wall,
            "batches": int(st["n_batches"]), "requests_total": int(st["n_requests"]),
            "resident_max_gb": st["resident_max_bytes"] / 1e9}


if __name__ == "__main__":
    import json
    print(json.dumps(run()))
