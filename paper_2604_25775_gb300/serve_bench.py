"""Serving measurement: open-loop Poisson streams of local-energy requests over open chains of
mixed lattices and models, submitted to the continuous-batching server. Each chain's walkers
stay on the device between requests. Reported per offered load (a fraction of the measured
capacity): p50 / p99 latency from submission to completion and throughput. Used by bench.py;
callable on its own:
    python -m paper_2604_25775_gb300.serve_bench [requests_per_load]
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import binding as Bd
from . import inputs as I

# the request mix: every lattice with both models, 1/8 doping (32x32: 448 + 448 electrons)
CLASSES = ["hubbard8x8", "tj8x8", "hubbard16x16", "tj16x16", "hubbard32x32", "tj32x32"]
LOADS = (0.3, 0.6, 0.9)


def _open_chains(srv, problems, sizes):
    """Open every chain (sizes[class][k] walkers) and wait for the loads."""
    chains, tickets = [], []
    for ci, pb in enumerate(problems):
        for k, n in enumerate(sizes[ci]):
            occ = I.random_configs(pb, n, 4000 + 10 * ci + k)
            t = srv.open(ci, occ)
            chains.append({"cls": ci, "id": t, "n": n})
            tickets.append(t)
    lat = []
    for t in tickets:
        r = srv.poll(t, 2_000_000_000)
        assert r is not None and r[0] == 0, r
        lat.append(r[1])
    return chains, np.array(lat)


def _stream(srv, chains, rate_hz, n_requests, rng):
    """Open-loop Poisson submission of n_requests local-energy requests, each to a chain drawn
    uniformly; returns (latencies_us, walkers_done, wall_s)."""
    pending, lat = [], []
    lock = threading.Lock()
    stop = {"flag": False}

    def poller():
        while True:
            with lock:
                item = pending.pop(0) if pending else None
            if item is None:
                if stop["flag"]:
                    return
                time.sleep(1e-4)
                continue
            r = srv.poll(item, 2_000_000_000)
            assert r is not None and r[0] == 0
            lat.append(r[1])

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    walkers = 0
    for _ in range(n_requests):
        now = time.perf_counter()
        while now < t_next:
            time.sleep(min(t_next - now, 1e-3))
            now = time.perf_counter()
        ch = chains[int(rng.integers(len(chains)))]
        t = srv.eloc(ch["id"], np.zeros(ch["n"]))
        with lock:
            pending.append(t)
        walkers += ch["n"]
        t_next += rng.exponential(1.0 / rate_hz)
    stop["flag"] = True
    th.join()
    return np.array(lat), walkers, time.perf_counter() - t0


def run(requests_per_load=2000, chains_per_class=4, walkers=(64, 4096), loads=LOADS, seed=0):
    rng = np.random.default_rng(seed)
    problems = [I.workload(n) for n in CLASSES]
    lo, hi = walkers
    sizes = [[int(np.exp(rng.uniform(np.log(lo), np.log(hi)))) for _ in range(chains_per_class)]
             for _ in problems]
    classes = [(pb, I.random_params(pb, 300 + i), I.plane_wave_M0(pb), sum(sizes[i]))
               for i, pb in enumerate(problems)]
    srv = Bd.Server(classes)
    t_open = time.perf_counter()
    chains, open_lat = _open_chains(srv, problems, sizes)
    t_open = time.perf_counter() - t_open
    # capacity: closed loop, every chain keeps one local-energy request in flight for 3 rounds
    t0 = time.perf_counter()
    done = 0
    for _ in range(3):
        ts = [srv.eloc(ch["id"], np.zeros(ch["n"])) for ch in chains]
        for t in ts:
            assert srv.poll(t, 2_000_000_000)[0] == 0
        done += sum(ch["n"] for ch in chains)
    capacity = done / (time.perf_counter() - t0)
    mean_walkers = float(np.mean([ch["n"] for ch in chains]))
    points = []
    for load in loads:
        rate = load * capacity / mean_walkers
        lat, w, wall = _stream(srv, chains, rate, requests_per_load, rng)
        points.append({"offered_load": load, "arrival_rate_hz": rate, "requests": int(len(lat)),
                       "p50_ms": float(np.percentile(lat, 50) / 1e3), "p99_ms": float(np.percentile(lat, 99) / 1e3),
                       "throughput_eloc_per_s": w / wall, "wall_s": wall})
    st = srv.stats()
    srv.destroy()
    return {"classes": CLASSES, "chains": len(chains),
            "walkers_per_chain": f"log-uniform in [{lo}, {hi}], drawn per chain: "
                                 + ", ".join(str(sum(s)) for s in sizes) + " walkers per class",
            "request": "local energies of every walker of the chain",
            "open_s": t_open, "open_p50_ms": float(np.percentile(open_lat, 50) / 1e3),
            "open_p99_ms": float(np.percentile(open_lat, 99) / 1e3),
            "capacity_eloc_per_s": capacity, "points": points,
            "batches": int(st["n_batches"]), "requests_total": int(st["n_requests"]),
            "resident_max_gb": st["resident_max_bytes"] / 1e9}


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(run(int(sys.argv[1]) if len(sys.argv) > 1 else 2000)))
