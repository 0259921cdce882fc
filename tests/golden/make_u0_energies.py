"""Writes u0_energies.json: the exact U = 0 (free-fermion) ground energy of Eq. H_h,
E0 = sum of the n_up lowest plus the n_dn lowest single-particle levels, with the levels
taken from the closed-form lattice dispersion
    torus:    eps(kx, ky) = -2t (cos kx + cos ky) - 4t' cos kx cos ky, k = 2 pi m / L
    open axis: cos k -> cos(pi m / (L + 1)), m = 1..L.
Closed form only; no call into the oracle or the CUDA library.

Usage: python tests/golden/make_u0_energies.py  (rewrites the json beside this file)
"""
import json
import math
import os

CASES = [
    # name, Lx, Ly, pbc_x, pbc_y, n_up, n_dn, t, tp
    ("hubbard4x4", 4, 4, 1, 1, 7, 7, 1.0, 0.0),
    ("hubbard8x8", 8, 8, 1, 1, 28, 28, 1.0, 0.0),
    ("hubbard16x16", 16, 16, 1, 1, 112, 112, 1.0, 0.0),
    ("hubbard32x32", 32, 32, 1, 1, 448, 448, 1.0, 0.0),
    ("cylinder16x4", 16, 4, 1, 0, 28, 28, 1.0, -0.2),
    ("open6x4_tp", 6, 4, 0, 0, 9, 8, 1.0, 0.3),
]


def cosines(L, periodic):
    if periodic:
        return [math.cos(2 * math.pi * m / L) for m in range(L)]
    return [math.cos(math.pi * m / (L + 1)) for m in range(1, L + 1)]


def e0(Lx, Ly, px, py, nu, nd, t, tp):
    lv = sorted(-2 * t * (a + b) - 4 * tp * a * b for a in cosines(Lx, px) for b in cosines(Ly, py))
    return sum(lv[:nu]) + sum(lv[:nd])


if __name__ == "__main__":
    out = {
        "_source": "closed-form U=0 ground energy of Eq. H_h (Sec. III), sum of lowest dispersion levels",
        "cases": {c[0]: {"Lx": c[1], "Ly": c[2], "pbc_x": c[3], "pbc_y": c[4], "n_up": c[5],
                         "n_dn": c[6], "t": c[7], "tp": c[8], "E0": e0(*c[1:])} for c in CASES},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "u0_energies.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))
