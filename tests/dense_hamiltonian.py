"""Independent dense Hamiltonian for tiny lattices (test helper, not the oracle).

Written separately from the oracle's operator code: basis states are integers whose bit
o is the occupation of orbital o = sigma*N + i, the Jordan-Wigner sign of an operator on
orbital o is the parity of the set bits below o (popcount), and the bonds are rebuilt here
from the lattice geometry. Used to pin the oracle's E_loc through <psi|H|psi> and to get
exact ground energies (Eq. H_h, Eq. ham-tj).
"""
from __future__ import annotations

import itertools

import numpy as np


def bonds(Lx, Ly, pbc_x, pbc_y, diagonal=False):
    """Unordered bonds; nearest neighbours, or next-nearest (diagonal) ones."""
    out = set()
    offs = [(1, 1), (1, -1)] if diagonal else [(1, 0), (0, 1)]
    for y in range(Ly):
        for x in range(Lx):
            for dx, dy in offs:
                xx, yy = x + dx, y + dy
                if not 0 <= xx < Lx:
                    if not pbc_x:
                        continue
                    xx %= Lx
                if not 0 <= yy < Ly:
                    if not pbc_y:
                        continue
                    yy %= Ly
                a, b = y * Lx + x, yy * Lx + xx
                if a == b:
                    continue
                out.add((min(a, b), max(a, b)))
    return sorted(out)


def _parity_below(state, o):
    return bin(state & ((1 << o) - 1)).count("1") & 1


def _c(state, o):
    if not (state >> o) & 1:
        return None, 0
    return state ^ (1 << o), (-1 if _parity_below(state, o) else 1)


def _cdag(state, o):
    if (state >> o) & 1:
        return None, 0
    return state | (1 << o), (-1 if _parity_below(state, o) else 1)


def basis(d):
    N = d["Lx"] * d["Ly"]
    states = []
    for up in itertools.combinations(range(N), d["n_up"]):
        for dn in itertools.combinations(range(N), d["n_dn"]):
            if d["model"] == 1 and set(up) & set(dn):
                continue
            s = 0
            for i in up:
                s |= 1 << i
            for i in dn:
                s |= 1 << (N + i)
            states.append(s)
    return states


def state_to_occ(s, N):
    occ = np.zeros(N, dtype=np.int8)
    for i in range(N):
        occ[i] = ((s >> i) & 1) | (((s >> (N + i)) & 1) << 1)
    return occ


def dense_h(d):
    """Dense H over the particle-number sector (t-J: Gutzwiller-projected sector)."""
    N = d["Lx"] * d["Ly"]
    states = basis(d)
    index = {s: k for k, s in enumerate(states)}
    H = np.zeros((len(states), len(states)))
    nn = bonds(d["Lx"], d["Ly"], d["pbc_x"], d["pbc_y"], False)
    nnn = bonds(d["Lx"], d["Ly"], d["pbc_x"], d["pbc_y"], True) if d["tp"] != 0 else []
    for k, s in enumerate(states):
        up = [(s >> i) & 1 for i in range(N)]
        dn = [(s >> (N + i)) & 1 for i in range(N)]
        if d["model"] == 0:
            H[k, k] += d["U"] * sum(u * v for u, v in zip(up, dn))
        elif d["model"] == 2:  # particle-hole transformed Hubbard: n_dn -> 1 - n_dn
            H[k, k] += d["U"] * sum(u * (1 - v) for u, v in zip(up, dn))
        else:
            for i, j in nn:
                H[k, k] += d["J"] * 0.25 * (up[i] - dn[i]) * (up[j] - dn[j])
        for amp, blist in ((d["t"], nn), (d["tp"], nnn)):
            for i, j in blist:
                for sg in (0, 1):
                    for a, b in ((i, j), (j, i)):
                        # -amp * c+_{b,sg} c_{a,sg}
                        s1, f1 = _c(s, sg * N + a)
                        if s1 is None:
                            continue
                        s2, f2 = _cdag(s1, sg * N + b)
                        if s2 is None:
                            continue
                        if s2 not in index:
                            continue  # left the (projected) sector
                        H[index[s2], k] += -amp * f1 * f2
        if d["model"] == 1:
            for i, j in nn:
                for a, b in ((i, j), (j, i)):
                    # (J/2) S+_a S-_b = (J/2) c+_{a up} c_{a dn} c+_{b dn} c_{b up}
                    st, f = s, 1
                    for op, o in ((_c, b), (_cdag, N + b), (_c, N + a), (_cdag, a)):
                        st, ff = op(st, o)
                        if st is None:
                            break
                        f *= ff
                    if st is None or st not in index:
                        continue
                    H[index[st], k] += 0.5 * d["J"] * f
    return H, states
