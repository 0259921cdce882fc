"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds no arithmetic of the method (no network, determinant or Hamiltonian
action). It only describes a problem (lattice, Hamiltonian constants, network shape) and
draws its inputs:

* occupation configurations, uniformly random among the valid ones
  (local states of Sec. II.B "Embedding Layer": 0 = empty, 1 = up, 2 = down, 3 = up+down);
* a flat float64 parameter vector, every entry i.i.d. N(0, scale^2) in a fixed tensor order;
* the plane-wave reference orbitals M0 (an input added to the orbital projection, not a
  learnable parameter), built from the closed-form eigenvectors of the hopping matrix;
* connected-move proposals for chain tests and benches.

Parameter layout (flat, float64, in this order; the C header documents the same order):
  embed   [N][4][h]   (per-site tables E_i, Sec. II.B) or [4][h] when shared
  for each layer l:  kernel [k_l][k_l][h][h] (ky, kx, c_in, c_out), bias [h]
  proj_w  [h][2*Ne]   columns [0,Ne) build rows (i, up), [Ne, 2Ne) rows (i, down)
  proj_b  [2*Ne]
The ACE family (Eq. ACE) uses the same order with per-layer widths: layers [0, n_conv) are
conv blocks h -> h followed by ln_gamma [h] and ln_beta [h] of the layer normalisation;
the site-wise layers after them map h -> h_mlp, then h_mlp -> h_mlp; proj_w is
[h_mlp][2*Ne]. The layer-normalisation gains are drawn as 1 + N(0, scale^2). The wide SCALE
family uses the same per-layer widths without normalisation. With the disk stencil a
kernel is stored for its taps only, [taps][c_in][c_out], taps in row-major box order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

MODEL_HUBBARD = 0
MODEL_TJ = 1
MODEL_HUBBARD_PH = 2  # Hubbard after the particle-hole transformation of the down spins
ACT_TANH = 0
ACT_SILU = 1
FAMILY_SCALE = 0
FAMILY_ACE = 1
FAMILY_WIDE = 2   # the SCALE layout at Table tab:model widths, full recompute only
STENCIL_BOX = 0   # k x k offsets
STENCIL_DISK = 1  # offsets of the k x k box within L2 distance (k-1)/2 (k = 5: SCALE-L's 13 sites)
PREC_FP64 = 0
PREC_MIXED = 1
PREC_MIXED_BF16 = 2
PREC_MIXED_FP16 = 3

LOWRANK_WARP = 0     # low-rank local-energy kernels of the library (same results)
LOWRANK_BATCHED = 1

MOVE_NONE = -1
MOVE_HOP = 0
MOVE_EXCHANGE = 1


@dataclasses.dataclass
class Problem:
    """Lattice + Hamiltonian + network shape. Plain data; see the module docstring."""

    Lx: int
    Ly: int
    pbc_x: int = 1
    pbc_y: int = 1
    n_up: int = 1
    n_dn: int = 1
    model: int = MODEL_HUBBARD
    t: float = 1.0
    tp: float = 0.0
    U: float = 8.0
    J: float = 0.0
    n_layers: int = 2
    h: int = 8
    ksize: Sequence[int] = (3, 1)
    residual: Sequence[int] = (1, 0)
    act: int = ACT_TANH
    per_site_embed: int = 1
    precision: int = PREC_FP64
    refresh_every: int = 64
    drift_tol: float = 1e-4
    family: int = FAMILY_SCALE
    n_conv: int = 0       # ACE: number of conv blocks with layer normalisation
    h_mlp: int = 0        # ACE: width of the site-wise layers (0 = h)
    ln_eps: float = 1e-5  # ACE: layer-normalisation epsilon
    stencil: int = STENCIL_BOX
    lowrank_kernel: int = 0  # LOWRANK_WARP or LOWRANK_BATCHED (a kernel choice of the library)

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    @property
    def Ne(self) -> int:
        return self.n_up + self.n_dn

    def as_dict(self) -> dict:
        d = dataclasses.asdict(self)
        d["ksize"] = list(self.ksize)
        d["residual"] = list(self.residual)
        return d

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def scale_layout(L: int, ksize_first: int = 3, conv_residual: int = 1):
    """Per-layer kernel sizes / residual flags for the SCALE layer layout of Sec. II.B:
    one k x k convolution with a residual (Eq. conv) followed by L-1 site-wise layers
    without residual (Eq. MLP)."""
    ks = [ksize_first] + [1] * (L - 1)
    rs = [conv_residual] + [0] * (L - 1)
    return ks, rs


def ace_layout(n_conv: int, n_mlp: int, ksize: int = 3):
    """Kernel sizes / residual flags of the ACE layout (Eq. ACE): n_conv residual k x k
    conv blocks (each followed by a layer normalisation), then n_mlp site-wise layers."""
    return [ksize] * n_conv + [1] * n_mlp, [1] * n_conv + [0] * n_mlp


def stencil_taps(k: int, stencil: int):
    """(dx, dy) offsets of a k x k layer's stencil in row-major box order."""
    r = (k - 1) // 2
    return [(dx, dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1)
            if stencil == STENCIL_BOX or dx * dx + dy * dy <= r * r]


def layer_widths(pb: Problem, l: int):
    """(c_in, c_out) of layer l."""
    hm = pb.h_mlp or pb.h
    if pb.family == FAMILY_SCALE:
        return pb.h, pb.h
    c_out = pb.h if l < pb.n_conv else hm
    c_in = pb.h if l <= pb.n_conv else hm
    return c_in, c_out


def param_shapes(pb: Problem) -> List[tuple]:
    """(name, shape) of every parameter tensor in flat-vector order."""
    N, h, Ne = pb.N, pb.h, pb.Ne
    shapes = [("embed", (N, 4, h) if pb.per_site_embed else (4, h))]
    c_last = h
    for l in range(pb.n_layers):
        k = int(pb.ksize[l])
        ci, co = layer_widths(pb, l)
        if pb.stencil == STENCIL_DISK:
            shapes.append((f"kernel{l}", (len(stencil_taps(k, pb.stencil)), ci, co)))
        else:
            shapes.append((f"kernel{l}", (k, k, ci, co)))
        shapes.append((f"bias{l}", (co,)))
        if pb.family == FAMILY_ACE and l < pb.n_conv:
            shapes.append((f"ln_gamma{l}", (co,)))
            shapes.append((f"ln_beta{l}", (co,)))
        c_last = co
    shapes.append(("proj_w", (c_last, 2 * Ne)))
    shapes.append(("proj_b", (2 * Ne,)))
    return shapes


def param_count(pb: Problem) -> int:
    return int(sum(int(np.prod(s)) for _, s in param_shapes(pb)))


def param_offsets(pb: Problem) -> dict:
    off, out = 0, {}
    for name, s in param_shapes(pb):
        n = int(np.prod(s))
        out[name] = (off, s)
        off += n
    return out


def random_params(pb: Problem, seed: int, scale: float = 0.05) -> np.ndarray:
    """Every learnable entry i.i.d. N(0, scale^2) from PCG64(seed), tensors in layout order."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, scale, size=int(np.prod(s))) + (1.0 if name.startswith("ln_gamma") else 0.0)
             for name, s in param_shapes(pb)]
    return np.concatenate(parts).astype(np.float64)


def random_configs(pb: Problem, B: int, seed: int) -> np.ndarray:
    """B uniformly random configurations with exactly n_up / n_dn electrons.

    Hubbard: up and down sites drawn independently without replacement.
    t-J: n_up + n_dn distinct sites, a uniformly random n_up-subset of them is up
    (no double occupancy, the Gutzwiller-projected space of Eq. ham-tj)."""
    rng = np.random.default_rng(seed)
    N = pb.N
    occ = np.zeros((B, N), dtype=np.int8)
    for b in range(B):
        if pb.model == MODEL_TJ:
            sites = rng.choice(N, pb.n_up + pb.n_dn, replace=False)
            perm = rng.permutation(pb.n_up + pb.n_dn)
            up = sites[perm[: pb.n_up]]
            dn = sites[perm[pb.n_up:]]
        else:
            up = rng.choice(N, pb.n_up, replace=False)
            dn = rng.choice(N, pb.n_dn, replace=False)
        occ[b, up] |= 1
        occ[b, dn] |= 2
    return occ


def _chain_modes(L: int, periodic: int):
    """Real one-dimensional modes of a chain of L sites (nearest-neighbour adjacency):
    returns (list of (cos-of-wavevector, label tuple), mode matrix [L][n_modes])."""
    x = np.arange(L)
    modes, labels = [], []
    if periodic:
        for m in range(L):
            mm = (L - m) % L
            if mm < m:
                continue  # pair {m, L-m} represented once
            k = 2.0 * math.pi * m / L
            if mm == m:  # k == -k (m = 0 or m = L/2)
                modes.append(np.cos(k * x) / math.sqrt(L))
                labels.append((math.cos(k), m, 0))
            else:
                modes.append(np.cos(k * x) * math.sqrt(2.0 / L))
                labels.append((math.cos(k), m, 0))
                modes.append(np.sin(k * x) * math.sqrt(2.0 / L))
                labels.append((math.cos(k), m, 1))
    else:
        for m in range(1, L + 1):
            q = math.pi * m / (L + 1)
            modes.append(np.sin(q * (x + 1)) * math.sqrt(2.0 / (L + 1)))
            labels.append((math.cos(q), m, 0))
    return labels, np.stack(modes, axis=1)


def plane_wave_orbitals(pb: Problem):
    """Single-particle eigenvectors of the hopping matrix of Eq. H_h (NN amplitude -t,
    NNN amplitude -t'), as real products of chain modes, sorted by energy.

    Energy of the product mode (a, b): -2t(ca + cb) - 4t' ca cb, with ca, cb the
    cosines of the two chain wave-vectors. Returns (energies [N], vectors [N][N]),
    site index i = y*Lx + x. Ties are ordered by the mode labels (cos before sin)."""
    lx, mx = _chain_modes(pb.Lx, pb.pbc_x)
    ly, my = _chain_modes(pb.Ly, pb.pbc_y)
    entries = []
    for a, (ca, ma, sa) in enumerate(lx):
        for b, (cb, mb, sb) in enumerate(ly):
            e = -2.0 * pb.t * (ca + cb) - 4.0 * pb.tp * ca * cb
            entries.append((round(e, 12), ma, mb, sa, sb, a, b, e))
    entries.sort(key=lambda r: r[:5])
    N = pb.N
    vecs = np.zeros((N, N))
    eps = np.zeros(N)
    for col, r in enumerate(entries):
        a, b = r[5], r[6]
        # site (x, y) -> y*Lx + x
        vecs[:, col] = np.outer(my[:, b], mx[:, a]).reshape(-1)
        eps[col] = r[7]
    return eps, vecs


def plane_wave_M0(pb: Problem) -> np.ndarray:
    """Reference orbital matrix M0 [2N][Ne]: block diagonal, rows (up, i) hold the n_up
    lowest plane waves in columns [0, n_up), rows (down, i) the n_dn lowest in
    columns [n_up, Ne). Orbital row index o = sigma*N + i."""
    _, vecs = plane_wave_orbitals(pb)
    N, Ne = pb.N, pb.Ne
    M0 = np.zeros((2 * N, Ne))
    M0[:N, : pb.n_up] = vecs[:, : pb.n_up]
    M0[N:, pb.n_up:] = vecs[:, : pb.n_dn]
    return M0


def metropolis_randoms(pb: Problem, B: int, S: int, seed: int):
    """Random inputs of S Metropolis steps for B chains: the electron pick [S][B] int32 in
    [0, Ne) (rank of the electron in ascending orbital order), the hop direction [S][B]
    int32 in [0, 4) (+x, -x, +y, -y) and the acceptance uniform [S][B] float64 in [0, 1)."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, pb.Ne, size=(S, B), dtype=np.int32)
    direction = rng.integers(0, 4, size=(S, B), dtype=np.int32)
    u = rng.random((S, B))
    return pick, direction, u


def symmetry_group(pb: Problem, translations: bool = True, reflections: bool = False,
                   spin_inversion: bool = False):
    """Orbital permutations [G][2N] int32 of a lattice symmetry group (o = s*N + i): the
    translations of the periodic axes, the reflections x -> -x and y -> -y (about the
    lattice centre on open axes), and the exchange of the two spins, all products of the
    chosen generators. Row 0 is the identity."""
    N, Lx, Ly = pb.N, pb.Lx, pb.Ly
    site_maps = []
    txs = range(Lx) if (translations and pb.pbc_x) else [0]
    tys = range(Ly) if (translations and pb.pbc_y) else [0]
    rxs = (False, True) if reflections else (False,)
    rys = (False, True) if reflections else (False,)
    for rx in rxs:
        for ry in rys:
            for tx in txs:
                for ty in tys:
                    m = np.zeros(N, dtype=np.int64)
                    for i in range(N):
                        x, y = i % Lx, i // Lx
                        if rx:
                            x = (-x) % Lx if pb.pbc_x else Lx - 1 - x
                        if ry:
                            y = (-y) % Ly if pb.pbc_y else Ly - 1 - y
                        m[i] = ((y + ty) % Ly) * Lx + (x + tx) % Lx
                    site_maps.append(m)
    perms = []
    for m in site_maps:
        for flip in ((False, True) if spin_inversion else (False,)):
            p = np.zeros(2 * N, dtype=np.int32)
            for s in range(2):
                for i in range(N):
                    p[s * N + i] = ((1 - s) if flip else s) * N + m[i]
            perms.append(p)
    return np.array(perms, dtype=np.int32)


def random_hop_moves(pb: Problem, occ: np.ndarray, seed: int) -> np.ndarray:
    """One proposed nearest-neighbour move per sample, int32 [B][4] = (kind, src, dst, spin).

    Hop: an electron of spin `spin` on `src` moves to the neighbour `dst` where that
    spin-orbital is empty (t-J: `dst` fully empty). kind = MOVE_NONE when the drawn
    site has no allowed move. Only used to drive chain benches and tests."""
    rng = np.random.default_rng(seed)
    B, N = occ.shape
    out = np.full((B, 4), MOVE_NONE, dtype=np.int32)
    for b in range(B):
        for _ in range(64):
            src = int(rng.integers(N))
            spin = int(rng.integers(2))
            if not (occ[b, src] >> spin) & 1:
                continue
            x, y = src % pb.Lx, src // pb.Lx
            d = int(rng.integers(4))
            dx, dy = [(1, 0), (-1, 0), (0, 1), (0, -1)][d]
            xx, yy = x + dx, y + dy
            if not (0 <= xx < pb.Lx):
                if not pb.pbc_x:
                    continue
                xx %= pb.Lx
            if not (0 <= yy < pb.Ly):
                if not pb.pbc_y:
                    continue
                yy %= pb.Ly
            dst = yy * pb.Lx + xx
            if (occ[b, dst] >> spin) & 1:
                continue
            if pb.model == MODEL_TJ and occ[b, dst] != 0:
                continue
            out[b] = (MOVE_HOP, src, dst, spin)
            break
    return out


def apply_moves(occ: np.ndarray, moves: np.ndarray) -> np.ndarray:
    """Occupations after the given moves (bookkeeping only; no amplitudes)."""
    out = occ.copy()
    for b in range(occ.shape[0]):
        kind, src, dst, spin = (int(v) for v in moves[b])
        if kind == MOVE_HOP:
            out[b, src] &= ~(1 << spin)
            out[b, dst] |= 1 << spin
        elif kind == MOVE_EXCHANGE:
            out[b, src], out[b, dst] = out[b, dst], out[b, src]
    return out


# ---------------------------------------------------------------------------------------
# Named workloads: the lattices, dopings and network shapes the method is exercised on.
# Seeds: parameters 1234 + index, configurations 5678 + index.
# ---------------------------------------------------------------------------------------

def workload(name: str) -> Problem:
    if name == "hubbard4x4":  # 4x4 torus, 7+7, 2 layers, 8 channels, FP64
        ks, rs = scale_layout(2)
        return Problem(4, 4, 1, 1, 7, 7, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 2, 8, ks, rs,
                       ACT_TANH, 1, PREC_FP64, 64, 1e-10)
    if name == "hubbard8x8":  # 8x8 torus, 1/8 doping 28+28, 4 layers, 16 channels
        ks, rs = scale_layout(4)
        return Problem(8, 8, 1, 1, 28, 28, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 4, 16, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    if name == "hubbard16x16":  # 16x16 torus, 112+112, 6 layers, 32 channels, mixed (FP16x3 site-wise)
        ks, rs = scale_layout(6)
        return Problem(16, 16, 1, 1, 112, 112, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 6, 32, ks, rs,
                       ACT_TANH, 1, PREC_MIXED_FP16, 64, 1e-4)
    if name == "cylinder16x4":  # periodic along 16, open along 4, t'=-0.2, 12 residual 3x3
        return Problem(16, 4, 1, 0, 28, 28, MODEL_HUBBARD, 1.0, -0.2, 8.0, 0.0, 12, 32,
                       [3] * 12, [1] * 12, ACT_TANH, 1, PREC_FP64, 64, 1e-10)
    if name == "tj8x8":
        ks, rs = scale_layout(4)
        return Problem(8, 8, 1, 1, 28, 28, MODEL_TJ, 1.0, 0.0, 0.0, 0.4, 4, 16, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    if name == "hubbard_ph8x8":  # attractive U=-4 at 28+28, after the particle-hole transformation: 28 + (64-28)
        ks, rs = scale_layout(4)
        return Problem(8, 8, 1, 1, 28, 36, MODEL_HUBBARD_PH, 1.0, 0.0, -4.0, 0.0, 4, 16, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    if name == "ace4x4":  # 4x4 torus, 7+7, 3 conv blocks + 2 site-wise layers, h 8 -> 12, FP64
        ks, rs = ace_layout(3, 2)
        return Problem(4, 4, 1, 1, 7, 7, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 5, 8, ks, rs,
                       ACT_SILU, 1, PREC_FP64, 64, 1e-10, FAMILY_ACE, 3, 12)
    if name == "ace8x8":  # 8x8 torus, 28+28, 16 conv blocks h=48, 2 site-wise layers h=64, mixed
        ks, rs = ace_layout(16, 2)
        return Problem(8, 8, 1, 1, 28, 28, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 18, 48, ks, rs,
                       ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_ACE, 16, 64)
    if name == "ace16x16":  # Table tab:model ACE: 16 conv blocks h=144, 2 site-wise layers h=256
        ks, rs = ace_layout(16, 2)
        return Problem(16, 16, 1, 1, 112, 112, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 18, 144, ks, rs,
                       ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_ACE, 16, 256)
    if name == "ace16x4":  # ACE on the periodic 16x4 lattice of the symmetry study, t'=0, 28+28
        ks, rs = ace_layout(16, 2)
        return Problem(16, 4, 1, 1, 28, 28, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 18, 144, ks, rs,
                       ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_ACE, 16, 256)
    if name == "scale_plus16x16":  # the bench network with SCALE-L's 13-site plus stencil (cached update)
        ks, rs = scale_layout(6, ksize_first=5)
        return Problem(16, 16, 1, 1, 112, 112, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 6, 32, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4, FAMILY_SCALE, 0, 0, 1e-5, STENCIL_DISK)
    if name == "scale_plus6x6":  # plus stencil, SCALE family, FP64 (parity of the cached update)
        ks, rs = scale_layout(2, ksize_first=5)
        return Problem(6, 6, 1, 1, 12, 12, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 2, 8, ks, rs,
                       ACT_TANH, 1, PREC_FP64, 64, 1e-10, FAMILY_SCALE, 0, 0, 1e-5, STENCIL_DISK)
    if name == "scale_l5x5":  # SCALE-L layout (13-site plus stencil), small widths, FP64
        return Problem(5, 5, 1, 1, 8, 8, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 3, 6, [5, 1, 1], [1, 0, 0],
                       ACT_SILU, 1, PREC_FP64, 64, 1e-10, FAMILY_WIDE, 1, 10, 1e-5, STENCIL_DISK)
    if name == "scale_l8x8":  # SCALE-L layout at 8x8, 28+28, widths 96 / 128, mixed
        return Problem(8, 8, 1, 1, 28, 28, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 5, 96, [5, 1, 1, 1, 1],
                       [1, 0, 0, 0, 0], ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_WIDE, 1, 128, 1e-5,
                       STENCIL_DISK)
    if name == "scale_l16x16":  # Table tab:model SCALE-L: plus stencil (L2 <= 2), h 384, 4 x 512
        return Problem(16, 16, 1, 1, 112, 112, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 5, 384, [5, 1, 1, 1, 1],
                       [1, 0, 0, 0, 0], ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_WIDE, 1, 512, 1e-5,
                       STENCIL_DISK)
    if name == "scale_xl32x32":  # Table tab:model SCALE-XL (32x32 only): 3x3, h 640, 4 x 1280
        return Problem(32, 32, 1, 1, 448, 448, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 5, 640, [3, 1, 1, 1, 1],
                       [1, 0, 0, 0, 0], ACT_SILU, 1, PREC_MIXED, 64, 1e-4, FAMILY_WIDE, 1, 1280)
    if name == "tj16x16":
        ks, rs = scale_layout(6)
        return Problem(16, 16, 1, 1, 112, 112, MODEL_TJ, 1.0, 0.0, 0.0, 0.4, 6, 32, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    if name == "hubbard32x32":
        ks, rs = scale_layout(4)
        return Problem(32, 32, 1, 1, 448, 448, MODEL_HUBBARD, 1.0, 0.0, 8.0, 0.0, 4, 16, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    if name == "tj32x32":
        ks, rs = scale_layout(4)
        return Problem(32, 32, 1, 1, 448, 448, MODEL_TJ, 1.0, 0.0, 0.0, 0.4, 4, 16, ks, rs,
                       ACT_TANH, 1, PREC_MIXED, 64, 1e-4)
    raise KeyError(name)


WORKLOAD_INDEX = {"hubbard4x4": 0, "hubbard8x8": 1, "hubbard16x16": 2, "cylinder16x4": 3,
                  "tj8x8": 4, "tj16x16": 4, "hubbard32x32": 4, "tj32x32": 4,
                  "hubbard_ph8x8": 5, "ace4x4": 6, "ace8x8": 6, "ace16x16": 6, "ace16x4": 6,
                  "scale_l5x5": 7, "scale_l8x8": 7, "scale_l16x16": 7, "scale_xl32x32": 7,
                  "scale_plus16x16": 2, "scale_plus6x6": 8}


def workload_seeds(name: str):
    i = WORKLOAD_INDEX[name]
    return 1234 + i, 5678 + i
