"""Timings of the paths beyond the SCALE chain step, used by bench.py and callable on
their own (one GPU, inputs resident on the device, CUDA events on the context's stream):

    python -m paper_2604_25775_gb300.next_bench ace [walkers]
        ACE (Sec. II "ACE", Table tab:model shape: 16 conv blocks at h = 144, two site-wise
        layers at 256) on the 16x16 torus, 112 + 112: the full-recompute local energy of
        `walkers` walkers (every psi(n') a fresh forward and FP64 LU), and the amplitudes of
        1024 configurations (forward + determinant).
    python -m paper_2604_25775_gb300.next_bench wide [walkers]
        Table tab:model SCALE-L (plus stencil, conv 384, site-wise 4 x 512) local energies on
        the 16x16 torus and SCALE-XL (conv 640, site-wise 4 x 1280) amplitudes on the 32x32
        torus, both by full recompute.
    python -m paper_2604_25775_gb300.next_bench plus [walkers]
        Low-rank local energies of the bench network with SCALE-L's plus stencil.
    python -m paper_2604_25775_gb300.next_bench symmetry [walkers]
        The symmetry-projected amplitude (App. "Symmetry Projection") over the 256
        translations of the SCALE 16x16 bench workload.
    python -m paper_2604_25775_gb300.next_bench grad [walkers]
        Per-sample d log|psi| / d theta on the gradient workload: the 16x4 cylinder (periodic
        along 16, open along 4), t' = -0.2, 28 + 28, 12 residual 3x3 layers of 32 channels
        (123,392 parameters), FP64 and mixed precision, with and without recomputation.
"""
from __future__ import annotations

import json
import sys

from . import binding as Bd
from . import inputs as I


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_ace(walkers: int = 16, chunk: int = 1024) -> dict:
    import torch
    pb = I.workload("ace16x16")
    params = I.random_params(pb, 1253, 0.02)
    M0 = I.plane_wave_M0(pb)
    ctx = Bd.make_context(pb, params, M0, chunk)
    occ = torch.from_numpy(I.random_configs(pb, chunk, 5703)).cuda()
    a, b = _events()
    ctx.scale_load(occ)  # warm-up
    torch.cuda.synchronize()
    a.record()
    ctx.scale_load(occ)
    b.record()
    torch.cuda.synchronize()
    load_ms = a.elapsed_time(b)
    ctx.scale_load(occ[:walkers].contiguous())
    e = torch.empty(walkers, dtype=torch.float64, device="cuda")
    ctx.scale_local_energy(e, Bd.PATH_FULL)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_local_energy(e, Bd.PATH_FULL)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    conv_flops = 2.0 * pb.n_conv * pb.N * 9 * pb.h * pb.h  # per configuration
    out = {"workload": "ace16x16: 16x16 torus, U=8, 112+112, 16 conv blocks h=144 + 2 site-wise h=256",
           "precision": "mixed (TF32x3 tensor-core layers, FP64 Slater matrices and LU)",
           "walkers": walkers, "ms": ms, "eloc_per_s": walkers / (ms / 1e3),
           "load_1024_ms": load_ms, "amplitudes_per_s": chunk / (load_ms / 1e3),
           "conv_gflop_per_amplitude": conv_flops / 1e9,
           "finite": bool(torch.isfinite(e).all().item())}
    ctx.close()
    return out


def run_symmetry(walkers: int = 1024) -> dict:
    import torch
    pb = I.workload("hubbard16x16")
    pseed, cseed = I.workload_seeds("hubbard16x16")
    ctx = Bd.make_context(pb, I.random_params(pb, pseed, 0.05), I.plane_wave_M0(pb), walkers)
    ctx.scale_load(torch.from_numpy(I.random_configs(pb, walkers, cseed)).cuda())
    perms = torch.from_numpy(I.symmetry_group(pb, translations=True)).cuda()
    chi = torch.ones(perms.shape[0], dtype=torch.float64, device="cuda")
    ctx.log_psi_sym(perms[:4].contiguous(), chi[:4].contiguous())  # warm-up
    a, b = _events()
    torch.cuda.synchronize()
    a.record()
    la, sg = ctx.log_psi_sym(perms, chi)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = {"walkers": walkers, "group": int(perms.shape[0]), "ms": ms,
           "amplitudes_per_s": walkers * perms.shape[0] / (ms / 1e3), "walkers_per_s": walkers / (ms / 1e3),
           "finite": bool(torch.isfinite(la).any().item())}
    ctx.close()
    return out


def run_wide(walkers: int = 8) -> dict:
    """SCALE-L (plus stencil, conv 384, site-wise 4 x 512) local energies on the 16x16 torus by
    full recompute and by the cached update; SCALE-XL (conv 640, site-wise 4 x 1280) on the
    32x32 torus: loads (forward, FP64 inverse, cache) and cached-update local energies."""
    import torch
    out = {}
    pl = I.workload("scale_l16x16")
    ctx = Bd.make_context(pl, I.random_params(pl, 1262, 0.02), I.plane_wave_M0(pl), 1024)
    occ = torch.from_numpy(I.random_configs(pl, 1024, 5712)).cuda()
    a, b = _events()
    ctx.scale_load(occ)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_load(occ)
    b.record()
    torch.cuda.synchronize()
    load_ms = a.elapsed_time(b)
    ctx.scale_load(occ[:walkers].contiguous())
    e = torch.empty(walkers, dtype=torch.float64, device="cuda")
    ctx.scale_local_energy(e, Bd.PATH_FULL)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_local_energy(e, Bd.PATH_FULL)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    # the cached update (low-rank local energies) on the same network and walkers, then on more
    lw = 256
    ctx.scale_load(occ[:lw].contiguous())
    el = torch.empty(lw, dtype=torch.float64, device="cuda")
    ctx.scale_local_energy(el, Bd.PATH_LOWRANK)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_local_energy(el, Bd.PATH_LOWRANK)
    b.record()
    torch.cuda.synchronize()
    lr_ms = a.elapsed_time(b)
    diff = ((el[:walkers] - e).abs() / e.abs().clamp(min=1.0)).cpu().numpy()
    out["scale_l16x16"] = {"walkers": walkers, "ms": ms, "eloc_per_s": walkers / (ms / 1e3),
                           "load_1024_ms": load_ms,
                           "lowrank_walkers": lw, "lowrank_ms": lr_ms, "lowrank_eloc_per_s": lw / (lr_ms / 1e3),
                           "speedup_lowrank_vs_full": (lw / lr_ms) / (walkers / ms),
                           "max_rel_diff_lowrank_vs_full": float(diff.max()),
                           "finite": bool(torch.isfinite(e).all().item() and torch.isfinite(el).all().item())}
    ctx.close()
    px = I.workload("scale_xl32x32")
    nx = 128
    ctx = Bd.make_context(px, I.random_params(px, 1264, 0.02), I.plane_wave_M0(px), nx)
    occ = torch.from_numpy(I.random_configs(px, nx, 5714)).cuda()
    ctx.scale_load(occ)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_load(occ)
    b.record()
    torch.cuda.synchronize()
    xl_ms = a.elapsed_time(b)
    xw = 4  # the cached update: low-rank local energies of the first walkers
    ctx.scale_load(occ[:xw].contiguous())
    ex = torch.empty(xw, dtype=torch.float64, device="cuda")
    ctx.scale_local_energy(ex, Bd.PATH_LOWRANK)
    torch.cuda.synchronize()
    a.record()
    ctx.scale_local_energy(ex, Bd.PATH_LOWRANK)
    b.record()
    torch.cuda.synchronize()
    xlr_ms = a.elapsed_time(b)
    out["scale_xl32x32"] = {"configurations": nx, "load_ms": xl_ms, "loads_per_s": nx / (xl_ms / 1e3),
                            "lowrank_walkers": xw, "lowrank_ms": xlr_ms, "lowrank_eloc_per_s": xw / (xlr_ms / 1e3),
                            "finite": bool(torch.isfinite(ex).all().item())}
    ctx.close()
    return out


def run_grad(walkers: int = 2048) -> dict:
    """Per-sample gradients on the 16x4 cylinder with the 12-layer residual stack, in FP64 and
    in mixed precision, with the activations kept and with recomputation."""
    import torch
    out = {"workload": "cylinder16x4: 16x4 cylinder, t'=-0.2, U=8, 28+28, 12 residual 3x3 layers, h=32",
           "walkers": walkers}
    for prec_name, prec in (("fp64", I.PREC_FP64), ("mixed", I.PREC_MIXED)):
        pb = I.workload("cylinder16x4").replace(precision=prec)
        pseed, cseed = I.workload_seeds("cylinder16x4")
        ctx = Bd.make_context(pb, I.random_params(pb, pseed), I.plane_wave_M0(pb), walkers)
        ctx.scale_load(torch.from_numpy(I.random_configs(pb, walkers, cseed)).cuda())
        g = torch.empty((walkers, ctx.P), dtype=torch.float64, device="cuda")
        a, b = _events()
        for rec in (0, 1):
            ctx.scale_grad_logpsi(g, rec)  # warm-up (scratch sized on first use)
            torch.cuda.synchronize()
            a.record()
            ctx.scale_grad_logpsi(g, rec)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            out[f"{prec_name}_{'recompute' if rec else 'stored'}_ms"] = ms
            out[f"{prec_name}_{'recompute' if rec else 'stored'}_grads_per_s"] = walkers / (ms / 1e3)
        out["params"] = ctx.P
        out[f"{prec_name}_finite"] = bool(torch.isfinite(g).all().item())
        del g
        ctx.close()
    return out


def run_plus(walkers: int = 8192) -> dict:
    """The SCALE chain step's local energies (cached update) on the bench network with
    SCALE-L's 13-site plus stencil in place of the 3x3 box, 16x16 torus."""
    import torch
    pb = I.workload("scale_plus16x16")
    pseed, cseed = I.workload_seeds("scale_plus16x16")
    ctx = Bd.make_context(pb, I.random_params(pb, pseed, 0.05), I.plane_wave_M0(pb), walkers)
    ctx.scale_load(torch.from_numpy(I.random_configs(pb, walkers, cseed)).cuda())
    e = torch.empty(walkers, dtype=torch.float64, device="cuda")
    ctx.scale_local_energy(e, Bd.PATH_LOWRANK)
    a, b = _events()
    torch.cuda.synchronize()
    a.record()
    ctx.scale_local_energy(e, Bd.PATH_LOWRANK)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = {"workload": "scale_plus16x16: 16x16 torus, U=8, 112+112, 5x5 plus conv + 5 site-wise, h=32",
           "walkers": walkers, "eloc_ms": ms, "eloc_per_s": walkers / (ms / 1e3),
           "finite": bool(torch.isfinite(e).all().item())}
    ctx.close()
    return out


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "ace"
    n = int(sys.argv[2]) if len(sys.argv) > 2 else None
    if what == "ace":
        print(json.dumps(run_ace(n or 16)))
    elif what == "wide":
        print(json.dumps(run_wide(n or 8)))
    elif what == "plus":
        print(json.dumps(run_plus(n or 8192)))
    elif what == "grad":
        print(json.dumps(run_grad(n or 2048)))
    else:
        print(json.dumps(run_symmetry(n or 1024)))
