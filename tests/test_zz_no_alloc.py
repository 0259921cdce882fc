"""The allocation-free log|psi| entry point (for callers that cannot call cudaMalloc: code
under an allocator owned by another runtime, or that may not allocate after setup) gives
the same log|psi| and signs as the context-based entry points, on two calls in a row.

Collected last on purpose (file name), so a run that stops at the first failure has run
every other test before this one. Passes alone in a fresh process and after the others."""
import numpy as np
import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,B,tol", [("hubbard4x4", 200, 1e-10), ("hubbard16x16", 300, 1e-10),
                                        ("tj8x8", 64, 1e-10)])
def test_noalloc_matches_context_path(name, B, tol):
    import torch
    pb = I.workload(name)
    pseed, cseed = I.workload_seeds(name)
    params = torch.from_numpy(I.random_params(pb, pseed)).cuda()
    M0 = torch.from_numpy(I.plane_wave_M0(pb)).cuda()
    occ_np = I.random_configs(pb, B, cseed)
    occ_np[-1, np.where(occ_np[-1] & 1)[0][0]] &= ~1  # one invalid sample: -inf, sign 0
    occ = torch.from_numpy(occ_np).cuda()
    ctx = Bd.Context(pb, B)
    ctx.scale_set_params(params, M0)
    ctx.scale_load(occ)
    la_ref, sg_ref = ctx.log_psi()
    torch.cuda.synchronize()
    for _ in range(2):  # the shared array keeps the previous call's contents
        la = torch.full((B,), 7.0, dtype=torch.float64, device="cuda")
        sg = torch.full((B,), 7, dtype=torch.int32, device="cuda")
        Bd.scale_log_psi_noalloc(pb, params, M0, occ, la, sg)
        torch.cuda.synchronize()
        assert torch.equal(sg, sg_ref)
        fin = torch.isfinite(la_ref)
        assert torch.equal(torch.isfinite(la), fin) and not fin[-1]
        assert (la[fin] - la_ref[fin]).abs().max().item() <= tol
    ctx.close()


def test_noalloc_rejects_oversized_shape_and_other_families():
    """A shape whose single sample does not fit the fixed array is refused with SCALE_EBUDGET
    before any work is queued (64x64, 1792 + 1792 electrons: one FP64 Slater matrix is 103 MB,
    the array 64 MiB), and the ACE family, which has no working set in the array, with
    SCALE_EUNSUPPORTED; an ordinary call still succeeds afterwards."""
    import torch
    big = I.workload("hubbard16x16").replace(Lx=64, Ly=64, n_up=1792, n_dn=1792)
    for pb, status in ((big, Bd.EBUDGET), (I.workload("ace4x4"), Bd.EUNSUPPORTED)):
        params = torch.zeros(I.param_count(pb), dtype=torch.float64, device="cuda")
        M0 = torch.zeros((2 * pb.N, pb.Ne), dtype=torch.float64, device="cuda")
        occ = torch.zeros((1, pb.N), dtype=torch.int8, device="cuda")
        la = torch.empty(1, dtype=torch.float64, device="cuda")
        sg = torch.empty(1, dtype=torch.int32, device="cuda")
        with pytest.raises(Bd.ScaleError) as e:
            Bd.scale_log_psi_noalloc(pb, params, M0, occ, la, sg)
        assert e.value.status == status
        del params, M0
    pb = I.workload("hubbard4x4")
    pseed, cseed = I.workload_seeds("hubbard4x4")
    params = torch.from_numpy(I.random_params(pb, pseed)).cuda()
    M0 = torch.from_numpy(I.plane_wave_M0(pb)).cuda()
    occ = torch.from_numpy(I.random_configs(pb, 8, cseed)).cuda()
    la = torch.empty(8, dtype=torch.float64, device="cuda")
    sg = torch.empty(8, dtype=torch.int32, device="cuda")
    Bd.scale_log_psi_noalloc(pb, params, M0, occ, la, sg)
    ctx = Bd.Context(pb, 8)
    ctx.scale_set_params(params, M0)
    ctx.scale_load(occ)
    la_ref, sg_ref = ctx.log_psi()
    torch.cuda.synchronize()
    fin = torch.isfinite(la_ref)
    assert fin.any() and torch.equal(sg, sg_ref) and torch.equal(torch.isfinite(la), fin)
    assert (la[fin] - la_ref[fin]).abs().max().item() <= 1e-10
    ctx.close()
