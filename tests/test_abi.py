"""C-ABI library: builds for sm_103a, loads, exports every entry point of include/scale.h,
and its host-only calls agree with the parameter layout (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2604_25775_gb300 import binding as Bd
from paper_2604_25775_gb300 import inputs as I

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "scale.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scale_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = Bd.load_library()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(Bd.EXPORTED)


@pytest.mark.parametrize("name", ["hubbard4x4", "hubbard16x16", "cylinder16x4", "tj8x8", "hubbard32x32",
                                  "scale_plus16x16",
                                  "ace4x4", "ace8x8", "ace16x16", "scale_l5x5", "scale_l16x16",
                                  "scale_xl32x32"])
def test_param_count_matches_layout(name):
    pb = I.workload(name)
    assert Bd.scale_param_count(pb) == I.param_count(pb)
    assert Bd.scale_footprint_bytes(pb, 16) > 0


def test_invalid_descriptors_rejected_on_host():
    bad = [
        I.workload("hubbard4x4").replace(Lx=2),          # periodic extent 2
        I.workload("hubbard4x4").replace(h=65),          # too many channels
        I.workload("hubbard4x4").replace(ksize=[2, 1]),  # even kernel
        I.workload("hubbard4x4").replace(n_up=17),       # more electrons than sites
        I.workload("tj8x8").replace(n_up=40, n_dn=40),   # t-J overfilled
        I.workload("hubbard4x4").replace(refresh_every=0),
        I.workload("hubbard_ph8x8").replace(tp=-0.2),    # PHT keeps its form on NN bonds only
        I.workload("hubbard4x4").replace(model=3),       # unknown model
        I.workload("hubbard4x4").replace(family=2),      # unknown network family
        I.workload("hubbard4x4").replace(lowrank_kernel=2),  # unknown low-rank kernel
        I.workload("ace4x4").replace(n_conv=0),          # ACE without conv blocks
        I.workload("ace4x4").replace(h=300),             # ACE conv width above 256
        I.workload("ace4x4").replace(residual=[1, 1, 0, 0, 0]),  # ACE conv block without residual
        I.workload("ace4x4").replace(ksize=[3, 3, 3, 3, 1]),     # ACE site-wise layer with a stencil
        I.workload("ace4x4").replace(ln_eps=-1.0),
        I.workload("scale_l5x5").replace(stencil=2),     # unknown stencil
        I.workload("scale_l5x5").replace(h=2000),        # wide SCALE conv above 1024
    ]
    for pb in bad:
        assert Bd.scale_param_count(pb) == -1
        assert Bd.scale_footprint_bytes(pb, 4) == 0


def test_package_star_import():
    """Every name the package lists in __all__ exists (a star import succeeds)."""
    import paper_2604_25775_gb300 as pkg
    ns = {}
    exec("from paper_2604_25775_gb300 import *", ns)
    for name in pkg.__all__:
        assert name in ns, name
