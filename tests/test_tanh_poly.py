"""The small-argument branch of the kernels' FP32 tanh (scale_internal.cuh) is a fitted cubic
in s = z^2. Its coefficients in the header must be the ones fit_tanh_poly.py produces, and the
polynomial must stay within 2e-8 relative of tanh on (0, 1/2] in exact arithmetic, with
q(0) near the Taylor coefficient -1/3."""
import importlib.util
import pathlib
import re

import numpy as np

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2604_25775_gb300" / "csrc"


def _header_coefs():
    src = (CSRC / "scale_internal.cuh").read_text()
    body = src[src.index("tanh_f32_small(float z)"):]
    body = body[:body.index("return")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1])  # the header runs from q3 down to q0


def test_header_matches_fit_and_bounds_error():
    spec = importlib.util.spec_from_file_location("fit_tanh_poly", CSRC / "fit_tanh_poly.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    err, c = mod.fit()
    q = _header_coefs()
    assert q.shape == (4,)
    assert np.allclose(q, c.astype(np.float32), rtol=0, atol=1e-9)
    assert err < 2e-8
    z = np.linspace(1e-6, 0.5, 200001)
    s = z * z
    approx = z + z * s * np.polyval(q[::-1], s)
    assert np.abs(approx / np.tanh(z) - 1).max() < 2e-8
    assert abs(q[0] + 1.0 / 3.0) < 1e-5
