"""Coefficients of the small-argument branch of the FP32 tanh in scale_internal.cuh.

For |z| < 1/2 the kernels take tanh z = z + z s q(s), s = z^2, with q a cubic fitted here to
minimise the largest relative error of tanh on (0, 1/2] (iteratively reweighted least squares
on a dense grid, Lawson's method). The fit reaches 1.5e-8 relative in exact arithmetic, below
the FP32 rounding of the evaluation; the degree-6 Taylor polynomial it replaces reached 1e-8.

    python fit_tanh_poly.py      # prints the coefficients q0..q3 and the fit's error
"""
import numpy as np


def fit(degree=3, zmax=0.5, iters=200):
    z = np.concatenate([np.linspace(1e-4, zmax, 20000), zmax * (1 - np.cos(np.linspace(0, np.pi / 2, 20000)))])
    z = z[z > 0]
    s = z * z
    target = (np.tanh(z) - z) / (z * s)  # the exact q(s)
    to_rel = (z * s) / np.tanh(z)  # relative error of tanh per unit error of q
    A = np.vander(s, degree + 1, increasing=True)
    w = np.ones_like(z)
    best = None
    for _ in range(iters):
        W = w * to_rel
        c, *_ = np.linalg.lstsq(A * W[:, None], target * W, rcond=None)
        err = (A @ c - target) * to_rel
        e = np.abs(err).max()
        if best is None or e < best[0]:
            best = (e, c)
        w = w * np.abs(err) ** 0.5 + 1e-300
        w /= w.max()
    return best


if __name__ == "__main__":
    e, c = fit()
    print("max relative error %.3e" % e)
    for k, v in enumerate(c):
        print("q%d = %.9ef" % (k, np.float32(v)))
