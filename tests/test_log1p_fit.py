"""The polynomial of the tensor-core sketch epilogue's log1p (0 <= r < 1):
the coefficients compiled into the CUDA source are the ones the committed fit
produces, and the fit evaluated in FP32 arithmetic is within 2e-7 relative of
log1p (the closed form, evaluated in FP64) on [0, 1], including r -> 0."""
import os
import re

import numpy as np

from paper_2110_12782_gb300 import fit_log1p

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_coefficients():
    src = open(os.path.join(ROOT, "paper_2110_12782_gb300", "csrc", "tc_ptx.cuh")).read()
    body = src[src.index("float log1p_poly(float t)"):]
    body = body[:body.index("}")]
    vals = [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]
    assert len(vals) == fit_log1p.DEGREE + 1
    return np.array(vals[::-1])  # Horner order c_8 .. c_0 in the source


def test_source_coefficients_are_the_fit():
    c = fit_log1p.fit()
    h = header_coefficients()
    assert np.all(np.abs(h - c.astype(np.float32)) <= 2 * np.spacing(np.abs(c).astype(np.float32)))


def test_fp32_evaluation_error():
    c = header_coefficients()
    r = np.concatenate([np.linspace(0.0, 1.0, 400001),
                        np.exp(np.linspace(np.log(2.0 ** -40), 0.0, 40001))]).astype(np.float32)
    y = fit_log1p.eval_f32(c, r).astype(np.float64)
    ref = np.log1p(r.astype(np.float64))
    nz = r > 0
    rel = np.abs(y[nz] - ref[nz]) / ref[nz]
    assert rel.max() < 2e-7, rel.max()
    assert y[r == 0].max() == 0.0
    # the polynomial (FP32 coefficients, exact arithmetic) approximates log1p(r)/r
    k = np.linspace(0.0, 1.0, 10001)
    g = np.where(k > 0, np.log1p(k) / np.where(k > 0, k, 1.0), 1.0)
    p = np.polynomial.polynomial.polyval(k - 0.5, c)
    assert np.max(np.abs(p - g) / g) < 1e-7
