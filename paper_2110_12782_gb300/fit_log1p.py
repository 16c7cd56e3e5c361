"""Coefficients of the polynomial that the tensor-core sketch epilogue uses
for log1p on [0, 1].

g(r) = log1p(r) / r is fitted by a polynomial of degree 8 in t = r - 1/2 (the
centred variable keeps the Horner evaluation well conditioned), minimising
the largest relative error over Chebyshev nodes on [0, 1] by iteratively
reweighted least squares (Lawson's algorithm).  The epilogue evaluates
log1p(r) = r p(r - 1/2) for 0 <= r < 1 and log(1 + r) from the hardware base-2
logarithm for r >= 1, where its absolute error is small against log(1 + r).

Run as a script to print the coefficients in the form the CUDA source holds
them (paper_2110_12782_gb300/csrc/tc_ptx.cuh, kLog1pPoly); the tests check
that the two agree and bound the error of the FP32 evaluation.
"""
import numpy as np

DEGREE = 8
NODES = 4000
ITERATIONS = 60


def g(r: np.ndarray) -> np.ndarray:
    r = np.asarray(r, dtype=np.float64)
    out = np.ones_like(r)
    nz = r != 0
    out[nz] = np.log1p(r[nz]) / r[nz]
    return out


def fit(degree: int = DEGREE) -> np.ndarray:
    """Coefficients c_0 .. c_degree of p(t) = sum c_i t^i, t = r - 1/2."""
    k = np.arange(NODES)
    r = (np.cos(np.pi * (k + 0.5) / NODES) + 1.0) / 2.0
    V = np.vander(r - 0.5, degree + 1, increasing=True)
    w = 1.0 / g(r)  # relative error
    wt = np.full(NODES, 1.0 / NODES)
    c = None
    for _ in range(ITERATIONS):
        s = w * np.sqrt(wt)
        c, *_ = np.linalg.lstsq(V * s[:, None], g(r) * s, rcond=None)
        e = np.abs(V @ c - g(r)) * w
        wt = wt * (e / e.max() + 1e-3)
        wt /= wt.sum()
    return c


def eval_f32(c: np.ndarray, r: np.ndarray) -> np.ndarray:
    """r p(r - 1/2) in FP32 arithmetic (each Horner step rounded once, as a
    fused multiply-add), for 0 <= r <= 1."""
    f32 = np.float32
    cf = np.asarray(c, dtype=f32)
    r = np.asarray(r, dtype=f32)
    t = (r - f32(0.5)).astype(f32)
    p = np.full_like(t, cf[-1])
    for ci in cf[-2::-1]:
        p = (p.astype(np.float64) * t.astype(np.float64) + np.float64(ci)).astype(f32)
    return (p * r).astype(f32)


if __name__ == "__main__":
    c = fit()
    print("constexpr float kLog1pPoly[%d] = {" % (DEGREE + 1))
    print(",\n".join("    %.9ef" % float(np.float32(x)) for x in c) + "};")
