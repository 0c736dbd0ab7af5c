"""Fits the two short polynomials of the FP32 solve kernel and prints them as
the kernel writes them (rt_kernels.cu: u_series_v and planck_nd).

  u(x) = (1 - e^-x) / x   on [-1/4, 1/4], degree 5  (the two-stream transmission
                          and the beam terms for small optical depth, Sec. 2.2)
  q(x) = (e^x - 1) / x    on [0, 1/2],    degree 4  (the Planck integrand
                          x^3 / (e^x - 1) = x^2 / q for small x)

Each is fitted for the least maximum RELATIVE error with the constant term
fixed at 1, by Lawson's iteratively reweighted least squares on Chebyshev
nodes, then rounded to FP32.  Run as a script to print the coefficients and
the error bounds: the maximum relative error of the rounded coefficients in
exact arithmetic, and evaluated by FP32 Horner with fused multiply-adds.
"""
import numpy as np

FITS = {
    # name: (function, interval, degree)
    "u_series": (lambda x: -np.expm1(-x) / x, (-0.25, 0.25), 5),
    "planck_q": (lambda x: np.expm1(x) / x, (0.0, 0.5), 4),
}


def _f(name, x):
    fn = FITS[name][0]
    x = np.asarray(x, np.float64)
    out = np.ones_like(x)
    nz = x != 0
    out[nz] = fn(x[nz])
    return out


def fit(name, n_nodes=4000, iters=300):
    """FP32 coefficients, constant term first."""
    _, (a, b), deg = FITS[name]
    k = np.arange(n_nodes)
    xs = 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n_nodes))
    fx = _f(name, xs)
    V = np.vander(xs, deg + 1, increasing=True)[:, 1:]
    y = fx - 1.0
    w = np.full(n_nodes, 1.0 / n_nodes)
    for _ in range(iters):
        W = np.sqrt(w) / fx
        c, *_ = np.linalg.lstsq(V * W[:, None], y * W, rcond=None)
        e = np.abs(V @ c - y) / fx
        w = w * e
        w /= w.sum()
    return np.concatenate([[1.0], c]).astype(np.float32)


def horner_fp32(c32, x):
    """Horner in FP32 with one rounding per multiply-add (the kernel's vfma)."""
    x = np.asarray(x, np.float32)
    p = np.full(x.shape, c32[-1], np.float32)
    for cc in c32[-2::-1]:
        p = (p.astype(np.float64) * x.astype(np.float64) + np.float64(cc)).astype(np.float32)
    return p


def errors(name, c32, n=400001):
    """(max relative error in exact arithmetic, max relative error of FP32 Horner)."""
    _, (a, b), _ = FITS[name]
    x32 = np.linspace(a, b, n).astype(np.float32)
    x = x32.astype(np.float64)
    f = _f(name, x)
    exact = np.polynomial.polynomial.polyval(x, c32.astype(np.float64))
    return float(np.abs(exact / f - 1).max()), float(np.abs(horner_fp32(c32, x32) / f - 1).max())


if __name__ == "__main__":
    for name in FITS:
        c = fit(name)
        ea, ef = errors(name, c)
        print(f"{name}: degree {len(c) - 1}, relative error {ea:.3g} exact, {ef:.3g} in FP32")
        print("  highest power first:", ", ".join(f"{float(v)!r}f" for v in c[::-1]))
