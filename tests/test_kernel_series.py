"""The short polynomials of the FP32 solve kernel, read from its source and
checked on the CPU against numpy's expm1 (no GPU, no oracle):

  u(x) = (1 - e^-x) / x on |x| < 1/4  -- the two-stream transmission terms and
         the beam terms for small optical depth (Sec. 2.2);
  q(x) = (e^x - 1) / x  on [0, 1/2)   -- the Planck integrand x^3/(e^x - 1) = x^2/q
         for small x (bin-integrated B, Sec. 2.2.1).

The bounds are those the kernel's comments state.  The fit script beside the
kernel must reproduce the coefficients that the kernel holds.
"""
import os
import re
import runpy

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_02293_b300", "csrc")


def kernel_coefficients(func):
    """FP32 coefficients of the Horner chain in `func`, constant term first."""
    src = open(os.path.join(CSRC, "rt_kernels.cu")).read()
    m = re.search(r"\b" + func + r"\(V x\) \{(.*?)\n\}", src, flags=re.S)
    assert m, func
    body = m.group(1)
    head = body.split("const V xx")[0]                      # planck_nd: the chain only
    vals = re.findall(r"V\((-?[0-9.e+-]+)f\)", head)
    return np.array([np.float32(v) for v in vals][::-1], np.float32)


def horner_fp32(c, x):
    p = np.full(x.shape, c[-1], np.float32)
    for cc in c[-2::-1]:
        p = (p.astype(np.float64) * x.astype(np.float64) + np.float64(cc)).astype(np.float32)
    return p


CASES = {
    # function in the kernel: (exact, interval, degree, bound exact, bound FP32)
    "u_series_v": (lambda x: -np.expm1(-x) / x, (-0.25, 0.25), 5, 3e-9, 7e-8),
    "planck_nd": (lambda x: np.expm1(x) / x, (0.0, 0.5), 4, 1.1e-7, 1.7e-7),
}


@pytest.mark.parametrize("func", sorted(CASES))
def test_kernel_polynomial_meets_its_stated_bound(func):
    f, (a, b), deg, bound, bound32 = CASES[func]
    c = kernel_coefficients(func)
    assert c.size == deg + 1 and c[0] == 1.0
    x32 = np.linspace(a, b, 200001).astype(np.float32)
    x32 = x32[x32 != 0]
    x = x32.astype(np.float64)
    want = f(x)
    exact = np.polynomial.polynomial.polyval(x, c.astype(np.float64))
    assert np.abs(exact / want - 1).max() < bound
    assert np.abs(horner_fp32(c, x32) / want - 1).max() < bound32


@pytest.mark.parametrize("func", sorted(CASES))
def test_kernel_polynomial_matches_the_series_at_the_origin(func):
    # first two Taylor coefficients: u = 1 - x/2 + ..., q = 1 + x/2 + ...
    c = kernel_coefficients(func)
    half = -0.5 if func == "u_series_v" else 0.5
    assert abs(c[1] - half) < 1e-5
    assert abs(c[2] - 1.0 / 6.0) < 2e-4


def test_fit_script_reproduces_the_kernel_coefficients():
    fs = runpy.run_path(os.path.join(CSRC, "fit_series.py"))
    np.testing.assert_array_equal(fs["fit"]("u_series"), kernel_coefficients("u_series_v"))
    np.testing.assert_array_equal(fs["fit"]("planck_q"), kernel_coefficients("planck_nd"))
