"""Host-side checks of constants baked into the CUDA kernels (no GPU needed).

The memristor current uses sinh(x) = x p(x^2) on |x| < 3/4 with a degree-6 polynomial p
(k_stencil.cu, where b is folded into the coefficients at handle creation).  Its coefficients are checked here against sinh itself in high precision,
and against the generator script that derives them (Chebyshev economisation of the Taylor
series), so that a mistyped digit or a wrong range cannot reach the residual unnoticed."""
import re
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2109_07929_gb300" / "csrc"


def _kernel_coefficients():
    src = (CSRC / "k_stencil.cu").read_text()
    body = src[src.index("kSinhPoly[7] = {"):]
    body = body[:body.index("};")]
    vals = {}
    for m in re.finditer(r"([0-9.]+e[-+][0-9]+|1\.0),\s*// t\^(\d)", body):
        vals[int(m.group(2))] = float(m.group(1))
    assert sorted(vals) == list(range(7)), vals
    return [vals[k] for k in range(7)]


def _range_limit():
    src = (CSRC / "k_stencil.cu").read_text()
    m = re.search(r"kSinhPolyX = ([0-9.]+);", src)
    return float(m.group(1))


def test_range_matches_the_generator():
    pytest.importorskip("sympy")
    gen = _generator()
    assert _range_limit() == float(gen.X2) ** 0.5 == 0.75


def test_sinh_polynomial_accuracy_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    c = [Fraction(v) for v in _kernel_coefficients()]
    worst = 0.0
    for x in np.linspace(0.0, 0.75, 2001)[1:]:
        t = Fraction(float(x)) ** 2
        p = sum(ck * t**k for k, ck in enumerate(c))            # exact in rationals
        ref = mpmath.sinh(mpmath.mpf(float(x))) / mpmath.mpf(float(x))
        err = abs((mpmath.mpf(p.numerator) / p.denominator - ref) / ref)
        worst = max(worst, float(err))
    # truncation < 2e-18 plus the rounding of the coefficients to FP64
    assert worst < 3e-17, worst


def test_sinh_polynomial_fp64_horner_within_two_ulp():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    c = _kernel_coefficients()
    xs = np.concatenate([np.linspace(-0.7499, 0.7499, 3001), [1e-300, -1e-8, 0.5, 0.74999999]])
    for x in xs:
        t = x * x
        ps = c[6]
        for k in range(5, -1, -1):      # separate multiply and add: at least the rounding
            ps = ps * t + c[k]            # of the kernel's FMAs
        val = x * ps
        ref = float(mpmath.sinh(mpmath.mpf(float(x))))
        assert abs(val - ref) <= 2 * np.spacing(abs(ref)) + 1e-320, (x, val, ref)


@pytest.mark.parametrize("b", [2.0, 0.025, 7.5, 2000.0])
def test_fp32_tail_of_the_polynomial(b):
    """The kernels evaluate the tail t^3 (c3 + c4 t + c5 t^2 + c6 t^3) of the folded
    polynomial in FP32 (coefficients pc_k = c_k b^2k rounded to FP32, t from dV rounded to
    FP32) and the rest in FP64.  That tail is at most x^6/5040 of P, so the current must stay
    within 1e-11 relative (plus FP64 rounding) of (1/b) sinh(b dV) over |b dV| < 3/4."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    c = _kernel_coefficients()
    pc = [c[k] * b ** (2 * k) for k in range(7)]
    assert all(1e-30 <= pc[k] <= 1e30 for k in range(3, 7))   # the kernels' FP32-tail range
    pcf = [np.float32(v) for v in pc]
    worst = 0.0
    for x in np.concatenate([np.linspace(-0.7499, 0.7499, 1501), [1e-12, 0.3, -0.6]]):
        dv = x / b
        t = dv * dv
        dvf = np.float32(dv)
        tf = np.float32(dvf * dvf)
        r = np.float32(np.float64(pcf[6]) * tf + pcf[5])
        r = np.float32(np.float64(r) * tf + pcf[4])
        r = np.float32(np.float64(r) * tf + pcf[3])
        ps = float(r) * t + pc[2]
        ps = ps * t + pc[1]
        ps = ps * t + pc[0]
        val = dv * ps
        ref = float(mpmath.sinh(mpmath.mpf(b) * mpmath.mpf(dv)) / mpmath.mpf(b))
        if ref == 0.0:
            assert val == 0.0
            continue
        err = abs(val - ref) - 4 * np.spacing(abs(ref))
        worst = max(worst, err / abs(ref))
    assert worst < 1e-11, worst


def _generator():
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_sinh_poly", CSRC / "gen_sinh_poly.py")
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    return gen


def test_generator_reproduces_kernel_coefficients():
    pytest.importorskip("sympy")
    coef, bound = _generator().coefficients()
    assert bound < 2e-18
    assert [float(v) for v in coef] == _kernel_coefficients()
