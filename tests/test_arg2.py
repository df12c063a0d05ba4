"""The FP32 argument function of the step kernels (arg2 in
paper_2211_15630_gb300/csrc/aap_device.cuh): the angle of the VM sum,
Eq. (collision_VM), replaces the library arctangent.  Its coefficients are read
from the header and its arithmetic is replayed in FP32 here (products and
sums rounded as the FMAs do), then compared with numpy's FP64 arctan2: the
error stays within 4e-7 rad (the fit's 1.4e-7 plus the fast quotient's two
ulp), far inside the kernels' 1e-5 rad tolerance, and the special cases
(the axes, the diagonals, a zero sum, signed zeros) come out right.  The GPU
parity tests check the compiled function through the whole step."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2211_15630_gb300", "csrc", "aap_device.cuh")
F32 = np.float32


def _coeffs():
    txt = open(HDR).read()
    return [F32(float(re.search(r"kAtan%d = ([-+0-9.eE]+)f" % k, txt).group(1))) for k in range(8)]


def _fma(a, b, c):
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def arg2(y, x, quotient_ulps=0):
    """FP32 replay of arg2; quotient_ulps perturbs t as the fast quotient may."""
    c = _coeffs()
    ax, ay = abs(F32(x)), abs(F32(y))
    hi, lo = max(ax, ay), min(ax, ay)
    t = F32(lo / hi) if hi > 0 else F32(0.0)
    if quotient_ulps and t > 0:
        t = F32(np.nextafter(t, F32(2.0)) if quotient_ulps > 0 else np.nextafter(t, F32(0.0)))
        t = min(t, F32(1.0))
    t2 = F32(t * t)
    r = c[7]
    for k in range(6, -1, -1):
        r = _fma(r, t2, c[k])
    r = F32(r * t)
    if ay > ax:
        r = F32(F32(1.57079632679490) - r)
    if F32(x) < 0:
        r = F32(F32(3.14159265358979) - r)
    return float(np.copysign(r, F32(y)))


def test_accuracy_over_the_circle():
    g = np.random.default_rng(1)
    ang = np.concatenate([g.uniform(-np.pi, np.pi, 4000), np.linspace(-np.pi, np.pi, 2001)])
    mag = np.concatenate([10.0 ** g.uniform(-3, 9, ang.size - 10), [1.0] * 10])
    worst = 0.0
    for a, m in zip(ang, mag):
        x, y = F32(m * np.cos(a)), F32(m * np.sin(a))
        ref = np.arctan2(np.float64(y), np.float64(x))
        for q in (0, 1, -1):
            d = abs(np.mod(arg2(y, x, q) - ref + np.pi, 2 * np.pi) - np.pi)
            worst = max(worst, d)
    assert worst < 4e-7, worst


def test_special_cases():
    assert arg2(0.0, 0.0) == 0.0
    assert arg2(0.0, 5.0) == 0.0
    assert abs(arg2(3.0, 0.0) - np.pi / 2) < 1e-7
    assert abs(arg2(-3.0, 0.0) + np.pi / 2) < 1e-7
    assert abs(arg2(0.0, -2.0) - np.pi) < 1e-6 and abs(arg2(-0.0, -2.0) + np.pi) < 1e-6
    for k in range(-3, 5):
        a = k * np.pi / 4
        x, y = F32(np.cos(a)), F32(np.sin(a))
        assert abs(np.mod(arg2(y, x) - np.arctan2(y, x) + np.pi, 2 * np.pi) - np.pi) < 4e-7
    # exact integer sums as the kernels pass them (units of 2^-22)
    for sc, ss in ((4194304 * 7, -1), (-3, 4194304 * 11), (123456789, -987654321)):
        assert abs(arg2(float(ss), float(sc)) - np.arctan2(ss, sc)) < 4e-7
