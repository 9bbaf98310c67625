"""Host checks of the control warp's FP64-free scalar helpers (scalar_bounds.cuh
compiled for the host behind cfet_selftest_i128_to_double,
cfet_selftest_ll_to_double_up and cfet_selftest_krylov_bounds; no GPU).

* The exact 128-bit reductions of the fixed-point kernels become doubles by
  integer operations: compared with Python's correctly rounded int -> float;
  the int64 maxima are converted rounding up (checked with exact fractions).
* The certain decisions on a Krylov dimension (Sec. 8.1's estimate
  beta0 beta_k |y_k|, y = exp(-i ts T_k) e_1) rest on lower and upper bounds
  of |y_k| from the leading Taylor term: checked against y computed in
  60-digit arithmetic on random Lanczos-like tridiagonals, and shown tight for
  small |ts| (so that they decide in practice), void where they cannot hold.
* The Gershgorin gate |ts| w <= 2k in FP32 must agree with the FP64 form
  whenever it decides.
"""

import ctypes as C
import math
import random

import numpy as np
import pytest

from paper_1102_5071_gb300 import _capi
from paper_1102_5071_gb300.build import build


@pytest.fixture(scope="module")
def lib():
    build()
    return _capi.load()


def _conv(lib, vals, shift):
    n = len(vals)
    lo = np.array([v & ((1 << 64) - 1) for v in vals], dtype=np.uint64)
    hi = np.array([(v >> 64) for v in vals], dtype=np.int64)
    out = np.zeros(n)
    assert lib.cfet_selftest_i128_to_double(lo.ctypes.data, hi.ctypes.data, n, shift, out.ctypes.data) == _capi.CFET_OK
    return out


def test_i128_to_double_is_correctly_rounded(lib):
    rng = random.Random(5)
    vals = [0, 1, -1, 2, -2, (1 << 127) - 1, -(1 << 127), 1 << 64, -(1 << 64), (1 << 64) - 1, (1 << 53) + 1,
            (1 << 54) + 2, (1 << 54) + 6, (1 << 100) + (1 << 47), (1 << 100) + (1 << 47) + 1, (1 << 100) + 3 * (1 << 47)]
    for bits in (3, 20, 52, 53, 54, 63, 64, 65, 90, 115, 126):
        for _ in range(40):
            v = rng.getrandbits(bits)
            if rng.random() < 0.3:  # exact halfway patterns
                v = (v >> 12 << 12) | (1 << 11)
            vals.append(v if rng.random() < 0.5 else -v)
    for shift in (0, 24, -37, 150):
        out = _conv(lib, vals, shift)
        for v, o in zip(vals, out):
            ref = math.ldexp(float(v), shift)  # float(int) rounds to nearest, ties to even
            assert o == ref, (v, shift, o, ref)


def test_ll_to_double_up_is_the_smallest_double_not_below(lib):
    # the int64 maxima of the fixed-point vectors enter the exponent bounds
    # rounded up: never below the integer, and the next double down is below it
    from fractions import Fraction
    rng = random.Random(6)
    vals = [0, 1, 2, 3, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 54) + 1, (1 << 62) - 1, (1 << 63) - 1,
            (1 << 60) + (1 << 7), -5]
    vals += [rng.getrandbits(b) for b in (10, 40, 53, 54, 58, 62, 63) for _ in range(30)]
    v = np.array(vals, dtype=np.int64)
    out = np.zeros(len(vals))
    assert lib.cfet_selftest_ll_to_double_up(v.ctypes.data, len(vals), out.ctypes.data) == _capi.CFET_OK
    for x, o in zip(vals, out):
        if x <= 0:
            assert o == 0.0
            continue
        assert Fraction(o) >= x, (x, o)
        assert Fraction(np.nextafter(o, 0.0)) < x, (x, o)


def _exact_y(a, b, ts, digits=60):
    # y = exp(-i ts T) e_0 by its Taylor series in high precision; returns |y_{k-1}|
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = digits
    k = len(a)
    A = [mp.mpf(x) for x in a]
    B = [mp.mpf(x) for x in b]
    t = [mp.mpc(1)] + [mp.mpc(0)] * (k - 1)
    y = list(t)
    c = mp.mpc(0, -ts)
    n = 0
    while True:
        n += 1
        z = []
        for r in range(k):
            s = A[r] * t[r]
            if r > 0:
                s += B[r - 1] * t[r - 1]
            if r < k - 1:
                s += B[r] * t[r + 1]
            z.append(s * c / n)
        t = z
        y = [u + v for u, v in zip(y, t)]
        if n > k + 20 and max(abs(v) for v in t) < mp.mpf(10) ** (-digits + 5) * max(abs(v) for v in y):
            break
    return abs(y[k - 1])


def _bounds(lib, a, b, ts, upper=False):
    lh = np.zeros(2)
    gate = C.c_int32()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b if len(b) else [0.0], dtype=np.float64)
    assert lib.cfet_selftest_krylov_bounds(len(a), a.ctypes.data, b.ctypes.data, ts, lh.ctypes.data,
                                           C.byref(gate)) == _capi.CFET_OK
    return (lh[0], lh[1], gate.value) if upper else (lh[0], gate.value)


def test_lead_bounds_enclose_the_exact_value_and_are_tight(lib):
    pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    tight = 0
    for case in range(120):
        k = int(rng.integers(2, 17))
        off = rng.uniform(-50, 50) if case % 3 == 0 else 0.0     # large diagonal offsets
        a = off + rng.uniform(-5, 5, k)
        b = rng.uniform(0.05, 5, k - 1)
        ts = float(rng.choice([-1, 1]) * 10 ** rng.uniform(-3.5, -0.5))
        lo, hi, _ = _bounds(lib, a, b, ts, upper=True)
        y = _exact_y(a, b, ts)
        assert hi < 1e29 and math.log2(y) <= hi, (k, ts, math.log2(y), hi)
        if lo > -1e29:
            assert math.log2(y) >= lo, (k, ts, math.log2(y), lo)
            # the leading term dominates for small |ts| ||T||: within a few percent
            if abs(ts) * (np.ptp(a) / 2 + 5) < 0.05:
                assert lo >= math.log2(y) - 0.2 and hi <= math.log2(y) + 0.2, (k, ts, math.log2(y), lo, hi)
                tight += 1
    assert tight >= 20


def test_lead_bound_void_cases(lib):
    # |ts| spread too large for the lower bound, a zero coupling (breakdown),
    # k = 1, a non-finite coupling
    a = np.array([0.0, 1.0, -2.0])
    assert _bounds(lib, a, [3.0, 4.0], 0.5)[0] < -1e29
    assert _bounds(lib, a, [3.0, 0.0], 0.01)[0] < -1e29
    assert _bounds(lib, a[:1], [], 0.01)[0] < -1e29
    assert _bounds(lib, a, [3.0, float("nan")], 0.01)[0] < -1e29
    # the bound at a small step equals the leading term to the margin
    lo, _ = _bounds(lib, a, [3.0, 4.0], 1e-3)
    lead = math.log2(1e-3 ** 2 * 3.0 * 4.0 / 2.0)
    assert lead - 0.01 < lo < lead


def _gersh_w(a, b):
    k = len(a)
    lo, hi = math.inf, -math.inf
    for r in range(k):
        rad = (abs(b[r - 1]) if r > 0 else 0.0) + (abs(b[r]) if r < k - 1 else 0.0)
        lo = min(lo, a[r] - rad)
        hi = max(hi, a[r] + rad)
    return hi - lo


def test_gersh_gate_agrees_with_fp64(lib):
    rng = np.random.default_rng(12)
    decided = 0
    for case in range(400):
        k = int(rng.integers(1, 40))
        a = rng.uniform(-1, 1, k) * 10 ** rng.uniform(-2, 3)
        b = rng.uniform(0, 1, max(k - 1, 0)) * 10 ** rng.uniform(-2, 2)
        w = _gersh_w(a, b)
        # steps around the threshold: far below, far above and within 1e-7 of it
        ts = 2.0 * k / w * float(rng.choice([0.3, 3.0, 1 - 1e-7, 1 + 1e-7, 1 - 1e-4, 1 + 1e-4])) if w > 0 else 0.1
        _, gate = _bounds(lib, a, b if k > 1 else [0.0], ts)
        ref = abs(ts) * w <= 2.0 * k
        if gate >= 0:
            assert gate == int(ref), (k, ts, w)
            decided += 1
        else:
            assert abs(abs(ts) * w / (2.0 * k) - 1) < 1e-4, (k, ts, w)
    assert decided >= 250
