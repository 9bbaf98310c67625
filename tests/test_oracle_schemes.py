"""Pins for oracle/schemes.py against facts the paper and mathematics fix."""

import math

import numpy as np
import pytest

from oracle import schemes as S

ALL = list(S.SCHEMES)


# --- shifted Legendre polynomials (Sec. 3.1) --------------------------------
def test_legendre_explicit_forms():
    # explicit P_2..P_4 printed in Sec. 3.1
    x = np.linspace(0.0, 1.0, 17)
    assert np.allclose(S.legendre_shifted(2, x), 6 * x**2 - 6 * x + 1, atol=1e-14)
    assert np.allclose(S.legendre_shifted(3, x), 20 * x**3 - 30 * x**2 + 12 * x - 1, atol=1e-14)
    assert np.allclose(S.legendre_shifted(4, x), 70 * x**4 - 140 * x**3 + 90 * x**2 - 20 * x + 1, atol=1e-13)


def test_legendre_parity_and_orthogonality():
    # Eq. (PSymm) and the scalar product int_0^1 P_m P_n = delta_mn / (2n+1),
    # evaluated with numpy's Gauss-Legendre nodes (library routine, 20 points)
    x = np.linspace(0.0, 1.0, 11)
    for n in range(7):
        assert np.allclose(S.legendre_shifted(n, 1 - x), (-1) ** n * S.legendre_shifted(n, x), atol=1e-13)
    t, wt = np.polynomial.legendre.leggauss(20)
    xq, wq = 0.5 * (t + 1.0), 0.5 * wt
    for m in range(6):
        for n in range(6):
            val = np.sum(wq * S.legendre_shifted(m, xq) * S.legendre_shifted(n, xq))
            assert abs(val - (1.0 / (2 * n + 1) if m == n else 0.0)) < 1e-14


# --- Gauss-Legendre rule (Sec. 7, Table tab:GaussLeg) -----------------------
@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_gauss_legendre_points_weights(M):
    x, w = S.gauss_legendre(M)
    # points are the zeros of P_M, symmetric about 1/2; weights symmetric
    assert np.max(np.abs(S.legendre_shifted(M, x))) < 1e-13
    assert np.allclose(x[::-1], 1 - x, atol=1e-15) and np.allclose(w[::-1], w, atol=1e-15)
    # exact for monomials of degree <= 2M-1, not for degree 2M
    for p in range(2 * M):
        assert abs(np.sum(w * x**p) - 1.0 / (p + 1)) < 1e-15
    assert abs(np.sum(w * x ** (2 * M)) - 1.0 / (2 * M + 1)) > 1e-6
    # matches numpy's Legendre-Gauss rule mapped to [0, 1]
    t, wt = np.polynomial.legendre.leggauss(M)
    assert np.allclose(x, 0.5 * (t + 1.0), atol=1e-15) and np.allclose(w, 0.5 * wt, atol=1e-15)


# --- order conditions (Sec. 4.1) ---------------------------------------------
@pytest.mark.parametrize("name", ALL)
def test_order1(name):
    # Eq. (Order1): sum_i f_{i,n} = delta_{n,1}
    f = S.full_table(S.SCHEMES[name])
    target = np.zeros(f.shape[1])
    target[0] = 1.0
    assert np.allclose(f.sum(axis=0), target, atol=1e-15)


@pytest.mark.parametrize("name", [n for n in ALL if S.SCHEMES[n].order >= 4])
def test_order2(name):
    # Eq. (Order2): sum_{i<j} f_{i,1} f_{j,2} - f_{j,1} f_{i,2} = -1/3
    f = S.full_table(S.SCHEMES[name])
    s = f.shape[0]
    val = sum(f[i, 0] * f[j, 1] - f[j, 0] * f[i, 1] for i in range(s) for j in range(i + 1, s))
    assert abs(val + 1.0 / 3.0) < 2e-15


def test_symmetric_expansion_rule():
    # Eq. (FSymm) on CF4:2: exp[A1/2 + A2/3] exp[A1/2 - A2/3]  (Eq. (UCF4:2))
    f = S.full_table(S.SCHEMES["CF4:2"])
    assert np.allclose(f, [[0.5, 1 / 3], [0.5, -1 / 3]], atol=0)
    # central exponential of CF4:3Opt carries odd n only (Eq. (CF4Optimal))
    f = S.full_table(S.SCHEMES["CF4:3Opt"])
    assert np.allclose(f, [[11 / 40, 20 / 87, 7 / 50], [9 / 20, 0, -7 / 25], [11 / 40, -20 / 87, 7 / 50]], atol=0)


def test_fourth_order_family():
    # Eq. (Coeff4th): f11 = (1 - f21)/2, f12 = 1/(3(1 + f21)); A3 condition
    # 2 f13 + f23 = 0 for CF4:3Opt (Sec. 5.2)
    for name in ("CF4:3", "CF4:3Opt"):
        f = S.full_table(S.SCHEMES[name])
        f21 = f[1, 0]
        assert abs(f[0, 0] - (1 - f21) / 2) < 1e-16
        assert abs(f[0, 1] - 1 / (3 * (1 + f21))) < 1e-16
    f = S.full_table(S.SCHEMES["CF4:3Opt"])
    assert abs(2 * f[0, 2] + f[1, 2]) < 1e-16


def _sixth_order_residuals(f):
    """The seven order conditions for s = 5 printed in Appendix C
    (Eq. (app:6thOrderConds)), as residuals (lhs - rhs)."""
    f11, f12, f13 = f[0, 0], f[0, 1], f[0, 2]
    f21, f22, f23 = f[1, 0], f[1, 1], f[1, 2]
    f31, f33 = f[2, 0], f[2, 2]
    r = []
    r.append(2 * f11 + 2 * f21 + f31 - 1)
    r.append(2 * f13 + 2 * f23 + f33)
    r.append(-f11 * f12 - 2 * f21 * f12 - f21 * f22 - f31 * f12 - f31 * f22 + 1 / 6)
    r.append(f12 * f13 + 2 * f12 * f23 + f12 * f33 + f22 * f23 + f22 * f33 + 1 / 30)
    a = (f11 * f21 * f13 / 3 - 2 * f11 * f21 * f23 / 3 - f11 * f21 * f33 / 3 + f11 * f31 * f13 / 6
         - f11 * f31 * f23 / 3 - f11 * f31 * f33 / 6 - f11**2 * f23 / 3 - f11**2 * f33 / 6
         + 2 * f21 * f31 * f13 / 3 + f21 * f31 * f23 / 6 - f21 * f31 * f33 / 6 + 2 * f21**2 * f13 / 3
         - f21**2 * f33 / 6 + f31**2 * f13 / 6 + f31**2 * f23 / 6)
    r.append(a - 1 / 60)
    b = (-f11 * f12**2 / 3 - f21 * f12 * f22 - f21 * f12**2 - f21 * f22**2 / 3 - f31 * f12 * f22
         - f31 * f12**2 / 2 - f31 * f22**2 / 2)
    r.append(b + 1 / 60)
    c = (f11 * f21 * f31 * f12 / 3 + f11 * f21 * f31 * f22 / 2 + f11 * f21**2 * f12 / 3
         + f11 * f21**2 * f22 / 3 + f11 * f31**2 * f12 / 12 + f11 * f31**2 * f22 / 6
         + f11**2 * f21 * f12 / 3 + f11**2 * f21 * f22 / 6 + f11**2 * f31 * f12 / 6
         + f11**2 * f31 * f22 / 6 + f11**3 * f12 / 12 + f21 * f31**2 * f22 / 12
         + f21**2 * f31 * f22 / 6 + f21**3 * f22 / 12)
    r.append(c - 1 / 360)
    return np.array(r)


@pytest.mark.parametrize("name,tol", [("CF6:5", 1e-15), ("CF6:5Imp", 1e-15), ("CF6:5Opt", 1e-15),
                                      ("CF6:5b", 1e-15)])
def test_sixth_order_conditions_s5(name, tol):
    f = S.full_table(S.SCHEMES[name])
    res = _sixth_order_residuals(f)
    assert np.max(np.abs(res)) < tol, res


def test_sixth_order_conditions_cf64():
    # CF6:4 is the s = 5 form with a vanishing central exponential
    f = S.full_table(S.SCHEMES["CF6:4"])
    f5 = np.zeros((5, 3))
    f5[0], f5[1], f5[3], f5[4] = f[0], f[1], f[2], f[3]
    assert np.max(np.abs(_sixth_order_residuals(f5))) < 1e-14


def test_cf65_quintic_root():
    # Appendix C: for f11 = 4/25, f21 is the single real root of the quintic
    f21 = S.full_table(S.SCHEMES["CF6:5"])[1, 0]
    c = [-126131602, 1646347450, -7919062500, 16950031250, -15834375000, 5498046875]
    roots = np.roots(c[::-1])
    real = roots[np.abs(roots.imag) < 1e-9].real
    assert len(real) == 1 and abs(real[0] - f21) < 1e-14
    # p(x, y) of Appendix C vanishes at (f11, f21) as well
    x, y = 0.16, f21
    p = (-2 + 30 * x - 192 * x**2 + 680 * x**3 - 1440 * x**4 + 1815 * x**5 - 1250 * x**6 + 360 * x**7
         + (18 - 232 * x + 1230 * x**2 - 3440 * x**3 + 5345 * x**4 - 4350 * x**5 + 1440 * x**6) * y
         + (-60 + 650 * x - 2740 * x**2 + 5655 * x**3 - 5710 * x**4 + 2250 * x**5) * y**2
         + (90 - 800 * x + 2535 * x**2 - 3450 * x**3 + 1710 * x**4) * y**3
         + (-60 + 425 * x - 920 * x**2 + 630 * x**3) * y**4 + (15 - 80 * x + 90 * x**2) * y**5)
    assert abs(p) < 1e-13


def test_cf65_remaining_coefficients():
    # Eq. (app:RemCoeff) reproduces the printed CF6:5 row entries from f11, f21
    f = S.full_table(S.SCHEMES["CF6:5"])
    f11, f21 = f[0, 0], f[1, 0]
    f22 = (1 + 5 * f11 * (f11 - 1)) / (30 * (f11 + f21 - 1) * (f11 + f21) * (2 * f11 + f21 - 1))
    f12 = (1 - 6 * f22 + 12 * f11 * f22 + 6 * f21 * f22) / (6 * (1 - f11))
    den = 30 * (f12 * (2 * f11 - 1) * (2 * f11 + f21 - 1)
                + f22 * (1 + 8 * f11**2 + 2 * (f21 - 2) * f21 + (8 * f21 - 7) * f11))
    f13 = ((2 * f11 - 1) * (2 * f11 + f21 - 1) - 3 * f22) / den
    f23 = (f11 + 3 * f12 + 4 * f11 * f21 + 2 * (f21 - 1) * f21 + 6 * f22 - 1) / den
    assert np.allclose([f12, f13, f22, f23], [f[0, 1], f[0, 2], f[1, 1], f[1, 2]], rtol=0, atol=2e-15)


def test_cf66opt_a1a4_condition():
    # Sec. 5.3: the [A1, A4] condition (s = 6 form) fixes f34
    f = S.full_table(S.SCHEMES["CF6:6Opt"])
    f11, f21, f31 = f[0, 0], f[1, 0], f[2, 0]
    f14, f24, f34 = f[0, 3], f[1, 3], f[2, 3]
    val = f11 * f14 + 2 * f21 * f14 + f21 * f24 + 2 * f31 * f14 + 2 * f31 * f24 + f31 * f34
    assert abs(val) < 1e-15


def test_cf64_closed_form_value():
    # f11 of CF6:4 from the closed form; sanity: it is real and the A1
    # condition with f21 = 1/2 - f11 holds by construction
    f = S.full_table(S.SCHEMES["CF6:4"])
    assert 0 < f[0, 0] < 1.5 and abs(2 * f[0, 0] + 2 * f[1, 0] - 1) < 1e-15


# --- g_{i,m} (Sec. 7) --------------------------------------------------------
def test_g_cf42_printed_weights():
    # Eq. (UCF4Gauss): left factor (3-2sqrt3)/12, (3+2sqrt3)/12; right factor
    # the mirror image; nodes 1/2 -+ sqrt(3)/6
    g, x, w, f = S.g_coefficients(S.SCHEMES["CF4:2"])
    a, b = (3 - 2 * math.sqrt(3)) / 12, (3 + 2 * math.sqrt(3)) / 12
    assert np.allclose(g, [[a, b], [b, a]], atol=1e-16)
    assert np.allclose(x, [0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6], atol=1e-16)


@pytest.mark.parametrize("name", ALL)
def test_g_sums(name):
    # sum_j g_{j,m} = w_m (from Order1 and GL exactness) and
    # sum_m g_{j,m} = f_{j,1} (orthogonality of P_{n-1} to P_0 under the rule)
    g, x, w, f = S.g_coefficients(S.SCHEMES[name])
    assert np.allclose(g.sum(axis=0), w, atol=5e-16)
    assert np.allclose(g.sum(axis=1), f[:, 0], atol=5e-16)


# ---------------------------------------------------------------- planted mistakes
def test_planted_mirror_sign_error_is_caught(monkeypatch):
    # rule (R1) with the sign (-1)^n instead of (-1)^(n+1): the second-order
    # condition and the printed CF4:2 factors must notice
    def bad(scheme):
        s, nA = scheme.s, scheme.nA
        f = np.zeros((s, nA))
        for i, row in enumerate(scheme.half):
            for n0, val in enumerate(row):
                f[i, n0] = val
                if s - 1 - i != i:
                    f[s - 1 - i, n0] = (-1.0) ** (n0 + 1) * val
        return f

    monkeypatch.setattr(S, "full_table", bad)
    f = S.full_table(S.SCHEMES["CF4:2"])
    s = f.shape[0]
    val = sum(f[i, 0] * f[j, 1] - f[j, 0] * f[i, 1] for i in range(s) for j in range(i + 1, s))
    assert abs(val + 1.0 / 3.0) > 1e-3
    assert not np.allclose(f, [[0.5, 1 / 3], [0.5, -1 / 3]], atol=0)


def test_planted_legendre_weight_error_is_caught(monkeypatch):
    # g_{i,m} without the factor (2n - 1): the printed CF4:2 weights of
    # Eq. (UCF4Gauss) must notice
    def bad(scheme):
        f = S.full_table(scheme)
        x, w = S.gauss_legendre(scheme.nA)
        g = np.zeros((scheme.s, len(x)))
        for i in range(scheme.s):
            for m in range(len(x)):
                g[i, m] = w[m] * sum(S.legendre_shifted(n, x[m]) * f[i, n] for n in range(scheme.nA))
        return g, x, w, f

    monkeypatch.setattr(S, "g_coefficients", bad)
    g, x, w, f = S.g_coefficients(S.SCHEMES["CF4:2"])
    a, b = (3 - 2 * math.sqrt(3)) / 12, (3 + 2 * math.sqrt(3)) / 12
    assert not np.allclose(g, [[a, b], [b, a]], atol=1e-12)
