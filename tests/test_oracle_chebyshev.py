"""Pins for oracle/chebyshev.py: dense library exponentials, the closed forms
of the harmonic-oscillator example (Sec. 8.2) and of the Jacobi-Anger
expansion, dense Gershgorin intervals, spectrum containment and unitarity."""

import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import cfet as OC, chebyshev as CH, operators as O


def _chain(N=6, nfields=1):
    pr = W.spin_chain(N)
    fields = [pr.xfield] + [W.uniform(50 + k, N, -1, 1) for k in range(1, nfields)]
    return pr, O.SpinChain(N, pr.J, pr.Delta, pr.h, fields), fields


def test_gershgorin_of_the_pauli_rows_matches_the_dense_matrix():
    # the row-sum construction from the Pauli-string applies against the
    # Kronecker-product matrix (an independent definition)
    pr, op, fields = _chain(7)
    assert np.allclose(CH.gershgorin_xxz(7, pr.J, pr.Delta, pr.h),
                       CH.gershgorin_dense(O.xxz_dense(7, pr.J, pr.Delta, pr.h)), rtol=0, atol=1e-12)
    assert np.allclose(CH.gershgorin_xfield(7, fields[0]), CH.gershgorin_dense(O.xfield_dense(7, fields[0])),
                       rtol=0, atol=1e-12)
    # a J with both signs and anisotropy
    h = W.uniform(9, 5, -2, 2)
    assert np.allclose(CH.gershgorin_xxz(5, -0.7, 2.5, h), CH.gershgorin_dense(O.xxz_dense(5, -0.7, 2.5, h)),
                       rtol=0, atol=1e-12)


def test_gershgorin_dia_matches_the_dense_matrix():
    p = W.grid_atom(Nr=40, L=3)
    dim = p.H0_values.shape[1]
    for offs, vals in ((p.H0_offsets, p.H0_values), (p.V_offsets, p.V_values)):
        D = np.zeros((dim, dim))
        for d, off in enumerate(offs):
            for r in range(dim):
                c = r + int(off)
                if 0 <= c < dim:
                    D[r, c] += vals[d, r]
        assert np.allclose(CH.gershgorin_dia(offs, vals), CH.gershgorin_dense(D), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("c", [(0.7, -0.4), (-0.3, 1.1), (1.0, 0.0)])
def test_stage_interval_contains_the_spectrum(c):
    pr, op, fields = _chain(6)
    lo, hi = CH.stage_interval(CH.operator_intervals(op), c)
    Hm = c[0] * O.xxz_dense(6, pr.J, pr.Delta, pr.h) + c[1] * O.xfield_dense(6, fields[0])
    ev = np.linalg.eigvalsh(Hm)
    assert lo <= ev[0] + 1e-12 and ev[-1] <= hi + 1e-12


def test_jacobi_anger_scalars_closed_form():
    # diagonal H = diag(x), x in [-1, 1]: the series must give exp(-i tau x)
    x = np.linspace(-1.0, 1.0, 41)
    op = O.Dense(np.diag(x), [])
    psi = np.ones(41, dtype=np.complex128)
    for tau in (0.3, 2.0, 17.5, -4.0):
        out, na, K, tail = CH.expv(lambda v: op.apply([1.0], v), psi, tau, -1.0, 1.0, 1e-14)
        assert np.max(np.abs(out - np.exp(-1j * tau * x))) < 1e-13
        assert na == K


def test_harmonic_oscillator_example():
    # Sec. 8.2: H_nn = n omega, 50 x 50, random psi, t = pi / (10 omega); exact
    # psi_n(t) = exp(-i t omega n) psi_n.  The error falls fast after 10-20 terms.
    omega = 1.0
    n = np.arange(50)
    H = np.diag(n * omega)
    psi = W.random_state(31, 50)
    t = math.pi / (10 * omega)
    exact = np.exp(-1j * t * omega * n) * psi
    lo, hi = CH.gershgorin_dense(H)
    assert (lo, hi) == (0.0, 49.0)
    errs = {}
    for tol in (1e-4, 1e-8, 1e-13):
        out, na, K, tail = CH.expv(lambda v: H @ v, psi, t, lo, hi, tol)
        errs[tol] = (np.linalg.norm(out - exact), K)
        assert errs[tol][0] <= tol
    assert 10 <= errs[1e-4][1] <= 30 and errs[1e-13][1] <= 45


@pytest.mark.parametrize("tau", [0.05, 0.5, 3.0, -0.7])
def test_expv_matches_dense_expm(tau):
    pr, op, fields = _chain(6, nfields=2)
    c = (0.8, -0.35, 0.2)
    Hm = c[0] * O.xxz_dense(6, pr.J, pr.Delta, pr.h) + sum(ck * O.xfield_dense(6, a) for ck, a in zip(c[1:], fields))
    lo, hi = CH.stage_interval(CH.operator_intervals(op), c)
    psi = W.random_state(3, 64)
    out, na, K, tail = CH.expv(lambda v: op.apply(c, v), psi, tau, lo, hi, 1e-12)
    ref = expm(-1j * tau * Hm) @ psi
    assert np.linalg.norm(out - ref) <= 1e-11
    assert abs(np.linalg.norm(out) - 1.0) <= 1e-11
    back, *_ = CH.expv(lambda v: op.apply(c, v), out, -tau, lo, hi, 1e-12)
    assert np.linalg.norm(back - psi) <= 2e-11


def test_truncation_rule_is_minimal():
    for z in (0.01, 0.7, 5.0, 80.0, -12.0):
        for tol in (1e-6, 1e-10, 0.0):
            r, K, tail = CH.coefficients(z, tol)
            eps = tol if tol > 0 else 2.0 ** -52
            assert tail <= eps
            if K > 0:
                _, K1, tail1 = CH.coefficients(z, 10 * tail + 1e-300)   # a looser bound never needs more
                assert K1 <= K
                # one term fewer violates the bound
                absJ = np.abs(np.array([r[0]] + [x / 2 for x in r[1:]]))
                assert tail + 2 * absJ[K] > eps
            assert len(r) == K + 1


def test_zero_and_constant_stage():
    # H_j = b I (zero width): only the phase exp(-i tau b); H_j = 0: identity
    psi = W.random_state(4, 16)
    out, na, K, _ = CH.expv(lambda v: 2.5 * v, psi, 0.3, 2.5, 2.5, 1e-12)
    assert na == 0 and np.allclose(out, np.exp(-0.75j) * psi, atol=1e-15)
    out, na, K, _ = CH.expv(lambda v: 0 * v, psi, 0.3, 0.0, 0.0, 1e-12)
    assert na == 0 and np.array_equal(out, psi)


def test_propagate_time_independent_is_exact():
    N = 6
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    psi = W.random_state(5, 1 << N)
    out = CH.propagate(op, psi, 0.0, 0.1, 5, 6, [lambda t: 0.0], 1e-12)
    ref = expm(-1j * 0.5 * O.xxz_dense(N, pr.J, pr.Delta, pr.h)) @ psi
    assert np.linalg.norm(out - ref) <= 1e-10


def test_propagate_agrees_with_the_krylov_oracle():
    N = 7
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    psi = W.neel_state(N)
    a, st = CH.propagate(op, psi, 0.0, 0.05, 20, 4, [pr.drive], 1e-12, return_stats=True)
    b = OC.propagate(op, psi, 0.0, 0.05, 20, 4, [pr.drive], 1e-12, 20)
    # both evaluate every stage exponential to 1e-12: the CFET steps agree
    assert np.linalg.norm(a - b) <= 40 * 2 * 1e-12
    assert st["n_applies"] == sum(st["K"]) and len(st["K"]) == 40


# ---------------------------------------------------------------- planted mistakes
def test_planted_missing_factor_two_is_caught(monkeypatch):
    # Jacobi-Anger with r_k = J_k(z) for every k (the factor 2 - delta_k0
    # dropped): the dense-expm pin must notice
    good = CH.coefficients

    def bad(z, tol):
        r, K, tail = good(z, tol)
        r = r.copy()
        r[1:] /= 2.0
        return r, K, tail

    monkeypatch.setattr(CH, "coefficients", bad)
    pr, op, fields = _chain(6, nfields=2)
    c = (0.8, -0.35, 0.2)
    Hm = c[0] * O.xxz_dense(6, pr.J, pr.Delta, pr.h) + sum(ck * O.xfield_dense(6, a) for ck, a in zip(c[1:], fields))
    lo, hi = CH.stage_interval(CH.operator_intervals(op), c)
    psi = W.random_state(3, 64)
    out, *_ = CH.expv(lambda v: op.apply(c, v), psi, 0.5, lo, hi, 1e-12)
    assert np.linalg.norm(out - expm(-0.5j * Hm) @ psi) > 1e-3


def test_planted_weyl_sign_error_is_caught(monkeypatch):
    # negative stage scalars without swapping the interval ends: the interval
    # no longer contains the spectrum
    def bad(intervals, coeffs):
        lo = hi = 0.0
        for (l, h), s in zip(intervals, coeffs):
            lo += s * l
            hi += s * h
        return lo, hi

    monkeypatch.setattr(CH, "stage_interval", bad)
    pr, op, fields = _chain(6, nfields=2)
    c = (-0.8, 0.35, -0.2)
    Hm = c[0] * O.xxz_dense(6, pr.J, pr.Delta, pr.h) + sum(ck * O.xfield_dense(6, a) for ck, a in zip(c[1:], fields))
    lo, hi = CH.stage_interval(CH.operator_intervals(op), c)
    ev = np.linalg.eigvalsh(Hm)
    assert not (lo <= ev.min() + 1e-12 and ev.max() <= hi + 1e-12)
