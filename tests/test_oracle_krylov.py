"""Pins for oracle/krylov.py against dense library exponentials and closed forms."""

import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import krylov as K
import workloads as W


def _herm(n, seed):
    a = W.complex_gaussian(seed, n * n).reshape(n, n)
    return 0.5 * (a + a.conj().T)


def test_tridiag_expm_matches_library():
    alpha = W.uniform(3, 9, -2, 2)
    beta = W.uniform(4, 8, 0.1, 1.5)
    T = K.tridiag_matrix(alpha, beta)
    for tau in (0.01, 0.3, 2.0):
        y = K.tridiag_expm_e1(alpha, beta, tau)
        ref = expm(-1j * tau * T)[:, 0]
        assert np.max(np.abs(y - ref)) < 1e-13


@pytest.mark.parametrize("tau", [0.05, 0.4, 3.0])
def test_expv_dense_random_hermitian(tau):
    # exp(-i tau H) psi vs scipy.linalg.expm on a 64-dimensional Hermitian H
    H = _herm(64, 11)
    psi = W.random_state(12, 64)
    out, log, na = K.expv(lambda v: H @ v, psi, tau, tol=1e-12, m_max=30)
    ref = expm(-1j * tau * H) @ psi
    assert np.linalg.norm(out - ref) < 1e-10
    assert abs(np.linalg.norm(out) - 1) < 1e-12


def test_expv_harmonic_oscillator_substeps():
    # Sec. 8.2: H_nn = n omega, exact psi_n(t) = exp(-i t omega n) psi_n; the
    # large spread forces substepping with a small Krylov space
    omega = 1.0
    n = np.arange(50)
    psi = W.random_state(5, 50)
    t = 2 * math.pi / omega
    out, log, na = K.expv(lambda v: n * omega * v, psi, t, tol=1e-11, m_max=20, max_substeps=200)
    exact = np.exp(-1j * t * omega * n) * psi
    assert len(log) > 1 and any(h > 0 for k, h in log)
    assert np.linalg.norm(out - exact) < 1e-9


def test_expv_fixed_k_error_order():
    # Sec. 8.1: for fixed K the Krylov error of exp(-i H dt) is of order dt^K
    H = _herm(40, 21)
    psi = W.random_state(22, 40)
    errs = []
    for tau in (0.08, 0.04):
        out, _, _ = K.expv(lambda v: H @ v, psi, tau, tol=0.0, m_max=4)
        errs.append(np.linalg.norm(out - expm(-1j * tau * H) @ psi))
    slope = math.log2(errs[0] / errs[1])
    assert 3.6 < slope < 4.4, slope


def test_expv_eigenvector_breakdown():
    H = _herm(16, 31)
    lam, Q = np.linalg.eigh(H)
    psi = Q[:, 3].astype(np.complex128)
    out, log, na = K.expv(lambda v: H @ v, psi, 0.7, tol=1e-12, m_max=10)
    assert log == [(1, 0)] and na == 1
    assert np.linalg.norm(out - np.exp(-0.7j * lam[3]) * psi) < 1e-13


def test_expv_zero_operator_is_identity():
    psi = W.random_state(7, 12)
    out, log, na = K.expv(lambda v: 0 * v, psi, 0.3, tol=1e-12, m_max=8)
    assert np.array_equal(out, psi) or np.linalg.norm(out - psi) < 1e-15


def test_expv_forced_replay_is_identical():
    H = _herm(48, 41)
    psi = W.random_state(42, 48)
    out, log, _ = K.expv(lambda v: H @ v, psi, 1.5, tol=1e-10, m_max=10, max_substeps=400)
    out2, log2, _ = K.expv(lambda v: H @ v, psi, 1.5, tol=1e-10, m_max=10, max_substeps=400, forced=log)
    assert any(h > 0 for _, h in log)
    assert log2 == log and np.array_equal(out, out2)


def test_expv_substep_cap_raises():
    n = np.arange(200)
    psi = W.random_state(5, 200)
    with pytest.raises(K.KrylovError):
        K.expv(lambda v: 50.0 * n * v, psi, 1.0, tol=1e-12, m_max=4, max_substeps=3)


# ---------------------------------------------------------------- full re-orthogonalisation (option)
def _gram_defect(V):
    M = np.array(V)
    return np.abs(M.conj() @ M.T - np.eye(len(V))).max()


def test_reorth_keeps_the_basis_orthonormal():
    # a spectrum with outliers: once the outlying Ritz values converge, the
    # three-term recurrence loses orthogonality (Paige); one classical
    # Gram-Schmidt sweep per step keeps the basis orthonormal to rounding
    lam = np.concatenate([np.linspace(0.0, 1.0, 300), [50.0, 100.0, 200.0]])
    psi = W.random_state(3, len(lam))
    V0, _, _ = K.lanczos(lambda v: lam * v, psi, 60)
    V1, _, _ = K.lanczos(lambda v: lam * v, psi, 60, reorth=True)
    assert _gram_defect(V0[:-1]) > 1e-2
    assert _gram_defect(V1) < 1e-13


@pytest.mark.parametrize("reorth", [False, True])
def test_lanczos_helper_is_the_expv_recurrence(reorth):
    # expv with a fixed K reconstructs beta_0 V_K exp(-i tau T_K) e_1 from the
    # same recurrence as the helper
    H = _herm(48, 31)
    psi = W.random_state(32, 48)
    out, _, _ = K.expv(lambda v: H @ v, psi, 0.3, tol=0.0, m_max=12, reorth=reorth)
    V, a, b = K.lanczos(lambda v: H @ v, psi, 12, reorth=reorth)
    y = K.tridiag_expm_e1(a, b[:11], 0.3)
    assert np.linalg.norm(out - np.linalg.norm(psi) * sum(y[i] * V[i] for i in range(12))) < 1e-14


@pytest.mark.parametrize("tau", [0.4, 3.0])
def test_expv_reorth_matches_expm_and_the_plain_recurrence(tau):
    # results agree with the dense exponential and across the two modes within
    # the tolerance
    H = _herm(64, 11)
    psi = W.random_state(12, 64)
    a, _, _ = K.expv(lambda v: H @ v, psi, tau, tol=1e-12, m_max=30, reorth=True)
    b, _, _ = K.expv(lambda v: H @ v, psi, tau, tol=1e-12, m_max=30)
    ref = expm(-1j * tau * H) @ psi
    assert np.linalg.norm(a - ref) < 1e-10 and np.linalg.norm(a - b) < 1e-10


def test_expv_reorth_on_the_outlier_spectrum():
    # the spectrum that breaks orthogonality: with a large Krylov space and a
    # long step both modes still meet the tolerance against the exact result
    lam = np.concatenate([np.linspace(0.0, 1.0, 300), [50.0, 100.0, 200.0]])
    psi = W.random_state(4, len(lam))
    exact = np.exp(-1j * 0.05 * lam) * psi
    for reorth in (False, True):
        out, log, _ = K.expv(lambda v: lam * v, psi, 0.05, tol=1e-12, m_max=60, reorth=reorth, max_substeps=50)
        assert np.linalg.norm(out - exact) < 1e-10, (reorth, log)


def test_planted_conjugation_error_in_gram_schmidt_is_caught(monkeypatch):
    # Gram-Schmidt coefficients <w, v_i> instead of <v_i, w>: the basis is no
    # longer orthonormal on the outlier spectrum
    def bad(V, w):
        for v in V:
            w = w - np.vdot(w, v) * v
        return w

    monkeypatch.setattr(K, "gram_schmidt", bad)
    lam = np.concatenate([np.linspace(0.0, 1.0, 300), [50.0, 100.0, 200.0]])
    psi = W.random_state(3, len(lam)) * np.exp(1j * np.linspace(0, 3, len(lam)))
    V, _, _ = K.lanczos(lambda v: lam * v, psi, 40, reorth=True)
    M = np.array(V)
    assert np.abs(M.conj() @ M.T - np.eye(len(V))).max() > 1e-8


@pytest.mark.parametrize("tau", [0.3, 1.0])
def test_expv_tolerance_is_absolute_for_unnormalised_states(tau):
    # the estimate carries beta_0 = ||psi||: for ||psi|| = 1000 the absolute
    # error still meets tol (without beta_0 the accepted Krylov spaces are
    # smaller and the error here exceeds 1e-9)
    a = W.complex_gaussian(11, 200 * 200).reshape(200, 200)
    H = 0.5 * (a + a.conj().T)
    psi = 1000.0 * W.random_state(12, 200)
    out, log, _ = K.expv(lambda v: H @ v, psi, tau, tol=1e-9, m_max=40)
    assert np.linalg.norm(out - expm(-1j * tau * H) @ psi) <= 1e-9


# ---------------------------------------------------------------- Gershgorin width
# The width gates when the estimate of Eq. (KryErr) is trusted (|tau| width
# <= 2k); it must never be smaller than the true eigenvalue spread of T_k.
# Pins: the dense eigenvalue spread (numpy eigvalsh) of random tridiagonals
# with either sign of beta, and closed forms where Gershgorin is exact.

def _width_bounds_spread(width_fn):
    cases = []
    for seed in range(40):
        k = 1 + seed % 12
        alpha = W.uniform(300 + seed, k, -3, 3)
        beta = W.uniform(400 + seed, max(k - 1, 1), -2, 2)[:k - 1]
        cases.append((alpha, beta))
    cases.append((np.zeros(3), np.ones(2)))                  # spread 2 sqrt(2)
    cases.append((np.array([5.0, -1.0, 2.0, 0.5]), np.array([0.0, 3.0, 0.0])))
    for alpha, beta in cases:
        lam = np.linalg.eigvalsh(K.tridiag_matrix(alpha, beta))
        if width_fn(list(alpha), list(beta)) < (lam[-1] - lam[0]) * (1 - 1e-14) - 1e-14:
            return False
    return True


def test_gershgorin_width_bounds_the_eigenvalue_spread():
    assert _width_bounds_spread(K.gershgorin_width)


def test_gershgorin_width_closed_forms():
    # one row: zero width; diagonal T: the exact spread of its entries;
    # [[a, b], [b, a]]: eigenvalues a -+ b, width 2|b| exactly; the k x k
    # tridiagonal with zero diagonal and unit off-diagonal: rows 2..k-1 reach
    # +-2, so the width is 4 (its spread is 4 cos(pi / (k + 1)) < 4)
    assert K.gershgorin_width([1.7], []) == 0.0
    assert K.gershgorin_width([3.0, -2.0, 0.5], [0.0, 0.0]) == 5.0
    assert K.gershgorin_width([0.3, 0.3], [-1.25]) == 2.5
    for k in (3, 7, 16):
        assert K.gershgorin_width([0.0] * k, [1.0] * (k - 1)) == 4.0
        lam = np.linalg.eigvalsh(K.tridiag_matrix(np.zeros(k), np.ones(k - 1)))
        assert abs((lam[-1] - lam[0]) - 4 * math.cos(math.pi / (k + 1))) < 1e-13


def test_planted_missing_neighbour_in_gershgorin_width_is_caught(monkeypatch):
    # a radius that counts only the next row's coupling underestimates the
    # spread (3 x 3 example: width 2 against 2 sqrt(2)); so does a width
    # taken from the signed couplings
    def one_sided(alpha, beta):
        k = len(alpha)
        lo, hi = np.inf, -np.inf
        for r in range(k):
            rad = abs(beta[r]) if r < k - 1 else 0.0
            lo, hi = min(lo, alpha[r] - rad), max(hi, alpha[r] + rad)
        return hi - lo

    def signed(alpha, beta):
        k = len(alpha)
        lo, hi = np.inf, -np.inf
        for r in range(k):
            rad = (beta[r - 1] if r > 0 else 0.0) + (beta[r] if r < k - 1 else 0.0)
            lo, hi = min(lo, alpha[r] - rad), max(hi, alpha[r] + rad)
        return hi - lo

    for bad in (one_sided, signed):
        monkeypatch.setattr(K, "gershgorin_width", bad)
        assert not _width_bounds_spread(K.gershgorin_width)
