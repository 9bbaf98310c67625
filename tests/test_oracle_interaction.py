"""Pins for oracle/interaction.py (Secs. 9.3, 9.4): closed forms where the
interaction picture is exact, convergence to the Schroedinger-picture
propagation, Hermitian stage operators."""

import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import cfet, interaction as IP, operators as O, schemes as S


def _exact_two_level(t, Dl, V, w):
    Om = math.sqrt((Dl - w) ** 2 + V**2)
    c, s = math.cos(Om * t), math.sin(Om * t)
    return np.array([[np.exp(-1j * w * t) * (c - 1j * (Dl - w) / Om * s), -1j * V / Om * np.exp(-1j * w * t) * s],
                     [-1j * V / Om * np.exp(1j * w * t) * s, np.exp(1j * w * t) * (c + 1j * (Dl - w) / Om * s)]])


def test_diagonal_hamiltonian_is_exact_for_any_step():
    # J = 0 and no drive: H = H_d, x^I is constant, so three coarse steps give
    # exp(-i H_d T) psi exactly
    N = 6
    h = W.uniform(3, N, -1, 1)
    op = O.SpinChain(N, 0.0, 0.7, h, [np.ones(N)])
    psi0 = W.random_state(2, 1 << N)
    out = IP.propagate(op, psi0, 0.3, 1.7, 3, "CF4:2", [lambda t: 0.0], 1e-13, 10)
    Hd = np.real(np.diag(O.xxz_dense(N, 0.0, 0.7, h)))
    assert np.linalg.norm(out - np.exp(-1j * Hd * 5.1) * psi0) <= 1e-13


@pytest.mark.parametrize("scheme", ["CF4:2", "CF6:5Opt", "CF8:11"])
def test_resonant_two_level_is_exact(scheme):
    # H = Dl sz + V (cos 2wt sx + sin 2wt sy) with Dl = w: in the interaction
    # picture of D = Dl sz the Hamiltonian is the constant V sx (Sec. 9.3), so a
    # few coarse CFET steps reproduce Eq. (TwoLevelU) to rounding; the
    # Schroedinger picture with the same steps does not
    Dl, V, w = 1.3, 0.4, 1.3
    op = O.Dense(Dl * O.SZ, [O.SX, O.SY])
    drives = [lambda t: V * math.cos(2 * w * t), lambda t: V * math.sin(2 * w * t)]
    psi0 = np.array([0.6, 0.8j])
    T = 4.0
    out = IP.propagate(op, psi0, 0.0, T / 4, 4, scheme, drives, 1e-14, 2)
    exact = _exact_two_level(T, Dl, V, w) @ psi0
    assert np.linalg.norm(out - exact) <= 1e-12
    sp = cfet.propagate(op, psi0, 0.0, T / 4, 4, scheme, drives, 1e-14, 2)
    assert np.linalg.norm(sp - exact) > 1e-6


def test_converges_to_the_schroedinger_picture_with_the_order():
    N = 6
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    psi0 = W.random_state(7, 1 << N)
    T = 2.0
    ref = cfet.propagate(op, psi0, 0.0, T / 400, 400, "CF8:11", [pr.drive], 1e-14, 30)
    errs = []
    for n in (20, 40):
        out = IP.propagate(op, psi0, 0.0, T / n, n, "CF4:2", [pr.drive], 1e-14, 30)
        errs.append(np.linalg.norm(out - ref))
    slope = math.log2(errs[0] / errs[1])
    assert 3.6 <= slope <= 4.4, (errs, slope)
    assert abs(np.linalg.norm(out) - 1.0) <= 1e-12


def test_stage_operator_is_hermitian_and_matches_the_dense_definition():
    N = 5
    pr = W.spin_chain(N)
    a2 = W.uniform(9, N, -1, 1)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield, a2])
    d, offdiag = IP.diagonal(op)
    g, x, _, _ = S.g_coefficients(S.get("CF6:5Opt"))
    t, dt = 0.4, 0.1
    tn = [t + xm * dt for xm in x]
    fv = [[math.cos(tm), 0.5 * math.sin(2 * tm)] for tm in tn]
    apply = IP.stage_apply(d, offdiag, g[1], tn, fv)
    # dense: sum_m g_m e^{i Hd t_m} (H0 - Hd + f1 V1 + f2 V2) e^{-i Hd t_m}
    H0 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    Hd = np.diag(np.diag(H0))
    M = np.zeros_like(H0)
    for gm, tm, fm in zip(g[1], tn, fv):
        U = expm(1j * Hd * tm)
        Hb = H0 - Hd + fm[0] * O.xfield_dense(N, pr.xfield) + fm[1] * O.xfield_dense(N, a2)
        M += gm * U @ Hb @ U.conj().T
    assert np.allclose(M, M.conj().T, atol=1e-13)
    u, v = W.random_state(1, 32), W.random_state(2, 32)
    assert np.allclose(apply(v), M @ v, atol=1e-13)
    assert abs(np.vdot(u, apply(v)) - np.conj(np.vdot(v, apply(u)))) <= 1e-13


# ---------------------------------------------------------------- planted mistakes
def test_planted_phase_sign_error_is_caught(monkeypatch):
    # stage operators built with e^{-i d t} H_b e^{+i d t} (the picture's
    # phases reversed): the resonant two-level system is no longer exact
    def bad(d, offdiag, g_row, t_nodes, fvals):
        def apply(v):
            out = np.zeros_like(v)
            for gm, tm, fm in zip(g_row, t_nodes, fvals):
                ph = np.exp(-1j * d * tm)
                out += gm * (ph * offdiag([1.0] + list(fm), np.conj(ph) * v))
            return out
        return apply

    monkeypatch.setattr(IP, "stage_apply", bad)
    Dl, V, w = 1.3, 0.4, 1.3
    op = O.Dense(Dl * O.SZ, [O.SX, O.SY])
    drives = [lambda t: V * math.cos(2 * w * t), lambda t: V * math.sin(2 * w * t)]
    psi0 = np.array([0.6, 0.8j])
    T = 4.0
    out = IP.propagate(op, psi0, 0.0, T / 4, 4, "CF4:2", drives, 1e-14, 2)
    assert np.linalg.norm(out - _exact_two_level(T, Dl, V, w) @ psi0) > 1e-6
