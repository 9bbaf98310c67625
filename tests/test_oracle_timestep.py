"""Pins for oracle/timestep.py (Sec. 6.6 time-step selection) against the
driven two-level system with its exact propagator (Eq. (TwoLevelU)) and a
fine-step reference for a chirped drive."""

import math

import numpy as np
import pytest

from oracle import cfet, operators as O, timestep as TS


def _exact(t, Dl, V, w):
    Om = math.sqrt((Dl - w) ** 2 + V**2)
    c, s = math.cos(Om * t), math.sin(Om * t)
    return np.array([[np.exp(-1j * w * t) * (c - 1j * (Dl - w) / Om * s), -1j * V / Om * np.exp(-1j * w * t) * s],
                     [-1j * V / Om * np.exp(1j * w * t) * s, np.exp(1j * w * t) * (c + 1j * (Dl - w) / Om * s)]])


def _problem(Dl=2.0, V=0.5, w=1.0):
    op = O.Dense(Dl * O.SZ, [O.SX, O.SY])
    drives = [lambda t: V * math.cos(2 * w * t), lambda t: V * math.sin(2 * w * t)]
    return op, drives


def _stepper(op, drives, scheme):
    return lambda psi, t, dt, n: cfet.propagate(op, psi, t, dt, n, scheme, drives, 1e-14, 2)


PSI0 = np.array([0.6, 0.8j])


@pytest.mark.parametrize("scheme,order", [("CF4:2", 4), ("CF6:5Opt", 6)])
def test_error_constant_predicts_the_true_error(scheme, order):
    # c from runs with n1 and n1 * 2^(1/N) steps predicts ||x_dt(T) - x(T)||
    # for a third, coarser step within 30 %
    Dl, V, w = 2.0, 0.5, 1.0
    op, drives = _problem(Dl, V, w)
    step = _stepper(op, drives, scheme)
    T = 5 * math.pi
    c, e, dt2 = TS.error_constant(step, PSI0, 0.0, T, 200, order)
    assert e > 0 and dt2 < T / 200
    exact = _exact(T, Dl, V, w) @ PSI0
    n = 120
    true_err = np.linalg.norm(step(PSI0, 0.0, T / n, n) - exact)
    pred = c * T * (T / n) ** order
    assert 0.7 <= pred / true_err <= 1.3, (pred, true_err)
    # the ratio dt1/dt2 = 3^(1/N) gives the same constant
    c3, _, _ = TS.error_constant(step, PSI0, 0.0, T, 200, order, ratio=3.0)
    assert abs(c3 / c - 1.0) <= 0.15


@pytest.mark.parametrize("target", [1e-5, 1e-7])
def test_selected_step_meets_the_goal(target):
    Dl, V, w = 2.0, 0.5, 1.0
    op, drives = _problem(Dl, V, w)
    step = _stepper(op, drives, "CF4:2")
    T = 20 * math.pi
    dt, n, c = TS.select_dt(step, PSI0, 0.0, T, target, 2 * math.pi, 60, 4)
    assert abs(n * dt - T) < 1e-12 * T
    err = np.linalg.norm(step(PSI0, 0.0, dt, n) - _exact(T, Dl, V, w) @ PSI0)
    assert 0.05 * target <= err <= 1.5 * target, (err, target)


@pytest.mark.parametrize("scheme,order", [("CF4:2", 4), ("CF6:5Opt", 6)])
def test_local_constant_is_time_invariant_for_the_rotating_drive(scheme, order):
    # H(t) of the rotating drive is H(0) rotated about z by 2wt, so the norm of
    # the one-step difference, hence c, is the same at every t; and the local
    # model scales as h^(N+1): halving h leaves c unchanged to O(h)
    op, drives = _problem()
    step = _stepper(op, drives, scheme)
    cs = [TS.local_error_constant(step, PSI0, t, 0.2, order)[0] for t in (0.0, 1.1, 2.5, 4.0)]
    assert max(cs) / min(cs) - 1.0 <= 1e-6   # rounding of a ~1e-9 difference
    c_half = TS.local_error_constant(step, PSI0, 0.0, 0.1, order)[0]
    assert abs(c_half / cs[0] - 1.0) <= 0.1


def _chirp_problem():
    # drive frequency grows linearly: steps must shrink over the run
    op = O.Dense(1.0 * O.SZ, [O.SX])
    drives = [lambda t: 0.8 * math.cos(0.5 * t + 0.15 * t * t)]
    return op, drives


def test_adaptive_steps_meet_the_goal_and_follow_the_drive():
    op, drives = _chirp_problem()
    step = _stepper(op, drives, "CF4:2")
    T, target = 12.0, 1e-7
    ref = cfet.propagate(op, PSI0, 0.0, T / 6000, 6000, "CF8:11", drives, 1e-14, 2)
    x, hs, trials = TS.propagate_adaptive(step, PSI0, 0.0, T, 4, target, 0.1, 1e-4, 1.0, 10000)
    assert abs(sum(hs) - T) < 1e-9
    err = np.linalg.norm(x - ref)
    # local errors add up less than coherently, so the per-step control is
    # conservative, but not by orders of magnitude
    assert target / 500 <= err <= target, err
    # the drive is ~4x faster at the end than at the start
    assert np.mean(hs[-5:]) < 0.6 * np.mean(hs[2:7])
    assert trials >= len(hs)


def test_adaptive_replay_is_identical_and_fixed_step_is_worse_at_equal_cost():
    op, drives = _chirp_problem()
    step = _stepper(op, drives, "CF4:2")
    T, target = 12.0, 1e-7
    x, hs, _ = TS.propagate_adaptive(step, PSI0, 0.0, T, 4, target, 0.1, 1e-4, 1.0, 10000)
    y, hs2, trials = TS.propagate_adaptive(step, PSI0, 0.0, T, 4, target, 0.1, 1e-4, 1.0, 10000, forced_h=hs)
    assert np.array_equal(x, y) and hs2 == hs and trials == 0
    # a uniform grid with as many half steps is less accurate (the error
    # concentrates where the drive is fast)
    ref = cfet.propagate(op, PSI0, 0.0, T / 6000, 6000, "CF8:11", drives, 1e-14, 2)
    n = 2 * len(hs)
    z = step(PSI0, 0.0, T / n, n)
    assert np.linalg.norm(x - ref) < np.linalg.norm(z - ref)


# ---------------------------------------------------------------- planted mistakes
def test_planted_missing_step_factor_is_caught(monkeypatch):
    # the local constant without its factor h (model h^N instead of h^(N+1)
    # per step): halving h no longer leaves c unchanged
    def bad(step, psi, t, h, order):
        N = int(order)
        x1 = step(np.array(psi, dtype=np.complex128), t, h, 1)
        x2 = step(np.array(psi, dtype=np.complex128), t, h / 2.0, 2)
        return float(np.linalg.norm(x1 - x2)) / (h ** N - (h / 2.0) ** N), x2

    monkeypatch.setattr(TS, "local_error_constant", bad)
    op, drives = _problem()
    step = _stepper(op, drives, "CF4:2")
    c1 = TS.local_error_constant(step, PSI0, 0.0, 0.2, 4)[0]
    c2 = TS.local_error_constant(step, PSI0, 0.0, 0.1, 4)[0]
    assert abs(c2 / c1 - 1.0) > 0.1


def test_planted_missing_run_length_is_caught(monkeypatch):
    # the two-run constant without the run length T in the model
    # eps = c T dt^N: it no longer predicts the true error of a third step
    def bad(step, psi0, t0, T, n1, order, ratio=2.0):
        N = int(order)
        n2 = int(round(n1 * ratio ** (1.0 / N)))
        dt1, dt2 = T / n1, T / n2
        x1 = step(np.array(psi0, dtype=np.complex128), t0, dt1, n1)
        x2 = step(np.array(psi0, dtype=np.complex128), t0, dt2, n2)
        e = float(np.linalg.norm(x1 - x2))
        return e / abs(dt1 ** N - dt2 ** N), e, dt2

    monkeypatch.setattr(TS, "error_constant", bad)
    Dl, V, w = 2.0, 0.5, 1.0
    op, drives = _problem(Dl, V, w)
    step = _stepper(op, drives, "CF4:2")
    T = 5 * math.pi
    c, _, _ = TS.error_constant(step, PSI0, 0.0, T, 200, 4)
    n = 120
    true_err = np.linalg.norm(step(PSI0, 0.0, T / n, n) - _exact(T, Dl, V, w) @ PSI0)
    assert not 0.7 <= c * T * (T / n) ** 4 / true_err <= 1.3
