"""Time-step selection for CFETs (oracle).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Sec. 6.6 (time-step selection) uses the error model of an Nth-order CFET,
epsilon = c T dt^N, and estimates the constant c from two propagations over
the same interval with steps dt_1 and dt_2:
    max_t ||x_1(t) - x_2(t)|| = c T |dt_1^N - dt_2^N|,
recommending dt_1 / dt_2 = (2 ... 3)^(1/N); from c the step for an accuracy
goal follows by extrapolation, and repeating the estimate at every step gives
adaptive step selection.  Readings taken here (the paper gives no more):

* the two grids meet only at the end of the interval, so the difference is
  taken at t0 + T (the model error grows linearly in t, so that is also its
  maximum); n_2 = round(n_1 ratio^(1/N)) steps give dt_2 = T / n_2;
* the step for a goal eps over a run of length T is dt = (eps / (c T))^(1/N),
  shortened to T / ceil(T / dt) so that whole steps end at T;
* adaptive stepping: from the state x at time t with trial step h, x_1 = one
  step of h, x_2 = two steps of h / 2; the model over one interval of length h
  gives c = ||x_1 - x_2|| / (h (h^N - (h/2)^N)) (``local_error_constant``);
  the run continues from x_2, so the step is accepted when the error the
  model gives for a whole run with steps of h / 2, c T (h/2)^N, is at most eps
  (or h has reached h_min); the next trial step is
  min(2 h, 1.8 (eps / (c T))^(1/N)) (0.9 times the h whose half meets the
  goal), clipped to [h_min, h_max] and to the remaining time.

Parity: pinned by ``tests/test_oracle_timestep.py`` against the driven
two-level system's exact propagator (Eq. (TwoLevelU)): the estimated c
predicts the true error of a third step size, the selected dt meets its goal,
the adaptive run meets its goal with steps that follow the drive.
"""

from __future__ import annotations

import math

import numpy as np


def error_constant(step, psi0, t0, T, n1, order, ratio=2.0):
    """c from two runs over [t0, t0 + T]: n1 steps and round(n1 ratio^(1/N)).
    step(psi, t, dt, nsteps) -> psi.  Returns (c, difference, dt2)."""
    N = int(order)
    n2 = int(round(n1 * ratio ** (1.0 / N)))
    if n2 <= n1:
        n2 = n1 + 1
    dt1, dt2 = T / n1, T / n2
    x1 = step(np.array(psi0, dtype=np.complex128), t0, dt1, n1)
    x2 = step(np.array(psi0, dtype=np.complex128), t0, dt2, n2)
    e = float(np.linalg.norm(x1 - x2))
    c = e / (T * abs(dt1 ** N - dt2 ** N))
    return c, e, dt2


def select_dt(step, psi0, t0, T, target, T_probe, n_probe, order, ratio=2.0):
    """dt and the number of steps for the goal `target` over a run of length T,
    with c estimated over [t0, t0 + T_probe].  Returns (dt, nsteps, c)."""
    N = int(order)
    c, _, _ = error_constant(step, psi0, t0, T_probe, n_probe, order, ratio)
    if c <= 0.0:
        return T, 1, c
    dt = (target / (c * T)) ** (1.0 / N)
    n = int(math.ceil(T / dt))
    return T / n, n, c


def local_error_constant(step, psi, t, h, order):
    """(c, x_2) from one step of h and two of h / 2 starting at (psi, t)."""
    N = int(order)
    x1 = step(np.array(psi, dtype=np.complex128), t, h, 1)
    x2 = step(np.array(psi, dtype=np.complex128), t, h / 2.0, 2)
    e = float(np.linalg.norm(x1 - x2))
    return e / (h * (h ** N - (h / 2.0) ** N)), x2


def propagate_adaptive(step, psi, t0, T, order, target, h0, h_min, h_max, max_steps, forced_h=None):
    """Adaptive CFET stepping over [t0, t0 + T] by the per-step estimate above.
    forced_h: replay these accepted steps (no estimate).  Returns
    (psi, accepted steps, number of trial steps)."""
    N = int(order)
    x = np.array(psi, dtype=np.complex128, copy=True)
    t, t_end = t0, t0 + T
    hs, trials = [], 0
    if forced_h is not None:
        for h in forced_h:
            x = step(x, t, h / 2.0, 2)
            t += h
        return x, list(forced_h), 0
    h = h0
    while t_end - t > 1e-12 * max(1.0, abs(t_end)):
        if len(hs) >= max_steps:
            raise RuntimeError("adaptive stepping: more than max_steps steps")
        rem = t_end - t
        h = min(h, rem)
        trials += 1
        c, x2 = local_error_constant(step, x, t, h, order)
        if c * T * (h / 2.0) ** N <= target or h <= h_min:
            x = x2
            t = t + h if h < rem else t_end
            hs.append(h)
        h_new = 2.0 * h if c <= 0.0 else min(2.0 * h, 1.8 * (target / (c * T)) ** (1.0 / N))
        h = min(max(h_new, h_min), h_max)
    return x, hs, trials
