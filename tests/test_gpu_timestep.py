"""GPU checks of the time-step selection entry points (Sec. 6.6):
cfet_error_constant, cfet_select_dt and cfet_propagate_adaptive against the
oracle's procedures (oracle/timestep.py) run with the oracle's CFET stepping.

The constants come from differences of two propagations (~1e-6 at order 4,
~2e-10 at order 6 here).  With the oracle's Krylov decisions the GPU and
oracle states differ only by rounding, at most 1e-14 over the few thousand
applies of the two runs, so c agrees to 1e-5 relative or to 1e-14 over the
difference, whichever is larger;
adaptive runs are compared by replaying the GPU's accepted steps in the oracle
(states within the usual 1e-10 parity) and by the step sequences themselves.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, operators as O, timestep as TS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1102_5071_gb300.build import build
    build()
    return torch


def _chain(N=8, drive=None, **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N)
    d = drive or pr.drive
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [d], **kw)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    return prop, op, [d]


def _oracle_step(op, drives, order, tol=1e-13, m=20):
    return lambda psi, t, dt, n: OC.propagate(op, psi, t, dt, n, order, drives, tol, m, max_substeps=400)


def chirp(t):
    return 0.8 * math.cos(0.5 * t + 0.15 * t * t)


@pytest.mark.parametrize("order", [4, 6])
def test_error_constant_matches_oracle(torch_cuda, order):
    prop, op, drives = _chain(m_max=20)
    psi0 = W.neel_state(8)
    x = torch_cuda.from_numpy(psi0).cuda()
    c, diff, dt2 = prop.error_constant(x, 0.0, 2.0, 20, order=order, tol=1e-13)
    c_o, diff_o, dt2_o = TS.error_constant(_oracle_step(op, drives, order), psi0, 0.0, 2.0, 20, order)
    assert dt2 == dt2_o
    assert abs(c / c_o - 1.0) <= max(1e-5, 1e-14 / diff_o), (c, c_o, diff_o)
    assert np.array_equal(x.cpu().numpy(), psi0)   # psi0 unchanged


def test_select_dt_matches_oracle_and_meets_the_goal(torch_cuda):
    prop, op, drives = _chain(m_max=20)
    psi0 = W.random_state(4, 256)
    x = torch_cuda.from_numpy(psi0).cuda()
    T, target = 4.0, 1e-7
    dt, n, c = prop.select_dt(x, 0.0, T, target, 1.0, 10, order=4, tol=1e-13)
    dt_o, n_o, c_o = TS.select_dt(_oracle_step(op, drives, 4), psi0, 0.0, T, target, 1.0, 10, 4)
    assert n == n_o and abs(dt - dt_o) <= 1e-12 and abs(c / c_o - 1.0) <= 1e-5
    prop.propagate(x, 0.0, dt, n, order=4, tol=1e-13)
    ref = OC.propagate(op, psi0, 0.0, T / 2000, 2000, 8, drives, 1e-14, 20)
    err = np.linalg.norm(x.cpu().numpy() - ref)
    assert 0.02 * target <= err <= 2.0 * target, err


def test_adaptive_matches_oracle(torch_cuda):
    prop, op, drives = _chain(drive=chirp, m_max=20)
    psi0 = W.random_state(5, 256)
    T, target = 6.0, 1e-8
    x = torch_cuda.from_numpy(psi0).cuda()
    hs, trials, st = prop.propagate_adaptive(x, 0.0, T, target, 0.1, 1e-4, 1.0, order=4, tol=1e-13)
    assert abs(sum(hs) - T) <= 1e-9 and trials >= len(hs) and st["n_exp"] > 0
    step = _oracle_step(op, drives, 4)
    # the oracle replaying the GPU's steps reaches the same state
    y, _, _ = TS.propagate_adaptive(step, psi0, 0.0, T, 4, target, 0.1, 1e-4, 1.0, 10000, forced_h=hs)
    assert np.linalg.norm(x.cpu().numpy() - y) <= 1e-10
    # and chooses the same steps itself
    _, hs_o, trials_o = TS.propagate_adaptive(step, psi0, 0.0, T, 4, target, 0.1, 1e-4, 1.0, 10000)
    assert len(hs_o) == len(hs) and trials_o == trials
    assert max(abs(a / b - 1.0) for a, b in zip(hs, hs_o)) <= 1e-4
    # steps shrink as the chirped drive speeds up, and the goal is met
    assert np.mean(hs[-4:]) < np.mean(hs[1:5])
    ref = OC.propagate(op, psi0, 0.0, T / 4000, 4000, 8, drives, 1e-14, 20)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= target


def test_adaptive_replay_and_errors(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, op, drives = _chain(drive=chirp)
    psi0 = W.random_state(6, 256)
    x = torch.from_numpy(psi0).cuda()
    hs, _, _ = prop.propagate_adaptive(x, 0.0, 3.0, 1e-8, 0.1, 1e-4, 1.0, order=6, tol=1e-12)
    y = torch.from_numpy(psi0).cuda()
    hs2, trials, _ = prop.propagate_adaptive(y, 0.0, 3.0, 1e-8, 0.1, 1e-4, 1.0, order=6, tol=1e-12, forced_h=hs)
    assert hs2 == hs and trials == 0 and torch.equal(x, y)
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.propagate_adaptive(y, 0.0, 1.0, 1e-8, 0.1, 0.2, 1.0)          # h0 < h_min
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.error_constant(y, 0.0, 1.0, 10, ratio=1.0)
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.select_dt(y, 0.0, 1.0, -1.0, 0.5, 5)
    with pytest.raises(P.CfetError, match="EKRYLOV"):
        prop.propagate_adaptive(y, 0.0, 5.0, 1e-12, 0.01, 0.01, 0.01, max_steps=3)


def test_full_size_chain_error_constant_predicts_the_error(torch_cuda):
    # N = 20 (the benchmark chain), CF4:2: c from 8 and 10 steps over T = 0.4
    # predicts the error of 5 steps against a fine CF8:11 run within 30 %
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, _, _ = _chain(20)
    psi0 = torch.from_numpy(W.random_state(2, 1 << 20)).cuda()
    T = 0.4
    c, _, _ = prop.error_constant(psi0, 0.0, T, 8, order=4, tol=1e-13, ratio=2.0)
    x = psi0.clone()
    prop.propagate(x, 0.0, T / 5, 5, order=4, tol=1e-13)
    ref = psi0.clone()
    prop.propagate(ref, 0.0, T / 80, 80, order=8, tol=1e-13)
    err = torch.linalg.vector_norm(x - ref).item()
    pred = c * T * (T / 5) ** 4
    assert 0.7 <= pred / err <= 1.3, (pred, err)
