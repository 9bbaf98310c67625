"""GPU checks of the fidelity gradient (cfet_fidelity_grad, the adjoint sweep).

* small chains: loss and gradient against the oracle's exact gradient
  (dense stage exponentials and Frechet derivatives), forward in the
  fixed-point and FP64 formats, with and without intermediate checkpoints;
* the full-size configuration (N = 18, 64 amplitude segments, T = 16,
  CF4:2, dt = 0.01, FP64): all 64 components against central finite
  differences (h = 1e-6) of the GPU fidelity, relative to the largest
  component, with a fixed Krylov dimension so that the loss is a smooth
  function of the amplitudes;
* the torch.autograd wrapper and argument validation.

Tolerances: the forward and backward Krylov exponentials are accurate to the
Krylov tolerance per stage, so loss and gradient differ from the exact ones by
a few times n_stages x tol; central differences have truncation error
O(h^2) and rounding error O(eps F / h), F the fidelity that is differenced.
"""


import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA, operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1102_5071_gb300.build import build
    build()
    return torch


def _prop(N, prec, m_max=16, a=None, nfields=1):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N)
    a = np.ones(N) if a is None else a
    V = [P.XField(N, a)] + [P.XField(N, np.ones(N))] * (nfields - 1)
    return P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), V, [lambda t: 0.0] * nfields, m_max=m_max,
                        precision=prec), pr


@pytest.mark.parametrize("prec", ["fx", "f64"])
@pytest.mark.parametrize("order,ce", [(4, 2), (6, 8), (2, 1)])
def test_gradient_matches_oracle_small(torch_cuda, prec, order, ce):
    torch = torch_cuda
    N, nseg, nsteps, dt, omega, phase = 4, 4, 8, 0.12, 2.0, 0.3
    a = W.uniform(41, N, 0.3, 1.2)
    prop, pr = _prop(N, prec, a=a)
    psi0, phi = W.random_state(1, 1 << N), W.random_state(11, 1 << N)
    amps = W.uniform(5, nseg, -1.0, 1.0)
    H0 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    V = O.xfield_dense(N, a)
    L_ref, g_ref = OA.grad_dense(H0, V, psi0, phi, amps, omega, phase, 0.0, dt, nsteps, order)
    L, g, st = prop.fidelity_grad(torch.from_numpy(psi0).cuda(), torch.from_numpy(phi).cuda(), 0.0, dt, nsteps,
                                  amps, omega, phase, order=order, tol=1e-13, checkpoint_every=ce)
    assert abs(L - L_ref) <= 1e-11, (L, L_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-9, (g, g_ref)
    assert st["max_drift"] <= 1e-10 and st["n_applies_backward"] > 0


@pytest.mark.parametrize("dt", [0.6, 2.0])
def test_gradient_with_long_stages_matches_oracle(torch_cuda, dt):
    # long stage exponentials make the stage integral oscillate fast:
    # om = |tau| (width_psi + width_lambda) selects the 24-node (dt 0.6) and
    # the 48-node rule (dt 2.0); the gradient still matches the oracle's exact
    # one (dense exponentials and Frechet derivatives)
    torch = torch_cuda
    N, nseg, nsteps, omega, phase = 4, 2, 4, 2.0, 0.3
    a = W.uniform(41, N, 0.3, 1.2)
    prop, pr = _prop(N, "f64", a=a)
    psi0, phi = W.random_state(1, 1 << N), W.random_state(11, 1 << N)
    amps = W.uniform(5, nseg, -1.0, 1.0)
    H0 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    V = O.xfield_dense(N, a)
    L_ref, g_ref = OA.grad_dense(H0, V, psi0, phi, amps, omega, phase, 0.0, dt, nsteps, 4)
    L, g, st = prop.fidelity_grad(torch.from_numpy(psi0).cuda(), torch.from_numpy(phi).cuda(), 0.0, dt, nsteps,
                                  amps, omega, phase, order=4, tol=1e-13, checkpoint_every=1)
    assert abs(L - L_ref) <= 1e-11, (L, L_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-9, (g, g_ref)


def test_gradient_beyond_the_largest_rule_reports_ekrylov(torch_cuda):
    # fixed Krylov dimension (tol <= 0) with a very long step: the stage
    # integral would need more than 48 nodes, the sweep gives up
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N = 4
    prop, pr = _prop(N, "f64")
    x = torch.from_numpy(W.random_state(1, 1 << N)).cuda()
    y = torch.from_numpy(W.random_state(11, 1 << N)).cuda()
    with pytest.raises(P.CfetError, match="EKRYLOV"):
        prop.fidelity_grad(x, y, 0.0, 20.0, 2, [0.5, -0.4], 2.0, order=4, tol=0.0)
    L, g, st = prop.fidelity_grad(x, y, 0.0, 0.1, 2, [0.5, -0.4], 2.0, order=4, tol=1e-12)   # still usable
    assert np.all(np.isfinite(g))


def test_checkpoint_spacing_does_not_change_the_gradient(torch_cuda):
    torch = torch_cuda
    N, nseg, nsteps, dt = 10, 5, 40, 0.02
    prop, _ = _prop(N, "fx")
    psi0 = torch.from_numpy(W.random_state(2, 1 << N)).cuda()
    phi = torch.from_numpy(W.random_state(12, 1 << N)).cuda()
    amps = W.uniform(6, nseg, -1.0, 1.0)
    out = [prop.fidelity_grad(psi0, phi, 0.0, dt, nsteps, amps, 2.0, order=4, tol=1e-12, checkpoint_every=ce)
           for ce in (1, 8, 40)]
    for L, g, st in out[1:]:
        assert abs(L - out[0][0]) <= 1e-12
        assert np.max(np.abs(g - out[0][1])) <= 1e-9
    assert out[2][2]["max_drift"] <= 1e-9   # recovery by the inverse step alone stays accurate


def test_full_size_gradient_matches_central_differences(torch_cuda):
    # N = 18 (dim 2^18), 64 segments over T = 16, CF4:2, dt = 0.01 (1600
    # steps), forward and backward in FP64 as the configuration names; every
    # one of the 64 components against a central difference (h = 1e-6) of the
    # loss, the differences taken with the fixed-point propagator (FP64-class,
    # within 1e-10 of the oracle) and the same fixed Krylov dimension, so that
    # the loss is a smooth function of the amplitudes
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N, nseg, T, dt, omega = 18, 64, 16.0, 0.01, 2.0
    nsteps = int(round(T / dt))
    m = 10
    prop, pr = _prop(N, "f64", m_max=m)
    psi0 = torch.from_numpy(W.random_state(3, 1 << N)).cuda()
    phi = torch.from_numpy(W.random_state(13, 1 << N)).cuda()
    amps = W.uniform(7, nseg, -1.0, 1.0)
    L, g, st = prop.fidelity_grad(psi0, phi, 0.0, dt, nsteps, amps, omega, order=4, tol=0.0, checkpoint_every=25)
    prop.close()
    # one forward propagator whose drive reads the amplitudes in place
    cur = amps.copy()
    f = OA.pwc_drive(cur, omega, 0.0, 0.0, dt, nsteps // nseg)
    fwd = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, np.ones(N))], [f], m_max=m, precision="fx")
    x = torch.empty_like(psi0)

    def fidelity(am):
        cur[:] = am
        x.copy_(psi0)
        fwd.propagate(x, 0.0, dt, nsteps, order=4, tol=0.0)
        return abs(torch.vdot(phi, x).item()) ** 2

    F0 = fidelity(amps)
    assert abs((1.0 - F0) - L) <= 1e-12
    # A random target in dim 2^18 has |<phi|psi>|^2 ~ 2^-18, so the gradient
    # components are ~1e-6: they are compared relative to the largest one.  The
    # fidelity itself is differenced (not 1 - F, whose rounding at 1 would
    # swamp differences of ~1e-12); its rounding noise is ~1e-19, i.e. ~1e-13
    # in a central difference with h = 1e-6, far below 1e-4 of the gradient.
    h = 1e-6
    fd = np.empty(nseg)
    for k in range(nseg):
        ap, am_ = amps.copy(), amps.copy()
        ap[k] += h
        am_[k] -= h
        fd[k] = -(fidelity(ap) - fidelity(am_)) / (2 * h)
    fwd.close()
    gmax = np.max(np.abs(g))
    worst = int(np.argmax(np.abs(fd - g)))
    assert gmax > 10 * F0 / nsteps                   # not trivially zero: ~F0 spread over the segments
    assert np.max(np.abs(fd - g)) <= 1e-4 * gmax, (worst, fd[worst], g[worst], gmax)
    assert st["max_drift"] <= 1e-9


def test_autograd_wrapper(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N, nseg, nsteps, dt = 4, 2, 6, 0.1
    prop, pr = _prop(N, "f64")
    psi0 = torch.from_numpy(W.random_state(1, 1 << N)).cuda()
    phi = torch.from_numpy(W.random_state(11, 1 << N)).cuda()
    amps = torch.tensor([0.3, -0.6], dtype=torch.float64, requires_grad=True)
    L = P.fidelity_loss(prop, amps, psi0, phi, 0.0, dt, nsteps, 2.0, tol=1e-13, checkpoint_every=3)
    L.backward()
    _, g, _ = prop.fidelity_grad(psi0, phi, 0.0, dt, nsteps, amps.detach().numpy(), 2.0, tol=1e-13,
                                 checkpoint_every=3)
    assert np.allclose(amps.grad.numpy(), g, rtol=0, atol=1e-15)


def test_fidelity_grad_validates(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, _ = _prop(4, "fx")
    x = torch.from_numpy(W.random_state(1, 16)).cuda()
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.fidelity_grad(x, x, 0.0, 0.1, 7, [0.1, 0.2], 2.0)          # 7 steps, 2 segments
    big, _ = _prop(4, "fx", m_max=20)
    with pytest.raises(P.CfetError, match="EINVAL"):
        big.fidelity_grad(x, x, 0.0, 0.1, 8, [0.1, 0.2], 2.0)           # m_max > 16
    two, _ = _prop(4, "fx", nfields=2)
    with pytest.raises(P.CfetError, match="EINVAL"):
        two.fidelity_grad(x, x, 0.0, 0.1, 8, [0.1, 0.2], 2.0)           # two drive operators
