"""Pins of the oracle's fidelity loss and its exact gradient (oracle/adjoint.py).

The gradient is assembled from Frechet derivatives of the stage exponentials
and adjoint states; it is checked against central finite differences of the
loss (matrix exponentials only, no derivative code), against the vanishing
gradient at an exact optimum, and the loss itself against the Krylov
propagation of oracle.cfet.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA, cfet as OC, operators as O, schemes as OS


def _problem(N, seed=1, nonuniform=False):
    pr = W.spin_chain(N)
    H0 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    a = W.uniform(40 + seed, N, 0.3, 1.2) if nonuniform else np.ones(N)
    V = O.xfield_dense(N, a)
    psi0 = W.random_state(seed, 1 << N)
    phi = W.random_state(seed + 10, 1 << N)
    return pr, a, H0, V, psi0, phi


@pytest.mark.parametrize("scheme,nonuniform", [("CF4:2", False), ("CF6:5Opt", True), ("CF2:1", False)])
def test_gradient_matches_central_differences(scheme, nonuniform):
    N, nseg, nsteps, dt, omega, phase = 3, 4, 8, 0.15, 2.0, 0.3
    _, _, H0, V, psi0, phi = _problem(N, nonuniform=nonuniform)
    amps = W.uniform(5, nseg, -1.0, 1.0)
    L, g = OA.grad_dense(H0, V, psi0, phi, amps, omega, phase, 0.0, dt, nsteps, scheme)
    h = 1e-6
    fd = np.zeros(nseg)
    for k in range(nseg):
        ap, am = amps.copy(), amps.copy()
        ap[k] += h
        am[k] -= h
        fd[k] = (OA.loss_dense(H0, V, psi0, phi, ap, omega, phase, 0.0, dt, nsteps, scheme)[0]
                 - OA.loss_dense(H0, V, psi0, phi, am, omega, phase, 0.0, dt, nsteps, scheme)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd))), (g, fd)
    assert abs(L - OA.loss_dense(H0, V, psi0, phi, amps, omega, phase, 0.0, dt, nsteps, scheme)[0]) < 1e-14


def test_gradient_vanishes_at_exact_optimum():
    N, nseg, nsteps, dt = 3, 2, 6, 0.1
    _, _, H0, V, psi0, _ = _problem(N)
    amps = np.array([0.7, -0.4])
    _, psiT = OA.loss_dense(H0, V, psi0, psi0, amps, 1.5, 0.0, 0.0, dt, nsteps, "CF4:2")
    L, g = OA.grad_dense(H0, V, psi0, psiT, amps, 1.5, 0.0, 0.0, dt, nsteps, "CF4:2")
    assert abs(L) < 1e-13 and np.max(np.abs(g)) < 1e-12


def test_loss_matches_krylov_propagation():
    N, nseg, nsteps, dt, omega = 4, 4, 8, 0.05, 2.0
    pr, a, H0, V, psi0, phi = _problem(N)
    amps = W.uniform(9, nseg, -1.0, 1.0)
    L, psiT = OA.loss_dense(H0, V, psi0, phi, amps, omega, 0.0, 0.0, dt, nsteps, "CF4:2")
    f = OA.pwc_drive(amps, omega, 0.0, 0.0, dt, nsteps // nseg)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [a])
    psiK = OC.propagate(op, psi0, 0.0, dt, nsteps, "CF4:2", [f], 1e-14, 24)
    assert np.linalg.norm(psiK - psiT) < 1e-12
    assert abs(L - (1 - abs(np.vdot(phi, psiK)) ** 2)) < 1e-12


def test_pwc_drive_maps_gauss_nodes_to_segments():
    amps = np.arange(1.0, 5.0)
    dt, sps = 0.01, 25
    f = OA.pwc_drive(amps, 0.0, 0.0, 0.0, dt, sps)   # omega = 0: f = amplitude
    x = OS.gauss_legendre(4)[0]
    for n in range(100):
        for xm in x:
            assert f(n * dt + xm * dt) == amps[n // sps]
