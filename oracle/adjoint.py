"""Fidelity loss of a CFET propagation and its exact gradient with respect to
piecewise-constant drive amplitudes (oracle).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

The paper has no gradients; this is the plain definition the device adjoint
is checked against.  Problem: H(t) = H0 + f(t) V with the drive
    f(t) = A_k cos(omega t + phase)  for t in segment k,
segments of nsteps / nseg CFET steps each (segment boundaries fall on step
boundaries, so the Gauss-Legendre nodes of a step, which are interior, all
belong to one segment).  psi(T) is the CFET propagation (Sec. 4, Eq. (Ucf);
Sec. 7, Eq. (OmGLeg)) with every stage exponential exp(-i dt H_{n,j}) taken
exactly (dense matrix exponential; small systems only), and
    L = 1 - |<phi|psi(T)>|^2.
With H_{n,j} = c_{j,0} H0 + c_{n,j} V and c_{n,j} = A_{seg(n)} gamma_{n,j},
gamma_{n,j} = sum_m g_{j,m} cos(omega (t_n + x_m dt) + phase), the chain rule
gives
    dL/dA_k = -2 Re( conj(o) sum_{n in k, j} gamma_{n,j} <lambda_{n,j}| dE_{n,j} |psi_{n,j}> ),
o = <phi|psi(T)>, psi_{n,j} the state before stage (n, j), lambda_{n,j} the
adjoint state (the product of all later stage exponentials, adjoint, applied
to phi), and dE the Frechet derivative of E = exp(-i dt H) in the direction
-i dt V (scipy.linalg.expm_frechet).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm, expm_frechet

from . import schemes


def pwc_drive(amps, omega, phase, t0, dt, steps_per_seg):
    """f(t) = amps[k] cos(omega t + phase), k = segment of the step containing t."""
    def f(t):
        n = int(math.floor((t - t0) / dt))
        k = min(max(n // steps_per_seg, 0), len(amps) - 1)
        return amps[k] * math.cos(omega * t + phase)
    return f


def _stage_tables(scheme, t0, dt, nsteps, omega, phase):
    """c0[j] and gamma[n, j] (stage order j = 0..s-1 as in the table)."""
    g, x, _w, _f = schemes.g_coefficients(scheme)
    s, M = g.shape
    c0 = g.sum(axis=1)
    gam = np.zeros((nsteps, s))
    for n in range(nsteps):
        t = t0 + n * dt
        for j in range(s):
            gam[n, j] = sum(g[j, m] * math.cos(omega * (t + x[m] * dt) + phase) for m in range(M))
    return c0, gam


def loss_dense(H0, V, psi0, phi, amps, omega, phase, t0, dt, nsteps, scheme):
    """L and psi(T) with exact stage exponentials (dense H0, V)."""
    if not isinstance(scheme, schemes.Scheme):
        scheme = schemes.get(scheme)
    nseg = len(amps)
    sps = nsteps // nseg
    c0, gam = _stage_tables(scheme, t0, dt, nsteps, omega, phase)
    psi = np.array(psi0, dtype=np.complex128)
    for n in range(nsteps):
        A = amps[n // sps]
        for j in range(scheme.s - 1, -1, -1):      # exp(Omega_s) first
            psi = expm(-1j * dt * (c0[j] * H0 + A * gam[n, j] * V)) @ psi
    o = np.vdot(phi, psi)
    return 1.0 - abs(o) ** 2, psi


def grad_dense(H0, V, psi0, phi, amps, omega, phase, t0, dt, nsteps, scheme):
    """(L, dL/dA) with exact stage exponentials and their Frechet derivatives."""
    if not isinstance(scheme, schemes.Scheme):
        scheme = schemes.get(scheme)
    nseg = len(amps)
    if nsteps % nseg:
        raise ValueError("nsteps must be a multiple of the number of segments")
    sps = nsteps // nseg
    c0, gam = _stage_tables(scheme, t0, dt, nsteps, omega, phase)
    # forward: the state before every stage, in application order
    psi = np.array(psi0, dtype=np.complex128)
    before = []
    for n in range(nsteps):
        A = amps[n // sps]
        for j in range(scheme.s - 1, -1, -1):
            before.append((n, j, psi))
            psi = expm(-1j * dt * (c0[j] * H0 + A * gam[n, j] * V)) @ psi
    o = np.vdot(phi, psi)
    # backward: lambda after each stage, derivative of that stage
    lam = np.array(phi, dtype=np.complex128)
    do = np.zeros(nseg, dtype=np.complex128)
    for n, j, psi_b in reversed(before):
        A = amps[n // sps]
        X = -1j * dt * (c0[j] * H0 + A * gam[n, j] * V)
        E, dE = expm_frechet(X, -1j * dt * V)
        do[n // sps] += gam[n, j] * np.vdot(lam, dE @ psi_b)
        lam = E.conj().T @ lam
    grad = -2.0 * np.real(np.conj(o) * do)
    return 1.0 - abs(o) ** 2, grad
