"""CFET propagation in the interaction picture (oracle).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Sec. 9.3: for A(t) = D + B(t) with a constant diagonal D, the interaction
picture x^I(t) = e^{-tD} x(t) obeys d/dt x^I = B^I(t) x^I with
B^I(t) = e^{-tD} B(t) e^{tD}, whose elements are B_mn multiplied by
e^{(D_nn - D_mm) t}: the diagonal and the sparsity pattern are kept.  Sec. 9.4
uses it to remove large diagonal entries from the Krylov matrices, at the
price of faster time dependence.  For the Schroedinger equation A = -i H with
H(t) = H_d + H_b(t), H_d the diagonal of H0:

    x^I(t) = e^{i H_d t} x(t),   H^I(t) = e^{i H_d t} H_b(t) e^{-i H_d t},

and a CFET step of x^I uses the stage operators (Sec. 7, Eq. (OmGLeg))
H^I_j = sum_m g_{j,m} H^I(t + x_m dt).  Here H^I_j v is evaluated by that
definition: for every node, multiply by the phases, apply H_b(t_m), multiply
by the conjugate phases.  Time is absolute (the picture is fixed at t = 0).

Parity: pinned by ``tests/test_oracle_interaction.py`` (exactness without an
off-diagonal part, exactness of the resonant two-level system whose
interaction-picture Hamiltonian is constant, Sec. 9.3, convergence to the
Schroedinger-picture result with the scheme's order, Hermitian stages).
"""

from __future__ import annotations

import numpy as np

from . import krylov, operators as O, schemes


def diagonal(op):
    """Diagonal d of H0 and an apply of the off-diagonal part:
    offdiag(coeffs, v) = (coeffs[0] (H0 - diag(d)) + sum_k coeffs[1+k] V_k) v."""
    if isinstance(op, O.SpinChain):
        N = op.N
        ones = np.ones(1 << N, dtype=np.complex128)
        d = np.zeros(1 << N)
        for i in range(N - 1):
            d += np.real(op.J * op.Delta * O.apply_z(O.apply_z(ones, i + 1, N), i, N))
        for i in range(N):
            d += np.real(op.h[i] * O.apply_z(ones, i, N))

        def offdiag(coeffs, v):
            out = np.zeros_like(v)
            for i in range(N - 1):
                out += op.J * O.apply_x(O.apply_x(v, i + 1, N), i, N)
                out += op.J * O.apply_y(O.apply_y(v, i + 1, N), i, N)
            out *= coeffs[0]
            for k, a in enumerate(op.xfields):
                out += coeffs[1 + k] * O.xfield_apply(v, N, a)
            return out

        return d, offdiag
    if isinstance(op, O.Dense):
        d = np.real(np.diag(op.H0)).copy()
        H0b = op.H0 - np.diag(np.diag(op.H0))

        def offdiag(coeffs, v):
            out = coeffs[0] * (H0b @ v)
            for k, V in enumerate(op.Vs):
                out = out + coeffs[1 + k] * (V @ v)
            return out

        return d, offdiag
    raise TypeError("interaction picture: spin chains and dense operators only")


def stage_apply(d, offdiag, g_row, t_nodes, fvals):
    """v -> H^I_j v = sum_m g_{j,m} e^{i d t_m} H_b(t_m) e^{-i d t_m} v."""
    def apply(v):
        out = np.zeros_like(v)
        for gm, tm, fm in zip(g_row, t_nodes, fvals):
            ph = np.exp(1j * d * tm)
            out += gm * (ph * offdiag([1.0] + list(fm), np.conj(ph) * v))
        return out
    return apply


def propagate(op, psi0, t0, dt, nsteps, scheme, drives, tol, m_max, m_min=2, max_substeps=64,
              forced_log=None, return_log=False):
    """CFET time stepping of psi0 (Schroedinger picture in and out) carried
    out in the interaction picture; arguments as ``oracle.cfet.propagate``."""
    if not isinstance(scheme, schemes.Scheme):
        scheme = schemes.get(scheme)
    if len(drives) != op.nV:
        raise ValueError("one drive function per drive operator")
    g, x, _w, _f = schemes.g_coefficients(scheme)
    d, offdiag = diagonal(op)
    psi = np.exp(1j * d * t0) * np.array(psi0, dtype=np.complex128)
    log, n_app, idx = [], 0, 0
    for n in range(nsteps):
        t = t0 + n * dt
        tn = [t + xm * dt for xm in x]
        fv = [[fk(tm) for fk in drives] for tm in tn]
        for j in range(scheme.s - 1, -1, -1):       # exp(Omega_s) first
            forced = forced_log[idx] if forced_log is not None else None
            psi, lg, na = krylov.expv(stage_apply(d, offdiag, g[j], tn, fv), psi, dt, tol, m_max, m_min=m_min,
                                      max_substeps=max_substeps, forced=forced)
            log.append(lg)
            n_app += na
            idx += 1
    psi = np.exp(-1j * d * (t0 + nsteps * dt)) * psi
    if return_log:
        return psi, log, n_app
    return psi
