"""CFET time stepping (oracle).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

One CFET step from t to t + dt (Sec. 4, Eq. (Ucf)):
    U(t + dt, t) ~= exp(Omega_1) exp(Omega_2) ... exp(Omega_s),
with, by Gauss-Legendre quadrature (Sec. 7, Eq. (OmGLeg)),
    Omega_j = dt * sum_m g_{j,m} A(t + x_m dt),   A(t) = -i H(t)   (Sec. 1).
For H(t) = H0 + sum_k f_k(t) V_k the stage operator is the weighted sum
    H_j = sum_m g_{j,m} H(t + x_m dt)
        = (sum_m g_{j,m}) H0 + sum_k (sum_m g_{j,m} f_k(t + x_m dt)) V_k,
which keeps the sparsity pattern of H (Sec. 8), and exp(Omega_j) psi =
exp(-i dt H_j) psi is evaluated by the Krylov method of ``oracle.krylov``.

Factor order: in exp(X) exp(Y) the right factor acts first (Sec. 2.2: e^X e^Y
is the exact propagator of a piecewise-constant A equal to Y on the first
interval and X on the second), so exp(Omega_s) is applied first and
exp(Omega_1) last.  Step n starts at t0 + n dt (Sec. 6.1 time stepping).
"""

from __future__ import annotations

import numpy as np

from . import krylov, schemes


def stage_coefficients(scheme, t, dt, drives):
    """c[j, 0] = sum_m g_{j,m};  c[j, k] = sum_m g_{j,m} f_k(t + x_m dt)."""
    g, x, _w, _f = schemes.g_coefficients(scheme)
    s, M = g.shape
    c = np.zeros((s, 1 + len(drives)), dtype=np.float64)
    for j in range(s):
        for m in range(M):
            c[j, 0] += g[j, m]
            for k, fk in enumerate(drives):
                c[j, 1 + k] += g[j, m] * fk(t + x[m] * dt)
    return c


def propagate(op, psi0, t0, dt, nsteps, scheme, drives, tol, m_max, m_min=2,
              max_substeps=64, forced_log=None, return_log=False, reorth=False):
    """Propagate psi0 from t0 over nsteps CFET steps of length dt.

    op: an operator family with .apply(coeffs, v) (oracle.operators).
    scheme: a Scheme, a scheme name, or an order (2, 4, 6, 8 -> default).
    drives: list of callables f_k(t), one per drive operator V_k.
    forced_log: optional decision log (list over stage exponentials, in
      execution order, of lists of (k, h)) to replay.
    reorth: full re-orthogonalisation of the Lanczos vectors (krylov.expv).
    Returns psi (and the decision log and the number of H applications when
    return_log is true).
    """
    if not isinstance(scheme, schemes.Scheme):
        scheme = schemes.get(scheme)
    if len(drives) != op.nV:
        raise ValueError("one drive function per drive operator")
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    log = []
    n_applies = 0
    idx = 0
    for n in range(nsteps):
        t = t0 + n * dt
        c = stage_coefficients(scheme, t, dt, drives)
        for j in range(scheme.s - 1, -1, -1):          # exp(Omega_s) first
            cj = c[j].copy()
            forced = forced_log[idx] if forced_log is not None else None
            psi, lg, na = krylov.expv(lambda v, cj=cj: op.apply(cj, v), psi, dt, tol, m_max,
                                      m_min=m_min, max_substeps=max_substeps, forced=forced, reorth=reorth)
            log.append(lg)
            n_applies += na
            idx += 1
    if return_log:
        return psi, log, n_applies
    return psi
