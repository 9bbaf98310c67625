"""Krylov (Lanczos) evaluation of exp(-i tau H) psi for Hermitian H.

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Sec. 8.1 of the paper: starting from psi, each multiplication by H gives a new
vector that is orthogonalised against the previous ones (Lanczos); the
exponential is then evaluated in the k-dimensional Krylov space, i.e. as the
exponential of the small k x k matrix (here the real symmetric tridiagonal
T_k of the Lanczos coefficients).  When the Krylov approximation is not yet
accurate enough at the largest allowed k, the paper prescribes time stepping,
exp(-i H tau) = exp(-i H tau_1) exp(-i H tau_2) ..., Eq. (KryErr) and the text
after it.

The paper does not fix a stopping rule; this oracle takes the following
reading (the CUDA path implements the same rule):

* Lanczos ordering (three-term recurrence, no re-orthogonalisation):
    u = H v_k - beta_{k-1} v_{k-1};  alpha_k = Re<v_k, u>;
    w = u - alpha_k v_k;             beta_k  = ||w||;  v_{k+1} = w / beta_k.
  Option (the paper is silent on it): full re-orthogonalisation by one
  classical Gram-Schmidt sweep, w <- w - sum_{i<=k} v_i <v_i, w> with all
  coefficients taken from the same w, before beta_k = ||w||; T_k keeps the
  recurrence's alpha and beta.
* a-posteriori estimate for the Krylov error of a (sub)step of length tau_s:
    y = exp(-i tau_s T_k) e_1   (eigendecomposition of T_k),
    err_k = beta_0 * beta_k * |y_k|   (beta_0 = ||psi||, y_k the last entry).
* acceptance: the smallest k >= m_min with err_k <= tol * tau_s / tau
  (tau the full stage time); a Lanczos breakdown beta_k <= bd_tol * (|alpha_k|
  + beta_{k-1} + 1) ends the iteration with err = 0 (invariant subspace).
* the estimate is evaluated only when |tau_s| width(T_k) <= 2 k, width the
  Gershgorin width of T_k (an upper bound of its eigenvalue spread); beyond
  that the bound Eq. (KryErr), which needs 2 rho <= K with 4 rho = tau times
  the spread, gives no assurance and the step counts as not converged.
* if no k <= m_max is accepted, the same basis is reused with tau_s halved
  (tau_s = remaining / 2^h, h = 1, 2, ...) until err <= tol * tau_s / tau;
  psi is advanced by tau_s, the basis is rebuilt from the new psi for the
  remaining time.  More than ``max_substeps`` substeps raise KrylovError.
* tol <= 0 selects the paper's fixed-K mode: exactly k = m_max Lanczos steps,
  one step of the full length, no error test (Sec. 8.2, 9.2, 11.1 use fixed K).

Every (sub)step appends (k, h) to a decision log; passing that log back as
``forced`` replays the same decisions (used for GPU/oracle parity runs, where
rounding could otherwise flip a decision that sits exactly at the threshold).
"""

from __future__ import annotations

import numpy as np


class KrylovError(RuntimeError):
    pass


BREAKDOWN_TOL = 1e-13
MAX_HALVINGS = 40


def tridiag_matrix(alpha, beta):
    k = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    for i in range(k - 1):
        T[i, i + 1] = beta[i]
        T[i + 1, i] = beta[i]
    return T


def tridiag_expm_e1(alpha, beta, tau):
    """y = exp(-i tau T) e_1 for the real symmetric tridiagonal T (diagonal
    alpha[0..k-1], off-diagonal beta[0..k-2]), by the eigendecomposition
    T = Q diag(lam) Q^T:  y = Q diag(exp(-i tau lam)) Q^T e_1."""
    T = tridiag_matrix(alpha, beta)
    lam, Q = np.linalg.eigh(T)
    return Q @ (np.exp(-1j * tau * lam) * Q[0, :])


def gershgorin_width(alpha, beta):
    """max_r (alpha_r + |beta_{r-1}| + |beta_r|) - min_r (alpha_r - |beta_{r-1}| - |beta_r|)."""
    k = len(alpha)
    lo, hi = np.inf, -np.inf
    for r in range(k):
        rad = (abs(beta[r - 1]) if r > 0 else 0.0) + (abs(beta[r]) if r < k - 1 else 0.0)
        lo = min(lo, alpha[r] - rad)
        hi = max(hi, alpha[r] + rad)
    return hi - lo


def gram_schmidt(V, w):
    """One classical Gram-Schmidt sweep: w - sum_i V_i <V_i, w>."""
    coeffs = [np.vdot(v, w) for v in V]
    for c, v in zip(coeffs, V):
        w = w - c * v
    return w


def lanczos(apply, psi, k, reorth=False):
    """k steps of the recurrence above from psi / ||psi|| without any test:
    the basis V (k + 1 vectors), alpha[k], beta[k]."""
    V = [np.asarray(psi, dtype=np.complex128) / np.linalg.norm(psi)]
    alpha, beta = [], []
    for j in range(1, k + 1):
        u = apply(V[j - 1])
        if j > 1:
            u = u - beta[j - 2] * V[j - 2]
        a = float(np.real(np.vdot(V[j - 1], u)))
        w = u - a * V[j - 1]
        if reorth:
            w = gram_schmidt(V, w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        V.append(w / b)
    return V, alpha, beta


def expv(apply, psi, tau, tol, m_max, m_min=2, max_substeps=64, forced=None, reorth=False):
    """exp(-i tau H) psi by Lanczos with substepping.

    apply(v) -> H v.  Returns (psi_new, log, n_applies) with log a list of
    (k, h) decisions.  ``forced``: optional list of (k, h) to replay.
    ``reorth``: full re-orthogonalisation (classical Gram-Schmidt) of every w.
    """
    psi = np.array(psi, dtype=np.complex128, copy=True)
    log = []
    n_applies = 0
    remaining = float(tau)
    fixed_k = tol <= 0.0
    forced_iter = iter(forced) if forced is not None else None
    while True:
        if forced_iter is not None:
            try:
                k_forced, h_forced = next(forced_iter)
            except StopIteration:
                raise KrylovError("forced decision log exhausted") from None
        else:
            k_forced = h_forced = None
        if len(log) >= max_substeps:
            raise KrylovError("substep limit reached")
        beta0 = np.linalg.norm(psi)
        if beta0 == 0.0:
            log.append((0, 0))
            return psi, log, n_applies
        V = [psi / beta0]
        alpha, beta = [], []
        accepted = None
        k_limit = k_forced if k_forced is not None else m_max
        for k in range(1, k_limit + 1):
            u = apply(V[k - 1])
            n_applies += 1
            if k > 1:
                u = u - beta[k - 2] * V[k - 2]
            a = float(np.real(np.vdot(V[k - 1], u)))
            w = u - a * V[k - 1]
            if reorth:
                w = gram_schmidt(V, w)
            b = float(np.linalg.norm(w))
            alpha.append(a)
            beta.append(b)
            prev_b = beta[k - 2] if k > 1 else 0.0
            breakdown = b <= BREAKDOWN_TOL * (abs(a) + prev_b + 1.0)
            if k_forced is not None:
                if k == k_forced:
                    accepted = (k, h_forced)
                    break
                V.append(w / b)
                continue
            if fixed_k:
                if k == m_max or breakdown:
                    accepted = (k, 0)
                    break
                V.append(w / b)
                continue
            if breakdown:
                accepted = (k, 0)
                break
            if k >= m_min and abs(remaining) * gershgorin_width(alpha, beta[:k - 1]) <= 2 * k:
                y = tridiag_expm_e1(alpha, beta[:k - 1], remaining)
                err = beta0 * b * abs(y[k - 1])
                if err <= tol * remaining / tau:
                    accepted = (k, 0)
                    break
            if k == m_max:
                break
            V.append(w / b)
        if accepted is None:
            # not converged at m_max: halve the substep on the same basis
            k = m_max
            width = gershgorin_width(alpha, beta[:k - 1])
            for h in range(1, MAX_HALVINGS + 1):
                ts = remaining / (2.0 ** h)
                if not abs(ts) * width <= 2 * k:
                    continue
                y = tridiag_expm_e1(alpha, beta[:k - 1], ts)
                err = beta0 * beta[k - 1] * abs(y[k - 1])
                if err <= tol * ts / tau:
                    accepted = (k, h)
                    break
            if accepted is None:
                raise KrylovError("no substep length meets the tolerance")
        k, h = accepted
        ts = remaining / (2.0 ** h)
        y = tridiag_expm_e1(alpha[:k], beta[:k - 1], ts)
        psi = beta0 * sum(y[i] * V[i] for i in range(k))
        log.append((k, h))
        if h == 0:
            return psi, log, n_applies
        remaining = remaining - ts
