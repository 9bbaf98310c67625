"""Chebyshev evaluation of exp(-i tau H) psi (oracle).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Sec. 8.1 names the Chebyshev technique (Tal-Ezer and Kosloff) as the second
way to compute the stage exponentials: expand exp(-i tau H) in Chebyshev
polynomials of H mapped onto [-1, 1], which needs a-priori bounds on the
eigenvalues of H (the paper's stated disadvantage) and only products H v.
The paper prints no formulas for it, so this module writes the standard
method out step by step:

* spectral bounds of a stage operator H_j = c_0 H0 + sum_k c_k V_k: each
  operator's Gershgorin interval [min_r (A_rr - R_r), max_r (A_rr + R_r)],
  R_r = sum_{c != r} |A_rc|, combined by Weyl's inequality (the interval of
  s A is s [lo, hi] for s >= 0 and s [hi, lo] for s < 0; intervals of a sum
  add);
* a = (hi - lo) / 2, b = (hi + lo) / 2 and Htilde = (H - b) / a, whose
  spectrum lies in [-1, 1];
* the Jacobi-Anger expansion exp(-i z x) = sum_k (2 - delta_k0) (-i)^k
  J_k(z) T_k(x), x in [-1, 1], gives
      exp(-i tau H) psi = exp(-i tau b) sum_k (2 - delta_k0) (-i)^k J_k(tau a) T_k(Htilde) psi;
* the series stops after the smallest K >= 0 whose tail bound
  2 sum_{k > K} |J_k(tau a)| is <= tol (||T_k(Htilde)|| <= 1); tol <= 0
  selects the tail bound 2^-52;
* T_k(Htilde) psi by the three-term recurrence v_0 = psi, v_1 = Htilde psi,
  v_{k+1} = 2 Htilde v_k - v_{k-1}.

The Bessel values come from ``scipy.special.jv`` (a library routine serving
as one step).  Parity: pinned by ``tests/test_oracle_chebyshev.py`` (dense
expm, the harmonic-oscillator example of Sec. 8.2 with its closed form,
Jacobi-Anger for scalars, bounds containing the spectrum, unitarity).
"""

from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import operators as O

TAIL_FLOOR = 2.0 ** -52


# ---------------------------------------------------------------------------
# Gershgorin intervals of single operators
# ---------------------------------------------------------------------------
def gershgorin_dense(A):
    """[min_r (A_rr - R_r), max_r (A_rr + R_r)] of a Hermitian matrix."""
    A = np.asarray(A)
    d = np.real(np.diag(A))
    R = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    return float(np.min(d - R)), float(np.max(d + R))


def gershgorin_xxz(N, J, Delta, h):
    """Gershgorin interval of the XXZ chain H0 (operators.xxz_apply), rows
    evaluated by the Pauli-string definitions: every bond term
    J (X_i X_{i+1} + Y_i Y_{i+1}) has at most one non-zero per row (column
    x ^ (3 << i)), so its entry in row x is (T_i 1)[x]; the diagonal comes from
    the Z Z and Z terms applied to the all-ones vector."""
    ones = np.ones(1 << N, dtype=np.complex128)
    diag = np.zeros(1 << N)
    R = np.zeros(1 << N)
    for i in range(N - 1):
        t = J * O.apply_x(O.apply_x(ones, i + 1, N), i, N) + J * O.apply_y(O.apply_y(ones, i + 1, N), i, N)
        R += np.abs(t)
        diag += np.real(J * Delta * O.apply_z(O.apply_z(ones, i + 1, N), i, N))
    for i in range(N):
        diag += np.real(h[i] * O.apply_z(ones, i, N))
    return float(np.min(diag - R)), float(np.max(diag + R))


def gershgorin_xfield(N, a):
    """V = sum_i a_i X_i: zero diagonal, one entry a_i per row and site."""
    ones = np.ones(1 << N, dtype=np.complex128)
    R = np.zeros(1 << N)
    for i in range(N):
        R += np.abs(a[i] * O.apply_x(ones, i, N))
    return float(np.min(-R)), float(np.max(R))


def gershgorin_dia(offsets, values):
    """DIA operator: diagonal = sum of the offset-0 diagonals, R_r = sum of
    |values| of the other stored diagonals whose column is inside [0, dim)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    dim = values.shape[1]
    r = np.arange(dim)
    diag = np.zeros(dim)
    R = np.zeros(dim)
    for d, off in enumerate(offsets):
        if off == 0:
            diag += values[d]
        else:
            c = r + int(off)
            ok = (c >= 0) & (c < dim)
            R[ok] += np.abs(values[d, ok])
    return float(np.min(diag - R)), float(np.max(diag + R))


def gershgorin_csr(row_ptr, col_idx, values):
    """CSR operator: diagonal = real part of the sum of the entries with
    column = row, R_r = sum of |value| of the row's other entries."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    values = np.asarray(values)
    dim = len(row_ptr) - 1
    diag = np.zeros(dim)
    R = np.zeros(dim)
    for r in range(dim):
        for e in range(row_ptr[r], row_ptr[r + 1]):
            if col_idx[e] == r:
                diag[r] += float(np.real(values[e]))
            else:
                R[r] += abs(values[e])
    return float(np.min(diag - R)), float(np.max(diag + R))


def operator_intervals(op):
    """Gershgorin interval of H0 and of every V_k of an operator family."""
    if isinstance(op, O.SpinChain):
        out = [gershgorin_xxz(op.N, op.J, op.Delta, op.h)]
        out += [gershgorin_xfield(op.N, a) for a in op.xfields]
        return out
    if isinstance(op, O.Banded):
        return [gershgorin_dia(*op.H0)] + [gershgorin_dia(o, v) for o, v in op.Vs]
    if isinstance(op, O.Dense):
        return [gershgorin_dense(op.H0)] + [gershgorin_dense(V) for V in op.Vs]
    if isinstance(op, O.Sparse):
        return [gershgorin_csr(*op.H0)] + [gershgorin_csr(*a) for a in op.Vs]
    raise TypeError("unknown operator family")


def stage_interval(intervals, coeffs):
    """Weyl: interval of sum_o coeffs[o] A_o from the intervals of the A_o."""
    lo = hi = 0.0
    for (l, h), s in zip(intervals, coeffs):
        if s >= 0.0:
            lo += s * l
            hi += s * h
        else:
            lo += s * h
            hi += s * l
    return lo, hi


# ---------------------------------------------------------------------------
# Expansion coefficients and truncation
# ---------------------------------------------------------------------------
def kmax_for(z):
    """Last Bessel order kept in the tail sums; J_k(z) beyond it is below 1e-30."""
    return int(math.ceil(z + 16.0 * z ** (1.0 / 3.0) + 40.0))


def coefficients(z, tol):
    """r_k = (2 - delta_k0) J_k(z) for k = 0..K with the truncation rule above
    (z may be negative: J_k(-z) = (-1)^k J_k(z)); returns (r, K, tail bound
    2 sum_{k>K} |J_k(z)|)."""
    eps = tol if tol > 0.0 else TAIL_FLOOR
    if z == 0.0:
        return np.array([1.0]), 0, 0.0
    km = kmax_for(abs(z))
    J = special.jv(np.arange(km + 1), z)
    absJ = np.abs(J)
    # tail[K] = 2 sum_{k=K+1}^{km} |J_k|
    tail = np.zeros(km + 1)
    acc = 0.0
    for k in range(km, -1, -1):
        tail[k] = 2.0 * acc
        acc += absJ[k]
    K = int(np.argmax(tail <= eps)) if np.any(tail <= eps) else km
    r = J[: K + 1].copy()
    r[1:] *= 2.0
    return r, K, float(tail[K])


def expv(apply, psi, tau, lo, hi, tol):
    """exp(-i tau H) psi for H with spectrum in [lo, hi]; apply(v) = H v.
    Returns (result, number of H applications, K, tail bound)."""
    a = 0.5 * (hi - lo)
    b = 0.5 * (hi + lo)
    phase = np.exp(-1j * tau * b)
    if a <= 0.0:
        return phase * psi, 0, 0, 0.0
    r, K, tail = coefficients(tau * a, tol)
    rot = -1j
    Ht = lambda v: (apply(v) - b * v) / a
    v_prev = np.array(psi, dtype=np.complex128, copy=True)
    out = r[0] * v_prev
    n_app = 0
    if K >= 1:
        v = Ht(v_prev)
        n_app += 1
        out = out + r[1] * rot * v
        for k in range(2, K + 1):
            v_next = 2.0 * Ht(v) - v_prev
            n_app += 1
            out = out + r[k] * rot ** k * v_next
            v_prev, v = v, v_next
    return phase * out, n_app, K, tail


def propagate(op, psi0, t0, dt, nsteps, scheme, drives, tol, return_stats=False):
    """CFET time stepping (as ``oracle.cfet.propagate``) with every stage
    exponential exp(-i dt H_j) evaluated by the Chebyshev expansion."""
    from . import cfet as C
    from . import schemes

    if not isinstance(scheme, schemes.Scheme):
        scheme = schemes.get(scheme)
    if len(drives) != op.nV:
        raise ValueError("one drive function per drive operator")
    iv = operator_intervals(op)
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    n_app, Ks, tails = 0, [], []
    for n in range(nsteps):
        c = C.stage_coefficients(scheme, t0 + n * dt, dt, drives)
        for j in range(scheme.s - 1, -1, -1):          # exp(Omega_s) first
            cj = c[j].copy()
            lo, hi = stage_interval(iv, cj)
            psi, na, K, tail = expv(lambda v, cj=cj: op.apply(cj, v), psi, dt, lo, hi, tol)
            n_app += na
            Ks.append(K)
            tails.append(tail)
    if return_stats:
        return psi, {"n_applies": n_app, "K": Ks, "tail": tails}
    return psi
