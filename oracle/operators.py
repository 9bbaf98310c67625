"""Hamiltonian application H v for the oracle (plain numpy, complex128).

TEST INFRASTRUCTURE (oracle): see ``oracle/__init__.py``.

Spin conventions (Sec. 6.2: Pauli matrices sigma_x, sigma_y, sigma_z in the
basis (spin up, spin down)):
  * basis index x in [0, 2^N); bit i of x is site i (little-endian);
  * bit value 0 = spin up (sigma_z = +1), bit value 1 = spin down;
  * hence sigma_z^(i) |x> = s_i(x) |x> with s_i = 1 - 2 b_i,
    sigma_x^(i) |x> = |x ^ 2^i>,
    sigma_y^(i) |x> = i s_i(x) |x ^ 2^i>   (sigma_y |up> = i |down>,
                                            sigma_y |down> = -i |up>).

The driven XXZ chain is the sum of Pauli strings
  H0 = sum_{i<N-1} [ J (X_i X_{i+1} + Y_i Y_{i+1}) + J Delta Z_i Z_{i+1} ]
       + sum_i h_i Z_i,          (open boundary)
  V  = sum_i a_i X_i            (the transverse drive operator),
the spin-chain form of Sec. 11.1, Eqs. (SpinChain1)-(SpinChain2), with the
XXZ anisotropy of the driven-chain workload.  The oracle applies every Pauli
string by the single-site definitions above; it does not use the fused
flip-if-antiparallel shortcut the CUDA kernel uses.
"""

from __future__ import annotations

import numpy as np


def _bits(N):
    return np.arange(1 << N, dtype=np.int64)


def apply_z(v, i, N):
    x = _bits(N)
    s = 1.0 - 2.0 * ((x >> i) & 1)
    return s * v


def apply_x(v, i, N):
    x = _bits(N)
    return v[x ^ (1 << i)]


def apply_y(v, i, N):
    # (Y v)[x] = sum_y <x|Y|y> v[y]; Y|y> = i s_i(y) |y ^ 2^i>, so the
    # component at x comes from y = x ^ 2^i with factor i s_i(x ^ 2^i).
    x = _bits(N)
    y = x ^ (1 << i)
    s_y = 1.0 - 2.0 * ((y >> i) & 1)
    return 1j * s_y * v[y]


def xxz_apply(v, N, J, Delta, h):
    """H0 v for the open XXZ chain with longitudinal fields h_i."""
    out = np.zeros_like(v)
    for i in range(N - 1):
        out += J * apply_x(apply_x(v, i + 1, N), i, N)
        out += J * apply_y(apply_y(v, i + 1, N), i, N)
        out += J * Delta * apply_z(apply_z(v, i + 1, N), i, N)
    for i in range(N):
        out += h[i] * apply_z(v, i, N)
    return out


def xfield_apply(v, N, a):
    """V v with V = sum_i a_i sigma_x^(i)."""
    out = np.zeros_like(v)
    for i in range(N):
        out += a[i] * apply_x(v, i, N)
    return out


def dia_apply(v, offsets, values):
    """Banded (DIA) operator: (D v)[r] = sum_d values[d, r] * v[r + offsets[d]],
    entries with r + offsets[d] outside [0, dim) contribute nothing."""
    dim = v.shape[0]
    out = np.zeros_like(v)
    r = np.arange(dim)
    for d, off in enumerate(offsets):
        c = r + int(off)
        ok = (c >= 0) & (c < dim)
        out[ok] += values[d, ok] * v[c[ok]]
    return out


def csr_apply(v, row_ptr, col_idx, values):
    """Compressed sparse rows: (A v)[r] = sum over the stored entries e of row
    r (e in [row_ptr[r], row_ptr[r+1])) of values[e] * v[col_idx[e]];
    duplicate entries of a row simply add."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    dim = len(row_ptr) - 1
    rows = np.repeat(np.arange(dim), np.diff(row_ptr))
    out = np.zeros(dim, dtype=np.complex128)
    np.add.at(out, rows, np.asarray(values) * v[np.asarray(col_idx, dtype=np.int64)])
    return out


# ---------------------------------------------------------------------------
# Operator families.  An operator family bundles H0 and the drive operators
# V_1..V_K; apply(coeffs, v) returns (c_0 H0 + sum_k c_k V_k) v, the stage
# operator of Sec. 8 (weighted sums of H(t) keep the sparsity pattern).
# ---------------------------------------------------------------------------
class SpinChain:
    """H(t) = H0 + sum_k f_k(t) V_k with H0 the XXZ chain and V_k transverse fields."""

    def __init__(self, N, J, Delta, h, xfields):
        self.N = int(N)
        self.dim = 1 << self.N
        self.J = float(J)
        self.Delta = float(Delta)
        self.h = np.asarray(h, dtype=np.float64)
        self.xfields = [np.asarray(a, dtype=np.float64) for a in xfields]

    @property
    def nV(self):
        return len(self.xfields)

    def apply(self, coeffs, v):
        out = coeffs[0] * xxz_apply(v, self.N, self.J, self.Delta, self.h)
        for k, a in enumerate(self.xfields):
            out = out + coeffs[1 + k] * xfield_apply(v, self.N, a)
        return out


def pauli_ops(label):
    """{site: letter} of a Pauli string given as a string over 'IXYZ'
    (character i acts on site i) or as a dict {site: letter}."""
    items = enumerate(label) if isinstance(label, str) else label.items()
    out = {}
    for site, letter in items:
        letter = letter.upper()
        if letter not in "IXYZ":
            raise ValueError(f"unknown Pauli letter {letter!r}")
        if letter != "I":
            out[int(site)] = letter
    return out


def pauli_string_apply(v, N, ops):
    """S v for the Pauli string S = product of the single-site operators in
    ops ({site: letter}); they act on different sites, so their order is free."""
    single = {"X": apply_x, "Y": apply_y, "Z": apply_z}
    out = v
    for site, letter in ops.items():
        out = single[letter](out, site, N)
    return out


class PauliSum:
    """H(t) = H0 + sum_k f_k(t) V_k with every operator a real combination of
    Pauli strings on N spins: terms = [(c, label), ...] (label as in pauli_ops).
    Real coefficients on tensor products of Hermitian Pauli matrices make every
    operator Hermitian."""

    def __init__(self, N, H0_terms, V_terms):
        self.N = int(N)
        self.dim = 1 << self.N
        self.H0 = [(float(c), pauli_ops(lb)) for c, lb in H0_terms]
        self.Vs = [[(float(c), pauli_ops(lb)) for c, lb in terms] for terms in V_terms]

    @property
    def nV(self):
        return len(self.Vs)

    def apply(self, coeffs, v):
        out = np.zeros_like(v)
        for k, terms in enumerate([self.H0] + self.Vs):
            for c, ops in terms:
                out = out + (coeffs[k] * c) * pauli_string_apply(v, self.N, ops)
        return out


class Banded:
    """H(t) = H0 + sum_k f_k(t) V_k with every operator in DIA form."""

    def __init__(self, H0, Vs):
        # H0, Vs[k]: (offsets [nd], values [nd, dim]) real
        self.H0 = (np.asarray(H0[0], dtype=np.int64), np.asarray(H0[1], dtype=np.float64))
        self.Vs = [(np.asarray(o, dtype=np.int64), np.asarray(val, dtype=np.float64)) for o, val in Vs]
        self.dim = self.H0[1].shape[1]

    @property
    def nV(self):
        return len(self.Vs)

    def apply(self, coeffs, v):
        out = coeffs[0] * dia_apply(v, *self.H0)
        for k, (o, val) in enumerate(self.Vs):
            out = out + coeffs[1 + k] * dia_apply(v, o, val)
        return out


class Sparse:
    """H(t) = H0 + sum_k f_k(t) V_k with every operator in CSR form, each given
    as (row_ptr [dim + 1], col_idx [nnz], values [nnz], real or complex)."""

    def __init__(self, H0, Vs):
        def conv(a):
            rp, ci, val = a
            return (np.asarray(rp, dtype=np.int64), np.asarray(ci, dtype=np.int64), np.asarray(val))
        self.H0 = conv(H0)
        self.Vs = [conv(a) for a in Vs]
        self.dim = len(self.H0[0]) - 1

    @property
    def nV(self):
        return len(self.Vs)

    def apply(self, coeffs, v):
        out = coeffs[0] * csr_apply(v, *self.H0)
        for k, a in enumerate(self.Vs):
            out = out + coeffs[1 + k] * csr_apply(v, *a)
        return out


class Dense:
    """H(t) = H0 + sum_k f_k(t) V_k with dense Hermitian matrices (tiny tests)."""

    def __init__(self, H0, Vs):
        self.H0 = np.asarray(H0, dtype=np.complex128)
        self.Vs = [np.asarray(V, dtype=np.complex128) for V in Vs]
        self.dim = self.H0.shape[0]

    @property
    def nV(self):
        return len(self.Vs)

    def matrix(self, coeffs):
        Hm = coeffs[0] * self.H0
        for k, V in enumerate(self.Vs):
            Hm = Hm + coeffs[1 + k] * V
        return Hm

    def apply(self, coeffs, v):
        return self.matrix(coeffs) @ v


# ---------------------------------------------------------------------------
# Dense construction of spin operators by Kronecker products of the 2x2 Pauli
# matrices of Sec. 6.2 (site 0 = least significant factor).  Independent of
# the bit formulas above; used to pin them on small chains.
# ---------------------------------------------------------------------------
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)


def site_op(op, i, N):
    """Dense 2^N x 2^N matrix of a single-site operator on site i."""
    out = np.ones((1, 1), dtype=np.complex128)
    for site in range(N - 1, -1, -1):          # most significant factor first
        out = np.kron(out, op if site == i else I2)
    return out


def xxz_dense(N, J, Delta, h):
    H = np.zeros((1 << N, 1 << N), dtype=np.complex128)
    for i in range(N - 1):
        H += J * (site_op(SX, i, N) @ site_op(SX, i + 1, N) + site_op(SY, i, N) @ site_op(SY, i + 1, N))
        H += J * Delta * site_op(SZ, i, N) @ site_op(SZ, i + 1, N)
    for i in range(N):
        H += h[i] * site_op(SZ, i, N)
    return H


def xfield_dense(N, a):
    H = np.zeros((1 << N, 1 << N), dtype=np.complex128)
    for i in range(N):
        H += a[i] * site_op(SX, i, N)
    return H


def pauli_dense(N, terms):
    """Dense sum_t c_t S_t from Kronecker products of the 2x2 Pauli matrices
    (independent of the bit formulas of pauli_string_apply)."""
    mats = {"X": SX, "Y": SY, "Z": SZ}
    H = np.zeros((1 << N, 1 << N), dtype=np.complex128)
    for c, label in terms:
        S = np.eye(1 << N, dtype=np.complex128)
        for site, letter in pauli_ops(label).items():
            S = S @ site_op(mats[letter], site, N)
        H += c * S
    return H
