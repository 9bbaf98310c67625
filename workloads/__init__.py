"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no arithmetic of the propagation method itself: it only
produces problem data (chain parameters, initial states, banded operator
arrays, drive functions) from fixed seeds, so that the CUDA path and the CPU
oracle are fed identical inputs.

Random numbers come from a counter-based splitmix64 stream: output i of the
stream with seed S is mix(S + (i + 1) * 0x9E3779B97F4A7C15) with the
splitmix64 finaliser (Steele, Lea & Flood, OOPSLA 2014).  Uniform variates are
the top 53 bits times 2^-53; Gaussian pairs use the Box-Muller transform.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+n-1 of the splitmix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, start: int = 0) -> np.ndarray:
    u = (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def complex_gaussian(seed: int, n: int) -> np.ndarray:
    """n complex numbers with independent N(0,1) real and imaginary parts."""
    u = uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]                         # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2) + 1j * r * np.sin(2.0 * np.pi * u2)


def random_state(seed: int, dim: int) -> np.ndarray:
    v = complex_gaussian(seed, dim)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# Driven XXZ chain:  H(t) = sum_i [J (X_i X_{i+1} + Y_i Y_{i+1}) + J Delta Z_i Z_{i+1}]
#                          + sum_i h_i Z_i + A cos(omega t) sum_i X_i   (open chain)
# ---------------------------------------------------------------------------
@dataclass
class SpinChainProblem:
    N: int
    J: float
    Delta: float
    h: np.ndarray
    A: float
    omega: float
    xfield: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.xfield is None:
            self.xfield = np.ones(self.N)

    @property
    def dim(self):
        return 1 << self.N

    def drive(self, t: float) -> float:
        return self.A * math.cos(self.omega * t)


def spin_chain(N: int, J: float = 1.0, Delta: float = 0.5, A: float = 1.0, omega: float = 2.0,
               h_seed: int = 1) -> SpinChainProblem:
    """Driven XXZ chain with fields h_i ~ U[-1, 1] drawn from ``h_seed``."""
    h = uniform(h_seed, N, -1.0, 1.0)
    return SpinChainProblem(N, J, Delta, h, A, omega)


def neel_state(N: int) -> np.ndarray:
    """Neel product state: even sites up (bit 0), odd sites down (bit 1)."""
    x = sum(1 << i for i in range(1, N, 2))
    psi = np.zeros(1 << N, dtype=np.complex128)
    psi[x] = 1.0
    return psi


# ---------------------------------------------------------------------------
# Hydrogen-like atom on a radial grid, m = 0 (index r = l * Nr + j, l-major,
# radius r_j = (j + 1) dr, Dirichlet walls at r = 0 and r = (Nr + 1) dr):
#   H0 = -1/2 d^2/dr^2 (3-point) + l(l+1)/(2 r^2) - Z/r
#   V  = dipole z: (l, j) <-> (l+1, j) with weight r_j (l+1)/sqrt((2l+1)(2l+3))
#   E(t) = E0 sin^2(pi t / Tp) cos(omega t)
# All operators are real symmetric and stored in DIA form:
#   (D v)[r] = sum_d values[d, r] * v[r + offsets[d]].
# ---------------------------------------------------------------------------
@dataclass
class GridAtomProblem:
    Nr: int
    L: int
    dr: float
    Z: float
    E0: float
    omega: float
    Tp: float
    H0_offsets: np.ndarray
    H0_values: np.ndarray
    V_offsets: np.ndarray
    V_values: np.ndarray

    @property
    def dim(self):
        return self.Nr * self.L

    def drive(self, t: float) -> float:
        return self.E0 * math.sin(math.pi * t / self.Tp) ** 2 * math.cos(self.omega * t)


def grid_atom(Nr: int = 2000, L: int = 100, dr: float = 0.1, Z: float = 1.0, E0: float = 0.05,
              omega: float = 0.057, Tp: float = 1000.0) -> GridAtomProblem:
    dim = Nr * L
    j = np.arange(Nr)
    r = (j + 1) * dr
    l_of = np.repeat(np.arange(L), Nr)
    r_of = np.tile(r, L)
    j_of = np.tile(j, L)
    diag = 1.0 / dr ** 2 + l_of * (l_of + 1) / (2.0 * r_of ** 2) - Z / r_of
    off = -0.5 / dr ** 2
    up = np.where(j_of < Nr - 1, off, 0.0)          # row (l, j) -> column (l, j+1)
    dn = np.where(j_of > 0, off, 0.0)               # row (l, j) -> column (l, j-1)
    H0_offsets = np.array([0, 1, -1], dtype=np.int64)
    H0_values = np.stack([diag, up, dn]).astype(np.float64)
    lf = l_of.astype(np.float64)
    w_up = np.where(l_of < L - 1, r_of * (lf + 1.0) / np.sqrt((2 * lf + 1) * (2 * lf + 3)), 0.0)
    w_dn = np.where(l_of > 0, r_of * lf / np.sqrt(np.maximum((2 * lf - 1) * (2 * lf + 1), 1.0)), 0.0)
    V_offsets = np.array([Nr, -Nr], dtype=np.int64)
    V_values = np.stack([w_up, w_dn]).astype(np.float64)
    assert H0_values.shape == (3, dim) and V_values.shape == (2, dim)
    return GridAtomProblem(Nr, L, dr, Z, E0, omega, Tp, H0_offsets, H0_values, V_offsets, V_values)


def atom_ground_state(p: GridAtomProblem):
    """Normalised ground state of the l = 0 block of H0 (the discrete '1s'
    state), embedded in the full grid; returns (psi, energy)."""
    from scipy.linalg import eigh_tridiagonal
    d = p.H0_values[0, :p.Nr]
    e = p.H0_values[1, :p.Nr - 1]
    lam, vec = eigh_tridiagonal(d, e, select="i", select_range=(0, 0))
    psi = np.zeros(p.dim, dtype=np.complex128)
    g = vec[:, 0]
    g = g * np.sign(g[np.argmax(np.abs(g))])
    psi[:p.Nr] = g / np.linalg.norm(g)
    return psi, float(lam[0])


# ---------------------------------------------------------------------------
# Batch of driven XXZ chains of uneven size: N uniform in {n_lo..n_hi},
# per-instance field seed, A ~ U[0.5, 2], omega ~ U[1, 3]; drive A cos(omega t)
# on sum_i X_i; psi0 a random normalised complex Gaussian state per instance.
# ---------------------------------------------------------------------------
@dataclass
class ChainInstance:
    N: int
    J: float
    Delta: float
    h: np.ndarray
    A: float
    omega: float
    psi_seed: int

    @property
    def xfield(self) -> np.ndarray:
        return np.ones(self.N)

    def drive(self, t: float) -> float:
        return self.A * math.cos(self.omega * t)


def chain_batch(n: int = 256, n_lo: int = 10, n_hi: int = 16, seed: int = 7, J: float = 1.0,
                Delta: float = 0.5):
    u = uniform(seed, 3 * n)
    out = []
    for i in range(n):
        N = n_lo + min(int(u[i] * (n_hi - n_lo + 1)), n_hi - n_lo)
        A = 0.5 + 1.5 * u[n + i]
        omega = 1.0 + 2.0 * u[2 * n + i]
        h = uniform(1000 + i, N, -1.0, 1.0)
        out.append(ChainInstance(N, J, Delta, h, A, omega, 5000 + i))
    return out


# ---------------------------------------------------------------------------
# Sparse Hermitian operators in compressed sparse row form
# ---------------------------------------------------------------------------
def _csr_from_entries(dim, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(dim + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), vals


def random_hermitian_csr(seed: int, dim: int, per_row: int = 6, complex_values: bool = True,
                         band: int = 0, duplicates: int = 0):
    """(row_ptr, col_idx, values) of a seeded sparse Hermitian matrix: a real
    diagonal U[-1, 1], and per row `per_row` upper-triangle partners (within
    `band` columns when band > 0, anywhere otherwise) with values whose real
    and imaginary parts are U[-1, 1] (real only without complex_values),
    mirrored with the conjugate value; `duplicates` entries are split into two
    stored halves (the same matrix, with repeated (row, column) pairs)."""
    u = uniform(seed, dim * (3 * per_row + 1) + 2 * duplicates + 1)
    pos = 0
    rows, cols, vals = [np.arange(dim)], [np.arange(dim)], [u[pos:pos + dim] * 2.0 - 1.0]
    pos += dim
    r = np.repeat(np.arange(dim), per_row)
    span = np.where(band > 0, np.minimum(band, dim - 1 - r), dim - 1 - r)
    off = 1 + np.floor(u[pos:pos + dim * per_row] * np.maximum(span, 1)).astype(np.int64)
    pos += dim * per_row
    ok = span >= 1
    c = np.minimum(r + off, dim - 1)
    re = u[pos:pos + dim * per_row] * 2.0 - 1.0
    pos += dim * per_row
    im = (u[pos:pos + dim * per_row] * 2.0 - 1.0) if complex_values else np.zeros(dim * per_row)
    pos += dim * per_row
    r, c, v = r[ok & (c > r)], c[ok & (c > r)], (re + 1j * im)[ok & (c > r)]
    rows += [r, c]
    cols += [c, r]
    vals += [v, np.conj(v)]
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    vals = np.concatenate([np.asarray(a, dtype=np.complex128) for a in vals])
    if duplicates:
        pick = (u[pos:pos + duplicates] * len(rows)).astype(np.int64)
        half = vals[pick] * 0.5
        vals[pick] = half
        rows, cols = np.concatenate([rows, rows[pick]]), np.concatenate([cols, cols[pick]])
        vals = np.concatenate([vals, half])
    rp, ci, vv = _csr_from_entries(dim, rows, cols, vals)
    return rp, ci, (vv if complex_values else vv.real.copy())


def dia_to_csr(offsets, values):
    """(row_ptr, col_idx, values) of a real DIA operator (stored diagonals,
    entries outside the matrix dropped, zeros kept)."""
    values = np.asarray(values, dtype=np.float64)
    dim = values.shape[1]
    r = np.arange(dim)
    rows, cols, vals = [], [], []
    for d, off in enumerate(offsets):
        c = r + int(off)
        ok = (c >= 0) & (c < dim)
        rows.append(r[ok])
        cols.append(c[ok])
        vals.append(values[d, ok])
    return _csr_from_entries(dim, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


# ---------------------------------------------------------------------------
# Named workloads (sizes of the driven-chain and grid-atom experiments)
# ---------------------------------------------------------------------------
CHAIN_SMALL = dict(N=8, J=1.0, Delta=0.5, A=1.0, omega=2.0, h_seed=1, order=4, dt=0.01, T=10.0,
                   m_max=16, tol=1e-12, psi0="neel")
CHAIN_LARGE = dict(N=20, J=1.0, Delta=0.5, A=1.0, omega=2.0, h_seed=1, orders=(4, 6, 8),
                   dts=(0.05, 0.02, 0.01), T=20.0, m_max=16, tol=1e-10, psi_seed=2)
BATCH = dict(n=256, n_lo=10, n_hi=16, order=6, dt=0.02, T=10.0, m_max=16, tol=1e-10)
ATOM = dict(Nr=2000, L=100, dr=0.1, E0=0.05, omega=0.057, Tp=1000.0, order=8, dt=0.1, m_max=64,
            tol=1e-10)
