"""Pins of the oracle's compressed-sparse-row operators (oracle/operators.py:
csr_apply, Sparse; oracle/chebyshev.py: gershgorin_csr).

The CSR operator kind is the boundary's general sparse Hermitian operator
(Sec. 8: the stage operator sum_k c_k H_k is applied term by term, so it keeps
the operators' sparsity).  Pins: scipy.sparse's CSR matrix-vector product, a
dense matrix filled entry by entry from the stored triples (brute force),
the DIA grid atom written as CSR against the oracle's DIA apply, dense expm
through the Krylov oracle, and dense Gershgorin intervals.  Planted mistakes
(conjugated values, a transposed operand, dropped duplicate entries) must each
fail a pin.
"""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.linalg import expm

import workloads as W
from oracle import cfet as OC, chebyshev as OCH, krylov as OK, operators as O


def _dense(rp, ci, v, dim):
    A = np.zeros((dim, dim), dtype=np.complex128)
    for r in range(dim):
        for e in range(rp[r], rp[r + 1]):
            A[r, ci[e]] += v[e]
    return A


def _pins_hold():
    # every pin of csr_apply in one predicate (used for the planted mistakes)
    ok = True
    for seed, dim, cplx, dup in ((1, 40, True, 6), (2, 33, False, 3), (3, 64, True, 0)):
        rp, ci, v = W.random_hermitian_csr(seed, dim, 5, cplx, duplicates=dup)
        x = W.random_state(seed + 10, dim)
        got = O.csr_apply(x, rp, ci, v)
        ok &= np.allclose(got, sp.csr_matrix((v, ci, rp), shape=(dim, dim)) @ x, rtol=0, atol=1e-13)
        ok &= np.allclose(got, _dense(rp, ci, v, dim) @ x, rtol=0, atol=1e-13)
    return bool(ok)


def test_csr_apply_matches_scipy_and_brute_force():
    assert _pins_hold()


def test_generated_operators_are_hermitian_with_duplicates():
    rp, ci, v = W.random_hermitian_csr(5, 80, 4, True, duplicates=9)
    A = _dense(rp, ci, v, 80)
    assert np.max(np.abs(A - A.conj().T)) == 0.0
    pairs = [(r, ci[e]) for r in range(80) for e in range(rp[r], rp[r + 1])]
    assert len(pairs) > len(set(pairs))                 # repeated (row, column) pairs exist
    assert np.any(np.abs(np.imag(v)) > 0.1)


def test_csr_empty_rows_and_empty_operator():
    rp = np.array([0, 0, 2, 2, 3])
    ci = np.array([1, 3, 2])
    v = np.array([2.0, 0.5j, -1.0])
    x = W.random_state(4, 4)
    out = O.csr_apply(x, rp, ci, v)
    assert out[0] == 0 and out[2] == 0
    assert np.allclose(out[1], 2.0 * x[1] + 0.5j * x[3]) and np.allclose(out[3], -x[2])
    assert np.all(O.csr_apply(x, np.zeros(5, dtype=np.int64), np.zeros(0, dtype=np.int64), np.zeros(0)) == 0)


def test_grid_atom_as_csr_matches_dia():
    p = W.grid_atom(Nr=150, L=6)
    dia = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    csr = O.Sparse(W.dia_to_csr(p.H0_offsets, p.H0_values), [W.dia_to_csr(p.V_offsets, p.V_values)])
    x = W.random_state(6, p.dim)
    c = np.array([0.7, -0.03])
    assert np.max(np.abs(csr.apply(c, x) - dia.apply(c, x))) <= 1e-12 * np.max(np.abs(dia.apply(c, x)))


def test_sparse_family_expv_matches_expm():
    dim = 120
    H0 = W.random_hermitian_csr(7, dim, 4, True)
    V1 = W.random_hermitian_csr(8, dim, 3, False, band=5)
    op = O.Sparse(H0, [V1])
    c = np.array([0.9, 0.4])
    Hm = c[0] * _dense(*H0, dim) + c[1] * _dense(*V1, dim)
    x = W.random_state(9, dim)
    for tau in (0.05, 0.6):
        out, _, _ = OK.expv(lambda v: op.apply(c, v), x, tau, 1e-12, 30, max_substeps=200)
        assert np.linalg.norm(out - expm(-1j * tau * Hm) @ x) <= 1e-10


def test_sparse_family_time_independent_propagation_matches_expm():
    dim = 64
    H0 = W.random_hermitian_csr(11, dim, 4, True)
    op = O.Sparse(H0, [W.random_hermitian_csr(12, dim, 2, True)])
    x = W.random_state(13, dim)
    out = OC.propagate(op, x, 0.0, 0.1, 5, 6, [lambda t: 0.0], 1e-13, 30)
    assert np.linalg.norm(out - expm(-0.5j * _dense(*H0, dim)) @ x) <= 1e-10


def test_gershgorin_csr_matches_dense_construction():
    # with unique (row, column) pairs the CSR interval is the dense one; with
    # repeated pairs (|a| + |b| >= |a + b|) it contains it; both contain the
    # spectrum
    for seed, cplx, dup in ((14, True, 5), (15, False, 0), (16, True, 0)):
        rp, ci, v = W.random_hermitian_csr(seed, 50, 4, cplx, duplicates=dup)
        A = _dense(rp, ci, v, 50)
        lo, hi = OCH.gershgorin_csr(rp, ci, v)
        dlo, dhi = OCH.gershgorin_dense(A)
        pairs = [(r, ci[e]) for r in range(50) for e in range(rp[r], rp[r + 1])]
        if len(pairs) == len(set(pairs)):
            assert abs(lo - dlo) <= 1e-13 and abs(hi - dhi) <= 1e-13
        assert lo <= dlo + 1e-13 and dhi <= hi + 1e-13
        lam = np.linalg.eigvalsh(A)
        assert lo <= lam[0] + 1e-12 and lam[-1] <= hi + 1e-12
    atom = W.grid_atom(Nr=60, L=3)                        # unique pairs, as the DIA form stores them
    rp, ci, v = W.dia_to_csr(atom.H0_offsets, atom.H0_values)
    A = _dense(rp, ci, v, 180)
    assert np.allclose(OCH.gershgorin_csr(rp, ci, v), OCH.gershgorin_dense(A), rtol=0, atol=1e-9)


@pytest.mark.parametrize("mistake", ["conjugate", "transpose", "drop_duplicates"])
def test_planted_csr_mistakes_are_caught(monkeypatch, mistake):
    good = O.csr_apply

    def bad(v, row_ptr, col_idx, values):
        row_ptr = np.asarray(row_ptr, dtype=np.int64)
        col_idx = np.asarray(col_idx, dtype=np.int64)
        values = np.asarray(values)
        dim = len(row_ptr) - 1
        rows = np.repeat(np.arange(dim), np.diff(row_ptr))
        out = np.zeros(dim, dtype=np.complex128)
        if mistake == "conjugate":
            np.add.at(out, rows, np.conj(values) * v[col_idx])
        elif mistake == "transpose":
            np.add.at(out, col_idx, values * v[rows])
        else:
            out[rows] = values * v[col_idx]          # repeated pairs overwrite instead of adding
        return out

    assert _pins_hold()
    monkeypatch.setattr(O, "csr_apply", bad)
    assert not _pins_hold()
    monkeypatch.setattr(O, "csr_apply", good)
