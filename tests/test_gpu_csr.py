"""GPU parity of the general sparse operator kind (CFET_OP_CSR) against the
CPU FP64 oracle (oracle.operators.Sparse, csr_apply).

Sec. 8: the stage operator c_0 H0 + sum_k c_k V_k is applied operator by
operator with the stage scalars (never formed), so any Hermitian sparse H0 and
V_k serve.  Cases: seeded random Hermitian matrices (complex values, repeated
(row, column) pairs, empty rows), a real banded one, and the grid atom written
in CSR form; FP64, fixed-point and complex64 vectors; Krylov and Chebyshev
stage exponentials.

Tolerances as in test_gpu_parity.py: apply elementwise 1e-13 relative to the
largest entry; expv and propagate ||psi_gpu - psi_oracle||_2 <= 1e-10 with
the oracle's Krylov decisions replayed (FP64-class formats), the complex64
rounding budget n_substeps * (4 sqrt(m_max) + 1) * 2^-24 (test_gpu_c64.py) for complex64.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, chebyshev as OCH, krylov as OK, operators as O

pytestmark = pytest.mark.gpu

PARITY = 1e-10
ULP32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1102_5071_gb300.build import build
    build()
    return torch


def _dev(torch, v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.complex128)).cuda()


def _problem(dim=3000, seed=21, nV=2):
    H0 = W.random_hermitian_csr(seed, dim, 6, True, duplicates=40)
    Vs = [W.random_hermitian_csr(seed + 1, dim, 3, False, band=40)]
    if nV > 1:
        Vs.append(W.random_hermitian_csr(seed + 2, dim, 2, True))
    drives = [lambda t: 0.8 * math.cos(1.3 * t), lambda t: 0.25 * math.sin(2.1 * t + 0.4)][:nV]
    return H0, Vs, drives


def _prop(H0, Vs, drives, **kw):
    import paper_1102_5071_gb300 as P
    return P.Propagator(P.CSR(*H0), [P.CSR(*v) for v in Vs], drives, **kw)


def test_csr_apply_matches_oracle(torch_cuda):
    torch = torch_cuda
    H0, Vs, drives = _problem()
    prop = _prop(H0, Vs, drives, precision="f64")
    op = O.Sparse(H0, Vs)
    x = W.random_state(3, op.dim)
    c = np.array([0.83, -1.1, 0.4])
    out = torch.empty(op.dim, dtype=torch.complex128, device="cuda")
    prop.apply(c, _dev(torch, x), out)
    ref = op.apply(c, x)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    prop.close()


@pytest.mark.parametrize("prec", ["f64", "fx", "c64"])
def test_csr_expv_matches_oracle(torch_cuda, prec):
    torch = torch_cuda
    H0, Vs, drives = _problem()
    prop = _prop(H0, Vs, drives, precision=prec, m_max=24, max_substeps=200)
    op = O.Sparse(H0, Vs)
    x = W.random_state(4, op.dim)
    c = np.array([0.9, 0.6, -0.3])
    ref, log, na = OK.expv(lambda v: op.apply(c, v), x, 0.4, 1e-11, 24, max_substeps=200)
    t = _dev(torch, x)
    st = prop.expv(c, 0.4, t, 1e-11)
    err = np.linalg.norm(t.cpu().numpy() - ref)
    bound = PARITY if prec != "c64" else st["n_substeps"] * (4 * math.sqrt(24) + 1) * ULP32 + 1e-11 * st["n_substeps"]
    assert err <= bound, (prec, err, log)
    prop.close()


@pytest.mark.parametrize("prec", ["f64", "fx", "c64"])
def test_csr_propagate_forced_matches_oracle(torch_cuda, prec):
    torch = torch_cuda
    H0, Vs, drives = _problem()
    prop = _prop(H0, Vs, drives, precision=prec, m_max=20, max_substeps=200)
    op = O.Sparse(H0, Vs)
    x = W.random_state(5, op.dim)
    ref, log, na = OC.propagate(op, x, 0.3, 0.05, 4, "CF6:5Opt", drives, 1e-11, 20, return_log=True,
                                max_substeps=200)
    t = _dev(torch, x)
    st = prop.propagate(t, 0.3, 0.05, 4, scheme="CF6:5Opt", tol=1e-11, forced=log)
    err = np.linalg.norm(t.cpu().numpy() - ref)
    assert st["n_applies"] == na
    bound = PARITY if prec != "c64" else st["n_substeps"] * (4 * math.sqrt(20) + 1) * ULP32
    assert err <= bound, (prec, err)
    if prec != "c64":
        # adaptive: the device's own decisions agree with the oracle's
        t2 = _dev(torch, x)
        st2, log2 = prop.propagate(t2, 0.3, 0.05, 4, scheme="CF6:5Opt", tol=1e-11, record=True)
        same = sum(a == b for a, b in zip(log, log2)) / len(log)
        assert same >= 0.95 and np.linalg.norm(t2.cpu().numpy() - ref) <= PARITY
    prop.close()


@pytest.mark.parametrize("prec", ["f64", "fx"])
def test_csr_every_order_with_substeps(torch_cuda, prec):
    # orders 2, 4, 8 with a small Krylov space: substeps (h > 0) occur
    torch = torch_cuda
    H0, Vs, drives = _problem(dim=700, seed=31, nV=1)
    prop = _prop(H0, Vs, drives, precision=prec, m_max=8, max_substeps=400)
    op = O.Sparse(H0, Vs)
    x = W.random_state(6, op.dim)
    for order in (2, 4, 8):
        ref, log, na = OC.propagate(op, x, 0.0, 0.3, 2, order, drives, 1e-10, 8, return_log=True,
                                    max_substeps=400)
        t = _dev(torch, x)
        prop.propagate(t, 0.0, 0.3, 2, order=order, tol=1e-10, forced=log)
        assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY, order
    assert any(h > 0 for lg in log for _, h in lg)
    prop.close()


@pytest.mark.parametrize("prec", ["fx", "f64"])
def test_grid_atom_as_csr_matches_dia_and_oracle(torch_cuda, prec):
    # the reduced grid atom (Nr = 120, l < 8) in CSR form: the oracle's DIA
    # propagation, and the device's DIA run with the same decisions
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=120, L=8)
    H0 = W.dia_to_csr(p.H0_offsets, p.H0_values)
    V = W.dia_to_csr(p.V_offsets, p.V_values)
    psi0, _ = W.atom_ground_state(p)
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    ref, log, _ = OC.propagate(op, psi0, 500.0, 0.1, 2, 8, [p.drive], 1e-10, 40, return_log=True, max_substeps=4000)
    csr = P.Propagator(P.CSR(*H0), [P.CSR(*V)], [p.drive], m_max=40, max_substeps=4000, precision=prec)
    dia = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive], m_max=40,
                       max_substeps=4000, precision=prec)
    a, b = _dev(torch, psi0), _dev(torch, psi0)
    csr.propagate(a, 500.0, 0.1, 2, order=8, tol=1e-10, forced=log)
    dia.propagate(b, 500.0, 0.1, 2, order=8, tol=1e-10, forced=log)
    assert np.linalg.norm(a.cpu().numpy() - ref) <= PARITY
    assert np.linalg.norm(a.cpu().numpy() - b.cpu().numpy()) <= PARITY
    csr.close()
    dia.close()


def test_csr_chebyshev_matches_oracle(torch_cuda):
    torch = torch_cuda
    H0, Vs, drives = _problem(dim=1500, seed=41)
    prop = _prop(H0, Vs, drives, expm="chebyshev", m_max=64, max_substeps=64)
    op = O.Sparse(H0, Vs)
    x = W.random_state(7, op.dim)
    ref, st_ref = OCH.propagate(op, x, 0.1, 0.05, 3, 6, drives, 1e-12, return_stats=True)
    t = _dev(torch, x)
    st = prop.propagate(t, 0.1, 0.05, 3, order=6, tol=1e-12)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY
    prop.close()


def test_csr_time_independent_matches_expm(torch_cuda):
    torch = torch_cuda
    from scipy.linalg import expm
    dim = 256
    H0 = W.random_hermitian_csr(51, dim, 5, True)
    V = W.random_hermitian_csr(52, dim, 2, False)
    A = np.zeros((dim, dim), dtype=np.complex128)
    rp, ci, v = H0
    for r in range(dim):
        for e in range(rp[r], rp[r + 1]):
            A[r, ci[e]] += v[e]
    x = W.random_state(8, dim)
    for prec in ("f64", "fx"):
        prop = _prop(H0, [V], [lambda t: 0.0], precision=prec, m_max=30)
        t = _dev(torch, x)
        prop.propagate(t, 0.0, 0.1, 5, order=8, tol=1e-13)
        assert np.linalg.norm(t.cpu().numpy() - expm(-0.5j * A) @ x) <= PARITY, prec
        prop.close()


def test_csr_validation(torch_cuda):
    import paper_1102_5071_gb300 as P
    rp = np.array([0, 1, 2], dtype=np.int64)
    good = P.CSR(rp, np.array([1, 0]), np.array([0.5 + 0.25j, 0.5 - 0.25j]))
    p = P.Propagator(good, [], [])
    p.close()
    bad_h = P.CSR(rp, np.array([1, 0]), np.array([0.5 + 0.25j, 0.5 + 0.25j]))     # not Hermitian
    with pytest.raises(P.CfetError, match="EINVAL"):
        P.Propagator(bad_h, [], [])
    bad_col = P.CSR(rp, np.array([2, 0]), np.array([1.0, 1.0]))                   # column out of range
    with pytest.raises(P.CfetError, match="EINVAL"):
        P.Propagator(bad_col, [], [])
    bad_rp = P.CSR(np.array([0, 2, 1], dtype=np.int64), np.array([0, 1]), np.array([1.0, 1.0]))
    with pytest.raises(P.CfetError, match="EINVAL"):
        P.Propagator(bad_rp, [], [])
    diag_im = P.CSR(np.array([0, 1], dtype=np.int64), np.array([0]), np.array([1.0 + 0.5j]))
    with pytest.raises(P.CfetError, match="EINVAL"):
        P.Propagator(diag_im, [], [])
    with pytest.raises(P.CfetError, match="EINVAL"):                               # mixed kinds
        P.Propagator(good, [P.DIA(np.array([0]), np.ones((1, 2)))], [lambda t: 0.0])
