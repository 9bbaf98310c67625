"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances: elementwise apply results agree to a few ulps of the operator
norm (1e-12 relative); whole propagations are compared by the 2-norm of the
difference, ||psi_gpu - psi_oracle||_2 <= 1e-10, with the oracle's Krylov
decisions replayed on the device (forced mode) so that the comparison measures
rounding only.  Adaptive-vs-adaptive runs are compared against the same bound
and their decision logs must agree.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, krylov as OK, operators as O

pytestmark = pytest.mark.gpu

PARITY = 1e-10


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


def _host(t):
    return t.cpu().numpy()


PRECS = ["fx", "f64"]


def _spin(torch, N, nfields=1, J=1.0, Delta=0.5, seed=1, **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N, J=J, Delta=Delta, h_seed=seed)
    fields = [pr.xfield] + [W.uniform(100 + k, N, -1, 1) for k in range(1, nfields)]
    prop = P.Propagator(P.XXZChain(N, J, Delta, pr.h), [P.XField(N, a) for a in fields],
                        [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)], **kw)
    op = O.SpinChain(N, J, Delta, pr.h, fields)
    drives = [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)]
    return prop, op, drives, pr


def _atom(torch, Nr, L, **kw):
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=Nr, L=L)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive], **kw)
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    return prop, op, [p.drive], p


# ---------------------------------------------------------------- apply (a4)
@pytest.mark.parametrize("N,nf", [(1, 1), (2, 1), (5, 2), (8, 1), (13, 3)])
def test_apply_spin(torch_cuda, N, nf):
    torch = torch_cuda
    prop, op, _, _ = _spin(torch, N, nfields=nf)
    v = W.random_state(7 + N, 1 << N)
    c = np.concatenate([[0.83], W.uniform(9, nf, -1.5, 1.5)])
    out = torch.empty(1 << N, dtype=torch.complex128, device="cuda")
    prop.apply(c, _dev(torch, v), out)
    torch.cuda.synchronize()
    ref = op.apply(c, v)
    scale = np.max(np.abs(ref)) + 1e-300
    assert np.max(np.abs(_host(out) - ref)) <= 1e-13 * max(scale, 1.0)


def test_apply_spin_full_size(torch_cuda):
    torch = torch_cuda
    prop, op, _, _ = _spin(torch, 20)
    v = W.random_state(2, 1 << 20)
    c = np.array([0.61, -0.47])
    out = torch.empty(1 << 20, dtype=torch.complex128, device="cuda")
    prop.apply(c, _dev(torch, v), out)
    ref = op.apply(c, v)
    assert np.max(np.abs(_host(out) - ref)) <= 1e-14 * max(np.max(np.abs(ref)), 1.0) * 20


@pytest.mark.parametrize("Nr,L", [(37, 7), (2000, 100)])
def test_apply_dia(torch_cuda, Nr, L):
    torch = torch_cuda
    prop, op, _, p = _atom(torch, Nr, L)
    v = W.random_state(11, p.dim)
    c = np.array([0.9, 0.04])
    out = torch.empty(p.dim, dtype=torch.complex128, device="cuda")
    prop.apply(c, _dev(torch, v), out)
    ref = op.apply(c, v)
    assert np.max(np.abs(_host(out) - ref)) <= 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------- expv (a5-a7)
@pytest.mark.parametrize("tau,tol,m", [(0.02, 1e-12, 16), (0.3, 1e-12, 24), (1.5, 1e-10, 12), (0.05, 0.0, 10)])
@pytest.mark.parametrize("prec", PRECS)
def test_expv_spin(torch_cuda, tau, tol, m, prec):
    torch = torch_cuda
    N = 10
    prop, op, _, _ = _spin(torch, N, m_max=m, max_substeps=200, precision=prec)
    psi0 = W.random_state(3, 1 << N)
    c = np.array([0.7, 0.45])
    t = _dev(torch, psi0)
    stats = prop.expv(c, tau, t, tol)
    ref, log, na = OK.expv(lambda v: op.apply(c, v), psi0, tau, tol, m, max_substeps=200)
    assert np.linalg.norm(_host(t) - ref) <= PARITY
    assert stats["n_substeps"] == len(log) and stats["n_applies"] == na


# ---------------------------------------------------------------- propagate (a1-a8)
def _parity_run(prop, op, drives, psi0, t0, dt, nsteps, scheme_or_order, tol, m, torch):
    ref, log, na = OC.propagate(op, psi0, t0, dt, nsteps, scheme_or_order, drives, tol, m, return_log=True,
                                max_substeps=200)
    kw = dict(scheme=scheme_or_order) if isinstance(scheme_or_order, str) else dict(order=scheme_or_order)
    t = _dev(torch, psi0)
    stats = prop.propagate(t, t0, dt, nsteps, tol=tol, forced=log, **kw)
    forced_err = np.linalg.norm(_host(t) - ref)
    t2 = _dev(torch, psi0)
    stats2, log2 = prop.propagate(t2, t0, dt, nsteps, tol=tol, record=True, **kw)
    adaptive_err = np.linalg.norm(_host(t2) - ref)
    return forced_err, adaptive_err, log, log2, stats, stats2, na


@pytest.mark.parametrize("prec", PRECS)
def test_propagate_chain_n8_full_run(torch_cuda, prec):
    # driven XXZ chain N = 8, Neel state, CF4:2, dt = 0.01, T = 10, m <= 16, tol 1e-12
    torch = torch_cuda
    cfg = W.CHAIN_SMALL
    prop, op, drives, _ = _spin(torch, cfg["N"], m_max=cfg["m_max"], max_substeps=200, precision=prec)
    psi0 = W.neel_state(cfg["N"])
    nsteps = int(round(cfg["T"] / cfg["dt"]))
    fe, ae, log, log2, st, st2, na = _parity_run(prop, op, drives, psi0, 0.0, cfg["dt"], nsteps, 4, cfg["tol"],
                                                 cfg["m_max"], torch)
    assert fe <= PARITY, fe
    assert ae <= PARITY, ae
    same = sum(a == b for a, b in zip(log, log2)) / len(log)
    assert same >= 0.99, same
    assert st["n_applies"] == na and st["n_exp"] == 2 * nsteps


@pytest.mark.parametrize("scheme", ["CF2:1", "CF4:2", "CF4:3", "CF4:3Opt", "CF6:4", "CF6:5", "CF6:5b", "CF6:6",
                                    "CF6:5Imp", "CF6:5Opt", "CF6:6Opt", "CF8:11"])
@pytest.mark.parametrize("prec", PRECS)
def test_propagate_every_scheme(torch_cuda, scheme, prec):
    torch = torch_cuda
    N = 9
    prop, op, drives, _ = _spin(torch, N, nfields=2, m_max=20, max_substeps=200, precision=prec)
    psi0 = W.random_state(5, 1 << N)
    fe, ae, log, log2, *_ = _parity_run(prop, op, drives, psi0, 0.37, 0.05, 6, scheme, 1e-11, 20, torch)
    assert fe <= PARITY and ae <= PARITY, (fe, ae)


@pytest.mark.parametrize("prec", PRECS)
def test_propagate_with_substeps(torch_cuda, prec):
    # large dt and a small Krylov space force substepping (h > 0 records)
    torch = torch_cuda
    N = 10
    prop, op, drives, _ = _spin(torch, N, m_max=8, max_substeps=400, precision=prec)
    psi0 = W.random_state(6, 1 << N)
    fe, ae, log, log2, *_ = _parity_run(prop, op, drives, psi0, 0.0, 0.6, 3, 6, 1e-10, 8, torch)
    assert any(h > 0 for lg in log for _, h in lg)
    assert fe <= PARITY and ae <= PARITY, (fe, ae)


@pytest.mark.parametrize("prec", PRECS)
def test_propagate_fixed_krylov_dimension(torch_cuda, prec):
    # tol <= 0: fixed K = m_max (the paper's K-vector runs)
    torch = torch_cuda
    N = 10
    prop, op, drives, _ = _spin(torch, N, m_max=10, precision=prec)
    psi0 = W.random_state(8, 1 << N)
    ref = OC.propagate(op, psi0, 0.0, 0.02, 15, 6, drives, 0.0, 10)
    t = _dev(torch, psi0)
    st = prop.propagate(t, 0.0, 0.02, 15, order=6, tol=0.0)
    assert np.linalg.norm(_host(t) - ref) <= PARITY
    assert st["n_applies"] == 15 * 5 * 10


@pytest.mark.parametrize("prec", PRECS)
def test_propagate_chain_n20_one_step(torch_cuda, prec):
    # full-size chain (dim 2^20), one CF4:2 step at dt = 0.05, fixed K = 10
    torch = torch_cuda
    prop, op, drives, pr = _spin(torch, 20, m_max=10, precision=prec)
    psi0 = W.random_state(2, 1 << 20)
    ref = OC.propagate(op, psi0, 0.0, 0.05, 1, 4, drives, 0.0, 10)
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.05, 1, order=4, tol=0.0)
    assert np.linalg.norm(_host(t) - ref) <= PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_chain_n20_zero_coupling_factorises(torch_cuda, prec):
    # J = 0: exact product of single-spin CFET results at full size (any-size property)
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N = 20
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=16, precision=prec)
    psi0 = W.neel_state(N)
    nsteps, dt = 40, 0.05
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, dt, nsteps, order=6, tol=1e-13)
    out = _host(t)
    x0 = int(np.argmax(np.abs(psi0)))
    single = []
    for i in range(N):
        e = np.zeros(2, dtype=np.complex128)
        e[(x0 >> i) & 1] = 1.0
        single.append(OC.propagate(O.Dense(pr.h[i] * O.SZ, [O.SX]), e, 0.0, dt, nsteps, 6, [pr.drive], 1e-14, 2))
    rng = np.random.default_rng(0)
    idx = rng.integers(0, 1 << N, 4000)
    amp = np.ones(len(idx), dtype=np.complex128)
    for i in range(N):
        amp *= np.where((idx >> i) & 1, single[i][1], single[i][0])
    assert np.max(np.abs(out[idx] - amp)) < 1e-12
    assert abs(np.linalg.norm(out) - 1.0) < 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_time_independent_matches_expm(torch_cuda, prec):
    torch = torch_cuda
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    N = 9
    pr = W.spin_chain(N)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [lambda t: 0.0], m_max=30, precision=prec)
    psi0 = W.random_state(4, 1 << N)
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.1, 5, order=8, tol=1e-13)
    ref = expm(-1j * 0.5 * O.xxz_dense(N, pr.J, pr.Delta, pr.h)) @ psi0
    assert np.linalg.norm(_host(t) - ref) < 1e-10


@pytest.mark.parametrize("Nr,L,nsteps,t0", [(120, 8, 3, 300.0)])
@pytest.mark.parametrize("prec", PRECS)
def test_propagate_atom_reduced(torch_cuda, Nr, L, nsteps, t0, prec):
    torch = torch_cuda
    prop, op, drives, p = _atom(torch, Nr, L, m_max=32, max_substeps=4000, precision=prec)
    psi0, _ = W.atom_ground_state(p)
    fe, ae, log, log2, *_ = _parity_run(prop, op, drives, psi0, t0, 0.1, nsteps, 8, 1e-10, 32, torch)
    assert fe <= PARITY and ae <= PARITY, (fe, ae)


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases(torch_cuda, prec):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, op, drives, _ = _spin(torch, 6, precision=prec)
    psi0 = W.random_state(1, 64)
    t = _dev(torch, psi0)
    st = prop.propagate(t, 0.0, 0.1, 0, order=4)                 # nsteps = 0: no-op
    assert np.array_equal(_host(t), psi0) and st["n_exp"] == 0
    z = torch.zeros(64, dtype=torch.complex128, device="cuda")  # zero state stays zero
    prop.propagate(z, 0.0, 0.1, 2, order=6)
    assert torch.count_nonzero(z).item() == 0
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.propagate(t, 0.0, 0.1, 1, order=5)
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.propagate(t, 0.0, 0.0, 1, order=4)
    bad = _dev(torch, psi0)
    bad[3] = complex(float("nan"), 0.0)
    with pytest.raises(P.CfetError, match="ENAN"):
        prop.propagate(bad, 0.0, 0.1, 1, order=4)
    # the context stays usable after an error
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.1, 1, order=4)
    # a spin chain of one site (dim 2)
    prop1, op1, dr1, _ = _spin(torch, 1, precision=prec)
    e = _dev(torch, np.array([0.6, 0.8j]))
    prop1.propagate(e, 0.0, 0.05, 10, order=8, tol=1e-13)
    ref = OC.propagate(op1, np.array([0.6, 0.8j]), 0.0, 0.05, 10, 8, dr1, 1e-13, 16)
    assert np.linalg.norm(_host(e) - ref) < PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_substep_cap_reports_ekrylov(torch_cuda, prec):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, op, drives, _ = _spin(torch, 8, m_max=4, max_substeps=2, precision=prec)
    t = _dev(torch, W.random_state(2, 256))
    with pytest.raises(P.CfetError, match="EKRYLOV"):
        prop.propagate(t, 0.0, 2.0, 1, order=4, tol=1e-12)


@pytest.mark.parametrize("prec", PRECS)
def test_e2e_host_entry_matches_device_entry(torch_cuda, prec):
    torch = torch_cuda
    prop, op, drives, _ = _spin(torch, 12, precision=prec)
    psi0 = W.random_state(3, 1 << 12)
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.02, 5, order=6, tol=1e-10)
    h = psi0.copy()
    prop.propagate_host(h, 0.0, 0.02, 5, order=6, tol=1e-10)
    assert np.array_equal(h, _host(t))


@pytest.mark.parametrize("prec", PRECS)
def test_full_size_atom_without_field_keeps_the_1s_state(torch_cuda, prec):
    # full-size grid atom (dim 200 000, CF8:11, dt = 0.1, m <= 64) with E0 = 0:
    # the discrete 1s state is an eigenvector of H0, so exp(-i H0 t) psi_1s =
    # exp(-i E_1s t) psi_1s exactly (an any-size property, checked at every
    # element)
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    a = W.ATOM
    p = W.grid_atom(Nr=a["Nr"], L=a["L"], dr=a["dr"], E0=0.0, omega=a["omega"], Tp=a["Tp"])
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=a["m_max"], max_substeps=4000, precision=prec)
    psi0, e1s = W.atom_ground_state(p)
    x = _dev(torch, psi0)
    nsteps = 3
    prop.propagate(x, 500.0, a["dt"], nsteps, order=a["order"], tol=1e-12)
    ref = np.exp(-1j * e1s * a["dt"] * nsteps) * psi0
    assert np.linalg.norm(_host(x) - ref) <= PARITY


@pytest.mark.parametrize("prec", PRECS + ["c64"])
def test_chain_n20_without_field_conserves_magnetisation(torch_cuda, prec):
    # with the x field switched off (A = 0) the XXZ chain conserves the number
    # of down spins: a random state on the half-filled sector of the N = 20
    # chain (popcount 10, 184 756 states) keeps every amplitude outside the
    # sector exactly zero and its norm to the Krylov tolerance (complex64: to
    # its FP32 rounding budget)
    import paper_1102_5071_gb300 as P
    torch = torch_cuda
    N = 20
    pr = W.spin_chain(N)
    x = np.arange(1 << N, dtype=np.int64)
    pop = np.zeros(1 << N, dtype=np.int64)
    for i in range(N):
        pop += (x >> i) & 1
    sector = pop == N // 2
    psi0 = W.random_state(13, 1 << N)
    psi0[~sector] = 0.0
    psi0 /= np.linalg.norm(psi0)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [lambda t: 0.0], m_max=16,
                        precision=prec)
    t = _dev(torch, psi0)
    st = prop.propagate(t, 0.0, 0.05, 10, order=6, tol=1e-10)
    out = t.cpu().numpy()
    assert np.count_nonzero(out[~sector]) == 0
    # (complex64: the rounding budget of tests/test_gpu_c64.py, 4 sqrt(16) + 1 = 17 FP32 ulps per substep)
    bound = st["n_substeps"] * (17 * 2.0 ** -24 if prec == "c64" else 1e-10)
    assert abs(np.linalg.norm(out[sector]) - 1.0) <= bound
