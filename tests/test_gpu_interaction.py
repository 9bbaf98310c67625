"""GPU parity of CFET stepping in the interaction picture of the diagonal of
H0 (CFET_PICTURE_INTERACTION, Secs. 9.3, 9.4) against oracle/interaction.py.

The device applies the stage operator from per-stage tables of complex
weights indexed by the local spin configuration (host-computed from the
phases e^{i (d(x) - d(y)) t_m}); the oracle applies the definition (phase,
H_b(t_m), conjugate phase at every node).  With the oracle's Krylov
decisions replayed the two agree to ||psi_gpu - psi_oracle||_2 <= 1e-10.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import interaction as IP, krylov as OK, operators as O

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


def _chain(N, nfields=1, J=1.0, Delta=0.5, picture="interaction", **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N, J=J, Delta=Delta)
    fields = [pr.xfield] + [W.uniform(100 + k, N, -1, 1) for k in range(1, nfields)]
    drives = [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)]
    prop = P.Propagator(P.XXZChain(N, J, Delta, pr.h), [P.XField(N, a) for a in fields], drives,
                        precision="f64", picture=picture, **kw)
    return prop, O.SpinChain(N, J, Delta, pr.h, fields), drives


def _compare(torch, prop, op, drives, psi0, t0, dt, nsteps, scheme, tol, m):
    ref, log, _ = IP.propagate(op, psi0, t0, dt, nsteps, scheme, drives, tol, m, return_log=True, max_substeps=200)
    kw = dict(scheme=scheme) if isinstance(scheme, str) else dict(order=scheme)
    x = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    st = prop.propagate(x, t0, dt, nsteps, tol=tol, forced=log, **kw)
    y = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    _, log2 = prop.propagate(y, t0, dt, nsteps, tol=tol, record=True, **kw)
    same = sum(a == b for a, b in zip(log, log2)) / len(log)
    return np.linalg.norm(x.cpu().numpy() - ref), same, st, np.linalg.norm(y.cpu().numpy() - ref)


def test_ip_chain_n8(torch_cuda):
    prop, op, drives = _chain(8, m_max=16, max_substeps=200)
    err, same, st, aerr = _compare(torch_cuda, prop, op, drives, W.neel_state(8), 0.0, 0.02, 50, 4, 1e-12, 16)
    assert err <= PARITY, err
    assert same >= 0.95 and aerr <= 1e-9


@pytest.mark.parametrize("scheme", ["CF2:1", "CF4:3Opt", "CF6:4", "CF6:5Opt", "CF8:11"])
def test_ip_schemes_two_fields(torch_cuda, scheme):
    prop, op, drives = _chain(9, nfields=2, m_max=20, max_substeps=200)
    err, same, st, _ = _compare(torch_cuda, prop, op, drives, W.random_state(5, 1 << 9), 0.37, 0.05, 6, scheme,
                                1e-11, 20)
    assert err <= PARITY, err


def test_ip_chain_n20_one_step(torch_cuda):
    prop, op, drives = _chain(20, m_max=16)
    err, same, st, _ = _compare(torch_cuda, prop, op, drives, W.random_state(2, 1 << 20), 0.5, 0.05, 1, 4,
                                1e-10, 16)
    assert err <= PARITY, err


def test_ip_diagonal_hamiltonian_is_exact(torch_cuda):
    # J = 0 and no drive: psi^I is constant, so coarse steps give exp(-i H_d T) psi
    torch = torch_cuda
    N = 10
    h = W.uniform(3, N, -1, 1)
    import paper_1102_5071_gb300 as P
    prop = P.Propagator(P.XXZChain(N, 0.0, 0.7, h), [P.XField(N, np.ones(N))], [lambda t: 0.0],
                        precision="f64", picture="interaction")
    psi0 = W.random_state(2, 1 << N)
    x = torch.from_numpy(psi0).cuda()
    st = prop.propagate(x, 0.3, 1.7, 3, order=4, tol=1e-12)
    Hd = np.real(np.diag(O.xxz_dense(N, 0.0, 0.7, h)))
    assert np.linalg.norm(x.cpu().numpy() - np.exp(-1j * Hd * 5.1) * psi0) <= 1e-12
    assert st["n_applies"] <= st["n_exp"] * 2     # zero stage operators: immediate breakdown


def test_ip_agrees_with_the_schroedinger_picture(torch_cuda):
    # both pictures converge to the same solution; at dt = 0.01 they agree to
    # the CFET error of the coarser of the two
    torch = torch_cuda
    N = 12
    ip, _, _ = _chain(N)
    sp, _, _ = _chain(N, picture="schroedinger")
    psi0 = W.random_state(7, 1 << N)
    x = torch.from_numpy(psi0).cuda()
    y = torch.from_numpy(psi0).cuda()
    ip.propagate(x, 0.0, 0.01, 200, order=6, tol=1e-12)
    sp.propagate(y, 0.0, 0.01, 200, order=6, tol=1e-12)
    assert torch.linalg.vector_norm(x - y).item() <= 1e-8
    assert abs(torch.linalg.vector_norm(x).item() - 1.0) <= 1e-11


def test_ip_context_rules(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    ip, op, drives = _chain(7)
    sp, _, _ = _chain(7, picture="schroedinger")
    psi0 = W.random_state(3, 128)
    x = torch.from_numpy(psi0).cuda()
    st = ip.propagate(x, 0.0, 0.1, 0, order=4)
    assert st["n_exp"] == 0 and np.array_equal(x.cpu().numpy(), psi0)
    # cfet_expv acts in the Schroedinger picture in both contexts
    c = np.array([0.7, 0.2])
    a = torch.from_numpy(psi0).cuda()
    b = torch.from_numpy(psi0).cuda()
    ip.expv(c, 0.3, a, tol=1e-12)
    sp.expv(c, 0.3, b, tol=1e-12)
    assert torch.equal(a, b)
    with pytest.raises(P.CfetError, match="EINVAL"):
        ip.fidelity_grad(x, x, 0.0, 0.1, 4, [0.1, 0.2], 2.0)
    z = torch.zeros(128, dtype=torch.complex128, device="cuda")
    ip.propagate(z, 0.0, 0.1, 2, order=6)
    assert torch.count_nonzero(z).item() == 0
