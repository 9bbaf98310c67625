"""GPU parity of the Pauli-sum operator family (CFET_OP_PAULI, FP64 kernel)
against the oracle's string-by-string apply (oracle/operators.py PauliSum).

Tolerances as in test_gpu_parity.py: applies to 1e-12 of the result's norm,
propagations ||psi_gpu - psi_oracle||_2 <= 1e-10 with the oracle's Krylov
decisions replayed (and adaptive runs within the same bound).
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, operators as O

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


def _random_terms(seed, N, n, max_weight=4):
    # strings of up to max_weight non-identity sites, coefficients U[-1, 1]
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(n):
        w = int(rng.integers(1, min(max_weight, N) + 1))
        sites = rng.choice(N, size=w, replace=False)
        label = {int(s): str(rng.choice(list("XYZ"))) for s in sites}
        terms.append((float(rng.uniform(-1, 1)), label))
    return terms


def _drives():
    return [lambda t: 0.9 * math.cos(1.7 * t), lambda t: 0.4 * math.sin(0.8 * t + 0.3)]


def _problem(N, seed=1, n0=40, nv=12):
    import paper_1102_5071_gb300 as P
    h0 = _random_terms(seed, N, n0)
    v1 = _random_terms(seed + 10, N, nv, max_weight=2)
    v2 = [(float(a), {i: "Y"}) for i, a in enumerate(W.uniform(seed + 20, N, -1, 1))]
    prop = P.Propagator(P.PauliSum(N, h0), [P.PauliSum(N, v1), P.PauliSum(N, v2)], _drives(), m_max=24,
                        max_substeps=200)
    return prop, O.PauliSum(N, h0, [v1, v2])


@pytest.mark.parametrize("N", [1, 7, 10])
def test_pauli_apply_matches_oracle(torch_cuda, N):
    prop, op = _problem(N)
    v = W.random_state(3, 1 << N)
    c = np.array([0.7, -0.45, 1.2])
    out_t = torch_cuda.zeros(1 << N, dtype=torch_cuda.complex128, device="cuda")
    prop.apply(c, _dev(torch_cuda, v), out_t)
    out = out_t.cpu().numpy()
    ref = op.apply(c, v)
    assert np.linalg.norm(out - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref))


@pytest.mark.parametrize("scheme", ["CF4:2", "CF6:5Opt", "CF8:11"])
def test_pauli_propagate_matches_oracle(torch_cuda, scheme):
    N = 9
    prop, op = _problem(N, seed=4)
    psi0 = W.random_state(5, 1 << N)
    ref, log, na = OC.propagate(op, psi0, 0.2, 0.05, 4, scheme, _drives(), 1e-11, 24, return_log=True,
                                max_substeps=200)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.2, 0.05, 4, scheme=scheme, tol=1e-11, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY and st["n_applies"] == na
    t2 = _dev(torch_cuda, psi0)
    _, log2 = prop.propagate(t2, 0.2, 0.05, 4, scheme=scheme, tol=1e-11, record=True)
    assert np.linalg.norm(t2.cpu().numpy() - ref) <= PARITY
    assert sum(a == b for a, b in zip(log, log2)) / len(log) >= 0.95


def test_pauli_form_of_the_chain_matches_the_chain_kernel(torch_cuda):
    # the driven XXZ chain given as Pauli strings runs the Pauli-sum kernel;
    # it agrees with the chain kernel (FP64) and with the oracle
    import paper_1102_5071_gb300 as P
    N = 12
    pr = W.spin_chain(N)
    terms = []
    for i in range(N - 1):
        terms += [(pr.J, {i: "X", i + 1: "X"}), (pr.J, {i: "Y", i + 1: "Y"}), (pr.J * pr.Delta, {i: "Z", i + 1: "Z"})]
    terms += [(float(pr.h[i]), {i: "Z"}) for i in range(N)]
    vterms = [(float(pr.xfield[i]), {i: "X"}) for i in range(N)]
    pauli = P.Propagator(P.PauliSum(N, terms), [P.PauliSum(N, vterms)], [pr.drive], m_max=20)
    chain = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=20,
                         precision="f64")
    psi0 = W.random_state(6, 1 << N)
    a, b = _dev(torch_cuda, psi0), _dev(torch_cuda, psi0)
    _, log = chain.propagate(b, 0.0, 0.02, 10, order=6, tol=1e-11, record=True)
    pauli.propagate(a, 0.0, 0.02, 10, order=6, tol=1e-11, forced=log)
    assert np.linalg.norm(a.cpu().numpy() - b.cpu().numpy()) <= 1e-12
    ref = OC.propagate(O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield]), psi0, 0.0, 0.02, 10, 6, [pr.drive], 1e-11,
                       20, forced_log=log)
    assert np.linalg.norm(a.cpu().numpy() - ref) <= PARITY


def test_chain_with_a_pauli_drive(torch_cuda):
    # an XXZ chain with a Y-field drive (not expressible as X fields): the
    # chain is expanded into strings, the context computes in FP64
    import paper_1102_5071_gb300 as P
    N = 8
    pr = W.spin_chain(N)
    ay = W.uniform(31, N, -1, 1)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.PauliSum(N, [(a, {i: "Y"}) for i, a in enumerate(ay)])],
                        [pr.drive], m_max=20)
    terms = []
    for i in range(N - 1):
        terms += [(pr.J, {i: "X", i + 1: "X"}), (pr.J, {i: "Y", i + 1: "Y"}), (pr.J * pr.Delta, {i: "Z", i + 1: "Z"})]
    terms += [(float(pr.h[i]), {i: "Z"}) for i in range(N)]
    op = O.PauliSum(N, terms, [[(a, {i: "Y"}) for i, a in enumerate(ay)]])
    psi0 = W.neel_state(N)
    ref, log, _ = OC.propagate(op, psi0, 0.0, 0.05, 20, 4, [pr.drive], 1e-12, 20, return_log=True)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 0.0, 0.05, 20, order=4, tol=1e-12, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY


def test_pauli_time_independent_matches_expm(torch_cuda):
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    N = 8
    terms = _random_terms(9, N, 30)
    prop = P.Propagator(P.PauliSum(N, terms), [], [], m_max=30)
    psi0 = W.random_state(7, 1 << N)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.0, 0.1, 8, order=8, tol=1e-12)
    ref = expm(-1j * 0.8 * O.pauli_dense(N, terms)) @ psi0
    assert np.linalg.norm(t.cpu().numpy() - ref) <= st["n_substeps"] * 1e-12 + 1e-12


def test_pauli_edge_cases(torch_cuda):
    import paper_1102_5071_gb300 as P
    torch = torch_cuda
    # an empty Pauli sum is the zero operator: psi unchanged
    prop = P.Propagator(P.PauliSum(5, []), [P.XField(5, np.zeros(5))], [lambda t: 1.0])
    psi0 = W.random_state(8, 32)
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.1, 3, order=4)
    assert np.allclose(t.cpu().numpy(), psi0, atol=1e-15)
    # the identity string only: a global phase exp(-i c T)
    prop = P.Propagator(P.PauliSum(5, [(0.7, "IIIII")]), [], [])
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.1, 3, order=4, tol=1e-13)
    assert np.allclose(t.cpu().numpy(), np.exp(-1j * 0.7 * 0.3) * psi0, atol=1e-13)
    # fixed point and complex64 are refused for Pauli sums
    with pytest.raises(P.CfetError, match="EINVAL"):
        P.Propagator(P.PauliSum(5, [(0.7, "XIIII")]), [], [], precision="fx")


def test_pauli_full_size_chain_one_step(torch_cuda):
    # the benchmark chain (N = 20) as Pauli strings: one CF4:2 step, fixed K = 10
    import paper_1102_5071_gb300 as P
    N = 20
    pr = W.spin_chain(N)
    terms = []
    for i in range(N - 1):
        terms += [(pr.J, {i: "X", i + 1: "X"}), (pr.J, {i: "Y", i + 1: "Y"}), (pr.J * pr.Delta, {i: "Z", i + 1: "Z"})]
    terms += [(float(pr.h[i]), {i: "Z"}) for i in range(N)]
    prop = P.Propagator(P.PauliSum(N, terms), [P.PauliSum(N, [(1.0, {i: "X"}) for i in range(N)])], [pr.drive],
                        m_max=10)
    psi0 = W.random_state(2, 1 << N)
    ref = OC.propagate(O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield]), psi0, 0.0, 0.05, 1, 4, [pr.drive], 0.0, 10)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 0.0, 0.05, 1, order=4, tol=0.0)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY
