"""GPU parity of the full re-orthogonalisation option (cfet_options.reorth,
FP64 kernel: one classical Gram-Schmidt sweep of every Lanczos vector against
all earlier ones) against the oracle in the same mode (krylov.expv with
reorth=True), and its behaviour on a spectrum where the plain three-term
recurrence loses orthogonality.  Bounds as in test_gpu_parity.py."""

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


@pytest.mark.parametrize("scheme", ["CF4:2", "CF6:5Opt"])
def test_reorth_chain_matches_oracle(torch_cuda, scheme):
    import paper_1102_5071_gb300 as P
    N = 10
    pr = W.spin_chain(N)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=24,
                        max_substeps=200, precision="f64", reorth=True)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    psi0 = W.random_state(5, 1 << N)
    ref, log, na = OC.propagate(op, psi0, 0.1, 0.1, 5, scheme, [pr.drive], 1e-12, 24, return_log=True,
                                max_substeps=200, reorth=True)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.1, 0.1, 5, scheme=scheme, tol=1e-12, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY and st["n_applies"] == na
    t2 = _dev(torch_cuda, psi0)
    prop.propagate(t2, 0.1, 0.1, 5, scheme=scheme, tol=1e-12)
    assert np.linalg.norm(t2.cpu().numpy() - ref) <= PARITY


def test_reorth_atom_matches_oracle(torch_cuda):
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=120, L=8)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive], m_max=40,
                        max_substeps=4000, precision="f64", reorth=True)
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    psi0, _ = W.atom_ground_state(p)
    ref, log, _ = OC.propagate(op, psi0, 300.0, 0.1, 2, 8, [p.drive], 1e-10, 40, return_log=True,
                               max_substeps=4000, reorth=True)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 300.0, 0.1, 2, order=8, tol=1e-10, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY


@pytest.mark.parametrize("reorth", [False, True])
def test_outlier_spectrum_both_modes_meet_the_tolerance(torch_cuda, reorth):
    # diag(lam) with outliers at 50, 100, 200 over a dense [0, 1] part: the
    # plain recurrence loses orthogonality at large k (pinned in the oracle);
    # with m = 60 and a long step both modes still reach the exact result
    import paper_1102_5071_gb300 as P
    lam = np.concatenate([np.linspace(0.0, 1.0, 300), [50.0, 100.0, 200.0]])
    prop = P.Propagator(P.DIA(np.array([0]), lam[None, :]), [], [], m_max=60, max_substeps=50, precision="f64",
                        reorth=reorth)
    psi0 = W.random_state(4, len(lam))
    t = _dev(torch_cuda, psi0)
    prop.expv(np.array([1.0]), 0.05, t, 1e-12)
    assert np.linalg.norm(t.cpu().numpy() - np.exp(-1j * 0.05 * lam) * psi0) <= PARITY


def test_reorth_pauli_sum_matches_oracle(torch_cuda):
    import paper_1102_5071_gb300 as P
    N = 7
    terms = [(0.8, {i: "X", i + 1: "Y"}) for i in range(N - 1)] + [(0.3 * (i + 1), {i: "Z"}) for i in range(N)]
    prop = P.Propagator(P.PauliSum(N, terms), [P.PauliSum(N, [(1.0, {i: "Y"}) for i in range(N)])],
                        [lambda t: math.cos(t)], m_max=24, reorth=True)
    op = O.PauliSum(N, terms, [[(1.0, {i: "Y"}) for i in range(N)]])
    psi0 = W.random_state(9, 1 << N)
    ref, log, _ = OC.propagate(op, psi0, 0.0, 0.1, 6, 6, [lambda t: math.cos(t)], 1e-12, 24, return_log=True,
                               reorth=True)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 0.0, 0.1, 6, order=6, tol=1e-12, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY
