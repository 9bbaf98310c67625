"""Propagations split over several persistent launches (steps_per_launch
smaller than nsteps) against one launch and against the oracle, for every
kernel: fixed point (Krylov and Chebyshev), complex64, FP64 and the FP64
interaction picture.  Each launch converts psi in and out of its format and
continues the exchange tags of the previous one."""

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, chebyshev as CH, interaction as IP, operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1102_5071_gb300.build import build
    build()
    return torch


CASES = [
    dict(precision="fx", expm="krylov", picture="schroedinger", tol=1e-10),
    dict(precision="fx", expm="chebyshev", picture="schroedinger", tol=1e-10),
    dict(precision="c64", expm="krylov", picture="schroedinger", tol=1.5e-4),   # 35 substeps x 64 x 2^-24
    dict(precision="f64", expm="krylov", picture="schroedinger", tol=1e-10),
    dict(precision="f64", expm="krylov", picture="interaction", tol=1e-10),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['precision']}-{c['expm']}-{c['picture']}")
def test_chunked_launches_match_one_launch_and_the_oracle(torch_cuda, case):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N = 10
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])

    def make(spl):
        return P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=16,
                            steps_per_launch=spl, precision=case["precision"], expm=case["expm"],
                            picture=case["picture"])

    psi0 = W.random_state(8, 1 << N)
    nsteps, dt, order, tol = 7, 0.03, 6, 1e-11
    outs = []
    for spl in (256, 2, 1):
        prop = make(spl)
        x = torch.from_numpy(psi0).cuda()
        st = prop.propagate(x, 0.2, dt, nsteps, order=order, tol=tol)
        assert st["n_exp"] == nsteps * 5
        outs.append(x.cpu().numpy())
        prop.close()
    for o in outs[1:]:
        assert np.linalg.norm(o - outs[0]) <= (1e-6 if case["precision"] == "c64" else 1e-13)
    if case["expm"] == "chebyshev":
        ref = CH.propagate(op, psi0, 0.2, dt, nsteps, order, [pr.drive], tol)
    elif case["picture"] == "interaction":
        ref = IP.propagate(op, psi0, 0.2, dt, nsteps, order, [pr.drive], tol, 16)
    else:
        ref = OC.propagate(op, psi0, 0.2, dt, nsteps, order, [pr.drive], tol, 16)
    for o in outs:
        assert np.linalg.norm(o - ref) <= case["tol"]
