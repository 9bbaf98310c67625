"""GPU parity of the staged apply of the fixed-point kernel (apply_form
"staged": each CTA's contiguous chunk of the current Krylov vector is also held
in shared memory, written by the pass that produced the vector, and
neighbours inside the chunk are read from there).

The neighbour sums of the fixed-point apply are exact integer additions and
every product is taken as in the element-wise form, so the staged and the
element-wise form must give bit-identical results for the same decisions; and
both must match the oracle within ||psi_gpu - psi_oracle||_2 <= 1e-10 (Sec.
8.1 Krylov exponentials, Eq. (Ucf) stepping).  Grid sizes that make chunk
boundaries fall at odd indices exercise the inside / outside test of every
neighbour; a single CTA holds the whole vector.
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


def _spin(N, nfields=1, **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N)
    fields = [pr.xfield] + [W.uniform(100 + k, N, -1, 1) for k in range(1, nfields)]
    drives = [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)]
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, a) for a in fields], drives,
                        precision="fx", **kw)
    return prop, O.SpinChain(N, pr.J, pr.Delta, pr.h, fields), drives


@pytest.mark.parametrize("N,nfields,grid", [(10, 1, 1), (12, 2, 7), (13, 1, 0), (15, 2, 19), (16, 1, 0)])
def test_staged_matches_oracle(torch_cuda, N, nfields, grid):
    torch = torch_cuda
    prop, op, drives = _spin(N, nfields, m_max=16, max_substeps=200, apply_form="staged", grid_size=grid)
    psi0 = W.random_state(11 + N, 1 << N)
    ref, log, na = OC.propagate(op, psi0, 0.2, 0.05, 2, "CF6:5Opt", drives, 1e-11, 16, return_log=True,
                                max_substeps=200)
    t = torch.from_numpy(psi0).cuda()
    st = prop.propagate(t, 0.2, 0.05, 2, scheme="CF6:5Opt", tol=1e-11, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY and st["n_applies"] == na
    t2 = torch.from_numpy(psi0).cuda()
    st2, log2 = prop.propagate(t2, 0.2, 0.05, 2, scheme="CF6:5Opt", tol=1e-11, record=True)
    assert sum(a == b for a, b in zip(log, log2)) / len(log) >= 0.95
    assert np.linalg.norm(t2.cpu().numpy() - ref) <= PARITY
    prop.close()


@pytest.mark.parametrize("N,grid", [(20, 0), (18, 100), (14, 3)])
def test_staged_is_bit_identical_to_elementwise(torch_cuda, N, grid):
    # the benchmark chain size and odd chunkings: same decisions, same bits
    torch = torch_cuda
    psi0 = W.random_state(2, 1 << N)
    outs, log = {}, None
    for form in ("elementwise", "staged"):
        prop, _, _ = _spin(N, 1, m_max=16, max_substeps=64, apply_form=form, grid_size=grid)
        x = torch.from_numpy(psi0).cuda()
        if log is None:
            _, log = prop.propagate(x, 0.0, 0.02, 3, order=6, tol=1e-10, record=True)
        else:
            prop.propagate(x, 0.0, 0.02, 3, order=6, tol=1e-10, forced=log)
        outs[form] = x.cpu().numpy()
        prop.close()
    assert np.array_equal(outs["staged"], outs["elementwise"])


def test_staged_zero_coupling_factorises_n20(torch_cuda):
    # J = 0 at full size with two site-dependent fields (the per-site table
    # path of the staged apply): product of single-spin propagations
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    N = 20
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    a1, a2 = W.uniform(21, N, 0.5, 1.5), W.uniform(22, N, -1, 1)

    def g(t):
        return 0.4 * math.sin(0.9 * t)

    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, a1), P.XField(N, a2)], [pr.drive, g],
                        m_max=16, precision="fx", apply_form="staged")
    psi0 = W.neel_state(N)
    nsteps, dt = 20, 0.05
    x = torch.from_numpy(psi0).cuda()
    prop.propagate(x, 0.0, dt, nsteps, order=6, tol=1e-13)
    out = x.cpu().numpy()
    x0 = int(np.argmax(np.abs(psi0)))
    single = []
    for i in range(N):
        e = np.zeros(2, dtype=np.complex128)
        e[(x0 >> i) & 1] = 1.0
        single.append(OC.propagate(O.Dense(pr.h[i] * O.SZ, [a1[i] * O.SX, a2[i] * O.SX]), e, 0.0, dt, nsteps, 6,
                                   [pr.drive, g], 1e-14, 2))
    idx = np.random.default_rng(2).integers(0, 1 << N, 4000)
    amp = np.ones(len(idx), dtype=np.complex128)
    for i in range(N):
        amp *= np.where((idx >> i) & 1, single[i][1], single[i][0])
    assert np.max(np.abs(out[idx] - amp)) < 1e-12
    prop.close()
