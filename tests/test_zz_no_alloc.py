"""The allocation-free entry point cfet_expv_chain_static against the oracle
and against cfet_expv.

cfet_expv_chain_static serves callers that cannot allocate device memory (all
of it owned by another allocator or a fixed budget, or loops that must not
take cudaMalloc's implicit synchronisation); its scratch lives in a static
device array shared by every call.  At each size this test calls it through
the C ABI twice in a row (different states, scalars and step lengths, so the
second call starts from the first call's leftover scratch) and compares each
result with the oracle's Lanczos exponential (oracle.krylov.expv on the
oracle's chain operator) and with the context-based cfet_expv on the same
operator, within the parity tolerance of the GPU tests
(||psi_a - psi_b||_2 <= 1e-10).  The sizes cover a chain shorter than the
diagonal table's low part (5 sites), the exact fit (10 sites) and the largest
accepted size (12 sites: the full basis region with m_max = 32).  The file is
named so that pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import krylov as OK, operators as O

pytestmark = pytest.mark.gpu

PARITY = 1e-10

# (sites, m_max, [(c0, c1, tau, tol, state seed), (...)]): two calls per size
CASES = [
    (5, 16, [(0.9, 0.35, 0.3, 1e-12, 5), (-0.4, 1.2, 0.7, 1e-10, 6)]),
    (10, 16, [(0.9, 0.35, 0.05, 1e-12, 5), (-0.4, 1.2, 0.7, 1e-10, 6)]),
    (12, 32, [(1.1, -0.6, 1.6, 1e-12, 7), (0.5, 0.9, 0.9, 1e-11, 8)]),
]


@pytest.mark.parametrize("N,m_max,calls", CASES)
def test_static_scratch_entry_matches_oracle_and_context_entry(N, m_max, calls):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_1102_5071_gb300 as P
    from paper_1102_5071_gb300 import _capi
    P.build()
    lib = _capi.load()
    pr = W.spin_chain(N)
    a = W.uniform(31, N, 0.5, 1.5)
    h = np.ascontiguousarray(pr.h, dtype=np.float64)
    op = O.SpinChain(N, pr.J, pr.Delta, h, [a])
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, h), [P.XField(N, a)], [pr.drive], m_max=m_max)
    kmax = 0
    for c0, c1, tau, tol, seed in calls:
        psi0 = W.random_state(seed, 1 << N)
        want, _, _ = OK.expv(lambda v: op.apply([c0, c1], v), psi0, tau, tol, m_max)
        ref = torch.from_numpy(psi0).cuda()
        prop.expv(np.array([c0, c1]), tau, ref, tol)
        out = torch.from_numpy(psi0).cuda()
        torch.cuda.synchronize()
        st = _capi.cfet_stats()
        rc = lib.cfet_expv_chain_static(N, pr.J, pr.Delta, h.ctypes.data_as(_capi.c_double_p),
                                        a.ctypes.data_as(_capi.c_double_p), c0, c1, tau,
                                        C.c_void_p(out.data_ptr()), tol, m_max,
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(st))
        assert rc == 0, rc
        assert st.n_exp == 1 and st.n_applies > 0
        kmax = max(kmax, st.max_k)
        got = out.cpu().numpy()
        assert np.linalg.norm(got - want) <= PARITY, np.linalg.norm(got - want)
        assert torch.linalg.vector_norm(out - ref).item() <= PARITY
    if m_max == 32:
        assert kmax > 16   # the upper half of the basis region is used
    prop.close()


def test_static_scratch_entry_rejects_sizes_beyond_its_limits():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_1102_5071_gb300 as P
    from paper_1102_5071_gb300 import _capi
    P.build()
    lib = _capi.load()
    big = torch.zeros(1 << 13, dtype=torch.complex128, device="cuda")
    hb = np.zeros(13)
    assert lib.cfet_expv_chain_static(13, 1.0, 0.5, hb.ctypes.data_as(_capi.c_double_p),
                                      hb.ctypes.data_as(_capi.c_double_p), 1.0, 0.0, 0.1,
                                      C.c_void_p(big.data_ptr()), 1e-10, 16, None, None) == _capi.CFET_EINVAL
    assert lib.cfet_expv_chain_static(10, 1.0, 0.5, hb.ctypes.data_as(_capi.c_double_p),
                                      hb.ctypes.data_as(_capi.c_double_p), 1.0, 0.0, 0.1,
                                      C.c_void_p(big.data_ptr()), 1e-10, 33, None, None) == _capi.CFET_EINVAL
