"""The allocation-free entry point cfet_expv_chain_static against cfet_expv.

cfet_expv_chain_static serves callers that cannot allocate device memory (all
of it owned by another allocator or a fixed budget, or loops that must not
take cudaMalloc's implicit synchronisation); its scratch lives in a static
device array shared by every call.  This test calls it through the C ABI twice
in a row (different states and step lengths, so the second call starts from
the first call's leftover scratch) and compares each result with the
context-based cfet_expv on the same operator, within the parity tolerance of
the GPU tests (||psi_a - psi_b||_2 <= 1e-10).  The file is named so that pytest
collects it last.
"""

import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_entry_matches_context_entry():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_1102_5071_gb300 as P
    from paper_1102_5071_gb300 import _capi
    P.build()
    lib = _capi.load()
    N = 10
    pr = W.spin_chain(N)
    a = W.uniform(31, N, 0.5, 1.5)
    h = np.ascontiguousarray(pr.h, dtype=np.float64)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, h), [P.XField(N, a)], [pr.drive], m_max=16)
    cases = [(0.9, 0.35, 0.05, 1e-12, 5), (-0.4, 1.2, 0.7, 1e-10, 6)]
    for c0, c1, tau, tol, seed in cases:
        psi0 = W.random_state(seed, 1 << N)
        ref = torch.from_numpy(psi0).cuda()
        prop.expv(np.array([c0, c1]), tau, ref, tol)
        out = torch.from_numpy(psi0).cuda()
        torch.cuda.synchronize()
        st = _capi.cfet_stats()
        rc = lib.cfet_expv_chain_static(N, pr.J, pr.Delta, h.ctypes.data_as(_capi.c_double_p),
                                        a.ctypes.data_as(_capi.c_double_p), c0, c1, tau,
                                        C.c_void_p(out.data_ptr()), tol, 16,
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(st))
        assert rc == 0, rc
        assert st.n_exp == 1 and st.n_applies > 0
        err = torch.linalg.vector_norm(out - ref).item()
        assert err <= 1e-10, err
    # sizes beyond the static limits are rejected
    big = torch.zeros(1 << 13, dtype=torch.complex128, device="cuda")
    hb = np.zeros(13)
    assert lib.cfet_expv_chain_static(13, 1.0, 0.5, hb.ctypes.data_as(_capi.c_double_p),
                                      hb.ctypes.data_as(_capi.c_double_p), 1.0, 0.0, 0.1,
                                      C.c_void_p(big.data_ptr()), 1e-10, 16, None, None) == _capi.CFET_EINVAL
    assert lib.cfet_expv_chain_static(N, 1.0, 0.5, h.ctypes.data_as(_capi.c_double_p),
                                      a.ctypes.data_as(_capi.c_double_p), 1.0, 0.0, 0.1,
                                      C.c_void_p(out.data_ptr()), 1e-10, 33, None, None) == _capi.CFET_EINVAL
    prop.close()
