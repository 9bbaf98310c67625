"""Bounded device waits: a grid-wide wait that one CTA never joins must give
up after its limit with CFET_ETIMEOUT, without a fault or a hang, and the
device must stay usable (failure detection tested by a flag nothing sets)."""

import ctypes as C
import time

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, operators as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1102_5071_gb300.build import build
    build()
    return torch


@pytest.mark.parametrize("which", [0, 1])
def test_wait_gives_up_with_etimeout(torch_cuda, which):
    from paper_1102_5071_gb300 import _capi
    lib = _capi.load()
    st = C.c_int32(-1)
    t = time.perf_counter()
    rc = lib.cfet_selftest_wait_timeout(which, 0.2, C.byref(st))
    el = time.perf_counter() - t
    assert rc == _capi.CFET_OK and st.value == _capi.CFET_ETIMEOUT
    assert 0.15 < el < 5.0
    # the device is still usable
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(6)
    prop = P.Propagator(P.XXZChain(6, pr.J, pr.Delta, pr.h), [P.XField(6, pr.xfield)], [pr.drive])
    psi0 = W.random_state(1, 64)
    x = torch_cuda.from_numpy(psi0).cuda()
    prop.propagate(x, 0.0, 0.05, 4, order=4, tol=1e-12)
    ref = OC.propagate(O.SpinChain(6, pr.J, pr.Delta, pr.h, [pr.xfield]), psi0, 0.0, 0.05, 4, 4, [pr.drive],
                       1e-12, 16)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-10
