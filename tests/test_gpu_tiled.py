"""GPU parity of the window-tiled apply of the fixed-point kernel (long XXZ
chains; tiles of 2^11 elements, one pass per window of index bits; two
windows for 12..18 sites, three for 19..25, four for 26..32).  The
option apply_form forces the tiled or the element-wise form (the default
takes the tiled form from 23 sites).

Tolerances as in test_gpu_parity.py: ||psi_gpu - psi_oracle||_2 <= 1e-10 with
the oracle's Krylov decisions replayed; the tiled and element-wise forms
differ only by the rounding of one extra product per sum and window (units
of 2^-57 relative), far below 1e-12 over a few steps.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, operators as O

pytestmark = pytest.mark.gpu

PARITY = 1e-10
FORMS = {"0": "elementwise", "1": "tiled"}


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


def _spin(N, nfields=1, J=1.0, Delta=0.5, **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N, J=J, Delta=Delta)
    fields = [pr.xfield] + [W.uniform(100 + k, N, -1, 1) for k in range(1, nfields)]
    drives = [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)]
    prop = P.Propagator(P.XXZChain(N, J, Delta, pr.h), [P.XField(N, a) for a in fields], drives, precision="fx",
                        **kw)
    return prop, O.SpinChain(N, J, Delta, pr.h, fields), drives


@pytest.mark.parametrize("N,nfields", [(13, 1), (14, 2), (16, 1)])
def test_fx_tiled_matches_oracle(torch_cuda, N, nfields):
    # two windows; forced (the oracle's decisions) and adaptive runs
    prop, op, drives = _spin(N, nfields=nfields, m_max=16, max_substeps=200, apply_form="tiled")
    psi0 = W.random_state(11, 1 << N)
    ref, log, na = OC.propagate(op, psi0, 0.2, 0.05, 2, "CF6:5Opt", drives, 1e-11, 16, return_log=True,
                                max_substeps=200)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.2, 0.05, 2, scheme="CF6:5Opt", tol=1e-11, forced=log)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY and st["n_applies"] == na
    t2 = _dev(torch_cuda, psi0)
    _, log2 = prop.propagate(t2, 0.2, 0.05, 2, scheme="CF6:5Opt", tol=1e-11, record=True)
    assert np.linalg.norm(t2.cpu().numpy() - ref) <= PARITY
    assert sum(a == b for a, b in zip(log, log2)) / len(log) >= 0.95


@pytest.mark.parametrize("N,nfields", [(19, 2), (20, 1)])
def test_fx_tiled_three_windows_match_oracle(torch_cuda, N, nfields):
    # three windows (19 sites with site-dependent fields; 20 sites, the
    # benchmark chain): one CF4:2 step with a fixed Krylov dimension 10
    prop, op, drives = _spin(N, nfields=nfields, m_max=10, apply_form="tiled")
    psi0 = W.random_state(2, 1 << N)
    ref = OC.propagate(op, psi0, 0.0, 0.05, 1, 4, drives, 0.0, 10)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 0.0, 0.05, 1, order=4, tol=0.0)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= PARITY


def _one_magnon_hamiltonian(N, J, Delta, h):
    # the XXZ chain restricted to the states with one spin down (bit k set):
    # diagonal J Delta sum_i z_i z_{i+1} + sum_i h_i z_i with z_k = -1, and the
    # exchange term moves the down spin by one site with amplitude 2J
    H = np.zeros((N, N))
    for k in range(N):
        z = np.ones(N)
        z[k] = -1.0
        H[k, k] = J * Delta * np.dot(z[:-1], z[1:]) + np.dot(h, z)
        if k + 1 < N:
            H[k, k + 1] = H[k + 1, k] = 2.0 * J
    return H


@pytest.mark.parametrize("N", [22, 26])
def test_fx_tiled_one_magnon_sector_is_exact(torch_cuda, N):
    # without an x field the one-magnon sector is closed: 22 sites (three
    # windows) and 26 sites (four) started with one spin down follow the N x N
    # problem to the Krylov tolerance, every other amplitude stays exactly zero
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    h6 = W.uniform(3, 6, -1, 1)
    idx6 = [1 << k for k in range(6)]
    assert np.allclose(O.xxz_dense(6, 0.8, 0.6, h6)[np.ix_(idx6, idx6)], _one_magnon_hamiltonian(6, 0.8, 0.6, h6),
                       atol=1e-14)
    J, Dl = 0.8, 0.6
    h = W.uniform(4, N, -1, 1)
    prop = P.Propagator(P.XXZChain(N, J, Dl, h), [P.XField(N, np.zeros(N))], [lambda t: 0.0], m_max=20,
                        max_substeps=400, precision="fx", apply_form="tiled")
    k0, T = N // 2 - 1, 2.0
    psi0 = np.zeros(1 << N, dtype=np.complex128)
    psi0[1 << k0] = 1.0
    x = _dev(torch_cuda, psi0)
    st = prop.propagate(x, 0.0, 0.25, 8, order=4, tol=1e-12)
    out = x.cpu().numpy()
    e = np.zeros(N)
    e[k0] = 1.0
    ref = expm(-1j * T * _one_magnon_hamiltonian(N, J, Dl, h)) @ e
    sector = np.array([1 << k for k in range(N)])
    bound = st["n_substeps"] * 1e-12 + 1e-12
    assert np.linalg.norm(out[sector] - ref) <= bound, (np.linalg.norm(out[sector] - ref), bound)
    rest = out.copy()
    rest[sector] = 0.0
    assert np.linalg.norm(rest) == 0.0


def test_fx_tiled_zero_coupling_factorises_n22(torch_cuda):
    # J = 0 with two site-dependent x fields: 22 sites (three windows)
    # factorise into driven two-level systems; sampled amplitudes against the
    # product of the oracle's single-site propagations
    import paper_1102_5071_gb300 as P
    N = 22
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    a1, a2 = W.uniform(21, N, 0.5, 1.5), W.uniform(22, N, -1, 1)

    def g(t):
        return 0.4 * math.sin(0.9 * t)

    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, a1), P.XField(N, a2)], [pr.drive, g],
                        m_max=16, precision="fx", apply_form="tiled")
    psi0 = W.neel_state(N)
    nsteps, dt = 30, 0.05
    x = _dev(torch_cuda, psi0)
    prop.propagate(x, 0.0, dt, nsteps, order=6, tol=1e-12)
    out = x.cpu().numpy()
    x0 = int(np.argmax(np.abs(psi0)))
    single = []
    for i in range(N):
        e = np.zeros(2, dtype=np.complex128)
        e[(x0 >> i) & 1] = 1.0
        single.append(OC.propagate(O.Dense(pr.h[i] * O.SZ, [a1[i] * O.SX, a2[i] * O.SX]), e, 0.0, dt, nsteps, 6,
                                   [pr.drive, g], 1e-14, 2))
    idx = np.random.default_rng(1).integers(0, 1 << N, 4000)
    amp = np.ones(len(idx), dtype=np.complex128)
    for i in range(N):
        amp *= np.where((idx >> i) & 1, single[i][1], single[i][0])
    assert np.max(np.abs(out[idx] - amp)) <= PARITY
    assert abs(np.linalg.norm(out) - 1.0) <= PARITY


def test_fx_tiled_matches_elementwise_n23(torch_cuda):
    # the driven chain of 23 sites: the element-wise run's decisions replayed
    # by the tiled form; the two results agree far below the parity bound
    N = 23
    psi0 = W.random_state(12, 1 << N)
    out = {}
    log = None
    for flag in ("0", "1"):
        prop, _, _ = _spin(N, m_max=16, max_substeps=200, apply_form=FORMS[flag])
        x = _dev(torch_cuda, psi0)
        if log is None:
            _, log = prop.propagate(x, 0.1, 0.04, 2, order=6, tol=1e-10, record=True)
        else:
            prop.propagate(x, 0.1, 0.04, 2, order=6, tol=1e-10, forced=log)
        out[flag] = x.cpu().numpy()
        prop.close()
    assert np.linalg.norm(out["1"] - out["0"]) <= 1e-12
