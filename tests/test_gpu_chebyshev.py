"""GPU parity of the Chebyshev stage exponentials (CFET_EXPM_CHEBYSHEV, the
fixed-point kernel k_cheb_fx) against the oracle's Chebyshev propagator.

Both sides use the same spectral interval (Gershgorin intervals combined by
Weyl's inequality), the same truncation rule and the same series; they differ
only by rounding (fixed point with a 2^-52 relative unit against FP64) and by
the Bessel values (Miller's recurrence against scipy, both ~1e-15 here), so
||psi_gpu - psi_oracle||_2 <= 1e-10 is required as for the Krylov path.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import chebyshev as CH, operators as O

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


def _spin(N, nfields=1, J=1.0, Delta=0.5, **kw):
    import paper_1102_5071_gb300 as P
    pr = W.spin_chain(N, J=J, Delta=Delta)
    fields = [pr.xfield] + [W.uniform(100 + k, N, -1, 1) for k in range(1, nfields)]
    drives = [pr.drive] + [(lambda t, k=k: 0.3 * math.sin((k + 1) * t)) for k in range(1, nfields)]
    prop = P.Propagator(P.XXZChain(N, J, Delta, pr.h), [P.XField(N, a) for a in fields], drives,
                        expm="chebyshev", **kw)
    return prop, O.SpinChain(N, J, Delta, pr.h, fields), drives


def _compare(torch, prop, op, drives, psi0, t0, dt, nsteps, scheme, tol):
    ref, ost = CH.propagate(op, psi0, t0, dt, nsteps, scheme, drives, tol, return_stats=True)
    kw = dict(scheme=scheme) if isinstance(scheme, str) else dict(order=scheme)
    x = _dev(torch, psi0)
    st = prop.propagate(x, t0, dt, nsteps, tol=tol, **kw)
    return np.linalg.norm(x.cpu().numpy() - ref), st, ost


def test_cheb_chain_n8(torch_cuda):
    cfg = W.CHAIN_SMALL
    prop, op, drives = _spin(cfg["N"], m_max=16)
    err, st, ost = _compare(torch_cuda, prop, op, drives, W.neel_state(cfg["N"]), 0.0, cfg["dt"], 100, 4, 1e-12)
    assert err <= PARITY, err
    assert st["n_applies"] == ost["n_applies"] and st["max_k"] == max(ost["K"])
    assert st["n_exp"] == st["n_substeps"] == 200


@pytest.mark.parametrize("scheme", ["CF2:1", "CF4:2", "CF4:3Opt", "CF6:4", "CF6:5Opt", "CF8:11"])
def test_cheb_schemes_two_fields(torch_cuda, scheme):
    # two drive operators with site-dependent fields (the per-site table path);
    # CF6:4 has an all-zero stage (K = 0, identity)
    prop, op, drives = _spin(9, nfields=2, m_max=20)
    err, st, ost = _compare(torch_cuda, prop, op, drives, W.random_state(5, 1 << 9), 0.37, 0.05, 6, scheme, 1e-10)
    assert err <= PARITY, err
    assert st["n_applies"] == ost["n_applies"]


def test_cheb_long_step_many_terms(torch_cuda):
    # dt = 0.6: tau * a ~ 10, over 20 terms per exponential
    prop, op, drives = _spin(10, m_max=16, max_substeps=16)
    err, st, ost = _compare(torch_cuda, prop, op, drives, W.random_state(6, 1 << 10), 0.0, 0.6, 3, 6, 1e-11)
    assert err <= PARITY, err
    assert st["max_k"] >= 20


def test_cheb_chain_n20_one_step(torch_cuda):
    prop, op, drives = _spin(20)
    err, st, ost = _compare(torch_cuda, prop, op, drives, W.random_state(2, 1 << 20), 0.0, 0.05, 1, 4, 1e-10)
    assert err <= PARITY, err


def test_cheb_full_size_chain_zero_coupling_factorises(torch_cuda):
    # N = 20, J = Delta = 0: the chain is a product of driven single spins whose
    # exact CFET propagation (oracle, dense 2x2 Krylov at 1e-14) gives every
    # amplitude; sampled amplitudes are bounded by the 2-norm of the error
    import paper_1102_5071_gb300 as P
    from oracle import cfet as OC
    N = 20
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, pr.xfield)], [pr.drive], expm="chebyshev")
    psi0 = W.neel_state(N)
    nsteps, dt = 40, 0.05
    x = _dev(torch_cuda, psi0)
    prop.propagate(x, 0.0, dt, nsteps, order=6, tol=1e-12)
    out = x.cpu().numpy()
    x0 = int(np.argmax(np.abs(psi0)))
    single = []
    for i in range(N):
        e = np.zeros(2, dtype=np.complex128)
        e[(x0 >> i) & 1] = 1.0
        single.append(OC.propagate(O.Dense(pr.h[i] * O.SZ, [O.SX]), e, 0.0, dt, nsteps, 6, [pr.drive], 1e-14, 2))
    idx = np.random.default_rng(0).integers(0, 1 << N, 4000)
    amp = np.ones(len(idx), dtype=np.complex128)
    for i in range(N):
        amp *= np.where((idx >> i) & 1, single[i][1], single[i][0])
    assert np.max(np.abs(out[idx] - amp)) <= 1e-9   # 240 exponentials at 1e-12 + CFET agreement of both
    assert abs(np.linalg.norm(out) - 1.0) <= 1e-10


def test_cheb_time_independent_matches_expm(torch_cuda):
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    N = 9
    pr = W.spin_chain(N)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [lambda t: 0.0],
                        expm="chebyshev")
    psi0 = W.random_state(4, 1 << N)
    x = _dev(torch_cuda, psi0)
    st = prop.propagate(x, 0.0, 0.1, 5, order=8, tol=1e-12)
    ref = expm(-1j * 0.5 * O.xxz_dense(N, pr.J, pr.Delta, pr.h)) @ psi0
    assert np.linalg.norm(x.cpu().numpy() - ref) <= st["n_exp"] * 1e-12 + 1e-12


def test_cheb_atom_reduced(torch_cuda):
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=120, L=8)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=64, max_substeps=4000, expm="chebyshev")
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    psi0, _ = W.atom_ground_state(p)
    err, st, ost = _compare(torch_cuda, prop, op, [p.drive], psi0, 300.0, 0.1, 2, 8, 1e-10)
    assert err <= PARITY, (err, st["max_k"])
    assert st["n_applies"] == ost["n_applies"]


def test_cheb_atom_long_expansion(torch_cuda):
    # a stiffer grid (l < 20, H0 up to ~2e4): about 500 terms per exponential,
    # where rounding in the recurrence would show (each vector keeps its own
    # exponent from its measured maximum)
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=400, L=20)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=64, max_substeps=4000, expm="chebyshev")
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    psi0, _ = W.atom_ground_state(p)
    err, st, ost = _compare(torch_cuda, prop, op, [p.drive], psi0, 500.0, 0.1, 1, 8, 1e-10)
    assert st["max_k"] >= 400
    assert err <= PARITY, err


def test_cheb_expv_matches_oracle(torch_cuda):
    prop, op, drives = _spin(11, nfields=2)
    c = np.array([0.8, -0.35, 0.2])
    psi0 = W.random_state(9, 1 << 11)
    lo, hi = CH.stage_interval(CH.operator_intervals(op), c)
    ref, na, K, tail = CH.expv(lambda v: op.apply(c, v), psi0, 0.7, lo, hi, 1e-11)
    x = _dev(torch_cuda, psi0)
    st = prop.expv(c, 0.7, x, tol=1e-11)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= PARITY
    assert st["n_applies"] == na and st["max_k"] == K


def test_cheb_host_entry_and_relaunch(torch_cuda):
    prop, op, drives = _spin(12)
    psi0 = W.random_state(3, 1 << 12)
    x = _dev(torch_cuda, psi0)
    prop.propagate(x, 0.0, 0.02, 5, order=6, tol=1e-10)
    h = psi0.copy()
    prop.propagate_host(h, 0.0, 0.02, 5, order=6, tol=1e-10)
    assert np.array_equal(h, x.cpu().numpy())
    y = _dev(torch_cuda, psi0)                      # the same call again: cached graph
    prop.propagate(y, 0.0, 0.02, 5, order=6, tol=1e-10)
    assert torch_cuda.equal(x, y)


def test_cheb_edge_cases(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, op, drives = _spin(6)
    psi0 = W.random_state(1, 64)
    x = _dev(torch, psi0)
    st = prop.propagate(x, 0.0, 0.1, 0, order=4)
    assert np.array_equal(x.cpu().numpy(), psi0) and st["n_exp"] == 0
    z = torch.zeros(64, dtype=torch.complex128, device="cuda")
    prop.propagate(z, 0.0, 0.1, 2, order=6)
    assert torch.count_nonzero(z).item() == 0
    bad = _dev(torch, psi0)
    bad[3] = complex(float("nan"), 0.0)
    with pytest.raises(P.CfetError, match="ENAN"):
        prop.propagate(bad, 0.0, 0.1, 1, order=4)
    with pytest.raises(P.CfetError, match="EINVAL"):          # no decision logs
        prop.propagate(_dev(torch, psi0), 0.0, 0.1, 1, order=4, record=True)
    small, _, _ = _spin(6, m_max=2, max_substeps=2)           # at most 4 terms
    with pytest.raises(P.CfetError, match="EKRYLOV"):
        small.propagate(_dev(torch, psi0), 0.0, 2.0, 1, order=4, tol=1e-12)
    # spectrum far from zero relative to its width: |b| > 1.5 a
    dim = 32
    vals = np.vstack([np.full(dim, 10.0), np.full(dim, 0.1), np.full(dim, 0.1)])
    far = P.Propagator(P.DIA(np.array([0, 1, -1]), vals), [], [], expm="chebyshev")
    with pytest.raises(P.CfetError, match="EINVAL"):
        far.propagate(_dev(torch, W.random_state(2, dim)), 0.0, 0.1, 1, order=4)
    x = _dev(torch, psi0)
    prop.propagate(x, 0.0, 0.1, 1, order=4)                   # the context stays usable
    with pytest.raises(P.CfetError, match="EINVAL"):
        prop.fidelity_grad(x, x, 0.0, 0.1, 4, [0.1, 0.2], 2.0)
    # a single spin
    prop1, op1, dr1 = _spin(1)
    e = _dev(torch, np.array([0.6, 0.8j]))
    prop1.propagate(e, 0.0, 0.05, 10, order=8, tol=1e-12)
    ref = CH.propagate(op1, np.array([0.6, 0.8j]), 0.0, 0.05, 10, 8, dr1, 1e-12)
    assert np.linalg.norm(e.cpu().numpy() - ref) <= PARITY
