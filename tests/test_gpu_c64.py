"""GPU parity of the mixed-precision path (complex64 Krylov vectors, FP32
apply, compensated FP64-class reductions, FP64 scalars) against the FP64
oracle.

Tolerance.  The method is the oracle's; only the storage and arithmetic of
the vectors change.  Per Krylov substep the result is a combination
beta0 sum_i y_i s_i q_i of k stored vectors (k <= m_max), each produced by at
most four FP32 roundings of relative size 2^-24 (store of psi, apply sum,
recurrence, store), weighted by y = exp(-i tau T_k) e_1 with ||y||_2 = 1, so
sum_i |y_i| <= sqrt(k); the combined result is rounded once more.  This
bounds the substep's relative error by (4 sqrt(k) + 1) 2^-24 (17 * 2^-24 for
k <= 16).  Unitary propagation does not amplify earlier errors, so they add at
most linearly over substeps:

    ||psi_c64 - psi_oracle||_2 <= n_substeps * (4 sqrt(m_max) + 1) * 2^-24 * ||psi0||.

(Measured errors are about 1.4 * 2^-24 per substep on the N = 20 chain.)

The oracle's Krylov decisions are replayed (forced mode) so that only
rounding is measured; adaptive runs must take the same decisions in at least
95 % of the stage exponentials.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import cfet as OC, operators as O

pytestmark = pytest.mark.gpu

ULP32 = 2.0 ** -24


FORMS = {"0": "elementwise", "1": "tiled"}


def budget(n_substeps, k=16):
    return n_substeps * (4.0 * math.sqrt(k) + 1.0) * ULP32


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
                        precision="c64", **kw)
    return prop, O.SpinChain(N, J, Delta, pr.h, fields), drives


def _run(torch, prop, op, drives, psi0, t0, dt, nsteps, scheme_or_order, tol, m):
    ref, log, _ = OC.propagate(op, psi0, t0, dt, nsteps, scheme_or_order, drives, tol, m, return_log=True,
                               max_substeps=4000)
    kw = dict(scheme=scheme_or_order) if isinstance(scheme_or_order, str) else dict(order=scheme_or_order)
    t = _dev(torch, psi0)
    st = prop.propagate(t, t0, dt, nsteps, tol=tol, forced=log, **kw)
    forced_err = np.linalg.norm(t.cpu().numpy() - ref)
    t2 = _dev(torch, psi0)
    _, log2 = prop.propagate(t2, t0, dt, nsteps, tol=tol, record=True, **kw)
    same = sum(a == b for a, b in zip(log, log2)) / len(log)
    return forced_err, same, st, np.linalg.norm(t2.cpu().numpy() - ref)


def test_c64_chain_n8(torch_cuda):
    cfg = W.CHAIN_SMALL
    prop, op, drives = _spin(cfg["N"], m_max=cfg["m_max"], max_substeps=200)
    err, same, st, aerr = _run(torch_cuda, prop, op, drives, W.neel_state(cfg["N"]), 0.0, cfg["dt"], 100, 4,
                               cfg["tol"], cfg["m_max"])
    assert err <= budget(st["n_substeps"]), (err, st["n_substeps"])
    assert same >= 0.95, same
    assert aerr <= budget(st["n_substeps"]) + 1e-9


@pytest.mark.parametrize("scheme", ["CF2:1", "CF4:2", "CF4:3Opt", "CF6:4", "CF6:5Opt", "CF8:11"])
def test_c64_schemes(torch_cuda, scheme):
    prop, op, drives = _spin(9, nfields=2, m_max=20, max_substeps=200)
    err, same, st, _ = _run(torch_cuda, prop, op, drives, W.random_state(5, 1 << 9), 0.37, 0.05, 6, scheme,
                            1e-9, 20)
    assert err <= budget(st["n_substeps"], 20), err
    assert same >= 0.95, same


def test_c64_substeps(torch_cuda):
    prop, op, drives = _spin(10, m_max=8, max_substeps=400)
    err, same, st, _ = _run(torch_cuda, prop, op, drives, W.random_state(6, 1 << 10), 0.0, 0.6, 3, 6, 1e-8, 8)
    assert st["n_substeps"] > st["n_exp"]
    assert err <= budget(st["n_substeps"], 8), err


def test_c64_fixed_krylov_dimension(torch_cuda):
    prop, op, drives = _spin(10, m_max=10)
    psi0 = W.random_state(8, 1 << 10)
    ref = OC.propagate(op, psi0, 0.0, 0.02, 15, 6, drives, 0.0, 10)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.0, 0.02, 15, order=6, tol=0.0)
    assert st["n_applies"] == 15 * 5 * 10
    assert np.linalg.norm(t.cpu().numpy() - ref) <= budget(st["n_substeps"], 10)


def test_c64_chain_n20_one_step(torch_cuda):
    prop, op, drives = _spin(20, m_max=10)
    psi0 = W.random_state(2, 1 << 20)
    ref = OC.propagate(op, psi0, 0.0, 0.05, 1, 4, drives, 0.0, 10)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.0, 0.05, 1, order=4, tol=0.0)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= budget(st["n_substeps"], 10)


def test_c64_chain_n20_zero_coupling_factorises(torch_cuda):
    import paper_1102_5071_gb300 as P
    N = 20
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, pr.xfield)], [pr.drive], m_max=16,
                        precision="c64")
    psi0 = W.neel_state(N)
    nsteps, dt = 40, 0.05
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.0, dt, nsteps, order=6, tol=1e-10)
    out = t.cpu().numpy()
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
    # every sampled amplitude is bounded by the 2-norm of the whole error
    assert np.max(np.abs(out[idx] - amp)) <= budget(st["n_substeps"])
    assert abs(np.linalg.norm(out) - 1.0) <= budget(st["n_substeps"])


def test_c64_time_independent_matches_expm(torch_cuda):
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    N = 9
    pr = W.spin_chain(N)
    prop = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [lambda t: 0.0],
                        m_max=30, precision="c64")
    psi0 = W.random_state(4, 1 << N)
    t = _dev(torch_cuda, psi0)
    st = prop.propagate(t, 0.0, 0.1, 5, order=8, tol=1e-9)
    ref = expm(-1j * 0.5 * O.xxz_dense(N, pr.J, pr.Delta, pr.h)) @ psi0
    # Krylov tolerance 1e-9 per substep plus the rounding budget
    assert np.linalg.norm(t.cpu().numpy() - ref) <= budget(st["n_substeps"], 30) + st["n_substeps"] * 1e-9


def test_c64_atom_reduced(torch_cuda):
    import paper_1102_5071_gb300 as P
    p = W.grid_atom(Nr=120, L=8)
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive], m_max=32,
                        max_substeps=4000, precision="c64")
    op = O.Banded((p.H0_offsets, p.H0_values), [(p.V_offsets, p.V_values)])
    psi0, _ = W.atom_ground_state(p)
    err, same, st, _ = _run(torch_cuda, prop, op, [p.drive], psi0, 300.0, 0.1, 2, 8, 1e-9, 32)
    assert err <= budget(st["n_substeps"], 32), (err, st["n_substeps"])


def test_c64_edge_cases(torch_cuda):
    torch = torch_cuda
    import paper_1102_5071_gb300 as P
    prop, op, drives = _spin(6)
    psi0 = W.random_state(1, 64)
    t = _dev(torch, psi0)
    st = prop.propagate(t, 0.0, 0.1, 0, order=4)
    assert np.array_equal(t.cpu().numpy(), psi0) and st["n_exp"] == 0
    z = torch.zeros(64, dtype=torch.complex128, device="cuda")
    prop.propagate(z, 0.0, 0.1, 2, order=6)
    assert torch.count_nonzero(z).item() == 0
    bad = _dev(torch, psi0)
    bad[3] = complex(float("nan"), 0.0)
    with pytest.raises(P.CfetError, match="ENAN"):
        prop.propagate(bad, 0.0, 0.1, 1, order=4)
    t = _dev(torch, psi0)
    prop.propagate(t, 0.0, 0.1, 1, order=4)   # the context stays usable
    prop1, op1, dr1 = _spin(1)
    e = _dev(torch, np.array([0.6, 0.8j]))
    st = prop1.propagate(e, 0.0, 0.05, 10, order=8, tol=1e-9)
    ref = OC.propagate(op1, np.array([0.6, 0.8j]), 0.0, 0.05, 10, 8, dr1, 1e-9, 16)
    assert np.linalg.norm(e.cpu().numpy() - ref) <= budget(st["n_substeps"])


def test_c64_host_entry_matches_device_entry(torch_cuda):
    prop, op, drives = _spin(12)
    psi0 = W.random_state(3, 1 << 12)
    t = _dev(torch_cuda, psi0)
    prop.propagate(t, 0.0, 0.02, 5, order=6, tol=1e-8)
    h = psi0.copy()
    prop.propagate_host(h, 0.0, 0.02, 5, order=6, tol=1e-8)
    assert np.array_equal(h, t.cpu().numpy())


def test_c64_full_size_atom_without_field_keeps_the_1s_state(torch_cuda):
    # stiff spectrum (H0 up to 5e5): the full-size grid atom with E0 = 0 keeps
    # its discrete 1s eigenstate up to the phase exp(-i E_1s t); the complex64
    # result must stay within single-precision rounding of it (a wrong beta
    # from cancellation would show up as a much larger error)
    import paper_1102_5071_gb300 as P
    a = W.ATOM
    p = W.grid_atom(Nr=a["Nr"], L=a["L"], dr=a["dr"], E0=0.0, omega=a["omega"], Tp=a["Tp"])
    prop = P.Propagator(P.DIA(p.H0_offsets, p.H0_values), [P.DIA(p.V_offsets, p.V_values)], [p.drive],
                        m_max=a["m_max"], max_substeps=4000, precision="c64")
    psi0, e1s = W.atom_ground_state(p)
    x = _dev(torch_cuda, psi0)
    st = prop.propagate(x, 500.0, a["dt"], 2, order=a["order"], tol=1e-9)
    ref = np.exp(-1j * e1s * a["dt"] * 2) * psi0
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-4, st


# ---------------------------------------------------------------- window-tiled apply
# Long chains take the window-tiled apply (shared-memory tiles of 2^12
# elements, one pass per window of index bits; the option apply_form forces it
# on or off).  Chains of
# 13..19 sites have two windows, 20..26 three, 27..30 four.

@pytest.mark.parametrize("N,nfields", [(13, 1), (14, 2), (16, 1), (17, 2)])
def test_c64_tiled_matches_oracle(torch_cuda, N, nfields):
    prop, op, drives = _spin(N, nfields=nfields, m_max=16, max_substeps=200, apply_form="tiled")
    err, same, st, aerr = _run(torch_cuda, prop, op, drives, W.random_state(11, 1 << N), 0.2, 0.05, 3, "CF6:5Opt",
                               1e-9, 16)
    assert err <= budget(st["n_substeps"]), (err, st["n_substeps"])
    assert same >= 0.95 and aerr <= budget(st["n_substeps"]) + 1e-9


def _one_magnon_hamiltonian(N, J, Delta, h):
    # XXZ chain (bit i of the index = site i, bit 1 = spin down) restricted to
    # the states with one spin down: site k down has the diagonal
    # J Delta sum_i z_i z_{i+1} + sum_i h_i z_i (z = +1 up, -1 down), and the
    # exchange term J (XX + YY) moves the down spin by one site with amplitude 2J
    H = np.zeros((N, N))
    for k in range(N):
        z = np.ones(N)
        z[k] = -1.0
        H[k, k] = J * Delta * np.dot(z[:-1], z[1:]) + np.dot(h, z)
        if k + 1 < N:
            H[k, k + 1] = H[k + 1, k] = 2.0 * J
    return H


@pytest.mark.parametrize("N", [22, 23, 27])
def test_c64_tiled_one_magnon_sector_is_exact(torch_cuda, N):
    # without an x field the one-magnon sector is closed: a chain of 22, 23
    # (three windows) or 27 sites (four) started with one spin down must follow the N x N
    # problem exactly and leave every other amplitude at zero; hops across all
    # window boundaries and the diagonal at every site enter
    from scipy.linalg import expm
    import paper_1102_5071_gb300 as P
    h6 = W.uniform(3, 6, -1, 1)
    H6 = O.xxz_dense(6, 0.8, 0.6, h6)
    idx6 = [1 << k for k in range(6)]
    assert np.allclose(H6[np.ix_(idx6, idx6)], _one_magnon_hamiltonian(6, 0.8, 0.6, h6), atol=1e-14)
    J, Dl = 0.8, 0.6
    h = W.uniform(4, N, -1, 1)
    prop = P.Propagator(P.XXZChain(N, J, Dl, h), [P.XField(N, np.zeros(N))], [lambda t: 0.0], m_max=24,
                        max_substeps=400, precision="c64", apply_form="tiled")
    k0, T = N // 2 - 1, 3.0
    psi0 = np.zeros(1 << N, dtype=np.complex128)
    psi0[1 << k0] = 1.0
    x = _dev(torch_cuda, psi0)
    st = prop.propagate(x, 0.0, 0.25, 12, order=4, tol=1e-9)
    out = x.cpu().numpy()
    e = np.zeros(N)
    e[k0] = 1.0
    ref = expm(-1j * T * _one_magnon_hamiltonian(N, J, Dl, h)) @ e
    sector = np.array([1 << k for k in range(N)])
    bound = budget(st["n_substeps"], 24) + st["n_substeps"] * 1e-9
    assert np.linalg.norm(out[sector] - ref) <= bound, (np.linalg.norm(out[sector] - ref), bound)
    rest = out.copy()
    rest[sector] = 0.0
    assert np.linalg.norm(rest) == 0.0


def test_c64_tiled_zero_coupling_factorises_n22(torch_cuda):
    # J = 0 with two site-dependent x fields: the chain of 22 sites (three
    # windows) factorises into driven two-level systems (flips of every bit,
    # per-site field coefficients, diagonal); sampled amplitudes against the
    # product of the oracle's single-site propagations
    import paper_1102_5071_gb300 as P
    N = 22
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    a1, a2 = W.uniform(21, N, 0.5, 1.5), W.uniform(22, N, -1, 1)

    def g(t):
        return 0.4 * math.sin(0.9 * t)

    prop = P.Propagator(P.XXZChain(N, 0.0, 0.0, pr.h), [P.XField(N, a1), P.XField(N, a2)], [pr.drive, g],
                        m_max=16, precision="c64", apply_form="tiled")
    psi0 = W.neel_state(N)
    nsteps, dt = 30, 0.05
    x = _dev(torch_cuda, psi0)
    st = prop.propagate(x, 0.0, dt, nsteps, order=6, tol=1e-10)
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
    assert np.max(np.abs(out[idx] - amp)) <= budget(st["n_substeps"])
    assert abs(np.linalg.norm(out) - 1.0) <= budget(st["n_substeps"])


def test_c64_tiled_matches_elementwise_and_fixed_point_n22(torch_cuda):
    # the driven chain of 22 sites: tiled and element-wise complex64 applies
    # replaying the fixed-point path's decisions agree within twice the
    # rounding budget, and each within the budget of the fixed-point result
    # (which matches the oracle to 1e-10 at the sizes the oracle reaches)
    import paper_1102_5071_gb300 as P
    N = 22
    pr = W.spin_chain(N)
    psi0 = W.random_state(12, 1 << N)
    kw = dict(m_max=16, max_substeps=200)
    fx = P.Propagator(P.XXZChain(N, pr.J, pr.Delta, pr.h), [P.XField(N, pr.xfield)], [pr.drive], precision="fx",
                      **kw)
    xf = _dev(torch_cuda, psi0)
    _, log = fx.propagate(xf, 0.1, 0.04, 2, order=6, tol=1e-9, record=True)
    outs = {}
    for flag in ("1", "0"):
        prop, _, _ = _spin(N, apply_form=FORMS[flag], **kw)
        x = _dev(torch_cuda, psi0)
        st = prop.propagate(x, 0.1, 0.04, 2, order=6, tol=1e-9, forced=log)
        outs[flag] = x.cpu().numpy()
    ref = xf.cpu().numpy()
    b = budget(st["n_substeps"])
    assert np.linalg.norm(outs["1"] - outs["0"]) <= 2 * b
    assert np.linalg.norm(outs["1"] - ref) <= b and np.linalg.norm(outs["0"] - ref) <= b
