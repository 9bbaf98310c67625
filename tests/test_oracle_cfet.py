"""Pins for oracle/cfet.py and oracle/operators.py (closed forms, library
routines, exact structural properties)."""

import math

import numpy as np
import pytest
from scipy.linalg import expm
import scipy.sparse as sp

from oracle import cfet, krylov, operators as O, schemes as S
import workloads as W

ORDER_OF = {n: S.SCHEMES[n].order for n in S.SCHEMES}


# --- driven two-level system, exact propagator Eq. (TwoLevelU), Sec. 6.2 ----
def _two_level_exact(t, Dl, V, w):
    Om = math.sqrt((Dl - w) ** 2 + V**2)
    c, s = math.cos(Om * t), math.sin(Om * t)
    return np.array([[np.exp(-1j * w * t) * (c - 1j * (Dl - w) / Om * s), -1j * V / Om * np.exp(-1j * w * t) * s],
                     [-1j * V / Om * np.exp(1j * w * t) * s, np.exp(1j * w * t) * (c + 1j * (Dl - w) / Om * s)]])


def _two_level_problem(Dl, V, w):
    # H(t) = [[Dl, V e^{-2iwt}], [V e^{2iwt}, -Dl]] = Dl sz + V cos(2wt) sx + V sin(2wt) sy
    op = O.Dense(Dl * O.SZ, [O.SX, O.SY])
    drives = [lambda t: V * math.cos(2 * w * t), lambda t: V * math.sin(2 * w * t)]
    return op, drives


def _cfet_propagator(op, drives, T, nsteps, scheme, run=cfet.propagate):
    U = np.zeros((2, 2), dtype=np.complex128)
    for b in range(2):
        e = np.zeros(2, dtype=np.complex128)
        e[b] = 1.0
        U[:, b] = run(op, e, 0.0, T / nsteps, nsteps, scheme, drives, tol=1e-14, m_max=2)
    return U


def _frob(U, Ut):
    # Eq. (Frob): ||U - U~||^2 = (1/L) sum |U_ij - U~_ij|^2
    return math.sqrt(np.sum(np.abs(U - Ut) ** 2) / U.shape[0])


def test_two_level_exact_propagator_is_a_solution():
    # sanity of the transcription: U(0) = 1, unitarity, and i dU/dt = H U
    Dl, V, w = 2.0, 0.5, 1.0
    assert np.allclose(_two_level_exact(0.0, Dl, V, w), np.eye(2))
    t, h = 0.7, 1e-6
    U = _two_level_exact(t, Dl, V, w)
    dU = (_two_level_exact(t + h, Dl, V, w) - _two_level_exact(t - h, Dl, V, w)) / (2 * h)
    H = np.array([[Dl, V * np.exp(-2j * w * t)], [V * np.exp(2j * w * t), -Dl]])
    assert np.allclose(U.conj().T @ U, np.eye(2), atol=1e-14)
    assert np.allclose(1j * dU, H @ U, atol=1e-8)


@pytest.mark.parametrize("name", list(S.SCHEMES))
def test_two_level_global_order(name):
    # Fig. 8 parameters (omega = 1, Delta = 2, V = 0.5, T = 5 pi): the global
    # error of an N-th order CFET falls as dt^N (Sec. 6.1: eps = c T dt^N)
    Dl, V, w = 2.0, 0.5, 1.0
    T = 5 * math.pi
    op, drives = _two_level_problem(Dl, V, w)
    Uex = _two_level_exact(T, Dl, V, w)
    N = ORDER_OF[name]
    steps = (40, 80) if N < 8 else (20, 40)
    e = [_frob(Uex, _cfet_propagator(op, drives, T, n, name)) for n in steps]
    slope = math.log2(e[0] / e[1])
    assert abs(slope - N) < 0.35, (name, e, slope)


def _propagate_reversed(op, psi0, t0, dt, nsteps, scheme, drives, tol, m_max):
    # planted mistake: exp(Omega_1) applied first instead of exp(Omega_s)
    scheme = S.get(scheme)
    psi = psi0.copy()
    for n in range(nsteps):
        c = cfet.stage_coefficients(scheme, t0 + n * dt, dt, drives)
        for j in range(scheme.s):
            psi, _, _ = krylov.expv(lambda v, cj=c[j]: op.apply(cj, v), psi, dt, tol, m_max)
    return psi


def test_two_level_detects_reversed_factor_order():
    Dl, V, w = 2.0, 0.5, 1.0
    T = 5 * math.pi
    op, drives = _two_level_problem(Dl, V, w)
    Uex = _two_level_exact(T, Dl, V, w)
    e = [_frob(Uex, _cfet_propagator(op, drives, T, n, "CF4:3Opt", run=_propagate_reversed)) for n in (40, 80)]
    assert math.log2(e[0] / e[1]) < 3.0


# --- Rosen-Zener pulse, Sec. 11.1 Eqs. (SpinChain2), (BPulse) -----------------
@pytest.mark.parametrize("detuning", [0.0, 0.25])
def test_rosen_zener_transition_probability(detuning):
    # single spin H = Delta sz + Re V(t) sx - Im V(t) sy with
    # V(t) = V e^{-2 i w t} / cosh(t / tau);  P_inf = sin^2(pi V tau) / cosh^2(pi (Delta - w) tau)
    tau, V = 1.0, 0.25
    Dl = 1.0
    w = Dl - detuning
    op = O.Dense(Dl * O.SZ, [O.SX, O.SY])
    drives = [lambda t: V * math.cos(2 * w * t) / math.cosh(t / tau),
              lambda t: V * math.sin(2 * w * t) / math.cosh(t / tau)]
    T0 = 40.0 * tau
    nsteps = 1600
    down = np.array([0, 1], dtype=np.complex128)
    psi = cfet.propagate(op, down, -T0, 2 * T0 / nsteps, nsteps, "CF6:5Opt", drives, tol=1e-14, m_max=2)
    p_up = abs(psi[0]) ** 2
    p_exact = math.sin(math.pi * V * tau) ** 2 / math.cosh(math.pi * detuning * tau) ** 2
    assert abs(p_up - p_exact) < 1e-8, (p_up, p_exact)


# --- operators vs independent constructions ----------------------------------
def test_xxz_apply_matches_kronecker():
    N = 5
    h = W.uniform(9, N, -1, 1)
    v = W.random_state(10, 1 << N)
    H = O.xxz_dense(N, 0.8, 0.37, h)
    assert np.allclose(H, H.conj().T)
    assert np.max(np.abs(O.xxz_apply(v, N, 0.8, 0.37, h) - H @ v)) < 1e-14
    a = W.uniform(11, N, -1, 1)
    assert np.max(np.abs(O.xfield_apply(v, N, a) - O.xfield_dense(N, a) @ v)) < 1e-14


def test_xxz_flip_term_is_antiparallel_hop():
    # X X + Y Y on a bond: 2 between |01> and |10>, 0 on aligned pairs
    N = 2
    H = O.xxz_dense(N, 1.0, 0.0, np.zeros(N))
    assert np.allclose(H, [[0, 0, 0, 0], [0, 0, 2, 0], [0, 2, 0, 0], [0, 0, 0, 0]])


def test_dia_apply_matches_scipy():
    p = W.grid_atom(Nr=30, L=5)
    v = W.random_state(13, p.dim)
    dim = p.dim
    for offs, vals in ((p.H0_offsets, p.H0_values), (p.V_offsets, p.V_values)):
        diags = [vals[d, : dim - o] if o >= 0 else vals[d, -o:] for d, o in enumerate(offs)]
        A = sp.diags(diags, list(offs), shape=(dim, dim), format="csr")
        assert np.max(np.abs(O.dia_apply(v, offs, vals) - A @ v)) < 1e-12
        assert abs(A - A.T).max() == 0.0       # real symmetric


def test_grid_atom_ground_energy():
    # l = 0 block: discrete hydrogen ground state, E -> -1/2 + O(dr^2)
    p = W.grid_atom()
    psi, E = W.atom_ground_state(p)
    Hpsi = O.Banded((p.H0_offsets, p.H0_values), []).apply([1.0], psi)
    rq = np.vdot(psi, Hpsi).real
    assert abs(rq - E) < 1e-10 and abs(E + 0.5) < 2e-3


# --- structural properties of the CFET ----------------------------------------
@pytest.mark.parametrize("name", ["CF2:1", "CF4:2", "CF4:3Opt", "CF6:5Opt", "CF8:11"])
def test_time_independent_hamiltonian_is_exact(name):
    # sum_i f_{i,1} = 1: with no drive, every scheme reproduces exp(-i H0 T)
    N = 6
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    psi0 = W.random_state(3, 1 << N)
    T, nsteps = 0.6, 4
    out = cfet.propagate(op, psi0, 0.0, T / nsteps, nsteps, name, [lambda t: 0.0], tol=1e-14, m_max=30)
    H0 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    assert np.linalg.norm(out - expm(-1j * T * H0) @ psi0) < 1e-11


@pytest.mark.parametrize("name", ["CF4:2", "CF6:5Opt", "CF8:11", "CF4:3Opt"])
def test_commuting_hamiltonian_is_gauss_legendre_quadrature(name):
    # H(t) = f(t) H1: every stage commutes, the step is exactly
    # exp(-i H1 dt sum_m w_m f(t + x_m dt))  (sum_j g_{j,m} = w_m)
    N = 5
    pr = W.spin_chain(N)
    H1 = O.xxz_dense(N, pr.J, pr.Delta, pr.h)
    op = O.Dense(np.zeros_like(H1), [H1])
    f = lambda t: math.cos(3.0 * t) + 0.5
    psi = W.random_state(4, 1 << N)
    t0, dt, nsteps = 0.3, 0.1, 3
    out = cfet.propagate(op, psi, t0, dt, nsteps, name, [f], tol=1e-14, m_max=32)
    x, w = S.gauss_legendre(S.SCHEMES[name].nA)
    ref = psi.copy()
    for n in range(nsteps):
        t = t0 + n * dt
        ref = expm(-1j * dt * sum(w[m] * f(t + x[m] * dt) for m in range(len(x))) * H1) @ ref
    assert np.linalg.norm(out - ref) < 1e-11


def test_zero_coupling_chain_factorises():
    # J = 0: sites decouple, each stage exponential is a tensor product, so the
    # chain result equals the product of single-spin CFET results
    N = 6
    pr = W.spin_chain(N, J=0.0, Delta=0.0, A=1.3, omega=1.7)
    op = O.SpinChain(N, 0.0, 0.0, pr.h, [pr.xfield])
    psi0 = W.neel_state(N)
    t0, dt, nsteps = 0.0, 0.05, 20
    out = cfet.propagate(op, psi0, t0, dt, nsteps, "CF6:5Opt", [pr.drive], tol=1e-14, m_max=40)
    single = []
    for i in range(N):
        op1 = O.Dense(pr.h[i] * O.SZ, [O.SX])
        e = np.zeros(2, dtype=np.complex128)
        e[(psi0.argmax() >> i) & 1] = 1.0
        single.append(cfet.propagate(op1, e, t0, dt, nsteps, "CF6:5Opt", [pr.drive], tol=1e-14, m_max=2))
    prod = np.ones(1, dtype=np.complex128)
    for i in range(N - 1, -1, -1):
        prod = np.kron(prod, single[i])
    assert np.linalg.norm(out - prod) < 1e-11


def test_unitarity_driven_chain():
    N = 6
    pr = W.spin_chain(N)
    op = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    out = cfet.propagate(op, W.neel_state(N), 0.0, 0.02, 50, 6, [pr.drive], tol=1e-12, m_max=16)
    assert abs(np.linalg.norm(out) - 1.0) < 1e-12
