"""Pins for the oracle's Pauli-sum operator (oracle/operators.py: PauliSum,
pauli_string_apply): the bit formulas against Kronecker products of the 2x2
Pauli matrices of Sec. 6.2, the XXZ chain written as Pauli strings, and closed
forms of exp(-i t H) for single strings."""

import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import cfet, operators as O


def _random_terms(rng, N, n):
    terms = []
    for _ in range(n):
        label = "".join(rng.choice(list("IXYZ"), size=N))
        terms.append((float(rng.uniform(-1, 1)), label))
    return terms


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_string_apply_matches_kronecker_products(seed):
    rng = np.random.default_rng(seed)
    N = 5
    terms = _random_terms(rng, N, 12)
    op = O.PauliSum(N, terms, [])
    H = O.pauli_dense(N, terms)
    assert np.allclose(H, H.conj().T, atol=1e-14)         # real combinations are Hermitian
    v = W.random_state(seed + 3, 1 << N)
    assert np.allclose(op.apply([1.0], v), H @ v, atol=1e-13)


def test_dict_and_string_labels_agree():
    N = 4
    a = O.PauliSum(N, [(0.7, "XYIZ"), (-0.2, "IIYY")], [])
    b = O.PauliSum(N, [(0.7, {0: "X", 1: "Y", 3: "Z"}), (-0.2, {2: "Y", 3: "Y"})], [])
    v = W.random_state(1, 16)
    assert np.array_equal(a.apply([1.0], v), b.apply([1.0], v))


def test_xxz_chain_as_pauli_strings():
    N = 6
    pr = W.spin_chain(N)
    terms = []
    for i in range(N - 1):
        for p2 in ("XX", "YY"):
            terms.append((pr.J, {i: p2[0], i + 1: p2[1]}))
        terms.append((pr.J * pr.Delta, {i: "Z", i + 1: "Z"}))
    terms += [(pr.h[i], {i: "Z"}) for i in range(N)]
    vterms = [(pr.xfield[i], {i: "X"}) for i in range(N)]
    op = O.PauliSum(N, terms, [vterms])
    chain = O.SpinChain(N, pr.J, pr.Delta, pr.h, [pr.xfield])
    v = W.random_state(2, 1 << N)
    c = [0.8, -0.35]
    assert np.allclose(op.apply(c, v), chain.apply(c, v), atol=1e-13)
    assert np.allclose(O.pauli_dense(N, terms), O.xxz_dense(N, pr.J, pr.Delta, pr.h), atol=1e-13)


def test_single_y_rotation_closed_form():
    # H = b Y on one spin: exp(-i t b Y)|up> = cos(bt)|up> + sin(bt)|down>
    b, T = 0.9, 1.3
    op = O.PauliSum(1, [(b, "Y")], [])
    out = cfet.propagate(op, np.array([1.0, 0.0], dtype=np.complex128), 0.0, T / 4, 4, 4, [], 1e-14, 2)
    assert np.allclose(out, [math.cos(b * T), math.sin(b * T)], atol=1e-13)


def test_yy_pair_closed_form():
    # H = J Y_0 Y_1: Y Y |up up> = (i)(i) |down down> = -|down down>, so
    # exp(-i t J Y Y)|up up> = cos(Jt)|up up> + i sin(Jt)|down down>
    J, T = 0.6, 2.1
    op = O.PauliSum(2, [(J, "YY")], [])
    psi0 = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.complex128)
    out = cfet.propagate(op, psi0, 0.0, T / 5, 5, 6, [], 1e-14, 4)
    assert np.allclose(out, [math.cos(J * T), 0.0, 0.0, 1j * math.sin(J * T)], atol=1e-13)


def test_time_independent_pauli_sum_matches_expm():
    rng = np.random.default_rng(7)
    N = 6
    terms = _random_terms(rng, N, 20)
    op = O.PauliSum(N, terms, [])
    psi0 = W.random_state(4, 1 << N)
    out = cfet.propagate(op, psi0, 0.0, 0.1, 6, 8, [], 1e-13, 30)
    ref = expm(-1j * 0.6 * O.pauli_dense(N, terms)) @ psi0
    assert np.linalg.norm(out - ref) <= 1e-11


# ---------------------------------------------------------------- planted mistakes
def test_planted_sign_error_in_y_is_caught(monkeypatch):
    # Y with the sign of its matrix elements flipped (i.e. -Y): the Kronecker
    # pin and the Y-rotation closed form must both notice
    good_y = O.apply_y
    monkeypatch.setattr(O, "apply_y", lambda v, i, N: -good_y(v, i, N))
    N = 3
    terms = [(0.7, "YIZ"), (0.4, "XYI")]
    v = W.random_state(5, 1 << N)
    assert not np.allclose(O.PauliSum(N, terms, []).apply([1.0], v), O.pauli_dense(N, terms) @ v, atol=1e-10)
    op = O.PauliSum(1, [(0.9, "Y")], [])
    out = cfet.propagate(op, np.array([1.0, 0.0], dtype=np.complex128), 0.0, 0.5, 2, 4, [], 1e-14, 2)
    assert not np.allclose(out, [math.cos(0.9), math.sin(0.9)], atol=1e-6)


def test_planted_site_reversal_is_caught(monkeypatch):
    # labels read from the last site backwards: the dict-against-string pin
    # and the chain-as-strings pin must notice
    good = O.pauli_ops
    monkeypatch.setattr(O, "pauli_ops",
                        lambda lb: good(lb[::-1]) if isinstance(lb, str) else good(lb))
    N = 4
    a = O.PauliSum(N, [(0.7, "XYIZ")], [])
    b = O.PauliSum(N, [(0.7, {0: "X", 1: "Y", 3: "Z"})], [])
    v = W.random_state(1, 16)
    assert not np.allclose(a.apply([1.0], v), b.apply([1.0], v), atol=1e-10)

