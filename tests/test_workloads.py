"""Pins for the seeded input generators (workloads/)."""

import numpy as np

import workloads as W


def test_splitmix64_reference_outputs():
    # first outputs of splitmix64 with seed 0, as published with the generator
    z = W.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_gaussian_statistics():
    u = W.uniform(1, 200000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    g = W.complex_gaussian(2, 200000)
    assert abs(g.real.mean()) < 0.01 and abs(g.real.var() - 1.0) < 0.02 and abs(g.imag.var() - 1.0) < 0.02
    assert abs(np.mean(g.real * g.imag)) < 0.01


def test_counter_based_stream_is_sliceable():
    a = W.splitmix64(7, 10)
    b = W.splitmix64(7, 4, start=6)
    assert np.array_equal(a[6:], b)


def test_neel_and_random_state():
    psi = W.neel_state(8)
    assert np.count_nonzero(psi) == 1 and psi[0b10101010] == 1.0
    v = W.random_state(2, 1 << 10)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-14


def test_grid_atom_shapes():
    p = W.grid_atom(Nr=50, L=4)
    assert p.dim == 200 and p.H0_values.shape == (3, 200) and p.V_values.shape == (2, 200)
    # radial hop cut at l-block edges, dipole zero outside the l range
    assert p.H0_values[1, 49] == 0.0 and p.H0_values[2, 50] == 0.0
    assert np.all(p.V_values[0, 150:] == 0.0) and np.all(p.V_values[1, :50] == 0.0)


def test_chain_batch_recipe():
    b = W.chain_batch()
    assert len(b) == 256
    assert {c.N for c in b} == set(range(10, 17))
    assert all(0.5 <= c.A <= 2.0 and 1.0 <= c.omega <= 3.0 for c in b)
    assert all(np.all(np.abs(c.h) <= 1.0) and c.h.shape == (c.N,) for c in b)
    b2 = W.chain_batch()
    assert all(np.array_equal(x.h, y.h) and x.A == y.A for x, y in zip(b, b2))   # seeded
    assert len({c.psi_seed for c in b}) == 256
