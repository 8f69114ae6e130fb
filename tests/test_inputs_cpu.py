"""The seeded input generators shared by the oracle and the GPU path: the
counter-based SplitMix64 stream against its published outputs, the derived
uniform and normal draws, and the lattice and tensor recipes of the
workloads (shapes, ranges, determinism)."""
import math

import numpy as np

from paper_2512_10910_gb300 import inputs as I


def test_splitmix64_matches_its_published_outputs():
    # the reference generator's first outputs for seeds 0 and 1234567
    assert [int(x) for x in I._splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in I._splitmix64(1234567, 3)] == [6457827717110365317, 3203168211198807973,
                                                           9817491932198370423]


def test_uniform_and_normal_draws():
    u = I.splitmix64_uniform(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    # (x >> 11) * 2^-53 of the raw stream
    assert u[0] == (int(I._splitmix64(7, 1)[0]) >> 11) * 2.0 ** -53
    z = I.splitmix64_normal(9, 200000, 1.0, 0.3)
    assert abs(z.mean() - 1.0) < 5e-3 and abs(z.std() - 0.3) < 5e-3


def test_lattice_bond_counts_and_degrees():
    for L in (2, 5, 16):
        g = I.square_lattice(L, L, 4)
        assert g.n_sites == L * L and g.n_bonds == 2 * L * (L - 1)
        assert max(len(g.legs(v)) for v in range(g.n_sites)) == (4 if L > 2 else 2)
    g = I.cubic_lattice(8, 8, 8, 2)
    assert g.n_sites == 512 and g.n_bonds == 3 * 64 * 7
    assert max(len(g.legs(v)) for v in range(g.n_sites)) == 6


def test_random_tensors_are_seeded_and_in_range():
    g = I.square_lattice(4, 4, 4)
    a, b, c = I.random_tensors(g, 3), I.random_tensors(g, 3), I.random_tensors(g, 4)
    fa, fb, fc = a.flat_data()[0], b.flat_data()[0], c.flat_data()[0]
    assert np.array_equal(fa, fb) and not np.array_equal(fa, fc)
    assert fa.min() >= 0.1 and fa.max() < 1.1
    assert fa.size == sum(int(np.prod(g.leg_dims(v))) for v in range(g.n_sites))
    # sites filled in id order from one stream
    np.testing.assert_array_equal(fa, I.splitmix64_uniform(3, fa.size) + 0.1)


def test_ising_square_root_weights():
    for beta in (0.2, 0.4, 0.2217):
        s = I.ising_sqrt_boltzmann(beta)
        w = np.array([[math.exp(beta), math.exp(-beta)], [math.exp(-beta), math.exp(beta)]])
        np.testing.assert_allclose(s @ s, w, rtol=1e-14)
        np.testing.assert_allclose(s, s.T)


def test_batched_workload_recipe():
    work = I.batched_workload(64, 1234)
    assert len(work) == 64
    again = I.batched_workload(64, 1234)
    assert [(k, L, D, b) for k, L, D, b, _ in work] == [(k, L, D, b) for k, L, D, b, _ in again]
    for kind, L, D, beta, net in work:
        assert 6 <= L <= 24 and net.n_sites == L * L
        if kind == "ising":
            assert D == 2 and 0.3 <= beta <= 0.5
        else:
            assert kind == "random" and 2 <= D <= 6 and beta is None
    assert {k for k, *_ in work} == {"ising", "random"}
