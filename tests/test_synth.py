"""The seeded input generators: determinism, SU(3) properties, distributions."""
import numpy as np

import synth


def test_splitmix64_is_counter_based_and_deterministic():
    a = synth.splitmix64(42, 10)
    b = synth.splitmix64(42, 6, offset=4)
    assert np.array_equal(a[4:], b)
    assert np.array_equal(a, synth.splitmix64(42, 10))
    assert not np.array_equal(a, synth.splitmix64(43, 10))
    assert len(set(a.tolist())) == 10


def test_uniform_and_gaussian_moments():
    u = synth.uniform(1, 200000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    g = synth.gaussian(2, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    assert abs(np.mean(g ** 4) - 3) < 0.1


def test_links_are_su3_and_reproducible():
    U = synth.random_links((3, 4, 2, 5), 0.7, 9)
    assert U.shape == (5, 2, 4, 3, 4, 3, 3)
    eye = np.einsum("...ab,...cb->...ac", U, U.conj())
    assert np.abs(eye - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    assert np.array_equal(U, synth.random_links((3, 4, 2, 5), 0.7, 9))
    # eps -> 0 approaches the unit field
    U0 = synth.random_links((2, 2, 2, 2), 1e-9, 9)
    assert np.abs(U0 - np.eye(3)).max() < 1e-8


def test_sources():
    b = synth.point_source((2, 3, 4, 5), site=7, spin=2, colour=1)
    assert b.shape == (5, 4, 3, 2, 4, 3) and b.sum() == 1 and b.reshape(-1, 4, 3)[7, 2, 1] == 1
    g = synth.gaussian_source((4, 4, 4, 4), 3)
    assert abs(np.mean(np.abs(g) ** 2) - 2) < 0.1


def test_workloads_describe_the_lattices():
    assert synth.WORKLOADS["16^3x32"]["dims"] == (16, 16, 16, 32)
    assert synth.WORKLOADS["4^3x8"]["eps"] == 0.3
