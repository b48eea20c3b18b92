"""Pins of the seeded input generators (workloads/), which both the oracle
and the CUDA path take their inputs from: SplitMix64 against its published
reference sequence, and the uniform and Box-Muller outputs against their
distributions."""
import math

import numpy as np

import workloads as W


def test_splitmix64_reference_sequence():
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014, in the form of Vigna's
    public-domain reference code) from state 0."""
    g = W.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_distributions():
    g = W.SplitMix64(W.DEFAULT_SEED)
    u = np.array([g.uniform() for _ in range(200000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    z = np.array(W.SplitMix64(7).normals(200001))
    assert len(z) == 200001
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    # the two members of a Box-Muller pair are uncorrelated
    pairs = np.array(W.SplitMix64(11).normals(200000)).reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 1e-2
    # tails of a standard normal: P(|z| > 2) = 0.0455
    assert abs((np.abs(z) > 2.0).mean() - math.erfc(2.0 / math.sqrt(2.0))) < 3e-3


def test_generators_are_deterministic_and_seed_dependent():
    a = W.uniform_array(123, 1000)
    b = W.uniform_array(123, 1000)
    c = W.uniform_array(124, 1000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    d1 = W.rti_adjoint(nx=64, ny=128).notes["a"]
    d2 = W.rti_adjoint(nx=64, ny=128).notes["a"]
    assert list(d1) == list(d2)
