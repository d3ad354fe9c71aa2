"""Seeded input generators: SplitMix64 against its published reference
outputs, and the droplet profile's stated properties."""
import numpy as np

from paper_1406_2686_gb300 import inputs


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (Vigna's reference splitmix64.c)
    got = inputs.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_determinism():
    a = inputs.uniform_pm1(7, 10000)
    b = inputs.uniform_pm1(7, 10000)
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.03


def test_droplet_profile():
    rA, rB = inputs.droplet_fields(40, 30, 20, R=8.0, seed=3, noise=1e-3)
    tot = rA + rB
    assert np.allclose(tot, 2.1, atol=1e-12)
    phi = (rA - rB) / tot
    assert phi[10, 15, 20] > 0.8 and phi[0, 0, 0] < -0.8
    rA0, rB0 = inputs.droplet_fields(40, 30, 20, R=8.0, seed=3, noise=0.0)
    dphi = phi - (rA0 - rB0) / 2.1
    assert np.max(np.abs(dphi)) <= 1e-3 + 1e-12
