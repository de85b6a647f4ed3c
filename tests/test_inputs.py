import numpy as np


def test_uniform_is_deterministic_and_uniform(inputs):
    a = inputs.uniform01(123, 100000, 3)
    b = inputs.uniform01(123, 100000, 3)
    np.testing.assert_array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.005 and abs(a.var() - 1 / 12) < 0.002
    c = inputs.uniform01(123, 1000, 4)
    assert np.corrcoef(a[:1000], c)[0, 1] < 0.1


def test_splitmix64_reference_values(inputs):
    # SplitMix64 outputs for state 0 (Steele, Lea, Flood 2014 reference stream)
    z = inputs._splitmix64(np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_bj_dispersion_ranges(inputs, params):
    x0 = inputs.dispersion(params, 4096, 7, "bj")
    n = params["x0_nominal"]
    assert np.all(np.abs(x0[:, 0] / n[0] - 1) <= 0.02 + 1e-15)
    for i in range(1, 7):
        assert np.all(np.abs(x0[:, i] / n[i] - 1) <= 0.1 + 1e-12)
    np.testing.assert_allclose(np.linalg.norm(x0[:, 7:11], axis=1), 1.0, atol=1e-14)
    tilt = 2 * np.arccos(np.clip(np.abs(x0[:, 7]), 0, 1))
    assert tilt.max() <= np.deg2rad(5) + 1e-12 and tilt.max() > np.deg2rad(4.5)
    assert np.all(np.abs(x0[:, 11:14]) <= np.deg2rad(2) + 1e-15)


def test_paper256_ranges_and_node_counts(inputs, params):
    x0 = inputs.dispersion(params, 256, 1, "paper256")
    for i, (lo, hi) in enumerate(((6, 9), (3, 6), (1, 2))):
        assert np.all((x0[:, 1 + i] >= lo) & (x0[:, 1 + i] < hi))
    Ns = inputs.node_counts(10000, 5)
    assert set(np.unique(Ns)) == {10, 15, 20, 30}
    assert np.all(np.abs(np.bincount(Ns)[[10, 15, 20, 30]] / 10000 - 0.25) < 0.03)
