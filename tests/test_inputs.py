"""The seeded input generator shared by the oracle and the library's tests and bench."""
import numpy as np

from paper_2502_14589_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    # first outputs of SplitMix64 (Vigna) from state 0, as printed by its reference code
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform01_is_53_bit_in_unit_interval():
    u = inputs.uniform01(7, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 0.01


def test_initial_state_recipe():
    y = inputs.initial_state((64, 48), 3, -0.05, 0.05)
    assert y.shape == (64 * 48,) and y.dtype == np.float64
    assert abs(y.mean()) < 1e-17
    assert y.min() > -0.06 and y.max() < 0.06
    z = inputs.initial_state((8, 8, 8), 0, -0.1, 0.1, 0.1)
    assert abs(z.mean() - 0.1) < 1e-15
    assert np.array_equal(y, inputs.initial_state((64, 48), 3, -0.05, 0.05))
    assert not np.array_equal(y, inputs.initial_state((64, 48), 4, -0.05, 0.05))


def test_batch_descriptors():
    n, eps = inputs.batch_descriptors(256, 0)
    assert len(n) == 256 and set(n.tolist()) <= set(inputs.BATCH_SIDES)
    assert eps.min() >= 0.01 and eps.max() < 0.05
    n2, eps2 = inputs.batch_descriptors(256, 0)
    assert np.array_equal(n, n2) and np.array_equal(eps, eps2)
    assert int((n.astype(np.int64) ** 2).sum()) == 17876992     # the benchmark batch's points
