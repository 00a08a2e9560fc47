"""Pins of the oracle's Philox4x64-10 and Gaussian test matrix (Alg. RSVD step 1).

The generator is pinned against numpy's own Philox bit generator - an
independent implementation of the same SC'11 definition (numpy advances its
counter by one before each block, hence the offset) - and the normals against
the standard normal law.
"""
import math

import numpy as np
import pytest

from oracle import philox


@pytest.mark.parametrize("key", [(0, 0), (201, 0), (0xFFFFFFFFFFFFFFFF, 7), (123456789, 987654321)])
@pytest.mark.parametrize("ctr", [0, 1, 5, 1000, 2**40 + 3])
def test_philox_matches_numpy_bit_generator(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array([ctr - 1 if ctr else 2**64 - 1, 0 if ctr else 2**64 - 1, 0 if ctr else 2**64 - 1, 0 if ctr else 2**64 - 1], dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    assert list(philox.philox4x64((ctr, 0, 0, 0), key)) == ref


def test_philox_full_counter_matches_numpy():
    c = (0x0123456789ABCDEF, 0xFEDCBA9876543210, 17, 2**63)
    key = (31337, 42)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array([c[0] - 1, c[1], c[2], c[3]], dtype=np.uint64))
    assert list(philox.philox4x64(c, key)) == [int(v) for v in bg.random_raw(4)]


def test_unit_interval_endpoints():
    # smallest value: half an ulp of the 53-bit grid, so log(u) stays finite
    assert philox.word_to_open_unit(0) == 0.5 * 2.0 ** -53
    # largest: (2^53 - 1/2) 2^-53 is a tie in FP64 and rounds to even, i.e. 1.0
    assert philox.word_to_open_unit(2**64 - 1) == 1.0
    assert 0.0 < philox.word_to_open_unit(0) < philox.word_to_open_unit(2**63) < 1.0


def test_box_muller_closed_form():
    # words whose top 53 bits encode u_a = 1/2 and u_b = 1/8 (+ the half-ulp offset)
    wa = (1 << 63)
    wb = (1 << 61)
    z = philox.box_muller_block((wa, wb, wa, wa))
    ua = 0.5 + 0.5 * 2.0 ** -53
    ub = 0.125 + 0.5 * 2.0 ** -53
    r = math.sqrt(-2.0 * math.log(ua))
    assert z[0] == pytest.approx(r * math.cos(math.pi / 4), rel=1e-14)
    assert z[1] == pytest.approx(r * math.sin(math.pi / 4), rel=1e-14)
    assert z[2] == pytest.approx(-r, rel=1e-14)  # u_b = 1/2 -> cos(pi) = -1
    assert abs(z[3]) < 1e-14


def test_columns_nest_and_layout():
    wide = philox.gaussian_test_matrix(37, 9, seed=5, stream=3)
    narrow = philox.gaussian_test_matrix(37, 4, seed=5, stream=3)
    np.testing.assert_array_equal(wide[:, :4], narrow)
    # element (r, c) is slot (c*n + r) % 4 of block (c*n + r) // 4
    r, c, n = 11, 6, 37
    e = c * n + r
    z = philox.box_muller_block(philox.philox4x64((e // 4, 0, 0, 0), (5, 3)))
    assert wide[r, c] == z[e % 4]


def test_streams_differ():
    a = philox.gaussian_test_matrix(16, 4, seed=1, stream=0)
    b = philox.gaussian_test_matrix(16, 4, seed=1, stream=1)
    assert not np.any(a == b)


def test_gaussian_moments_and_ks():
    from scipy import stats
    z = philox.gaussian_test_matrix(4000, 30, seed=201, stream=0).ravel()  # 1.2e5 draws
    n = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
