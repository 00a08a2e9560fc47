"""Pins of the oracle's block-wise truncation with global post-selection (Sec. III.A).

The plain definition - the chi largest singular values of the whole
block-diagonal matrix - is computed here by brute force on the assembled
matrix and compared with the block-wise result.
"""
import numpy as np
import pytest
from scipy.linalg import block_diag

from oracle.sectors import block_rsvd_adaptive, block_rsvd_global, block_tsvd_global, global_select, trial_ranks
from paper_1710_01463_gb300 import inputs


def small_blocks(seed=3):
    shapes, f = inputs.sector_shapes(N=6, lo=5, hi=30, seed=seed)
    return [inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.2, fb), 100 + b)
            for b, ((m, n), fb) in enumerate(zip(shapes, f))]


@pytest.mark.parametrize("chi", [1, 7, 20, 40])
def test_blockwise_equals_assembled_truncation(chi):
    blocks = small_blocks()
    res, kept = block_tsvd_global(blocks, chi)
    s_all = np.linalg.svd(block_diag(*blocks), compute_uv=False)[:chi]
    got = np.sort(np.concatenate([r[1] for r in res]))[::-1]
    np.testing.assert_allclose(got, s_all, rtol=1e-12)
    assert sum(kept) == chi
    # the block-wise factors reproduce the best rank-chi approximation of the whole matrix
    approx = block_diag(*[(U * s) @ Vt if s.size else np.zeros(A.shape) for (U, s, Vt), A in zip(res, blocks)])
    err = np.linalg.norm(block_diag(*blocks) - approx, "fro")
    s_full = np.linalg.svd(block_diag(*blocks), compute_uv=False)
    assert err == pytest.approx(np.sqrt(np.sum(s_full[chi:] ** 2)), rel=1e-10)


def test_tie_break_lowest_block_then_index():
    kept = global_select([np.array([3.0, 1.0]), np.array([2.0, 1.0]), np.array([1.0])], 3)
    assert kept == [2, 1, 0]
    kept = global_select([np.array([1.0]), np.array([1.0]), np.array([1.0])], 2)
    assert kept == [1, 1, 0]


def test_rsvd_maximal_policy_matches_plain_definition():
    blocks = small_blocks(5)
    chi = 12
    res_t, kept_t = block_tsvd_global(blocks, chi)
    res_r, kept_r, ranks = block_rsvd_global(blocks, chi, p=30, q=2, seed=9)
    assert ranks == trial_ranks([b.shape for b in blocks], chi, "maximal")
    assert kept_r == kept_t       # l >= min(m_b, n_b) for these blocks: exact
    for (_, st, _), (_, sr, _) in zip(res_t, res_r):
        np.testing.assert_allclose(sr, st, rtol=1e-11)


def test_even_policy_ranks():
    assert trial_ranks([(100, 80), (10, 50)], 64, "even", c=3) == [35, 10]


@pytest.mark.parametrize("start", ["ones", "even", "maximal"])
def test_adaptive_ranks_reach_the_plain_definition_from_any_guess(start):
    # with p large enough that every trial is exact, the adaptive ranks keep exactly the
    # plain definition's values whatever the first guess; a saturated guess grows
    blocks = small_blocks(5)
    chi = 12
    res_t, kept_t = block_tsvd_global(blocks, chi)
    shapes = [b.shape for b in blocks]
    r0 = {"ones": [1] * len(blocks), "even": trial_ranks(shapes, chi, "even", c=0),
          "maximal": trial_ranks(shapes, chi, "maximal")}[start]
    res, kept, ranks, rounds = block_rsvd_adaptive(blocks, chi, 30, 2, 9, r0)
    assert kept == kept_t
    for (_, st, _), (_, sr, _) in zip(res_t, res):
        np.testing.assert_allclose(sr, st, rtol=1e-11)
    # no block ends saturated below its cap, and the maximal guess needs one round
    for kb, r, A in zip(kept, ranks, blocks):
        assert kb < r or r == min(chi, *A.shape)
    if start == "maximal":
        assert rounds == 1
    if start == "ones":
        assert rounds > 1


def test_adaptive_ranks_on_rsvd_samples():
    # blocks larger than the samples (inexact RSVD): the kept values still equal the plain
    # definition's to RSVD accuracy on this fast-decaying spectrum
    shapes, f = inputs.sector_shapes(N=5, lo=40, hi=120, seed=8)
    blocks = [inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 4.0) * fb, 200 + b)
              for b, ((m, n), fb) in enumerate(zip(shapes, f))]
    chi = 30
    res_t, kept_t = block_tsvd_global(blocks, chi)
    res, kept, ranks, rounds = block_rsvd_adaptive(blocks, chi, 10, 2, 4, [2] * len(blocks))
    assert kept == kept_t
    for (_, st, _), (_, sr, _) in zip(res_t, res):
        np.testing.assert_allclose(sr, st, rtol=1e-8, atol=1e-12 * max(s[0] for _, s, _ in res_t if s.size))
