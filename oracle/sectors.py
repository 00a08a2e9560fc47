"""Oracle: block-wise (symmetry-sector) truncation with global post-selection.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. III.A: with Abelian symmetries the matrix to compress is block diagonal
over N sectors; the factorization is done block by block, and the chi largest
singular values over all blocks are kept ("post-select the chi largest").

Plain definition (TSVD form): take every singular value of every block, sort
all of them descending, keep the first chi.  Ties are broken by (block index,
index within the block) ascending - the paper is silent on ties.

RSVD form: each block b is compressed by Alg. RSVD at a trial rank k'_b chosen
beforehand (the paper's two policies: "maximal" k'_b = min(chi, m_b, n_b) as in
its TTN runs, and k'_b = chi / N + c as in its TEBD runs), then the same global
selection runs over the k'_b returned values of each block.
"""
import numpy as np

from .rsvd import rsvd, tsvd


def trial_ranks(shapes, chi, policy="maximal", c=0):
    """Per-block trial ranks k'_b (Sec. III.A)."""
    out = []
    N = len(shapes)
    for (m, n) in shapes:
        if policy == "maximal":
            kb = min(chi, m, n)
        elif policy == "even":
            kb = min(chi // N + c, m, n)
        else:
            raise ValueError(policy)
        out.append(kb)
    return out


def global_select(svals, chi):
    """Number of values kept per block when the chi largest over all blocks are kept.

    ``svals`` is a list of descending 1-D arrays (one per block).
    """
    pool = []
    for b, s in enumerate(svals):
        for i, v in enumerate(np.asarray(s, dtype=np.float64)):
            pool.append((-float(v), b, i))
    pool.sort()
    kept = [0] * len(svals)
    for (_, b, _) in pool[:chi]:
        kept[b] += 1
    return kept


def block_tsvd_global(blocks, chi):
    """Plain definition: TSVD of every block, then global top-chi selection."""
    full = [tsvd(A, min(A.shape)) for A in blocks]
    kept = global_select([f[1] for f in full], chi)
    return [(U[:, :kb], s[:kb], Vt[:kb]) for (U, s, Vt), kb in zip(full, kept)], kept


def block_rsvd_global(blocks, chi, p, q, seed, ranks=None, policy="maximal", c=0):
    """RSVD form: per-block RSVD at trial rank k'_b, then global top-chi selection.

    Block b uses the Philox stream b.
    """
    shapes = [A.shape for A in blocks]
    if ranks is None:
        ranks = trial_ranks(shapes, chi, policy, c)
    res = [rsvd(A, kb, p, q, seed, stream=b) for b, (A, kb) in enumerate(zip(blocks, ranks))]
    kept = global_select([r[1] for r in res], chi)
    return [(U[:, :kb], s[:kb], Vt[:kb]) for (U, s, Vt), kb in zip(res, kept)], kept, ranks


def block_rsvd_adaptive(blocks, chi, p, q, seed, ranks0):
    """Adaptive per-block trial ranks (the fixed-error route to the sector sizes that
    Sec. V proposes, here for the global top-chi cut): start from any trial ranks, select
    the chi largest over all blocks; a block all of whose k'_b values were kept while
    k'_b < min(chi, m_b, n_b) may hold more values above the cut, so its trial rank is
    doubled (capped there) and the block compressed again (same Philox stream b: the
    larger test matrix extends the previous one); repeat until no block is saturated.
    Returns (factors, kept, ranks, rounds)."""
    caps = [min(chi, *A.shape) for A in blocks]
    ranks = [max(1, min(k, c)) for k, c in zip(ranks0, caps)]
    res = [rsvd(A, kb, p, q, seed, stream=b) for b, (A, kb) in enumerate(zip(blocks, ranks))]
    rounds = 1
    while True:
        kept = global_select([r[1] for r in res], chi)
        grow = [b for b in range(len(blocks)) if kept[b] == ranks[b] and ranks[b] < caps[b]]
        if not grow:
            break
        for b in grow:
            ranks[b] = min(2 * ranks[b], caps[b])
            res[b] = rsvd(blocks[b], ranks[b], p, q, seed, stream=b)
        rounds += 1
    return [(U[:, :kb], s[:kb], Vt[:kb]) for (U, s, Vt), kb in zip(res, kept)], kept, ranks, rounds
