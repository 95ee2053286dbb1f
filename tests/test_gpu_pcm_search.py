"""Device-side H_o search (bch_search_pcm): step 6 of Sec. III-A as parallel annealing
chains on the GPU.  Every chain's matrix is bit-exact against the oracle's annealing of
that chain (the same PRNG stream, the same proposals and acceptance tests, the same rank
repair), chain 0 is the matrix bch_build_pcm builds, and the kept chain is the one with
the lowest loss (#4-cycles + lambda Var(column weights), lambda = n) among the chains
that reach rank n - k, recomputed here from the matrices themselves."""
import numpy as np
import pytest

import oracle as O
from paper_2412_20828_gb300 import bchdec as B

pytestmark = pytest.mark.gpu


def _loss_terms(H):
    ov = H.astype(np.int64) @ H.T.astype(np.int64)
    iu = np.triu_indices(H.shape[0], 1)
    c4 = int((ov[iu] * (ov[iu] - 1) // 2).sum())
    col = H.sum(axis=0).astype(np.int64)
    return c4, int((col * col).sum()), int(col.sum())


@pytest.mark.parametrize("nk,chains,m_rows", [((63, 45), 6, 0), ((63, 36), 6, 0), ((63, 36), 3, 47),
                                              ((127, 99), 3, 0)])
def test_search_chains_match_oracle(nk, chains, m_rows):
    from paper_2412_20828_gb300 import build
    build.build()
    n, k = nk
    code, best, stats, dense = B.search_pcm(n, k, chains, m_rows=m_rows, return_all=True)
    assert np.array_equal(dense[0], B.build_pcm_host(n, k, m_rows=m_rows))
    losses = []
    for c in range(chains):
        H, c4, ss = O.build_ho_chain(n, k, c, m_rows=m_rows)
        assert np.array_equal(dense[c], H), f"chain {c}"
        assert (stats[c, 0], stats[c, 1], stats[c, 2]) == (c4, ss, 1)
        c4b, ssb, e = _loss_terms(H)
        assert (c4b, ssb) == (c4, ss)
        losses.append(c4b + n * (ssb - e * e / n) / n)
    assert best == int(np.argmin(losses))
    assert np.array_equal(code.dense(), dense[best])
    # a chain is a different annealing run: the chains do not all end in one matrix
    assert len({d.tobytes() for d in dense}) > 1


def test_search_rejects_bad_arguments():
    with pytest.raises(B.BchError) as e:
        B.search_pcm(63, 45, 0)
    assert e.value.status == B.EINVAL
