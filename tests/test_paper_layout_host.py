"""Host logic of the paper's own decoder layout: the 9-member automorphism block of
Sec. III-B, checked against the three maps as the paper defines them (interleaving =
even-index bits then odd-index bits; Frobenius i -> 2i mod N; cyclic shifts
s d_p + d_o with d_p = 21 / 42 and d_o in [0, d_p)), built here with numpy slicing."""
import numpy as np
import pytest

from paper_2412_20828_gb300.paper_layout import PRINTED_LADDER, paper_block


def _apply(v, y):
    # the library's map: z[(2^j i + s) mod n] = y[i]
    n = len(y)
    s, j = int(v) & 0xFF, int(v) >> 8
    z = np.empty_like(y)
    z[(pow(2, j, n) * np.arange(n) + s) % n] = y
    return z


@pytest.mark.parametrize("n,m,d_p", [(63, 6, 21), (127, 7, 42)])
def test_paper_block_is_the_nine_automorphisms(n, m, d_p):
    y = np.arange(1000, 1000 + n)
    inter = np.concatenate([y[0::2], y[1::2]])
    frob = np.empty_like(y)
    frob[(2 * np.arange(n)) % n] = y
    blk = paper_block(n, m, 64, 5, seed=11)
    assert blk.shape == (64, 9)
    offsets = set()
    for row in blk:
        got = [tuple(_apply(v, y)) for v in row]
        # the offset is the shift of the identity member with the smallest amount
        d_o = min(int(v) & 0xFF for v in row[:3])
        assert 0 <= d_o < d_p
        offsets.add(d_o)
        want = [tuple(np.roll(w, d_o + q * d_p)) for w in (y, inter, frob) for q in range(3)]
        assert got == want
    assert len(offsets) > 5  # the offset is drawn per frame
    # stateless in (seed, frame0)
    assert np.array_equal(paper_block(n, m, 64, 5, seed=11), blk)
    assert not np.array_equal(paper_block(n, m, 64, 6, seed=11), blk)


def test_printed_ladder_is_monotone_in_rows():
    # Sec. III-A: (beta, M_o, FER) pairs; M_o grows with beta and starts at n - k
    for (n, k), ladder in PRINTED_LADDER.items():
        assert ladder[0][1] == n - k
        assert all(a[0] < b[0] and a[1] < b[1] for a, b in zip(ladder, ladder[1:]))
