"""The work split of a wide-basis pass (frsvt_wide_pass_plan, host arithmetic, no GPU): the
tile-major (tile, K-chunk) units of Alg. 1's passes over A cut into contiguous CTA ranges.  The
pass kernel keeps two TMEM accumulators (a range may touch at most two tiles) and the workspace
eight partial planes per tile; the plan reported by the library is checked against those limits
and against a direct enumeration of the ranges."""
import itertools

import pytest

from paper_1509_00296_gb300 import frsvt

TILE = 256


def enumerate_plan(nlong, nk, kc, grid):
    """Ranges [b U / G, (b + 1) U / G) of the U = ntiles * nkc units, enumerated unit by unit."""
    ntiles, nkc = -(-nlong // TILE), -(-nk // kc)
    units = ntiles * nkc
    owner = [None] * units
    tiles_of_cta = []
    for b in range(grid):
        u0, u1 = b * units // grid, (b + 1) * units // grid
        assert u1 > u0, "empty range"
        for u in range(u0, u1):
            assert owner[u] is None
            owner[u] = b
        tiles_of_cta.append({u // nkc for u in range(u0, u1)})
    assert all(o is not None for o in owner)                       # every unit once
    parts = [len({owner[t * nkc + c] for c in range(nkc)}) for t in range(ntiles)]
    for t in range(ntiles):                                        # a tile's CTAs are consecutive
        ctas = sorted({owner[t * nkc + c] for c in range(nkc)})
        assert ctas == list(range(ctas[0], ctas[-1] + 1))
    return max(parts), max(len(s) for s in tiles_of_cta)


@pytest.mark.parametrize("nlong,nk,prec,sms", list(itertools.product(
    [33, 256, 300, 1031, 2048, 8192, 12000, 40000], [33, 130, 517, 2048, 8192], [0, 1, 2], [152, 148, 16])))
def test_plan_matches_enumeration(nlong, nk, prec, sms):
    grid, max_parts, max_tiles = frsvt.wide_pass_plan(nlong, nk, prec, sms)
    ntiles, kc = -(-nlong // TILE), (32 if prec == 0 else 64)
    units = ntiles * -(-nk // kc)
    assert ntiles <= grid <= max(ntiles, sms)
    assert grid <= max(ntiles, units // 2)                        # at least two units per CTA unless one tile each
    assert max_parts <= 8 and max_tiles <= 2
    assert (max_parts, max_tiles) == enumerate_plan(nlong, nk, kc, grid)


def test_plan_of_the_recovery_matrix():
    """8192 x 8192: 32 tiles x 256 K-chunks on 152 SMs, 5-6 partials per tile."""
    assert frsvt.wide_pass_plan(8192, 8192, 0, 152) == (152, 6, 2)
    assert frsvt.wide_pass_plan(8192, 8192, 1, 152) == (152, 6, 2)


def test_plan_invalid_arguments():
    for args in ((0, 100, 0, 152), (100, 0, 0, 152), (100, 100, 3, 152), (100, 100, 0, 0)):
        with pytest.raises(frsvt.FrsvtError):
            frsvt.wide_pass_plan(*args)
