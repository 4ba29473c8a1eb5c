"""The tolerance rules of the GPU parity tests (parity.py), on planted records.

A different triangle is accepted only as a near-edge tie (the oracle's hit
within 1e-6 of an edge and t within 1e-5 relative); the same triangle must
keep its bits; a key mismatch is accepted only on a marginal ray.
"""
import numpy as np
import pytest

import parity
from paper_2305_16652_gb300 import hcc


def _hits(rows):
    a = np.zeros(len(rows), dtype=hcc.HIT_DTYPE)
    for i, (p, t, u, v) in enumerate(rows):
        a[i] = (p, t, u, v)
    return a


MISS = (-1, np.inf, 0.0, 0.0)


@pytest.fixture(autouse=True)
def _own_tally():
    """Planted records stay out of the session's exception report."""
    saved = dict(parity.TALLY)
    parity.TALLY.clear()
    yield
    parity.TALLY.clear()
    parity.TALLY.update(saved)


def test_identical_records_have_no_exception():
    h = _hits([(3, 1.5, 0.2, 0.3), MISS])
    assert parity.hit_exceptions(h, h.copy()) == 0


def test_same_triangle_must_keep_its_bits():
    o = _hits([(3, 1.5, 0.2, 0.3)])
    g = _hits([(3, np.nextafter(np.float32(1.5), np.float32(2)), 0.2, 0.3)])
    with pytest.raises(AssertionError, match="same triangle"):
        parity.hit_exceptions(g, o)


def test_near_edge_tie_with_close_t_is_allowed():
    o = _hits([(3, 2.0, 5e-7, 0.5)])                  # oracle hit 5e-7 from the edge v0-v2
    g = _hits([(4, 2.0 * (1 + 5e-6), 0.4, 0.3)])      # its neighbour, t within 1e-5 relative
    assert parity.hit_exceptions(g, o) == 1


def test_tie_needs_the_oracle_hit_near_an_edge():
    o = _hits([(3, 2.0, 0.1, 0.5)])                   # well inside its triangle
    g = _hits([(4, 2.0, 5e-7, 0.5)])
    with pytest.raises(AssertionError):
        parity.hit_exceptions(g, o)


def test_tie_needs_t_within_relative_tolerance():
    o = _hits([(3, 0.01, 5e-7, 0.5)])                 # below t = 1 the tolerance stays relative
    g = _hits([(4, 0.01 + 2e-7, 0.4, 0.3)])
    with pytest.raises(AssertionError):
        parity.hit_exceptions(g, o)
    g_ok = _hits([(4, 0.01 * (1 + 9e-6), 0.4, 0.3)])
    assert parity.hit_exceptions(g_ok, o) == 1


def test_hit_against_miss_only_at_an_edge():
    o = _hits([(3, 2.0, 1 - 1e-7, 0.0)])              # on the mesh border
    assert parity.hit_exceptions(_hits([MISS]), o) == 1
    assert parity.hit_exceptions(o, _hits([MISS])) == 1
    inner = _hits([(3, 2.0, 0.3, 0.3)])
    with pytest.raises(AssertionError):
        parity.hit_exceptions(_hits([MISS]), inner)


def test_compare_hits_bounds_and_records_the_count():
    n = 100
    o = _hits([(3, 2.0, 5e-7, 0.5)] * n)
    g = _hits([(4, 2.0, 0.4, 0.3)] * n)
    with pytest.raises(AssertionError):  # 100 ties among 100 rays: far above 1e-3
        parity.compare_hits(g, o)
    g[:99] = o[:99]
    assert parity.compare_hits(g, o) == 1
    assert any("hits" in k for row in parity.TALLY.values() for k in row)


def test_compare_keys_accepts_only_marginal_rays():
    o = np.arange(2000, dtype=np.uint64)
    g = o.copy()
    g[7] ^= np.uint64(4)
    assert parity.compare_keys(g, o, lambda b: np.full(len(b), 1e-9)) == 1
    with pytest.raises(AssertionError, match="non-marginal"):
        parity.compare_keys(g, o, lambda b: np.full(len(b), 1e-3))
    lines = parity.summary_lines()
    assert any(line.startswith("total keys") for line in lines)
