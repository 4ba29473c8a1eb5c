"""Comparison rules of the GPU parity tests, and the tally of their exceptions.

Keys (Algorithm 1 and the other encoders' box tests): a GPU key must equal
the oracle's bit for bit, except on a ray whose slab-test margin
(``oracle.key_margin``: the smallest relative gap |tfar - tnear| /
max(1, |tnear|, |tfar|) over the boxes that drive key bits) is below 1e-6.
Such a ray sits on a box boundary, where the inclusive test of the paper's
intersection step could go either way under a rounding change.

Hit records (closest hit by Moller-Trumbore): a GPU record must equal the
oracle's bit for bit.  The only exceptions are near-edge ties:
  * both hit different triangles, the oracle's hit lies within 1e-6 of an
    edge in barycentric terms (min(u, v, 1 - u - v) < 1e-6) and the two t
    agree within 1e-5 relative to the oracle's t;
  * one side hits and the other misses, and the hit lies within 1e-6 of an
    edge (a ray grazing the border of the mesh).
The same triangle must always give the same (t, u, v) bits.

Every comparison adds what it checked and the exceptions it allowed to a
tally keyed by the running test; ``summary_lines`` prints it at the end of
the session (see conftest.py), so each run reports its exception counts.
"""
from __future__ import annotations

import os

import numpy as np

MARGIN_KEY = 1e-6     # slab-test margin below which a key bit may differ
TOL_T = 1e-5          # relative agreement of t on a near-edge tie
TOL_BARY = 1e-6       # barycentric margin of a near-edge hit

TALLY: dict = {}


def _test_id() -> str:
    cur = os.environ.get("PYTEST_CURRENT_TEST", "outside a test")
    return cur.rsplit(" (", 1)[0]


def record(kind: str, checked: int, exceptions: int) -> None:
    row = TALLY.setdefault(_test_id(), {})
    c, e = row.get(kind, (0, 0))
    row[kind] = (c + int(checked), e + int(exceptions))


def summary_lines() -> list:
    out = []
    tot = {}
    for test, row in sorted(TALLY.items()):
        for kind, (c, e) in sorted(row.items()):
            tc, te = tot.get(kind, (0, 0))
            tot[kind] = (tc + c, te + e)
            if e:
                out.append(f"{test}: {kind}: {e} exceptions of {c} checked")
    for kind, (c, e) in sorted(tot.items()):
        out.append(f"total {kind}: {e} exceptions of {c} checked")
    return out


def bary_margin(h) -> float:
    u, v = float(h["u"]), float(h["v"])
    return min(u, v, 1.0 - u - v)


def hit_exceptions(g, o, tol_t: float = TOL_T, tol_b: float = TOL_BARY) -> int:
    """Number of allowed near-edge ties between GPU records g and oracle
    records o; raises AssertionError on any other difference."""
    gi32 = np.ascontiguousarray(g).view(np.int32).reshape(-1, 4)
    oi32 = np.ascontiguousarray(o).view(np.int32).reshape(-1, 4)
    assert gi32.shape == oi32.shape
    bad = np.nonzero(np.any(gi32 != oi32, axis=1))[0]
    exceptions = 0
    for i in bad:
        gi, oi = g[i], o[i]
        gh, oh = int(gi["prim"]) >= 0, int(oi["prim"]) >= 0
        if gh and oh:
            if int(gi["prim"]) == int(oi["prim"]):
                raise AssertionError(f"ray {i}: same triangle, different numbers {gi} vs {oi}")
            ot, gt = float(oi["t"]), float(gi["t"])
            if bary_margin(oi) < tol_b and abs(gt - ot) <= tol_t * abs(ot):
                exceptions += 1
                continue
        elif gh or oh:
            if bary_margin(gi if gh else oi) < tol_b:
                exceptions += 1
                continue
        raise AssertionError(f"ray {i}: GPU {gi} vs oracle {oi}")
    return exceptions


def compare_hits(g, o, max_frac: float = 1e-3) -> int:
    """Bit-exact except counted near-edge ties (bounded to max_frac of the
    rays); records the count and returns it."""
    e = hit_exceptions(g, o)
    record("hits (near-edge ties)", len(g), e)
    assert e <= max(1, max_frac * len(g)), e
    return e


def compare_keys(g, o, margin_of, max_frac: float = 1e-3) -> int:
    """Keys g (GPU) against o (oracle): every mismatch must be on a ray whose
    margin_of(indices) is below 1e-6; records the count and returns it."""
    g = np.asarray(g, np.uint64)
    o = np.asarray(o, np.uint64)
    assert g.shape == o.shape
    bad = np.nonzero(g != o)[0]
    if len(bad):
        m = np.asarray(margin_of(bad))
        assert np.all(m < MARGIN_KEY), f"{int(np.sum(m >= MARGIN_KEY))} key mismatches on non-marginal rays"
    record("keys (marginal rays)", len(g), len(bad))
    assert len(bad) <= max(1, max_frac * len(g)), len(bad)
    return len(bad)
