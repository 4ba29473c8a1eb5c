"""Pins of the CPU oracle against facts outside itself (no GPU needed).

Each test checks the oracle against what the paper or plain mathematics
fixes: the worked codes printed in the paper, hand-computed examples,
closed forms, textbook special cases, brute force on tiny inputs and
invariants that characterise the result completely.
"""
import os
from dataclasses import dataclass
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            rows[k] = v
    return rows


# ---------------------------------------------------------------- HCC codes

def _grid_cut():
    """Sixteen unit cells of a 4 x 4 grid in the z = [0, 1] slab, numbered row by row."""
    lo, hi = [], []
    for r in range(4):
        for c in range(4):
            lo.append((c, r, 0.0))
            hi.append((c + 1, r + 1, 1.0))
    return np.array(lo, np.float32), np.array(hi, np.float32)


def _segment(o, d):
    """A ray segment o + t d, t in [0, 1], in the z = 0.5 plane (d.z = 0)."""
    return (np.array([[o[0], o[1], 0.5, 0.0]], np.float32), np.array([[d[0], d[1], 0.0, 1.0]], np.float32))


# Segments re-creating the four rays of the SpaceAnchor figure; the cells each
# one crosses are worked out by hand in the comments (x = column, y = row).
SPACE_ANCHOR_RAYS = {
    # (0.95, 0.02) -> (1.30, 2.95): x = 1 at y = 0.44; y = 1 at x = 1.07; y = 2 at x = 1.19
    "ray1": ((0.95, 0.02), (0.35, 2.93)),   # cells 0, 1, 5, 9
    # (0.97, 0.05) -> (1.27, 2.90): x = 1 at y = 0.34; y = 1 at x = 1.07; y = 2 at x = 1.18
    "ray2": ((0.97, 0.05), (0.30, 2.85)),   # cells 0, 1, 5, 9
    # (2.60, 2.90) -> (0.30, 3.70): y = 3 at x = 2.31; x = 2 at y = 3.11; x = 1 at y = 3.46
    "ray3": ((2.60, 2.90), (-2.30, 0.80)),  # cells 10, 14, 13, 12
    # (1.80, 3.90) -> (3.40, 0.20): x = 2 at y = 3.44; y = 3 at x = 2.19; y = 2 at x = 2.62;
    #                                x = 3 at y = 1.13; y = 1 at x = 3.05
    "ray4": ((1.80, 3.90), (1.60, -3.70)),  # cells 13, 14, 10, 6, 7, 3
}


def test_hcc_codes_of_space_anchor_figure():
    golden = _read_golden("spaceanchor_codes.txt")
    lo, hi = _grid_cut()
    for name, (o, d) in SPACE_ANCHOR_RAYS.items():
        org, dir_ = _segment(o, d)
        key = int(oracle.encode_hcc(org, dir_, lo, hi, 16)[0])
        assert format(key, "016b") == golden[name], name


def test_hcc_bit_order_single_cells():
    # a segment inside one cell sets exactly that cell's bit, counted from the MSB
    lo, hi = _grid_cut()
    for r in range(4):
        for c in range(4):
            org, dir_ = _segment((c + 0.4, r + 0.4), (0.2, 0.2))
            key = int(oracle.encode_hcc(org, dir_, lo, hi, 16)[0])
            assert key == 1 << (15 - (r * 4 + c))
            key32 = int(oracle.encode_hcc(org, dir_, lo, hi, 32)[0])
            assert key32 == 1 << (31 - (r * 4 + c))  # bits below the cut size stay 0
            key8 = int(oracle.encode_hcc(org, dir_, lo, hi, 8)[0])
            idx = r * 4 + c
            assert key8 == ((1 << (7 - idx)) if idx < 8 else 0)  # only min(C, k) nodes drive bits


def _clip_double(o, d, tmin, tmax, lo, hi):
    """Liang-Barsky clip of the segment against the box in exact rationals."""
    t0, t1 = Fraction(float(tmin)), Fraction(float(tmax)) if np.isfinite(tmax) else None
    for a in range(3):
        oa, da = Fraction(float(o[a])), Fraction(float(d[a]))
        la, ha = Fraction(float(lo[a])), Fraction(float(hi[a]))
        if da == 0:
            if oa < la or oa > ha:
                return False
            continue
        ta, tb = (la - oa) / da, (ha - oa) / da
        if ta > tb:
            ta, tb = tb, ta
        t0 = max(t0, ta)
        t1 = tb if t1 is None else min(t1, tb)
        if t0 > t1:
            return False
    return True


def test_hcc_slab_matches_exact_clipping():
    rng = np.random.default_rng(7)
    n, C = 400, 24
    c = rng.uniform(0, 1, (C, 3))
    e = rng.uniform(0.02, 0.5, (C, 3))
    lo = (c - e).astype(np.float32)
    hi = (c + e).astype(np.float32)
    org = np.concatenate([rng.uniform(-0.5, 1.5, (n, 3)), rng.uniform(0, 0.3, (n, 1))], 1).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d[rng.uniform(size=(n, 3)) < 0.05] = 0.0  # some zero direction components
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-30)
    tmax = np.where(rng.uniform(size=(n, 1)) < 0.5, np.inf, rng.uniform(0.2, 2.0, (n, 1)))
    dir_ = np.concatenate([d, tmax], 1).astype(np.float32)
    keys = oracle.encode_hcc(org, dir_, lo, hi, 32)
    margin = oracle.key_margin(org, dir_, lo, hi, 32)
    checked = 0
    for i in range(n):
        if margin[i] < 1e-6:
            continue
        for r in range(C):
            exact = _clip_double(org[i], dir_[i], org[i, 3], dir_[i, 3], lo[r], hi[r])
            assert bool((int(keys[i]) >> (31 - r)) & 1) == exact, (i, r)
            checked += 1
    assert checked > 0.9 * n * C


# ------------------------------------------------------- slab-test margin
#
# A key bit may differ from the oracle only on a ray whose smallest relative
# slab gap |tfar - tnear| / max(1, |tnear|, |tfar|) over the boxes that drive
# key bits (the first min(cut size, k) in key order) is below 1e-6 (the
# reading of Algorithm 1's intersection test at a box boundary).  Boxes the
# ray misses through a zero direction component (an infinite distance) do
# not count.  These pins fix that function by hand-worked rays and by exact
# rational arithmetic.

UNIT_LO = np.zeros((1, 3), np.float32)
UNIT_HI = np.ones((1, 3), np.float32)


def _margin1(o, d, tmin=0.0, tmax=np.inf, lo=UNIT_LO, hi=UNIT_HI, k=32):
    org = np.array([[o[0], o[1], o[2], tmin]], np.float32)
    dir_ = np.array([[d[0], d[1], d[2], tmax]], np.float32)
    return float(oracle.key_margin(org, dir_, lo, hi, k)[0])


def test_key_margin_hand_worked_unit_box():
    # along x through the middle: the box spans t in [1, 2]: gap 1 over max(1, 1, 2) = 2
    assert _margin1((-1, 0.5, 0.5), (1, 0, 0)) == 0.5
    # through the corners (0,0,0) -> (1,1,1): t in [1, 2] on every axis
    assert _margin1((-1, -1, -1), (1, 1, 1)) == 0.5
    # touching the corner (1, 1, 1) only: x, y in [0, 1], z in [1, 2]: tnear = tfar = 1
    assert _margin1((0, 0, 2), (1, 1, -1)) == 0.0
    # origin inside, distances below 1: [max(-0.25, tmin 0), 0.75] -> 0.75 / max(1, 0, 0.75)
    assert _margin1((0.25, 0.5, 0.5), (1, 0, 0)) == 0.75
    # the interval end clips the box: [1, min(2, tmax 1.5)] -> 0.5 / 1.5
    assert abs(_margin1((-1, 0.5, 0.5), (1, 0, 0), tmax=1.5) - 1.0 / 3.0) < 1e-7
    # ... and so does its start: [max(1, tmin 1.75), 2] -> 0.25 / 2
    assert _margin1((-1, 0.5, 0.5), (1, 0, 0), tmin=1.75) == 0.125
    # a miss counts as well: the interval [1.75, 2] lies beyond tmax 1.25 -> tnear - tfar = 0.5 over 1.75
    assert abs(_margin1((-1, 0.5, 0.5), (1, 0, 0), tmin=1.75, tmax=1.25) - 0.5 / 1.75) < 1e-7
    # parallel to the x faces, outside the slab: an infinite distance, so no box counts
    assert _margin1((-1, 2, 0.5), (1, 0, 0)) == np.inf
    assert _margin1((-1, 0.5, -3), (1, 0, -0.0)) == np.inf


def test_key_margin_grazing_a_face():
    # o = (-1, 0.5, 1 - a), d = (1, 0, b) enters through x = 0 at t = 1 and leaves
    # through z = 1 at t = a / b; for a / b slightly above 1 the gap is a / b - 1
    for a, b in ((0.5, 0.49), (0.25, 0.2499), (0.5, 0.5 - 2.0 ** -20)):
        a32, b32 = float(np.float32(a)), float(np.float32(b))
        o, d = (-1.0, 0.5, float(np.float32(1.0 - a32))), (1.0, 0.0, b32)
        exact = _exact_gap(o, d, 0.0, np.inf, UNIT_LO[0], UNIT_HI[0])
        m = _margin1(o, d)
        assert exact is not None and abs(m - float(exact)) <= 4e-7 * (1 + float(exact)), (a, b, m, float(exact))
        assert 0 < m < 0.05
    # the last one is within 1e-6 of the edge: a marginal ray
    assert _margin1((-1.0, 0.5, 0.5), (1.0, 0.0, 0.5 - 2.0 ** -22)) < 1e-6


def test_key_margin_counts_only_the_boxes_that_drive_bits():
    # box 0 gives gap 0.5; box 2 (touched at a corner) gives 0: it drives a bit
    # only when the key has at least 3 bits
    lo = np.array([[0, 0, 0], [5, 5, 5], [1, 1, 1]], np.float32)
    hi = np.array([[1, 1, 1], [6, 6, 6], [2, 2, 2]], np.float32)
    o, d = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    # box 1 spans t in [6, 7] (gap 1 / 7), box 2 spans [2, 3] (gap 1 / 3)
    assert abs(_margin1(o, d, lo=lo, hi=hi, k=1) - 0.5) < 1e-7
    assert abs(_margin1(o, d, lo=lo, hi=hi, k=2) - 1.0 / 7.0) < 1e-7
    assert abs(_margin1(o, d, lo=lo, hi=hi, k=3) - 1.0 / 7.0) < 1e-7
    # a ray touching box 2's corner only: margin 0 once box 2 drives a bit
    o2, d2 = (1.0, 1.0, 3.0), (1.0, 1.0, -1.0)  # box 2: x, y in [0, 1], z in [1, 2]; boxes 0, 1: gaps 1, 1.5
    assert _margin1(o2, d2, lo=lo, hi=hi, k=3) == 0.0
    assert _margin1(o2, d2, lo=lo, hi=hi, k=2) > 0.1


def _exact_gap(o, d, tmin, tmax, lo, hi):
    """The relative slab gap in exact rationals; None for a box missed by an infinite distance."""
    tn, tf = [Fraction(float(np.float32(tmin)))], []
    if np.isfinite(tmax):
        tf.append(Fraction(float(np.float32(tmax))))
    for a in range(3):
        oa, da = Fraction(float(np.float32(o[a]))), Fraction(float(np.float32(d[a])))
        la, ha = Fraction(float(lo[a])), Fraction(float(hi[a]))
        if da == 0:
            assert oa != la and oa != ha, "origin on a slab plane: not a case for this pin"
            if not (la < oa < ha):
                return None
            continue
        ta, tb = (la - oa) / da, (ha - oa) / da
        tn.append(min(ta, tb))
        tf.append(max(ta, tb))
    if not tf:
        return None
    near, far = max(tn), min(tf)
    return abs(far - near) / max(Fraction(1), abs(near), abs(far))


def test_key_margin_matches_exact_rationals():
    rng = np.random.default_rng(11)
    n, C = 300, 12
    c = rng.uniform(0, 1, (C, 3))
    e = rng.uniform(0.02, 0.5, (C, 3))
    lo = (c - e).astype(np.float32)
    hi = (c + e).astype(np.float32)
    org = np.concatenate([rng.uniform(-0.5, 1.5, (n, 3)), rng.uniform(0, 0.3, (n, 1))], 1).astype(np.float32)
    d = rng.normal(size=(n, 3)) * rng.choice([1e-3, 1.0, 30.0], size=(n, 1))
    d[rng.uniform(size=(n, 3)) < 0.07] = 0.0  # some zero direction components
    tmax = np.where(rng.uniform(size=(n, 1)) < 0.5, np.inf, rng.uniform(0.2, 4.0, (n, 1)))
    dir_ = np.concatenate([d, tmax], 1).astype(np.float32)
    for k in (1, 5, 12, 32):
        m = oracle.key_margin(org, dir_, lo, hi, k)
        for i in range(n):
            gaps = [g for r in range(min(C, k))
                    if (g := _exact_gap(org[i, :3], dir_[i, :3], org[i, 3], dir_[i, 3], lo[r], hi[r])) is not None]
            if not gaps:
                assert m[i] == np.inf, (k, i)
                continue
            g = float(min(gaps))
            # three roundings per distance (reciprocal, difference, product): 4e-7 covers them
            assert abs(m[i] - g) <= 4e-7 * (1 + g), (k, i, m[i], g)


# ----------------------------------------------------------- HAD and the cut

@dataclass
class HandTree:
    lo: np.ndarray
    hi: np.ndarray
    left: np.ndarray
    right: np.ndarray
    count: np.ndarray


def _hand_tree():
    """An unbalanced BVH2 (in the spirit of Fig. BF) with cubic node boxes.

    id: (side, triangle count for a leaf, children)
      0 root side 4        1 A side 3          2 leaf side 2, TC 4
      3 A2 side 2          4 leaf side 1, TC 1 5 leaf side 1, TC 2
      6 B side 3           7 B1 side 2         8 leaf side 1, TC 3
      9 leaf side 1, TC 4  10 B2 side 2        11 leaf side 1, TC 1
      12 B3 side 1         13 leaf side .5, TC 2   14 leaf side .5, TC 4
    """
    side = [4, 3, 2, 2, 1, 1, 3, 2, 1, 1, 2, 1, 1, 0.5, 0.5]
    kids = {0: (1, 6), 1: (2, 3), 3: (4, 5), 6: (7, 10), 7: (8, 9), 10: (11, 12), 12: (13, 14)}
    tc = {2: 4, 4: 1, 5: 2, 8: 3, 9: 4, 11: 1, 13: 2, 14: 4}
    n = len(side)
    lo = np.zeros((n, 3), np.float32)
    hi = np.array([[s, s, s] for s in side], np.float32)
    left = np.array([kids.get(i, (-1, -1))[0] for i in range(n)], np.int32)
    right = np.array([kids.get(i, (-1, -1))[1] for i in range(n)], np.int32)
    count = np.array([tc.get(i, 0) for i in range(n)], np.uint32)
    return HandTree(lo, hi, left, right, count)


def test_surface_area_closed_forms():
    assert oracle.surface_area([0, 0, 0], [1, 1, 1]) == 6.0
    assert oracle.surface_area([0, 0, 0], [2, 3, 4]) == 2 * (6 + 12 + 8)
    assert oracle.surface_area([1, 1, 1], [1, 1, 1]) == 0.0


def test_had_hand_computed():
    # SA of a cube of side s is 6 s^2.  Leaves: TC * SA.  Internal (lambda = 1/8):
    #   A2 = 6 + 12 + 3 = 21;  A = 96 + 21 + 6.75 = 123.75
    #   B1 = 18 + 24 + 3 = 45; B3 = 3 + 6 + 0.75 = 9.75; B2 = 6 + 9.75 + 3 = 18.75
    #   B = 45 + 18.75 + 6.75 = 70.5; root = 123.75 + 70.5 + 12 = 206.25
    h = oracle.had(_hand_tree(), 0.125)
    expect = [206.25, 123.75, 96, 21, 6, 12, 70.5, 45, 18, 24, 18.75, 6, 9.75, 3, 6]
    assert h.tolist() == expect


def test_had_lambda_zero_is_leaf_sum():
    w = gen.tiny_workload(0, ntris=3000, nrays=64)
    b = w.bvh
    h = oracle.had(b, 0.0)
    leaves = b.left < 0
    ex = b.hi.astype(np.float64) - b.lo.astype(np.float64)
    sa = 2 * (ex[:, 0] * ex[:, 1] + ex[:, 1] * ex[:, 2] + ex[:, 2] * ex[:, 0])
    # same terms, different summation order
    np.testing.assert_allclose(h[0], np.sum(b.count[leaves] * sa[leaves]), rtol=1e-10)
    # with lambda > 0 a parent's HAD exceeds each child's whenever its box has area
    h = oracle.had(b, 0.125)
    inner = np.nonzero(~leaves)[0]
    assert np.all(h[inner] > h[b.left[inner]]) and np.all(h[inner] > h[b.right[inner]])


def test_cut_hand_example():
    t = _hand_tree()
    # Worked by hand from Algorithm 2 with the HADs above (see test_had_hand_computed):
    # C = 5: pop 0, pop A, pop leaf 2 (cut, max 4), pop B, pop B1 -> queue {9, 3, 10, 8}
    assert oracle.select_cut(t, 5).tolist() == [2, 9, 3, 10, 8]
    # C = 7: ... pop leaf 9 (cut, max 5), pop A2, pop B2 -> queue {8, 5, 12, 4, 11};
    # leaves 4 and 11 tie at HAD 6 and keep index order.
    assert oracle.select_cut(t, 7).tolist() == [2, 9, 8, 5, 12, 4, 11]
    assert oracle.select_cut(t, 1).tolist() == [0]
    assert oracle.select_cut(t, 2).tolist() == [1, 6]
    # more nodes than leaves: the queue empties and the cut is every leaf
    assert oracle.select_cut(t, 100).tolist() == [2, 9, 8, 5, 4, 11, 14, 13]


def _cut_invariants(b, cut, C, lam):
    h = oracle.had(b, lam)
    n = b.num_nodes if hasattr(b, "num_nodes") else len(b.left)
    parent = np.full(n, -1)
    inner = np.nonzero(b.left >= 0)[0]
    parent[b.left[inner]] = inner
    parent[b.right[inner]] = inner
    in_cut = np.zeros(n, bool)
    in_cut[cut] = True
    nleaves = int(np.sum(b.left < 0))
    assert len(cut) == min(C, nleaves) or (C == 1 and len(cut) == 1)
    # every leaf has exactly one cut node on its path to the root
    for leaf in np.nonzero(b.left < 0)[0]:
        k, m = leaf, 0
        while k >= 0:
            m += in_cut[k]
            k = parent[k]
        assert m == 1
    # ordered by HAD descending, ties by index
    key = [(-h[c], c) for c in cut]
    assert key == sorted(key)
    # greedy property: every expanded (strict ancestor of a cut node) node has
    # HAD >= every internal cut node's HAD
    expanded = set()
    for c in cut:
        k = parent[c]
        while k >= 0:
            expanded.add(k)
            k = parent[k]
    inner_cut = [c for c in cut if b.left[c] >= 0]
    if expanded and inner_cut:
        assert min(h[list(expanded)]) >= max(h[inner_cut])


@pytest.mark.parametrize("C", [1, 2, 3, 32, 64, 257])
def test_cut_invariants_on_generated_bvh(C):
    w = gen.tiny_workload(0, ntris=2000, nrays=64)
    cut = oracle.select_cut(w.bvh, C)
    _cut_invariants(w.bvh, cut, C, 0.125)


def test_cut_invariants_room_scene():
    tris = gen.room_tris(5, target_tris=20_000, clusters=6)
    b = gen.build_bvh(tris)
    for C in (32, 256, 4096):
        _cut_invariants(b, oracle.select_cut(b, C), C, 0.125)


# --------------------------------------------------------------- TwoPoint key

def test_twopoint_hand_computed():
    lo, hi = np.zeros(3, np.float32), np.ones(3, np.float32)
    # k = 32 -> 5 bits per coordinate, L = 0.25
    # ray A: o = (.5, .25, .75), d = +x -> t = (.75, .25, .75)
    #   q_o = (16, 8, 24), q_t = (24, 8, 24); level 4: 1 0 1 1 0 1, level 3: 0 1 1 1 1 1
    #   30-bit key 101101 011111 0...0, shifted left by 2 -> 0xB5F00000
    # ray B: o = 0, d = +z -> t = (0, 0, .25): only q_tz = 8 (level 3) -> bit 18 << 2 = 0x00100000
    # ray C: o = (1, 1, 1), d = 0 -> every q clamps to 31 -> 0xFFFFFFFC
    org = np.array([[.5, .25, .75, 0], [0, 0, 0, 0], [1, 1, 1, 0]], np.float32)
    dir_ = np.array([[1, 0, 0, np.inf], [0, 0, 1, np.inf], [0, 0, 0, np.inf]], np.float32)
    keys = oracle.encode_twopoint(org, dir_, lo, hi, 32)
    assert [int(k) for k in keys] == [0xB5F00000, 0x00100000, 0xFFFFFFFC]


def _morton3_magic(x, y, z):
    """Textbook 30-bit 3D Morton code via bit-spreading masks (10 bits per axis)."""
    def spread(v):
        v &= 0x3FF
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        return v
    return (spread(x) << 2) | (spread(y) << 1) | spread(z)


def test_twopoint_reduces_to_morton_when_termination_equals_origin():
    # With a zero direction the termination estimate equals the origin, so the
    # 6D key is the 3D Morton code of the origin with each 3-bit group doubled.
    rng = np.random.default_rng(3)
    n = 500
    org = np.concatenate([rng.uniform(0, 1, (n, 3)), np.zeros((n, 1))], 1).astype(np.float32)
    dir_ = np.zeros((n, 4), np.float32)
    dir_[:, 3] = np.inf
    lo, hi = np.zeros(3, np.float32), np.ones(3, np.float32)
    keys = oracle.encode_twopoint(org, dir_, lo, hi, 64)  # 10 bits per coordinate, 4 spare bits
    for i in range(n):
        q = [min(int(np.float32(org[i, a]) * np.float32(1024.0)), 1023) for a in range(3)]
        m3 = _morton3_magic(*q)
        expect = 0
        for j in range(10):
            g = (m3 >> (3 * j)) & 7
            expect |= ((g << 3) | g) << (6 * j)
        assert int(keys[i]) == expect << 4


# ---------------------------------------------------------------------- sort

@pytest.mark.parametrize("n,kmax", [(0, 1), (1, 1), (33, 1), (4097, 16), (5000, 2 ** 32), (3000, 2 ** 64 - 1)])
def test_stable_sort_characterisation(n, kmax):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, kmax, n, dtype=np.uint64, endpoint=True) if n else np.zeros(0, np.uint64)
    perm = oracle.stable_sort(keys)
    # a permutation ...
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
    sk = keys[perm]
    # ... that orders the keys ...
    assert np.all(sk[1:] >= sk[:-1])
    # ... and keeps equal keys in input order, which makes it unique
    same = sk[1:] == sk[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])


def test_gather_is_permutation_of_records():
    rng = np.random.default_rng(1)
    org = rng.normal(size=(1000, 4)).astype(np.float32)
    dir_ = rng.normal(size=(1000, 4)).astype(np.float32)
    perm = rng.permutation(1000).astype(np.uint32)
    oo, od = oracle.gather(org, dir_, perm)
    for j in (0, 1, 499, 999):
        assert oo[j].tobytes() == org[perm[j]].tobytes() and od[j].tobytes() == dir_[perm[j]].tobytes()


# --------------------------------------------------------------------- trace

def test_moller_trumbore_closed_forms():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    down = np.array([0, 0, -1], np.float32)
    assert oracle.intersect([0.25, 0.25, 1], down, 0, np.inf, tri) == (True, 1.0, 0.25, 0.25)
    assert oracle.intersect([0.5, 0.25, 3], down, 0, np.inf, tri) == (True, 3.0, 0.5, 0.25)
    assert oracle.intersect([-0.1, 0.25, 1], down, 0, np.inf, tri)[0] is False   # u < 0
    assert oracle.intersect([0.25, -0.1, 1], down, 0, np.inf, tri)[0] is False   # v < 0
    assert oracle.intersect([0.6, 0.6, 1], down, 0, np.inf, tri)[0] is False     # u + v > 1
    assert oracle.intersect([0.25, 0.25, 1], [1, 0, 0], 0, np.inf, tri)[0] is False  # parallel: det = 0
    assert oracle.intersect([0.25, 0.25, 1], down, 1.0, np.inf, tri)[0] is False  # t = tmin excluded
    assert oracle.intersect([0.25, 0.25, 1], down, 0, 1.0, tri)[0] is False       # t = tmax excluded
    assert oracle.intersect([0.25, 0.25, -1], down, 0, np.inf, tri)[0] is False   # behind the origin
    assert oracle.intersect([0.25, 0.25, -1], -down, 0, np.inf, tri)[:2] == (True, 1.0)  # two-sided


def _cramer(o, d, tri):
    """Ray/triangle by Cramer's rule in exact rationals: (t, u, v) or None."""
    F = lambda a: [Fraction(float(x)) for x in a]
    o, d = F(o), F(d)
    v0, v1, v2 = F(tri[0:3]), F(tri[3:6]), F(tri[6:9])
    e1 = [v1[i] - v0[i] for i in range(3)]
    e2 = [v2[i] - v0[i] for i in range(3)]
    s = [o[i] - v0[i] for i in range(3)]
    # solve [-d e1 e2] [t u v]^T = s
    def det3(a, b, c):
        return (a[0] * (b[1] * c[2] - b[2] * c[1]) - b[0] * (a[1] * c[2] - a[2] * c[1])
                + c[0] * (a[1] * b[2] - a[2] * b[1]))
    nd = [-x for x in d]
    D = det3(nd, e1, e2)
    if D == 0:
        return None
    return det3(s, e1, e2) / D, det3(nd, s, e2) / D, det3(nd, e1, s) / D


def test_moller_trumbore_against_exact_cramer():
    rng = np.random.default_rng(11)
    agree = 0
    for _ in range(1500):
        tri = rng.uniform(-1, 1, 9).astype(np.float32)
        o = rng.uniform(-1, 1, 3).astype(np.float32)
        target = (tri[0:3] * 0.3 + tri[3:6] * 0.3 + tri[6:9] * 0.4) + rng.normal(0, 0.3, 3)
        d = (target - o)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        hit, t, u, v = oracle.intersect(o, d, 0, np.inf, tri)
        ex = _cramer(o, d, tri)
        if ex is None:
            assert not hit
            continue
        te, ue, ve = (float(x) for x in ex)
        margin = min(ue, ve, 1 - ue - ve)
        if abs(margin) < 1e-4 or abs(te) < 1e-4:
            continue  # near an edge or the origin: rounding may decide
        assert hit == (margin > 0 and te > 0)
        if hit:
            assert abs(t - te) <= 1e-4 * max(1.0, abs(te))
            assert abs(u - ue) <= 1e-4 and abs(v - ve) <= 1e-4
        agree += 1
    assert agree > 1000


def test_trace_plane_closed_form():
    h = 2.5
    tris = np.array([[-100, -100, h, 100, -100, h, 100, 100, h],
                     [-100, -100, h, 100, 100, h, -100, 100, h]], np.float32)
    rng = np.random.default_rng(5)
    n = 2000
    o = np.concatenate([rng.uniform(-5, 5, (n, 2)), rng.uniform(-3, 2, (n, 1)), np.full((n, 1), 1e-4)], 1)
    d = np.concatenate([rng.normal(size=(n, 2)) * 0.3, rng.uniform(0.2, 1, (n, 1))], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o, d4 = o.astype(np.float32), np.concatenate([d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    hits = oracle.trace_brute(tris, o, d4)
    assert np.all(hits["prim"] >= 0)
    t_exact = (h - o[:, 2].astype(np.float64)) / d4[:, 2].astype(np.float64)
    np.testing.assert_allclose(hits["t"], t_exact, rtol=2e-6)


def _uv_sphere(r, seg=32, ring=16):
    tris = []
    for i in range(ring):
        th0, th1 = np.pi * i / ring, np.pi * (i + 1) / ring
        for j in range(seg):
            ph0, ph1 = 2 * np.pi * j / seg, 2 * np.pi * (j + 1) / seg
            P = lambda th, ph: (r * np.sin(th) * np.cos(ph), r * np.cos(th), r * np.sin(th) * np.sin(ph))
            a, b, c, d = P(th0, ph0), P(th0, ph1), P(th1, ph1), P(th1, ph0)
            if i > 0:
                tris.append(a + b + c)
            if i < ring - 1:
                tris.append(a + c + d)
    return np.array(tris, np.float32)


def test_trace_sphere_from_centre():
    r = 2.0
    tris = _uv_sphere(r)
    rng = np.random.default_rng(9)
    n = 3000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    org = np.zeros((n, 4), np.float32)
    dir_ = np.concatenate([d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    hits = oracle.trace_brute(tris, org, dir_)
    hit = hits["prim"] >= 0
    assert hit.mean() >= 0.999  # Moller-Trumbore is not watertight on shared edges
    # every point of a triangle inscribed in the sphere lies between the plane
    # distance r cos(max vertex spread) and r; the spread here is below 17 deg.
    assert np.all(hits["t"][hit] <= r * (1 + 1e-6))
    assert np.all(hits["t"][hit] >= r * np.cos(np.radians(17)))


def _tiny_scene(seed, ntris, nrays, mu=-2.0):
    """Random triangles large enough (median edge ~0.13) that many rays hit."""
    tris = gen.random_tris(seed, ntris, mu=mu)
    bvh = gen.build_bvh(tris)
    sec, _, prim = gen.camera_rays(tris, (0.5, 0.5, -1.2), (0.5, 0.5, 0.5), 45.0, 32, 32, 16, seed,
                                   sample_major=True, max_rays=nrays)
    return gen.Workload("tiny", tris, bvh, sec, None, prim)


@pytest.mark.parametrize("seed,ntris", [(0, 800), (1, 2000)])
def test_trace_bvh_equals_brute_force(seed, ntris):
    w = _tiny_scene(seed, ntris, 1500)
    org, dir_ = w.rays.org, w.rays.dir.copy()
    dir_[::3, 3] = np.float32(0.05)  # some finite tmax
    brute = oracle.trace_brute(w.tris, org, dir_)
    bvh = oracle.trace_bvh(w.bvh, org, dir_)
    assert brute.tobytes() == bvh.tobytes()
    assert (brute["prim"] >= 0).mean() > 0.2
    any_b = oracle.trace_bvh(w.bvh, org, dir_, any_hit=True)
    assert np.array_equal(any_b["prim"] >= 0, brute["prim"] >= 0)
    # any-hit reports some valid hit of the ray
    for i in np.nonzero(any_b["prim"] >= 0)[0][:200]:
        ok, t, u, v = oracle.intersect(org[i, :3], dir_[i, :3], org[i, 3], dir_[i, 3],
                                       w.tris[any_b["prim"][i]])
        assert ok and t == any_b["t"][i]


def test_trace_reorder_invariance():
    w = _tiny_scene(2, 1500, 1024)
    rng = np.random.default_rng(2)
    perm = rng.permutation(w.rays.n).astype(np.uint32)
    o2, d2 = oracle.gather(w.rays.org, w.rays.dir, perm)
    a = oracle.trace_bvh(w.bvh, w.rays.org, w.rays.dir)
    b = oracle.trace_bvh(w.bvh, o2, d2)
    assert a[perm].tobytes() == b.tobytes()


# ------------------------------------------------- Origin, Origin-Direction

def test_origin_key_is_textbook_morton():
    rng = np.random.default_rng(21)
    n = 400
    org = np.concatenate([rng.uniform(0, 1, (n, 3)), np.zeros((n, 1))], 1).astype(np.float32)
    lo, hi = np.zeros(3, np.float32), np.ones(3, np.float32)
    keys = oracle.encode_origin(org, lo, hi, 32)  # 10 bits per axis, 2 spare bits
    for i in range(n):
        q = [min(int(np.float32(org[i, a]) * np.float32(1024.0)), 1023) for a in range(3)]
        assert int(keys[i]) == _morton3_magic(*q) << 2


@pytest.mark.parametrize("d,uv", [((0, 0, 1), (0.5, 0.5)), ((1, 0, 0), (1.0, 0.5)), ((-1, 0, 0), (0.0, 0.5)),
                                  ((0, 1, 0), (0.5, 1.0)), ((0, -1, 0), (0.5, 0.0)), ((0, 0, -1), (1.0, 1.0)),
                                  ((1, 1, 1), (2 / 3, 2 / 3)), ((0, 0, 0), (0.5, 0.5))])
def test_octahedral_map_closed_forms(d, uv):
    u, v = oracle.octahedral(np.array(d, np.float32))
    assert abs(u - uv[0]) < 1e-6 and abs(v - uv[1]) < 1e-6


def test_octahedral_map_inverts():
    """Decode (u, v) with the inverse octahedral map and recover the direction."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        u, v = oracle.octahedral(d.astype(np.float32))
        x, y = 2 * u - 1, 2 * v - 1
        z = 1 - abs(x) - abs(y)
        if z < 0:
            x, y = (1 - abs(y)) * np.sign(x if x != 0 else 1), (1 - abs(x)) * np.sign(y if y != 0 else 1)
        r = np.array([x, y, z])
        r /= np.linalg.norm(r)
        assert np.allclose(r, d, atol=1e-5)


def test_origin_dir_hand_computed():
    # k = 16: bd = 2 bits per direction coordinate, bo = 4 bits per origin axis.
    # o = (.5, .25, .75) -> q = (8, 4, 12): levels x y z: 101, 011, 000, 000 -> 101011000000
    # d = +z -> (u, v) = (.5, .5) -> q = (2, 2): levels u v: 11, 00 -> 1100
    # key = 101011000000 1100 = 0xAC0C
    org = np.array([[.5, .25, .75, 0]], np.float32)
    dir_ = np.array([[0, 0, 1, np.inf]], np.float32)
    k = oracle.encode_origin_dir(org, dir_, np.zeros(3, np.float32), np.ones(3, np.float32), 16)
    assert int(k[0]) == 0xAC0C
    # 32 bits: bd = 5, bo = 7 -> 31 bits used, one pad bit at the bottom
    k32 = int(oracle.encode_origin_dir(org, dir_, np.zeros(3, np.float32), np.ones(3, np.float32), 32)[0])
    assert k32 & 1 == 0 and k32 >> 11 == _morton3_magic(64, 32, 96)  # origin part: 7-bit coords


def test_anc_closed_forms():
    perm = np.arange(64, dtype=np.uint32)
    assert oracle.anc(np.zeros(64, np.uint64), perm) == 1.0
    assert oracle.anc(np.arange(64, dtype=np.uint64), perm) == 32.0
    keys = np.repeat(np.arange(8, dtype=np.uint64), 8)  # each warp of 32 holds 4 codes
    assert oracle.anc(keys, perm) == 4.0


# ------------------------------------------------------------- next bounce

def test_spawn_rays_are_cosine_distributed_on_the_visible_side():
    """Spawned directions are unit, on the side facing the incoming ray, and
    cosine-distributed: E[cos] = 2/3 and E[cos^2] = 1/2 about the normal."""
    tri = np.array([[0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)  # normal +z
    n = 20000
    org = np.tile(np.array([[0.25, 0.25, 1.0, 1e-4]], np.float32), (n, 1))
    dir_ = np.tile(np.array([[0, 0, -1, np.inf]], np.float32), (n, 1))
    hits = np.zeros(n, oracle.HIT_DTYPE)
    hits["prim"], hits["t"] = 0, 1.0
    oo, od = oracle.spawn(org, dir_, hits, tri, seed=7, tmin=1e-4)
    assert np.allclose(oo[:, :3], [0.25, 0.25, 0.0]) and np.all(oo[:, 3] == np.float32(1e-4))
    c = od[:, 2].astype(np.float64)
    assert np.all(c >= 0) and np.allclose(np.linalg.norm(od[:, :3], axis=1), 1, atol=1e-5)
    assert abs(c.mean() - 2 / 3) < 0.01 and abs((c ** 2).mean() - 0.5) < 0.01
    # incoming from below: the normal flips, directions go to -z
    _, od2 = oracle.spawn(org * [1, 1, -1, 1], -dir_ * [1, 1, 1, -1], hits, tri, seed=7, tmin=1e-4)
    assert np.all(od2[:, 2] <= 0)
    # misses become empty rays, and the draw depends on the seed
    hits["prim"][::2] = -1
    oo3, od3 = oracle.spawn(org, dir_, hits, tri, seed=7, tmin=1e-4)
    assert np.all(oo3[::2, 3] == 1) and np.all(od3[::2, 3] == 0)
    _, od4 = oracle.spawn(org, dir_, hits, tri, seed=8, tmin=1e-4)
    assert not np.array_equal(od3[1::2], od4[1::2])


def test_twopoint_length_fraction_scales_the_direction():
    # termination o + (f * E) d: for powers of two, f = 0.5 with d equals f = 0.25 with 2 d
    # bit for bit (the scalings are exact), and f = 0 puts the termination on the origin
    w = gen.tiny_workload(0, ntris=2000, nrays=1500)
    o, d = w.rays.org, w.rays.dir
    lo, hi = w.bvh.lo[0], w.bvh.hi[0]
    base = oracle.encode_twopoint(o, d, lo, hi, 60)
    assert np.array_equal(base, oracle.encode_twopoint(o, d, lo, hi, 60, fraction=0.25))
    for f, s in ((0.5, 2.0), (1.0, 4.0), (0.125, 0.5)):
        d2 = d.copy()
        d2[:, :3] *= s
        assert np.array_equal(oracle.encode_twopoint(o, d, lo, hi, 60, fraction=f),
                              oracle.encode_twopoint(o, d2, lo, hi, 60))
    zero = d.copy()
    zero[:, :3] = 0.0
    assert np.array_equal(oracle.encode_twopoint(o, d, lo, hi, 60, fraction=0.0),
                          oracle.encode_twopoint(o, zero, lo, hi, 60))
    assert not np.array_equal(oracle.encode_twopoint(o, d, lo, hi, 60, fraction=0.75), base)
