"""Pins for the oracle's method variants (CPU only): the multi-level
hierarchy cut code (Sec. 4.3, Algorithm 3), regular grid encoding (Sec. 5)
and the prefix path code (Sec. 4.1)."""
import os

import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen
from test_oracle_pins import HandTree, _hand_tree, _read_golden

# ------------------------------------------------------------------ MLHCC cut


def _ids(a):
    return [list(map(int, r)) for r in a]


def test_mlhcc_cut_hand_example():
    t = _hand_tree()
    # HADs (test_had_hand_computed): 0 206.25, A=1 123.75, 2 96, A2=3 21, 4 6, 5 12, B=6 70.5,
    # B1=7 45, 8 18, 9 24, B2=10 18.75, 11 6, B3=12 9.75, 13 3, 14 6.
    # Leaves under: 0:8, 1:3, 3:2, 6:5, 7:2, 10:3, 12:2, leaves:1.
    # T=2, L=2: pop 0 -> {1, 6}; low cuts by Algorithm 2 on each subtree.
    top, low = oracle.select_cut_ml(t, 2, 2)
    assert top.tolist() == [1, 6] and _ids(low) == [[2, 3], [7, 10]]
    # T=4, L=2: pop 0 -> {1, 6}; pop 1 -> leaf 2 discarded, push 3; pop 6 -> {3, 7, 10};
    # pop 7 (no eligible child) -> list, max 3; pop 3 -> list, max 2; pop 10 -> leaf 11
    # discarded, push 12; pop 12 -> list, max 1; queue empty.
    top, low = oracle.select_cut_ml(t, 4, 2)
    assert top.tolist() == [7, 3, 12] and _ids(low) == [[9, 8], [5, 4], [14, 13]]
    # T=3, L=3: eligible nodes 0, 1, 6, 10.  pop 0 -> {1, 6}; pop 1 -> list, max 2;
    # pop 6 -> push 10 (7 discarded); pop 10 -> list, max 1.
    # Low cut of 1 with 3 nodes: pop 1 -> {2, 3}; pop leaf 2 -> cut, max 2; pop 3 -> {4, 5}.
    # Low cut of 10: pop 10 -> {11, 12}; pop 12 -> {11, 13, 14}; 11 and 14 tie at HAD 6.
    top, low = oracle.select_cut_ml(t, 3, 3)
    assert top.tolist() == [1, 10] and _ids(low) == [[2, 5, 4], [11, 14, 13]]
    # a low level larger than the whole tree leaves no eligible top node
    top, low = oracle.select_cut_ml(t, 4, 9)
    assert top.size == 0
    # one top node: the root, whose low cut is the cut of Algorithm 2
    top, low = oracle.select_cut_ml(t, 1, 8)
    assert top.tolist() == [0] and low[0].tolist() == oracle.select_cut(t, 8).tolist()


@pytest.mark.parametrize("T", [1, 2, 8, 16, 33])
def test_mlhcc_with_single_low_nodes_reduces_to_hcc_cut(T):
    w = gen.tiny_workload(0, ntris=2000, nrays=64)
    top, low = oracle.select_cut_ml(w.bvh, T, 1)
    assert top.tolist() == oracle.select_cut(w.bvh, T).tolist()
    assert low[:, 0].tolist() == top.tolist()


def _subtree(b, n):
    out, stack = [], [n]
    while stack:
        k = stack.pop()
        out.append(k)
        if b.left[k] >= 0:
            stack += [int(b.left[k]), int(b.right[k])]
    return out


@pytest.mark.parametrize("T,L", [(8, 8), (16, 16), (4, 32), (32, 2)])
def test_mlhcc_cut_invariants(T, L):
    tris = gen.room_tris(5, target_tris=20_000, clusters=6)
    b = gen.build_bvh(tris)
    h = oracle.had(b, 0.125)
    top, low = oracle.select_cut_ml(b, T, L)
    assert 1 <= top.size <= T and low.shape == (top.size, L)
    assert [(-h[c], c) for c in top] == sorted((-h[c], c) for c in top)
    subs = {int(t): set(_subtree(b, int(t))) for t in top}
    for i, t in enumerate(top):
        leaves = [k for k in subs[int(t)] if b.left[k] < 0]
        assert len(leaves) >= L  # eligible: its subtree supplies L low nodes
        for u in top[i + 1:]:
            assert int(u) not in subs[int(t)] and int(t) not in subs[int(u)]  # top nodes are disjoint
        # the low cut covers the top node's leaves once each and lies in its subtree
        assert set(low[i].tolist()) <= subs[int(t)] and len(set(low[i].tolist())) == L
        low_subs = [set(_subtree(b, int(c))) for c in low[i]]
        for leaf in leaves:
            assert sum(leaf in sub for sub in low_subs) == 1
        assert [(-h[c], c) for c in low[i]] == sorted((-h[c], c) for c in low[i])


# --------------------------------------------------------------- MLHCC keys

def _mlhcc_figure_boxes():
    """Eight top boxes in a row along x (unit cells, id order permuted so that
    a segment can cross ids 1, 3, 4, 5 only), each holding eight low boxes of
    width 1/8 in x, in the lower (y in [0, .5]) or upper half of the cell."""
    pos = {0: 0, 2: 1, 1: 2, 3: 3, 4: 4, 5: 5, 6: 6, 7: 7}  # top id -> cell position
    lower = {1: {1, 2, 4, 5}, 6: {2, 3, 4, 5, 6}}
    top_lo = np.array([[pos[t], 0, 0] for t in range(8)], np.float32)
    top_hi = np.array([[pos[t] + 1, 1, 1] for t in range(8)], np.float32)
    low_lo = np.zeros((8, 8, 3), np.float32)
    low_hi = np.zeros((8, 8, 3), np.float32)
    for t in range(8):
        for j in range(8):
            y0 = 0.0 if j in lower.get(t, set()) else 0.5
            low_lo[t, j] = (pos[t] + j / 8, y0, 0)
            low_hi[t, j] = (pos[t] + (j + 1) / 8, y0 + 0.5, 1)
    return top_lo, top_hi, low_lo, low_hi


def test_mlhcc_codes_of_the_figure():
    golden = _read_golden("mlhcc_codes.txt")
    top_lo, top_hi, low_lo, low_hi = _mlhcc_figure_boxes()
    # horizontal segments at y = 0.25, z = 0.5: ray1 spans x 2.2 .. 5.8 (top cells at
    # positions 2-5 = ids 1, 3, 4, 5; inside id 1 the low boxes at x >= 2.2 in the lower
    # half are 1, 2, 4, 5); ray2 spans x 6.2 .. 7.8 (ids 6, 7; low boxes 2-6 of id 6)
    segs = {"ray1": (2.2, 3.6), "ray2": (6.2, 1.6)}
    for name, (x0, dx) in segs.items():
        org = np.array([[x0, 0.25, 0.5, 0.0]], np.float32)
        dir_ = np.array([[dx, 0.0, 0.0, 1.0]], np.float32)
        key = int(oracle.encode_mlhcc(org, dir_, 8, top_lo, top_hi, low_lo, low_hi, 16)[0])
        assert format(key, "016b") == golden[name], name


def test_mlhcc_key_reductions():
    w = gen.tiny_workload(0, ntris=3000, nrays=2000)
    b, r = w.bvh, w.rays
    # one low node per top node (the node itself): the key is HCC of the top cut with
    # one more bit that says whether any top node was met
    top, low = oracle.select_cut_ml(b, 12, 1)
    k = oracle.encode_mlhcc(r.org, r.dir, 12, b.lo[top], b.hi[top], b.lo[low], b.hi[low], 16)
    h = oracle.encode_hcc(r.org, r.dir, b.lo[top], b.hi[top], 16)
    any_top = (h != 0).astype(np.uint64)
    assert np.array_equal(k, h | (any_top << np.uint64(3)))
    # the low field of the representative equals HCC of that node's low cut
    top, low = oracle.select_cut_ml(b, 8, 8)
    k = oracle.encode_mlhcc(r.org, r.dir, 8, b.lo[top], b.hi[top], b.lo[low], b.hi[low], 24)
    h = oracle.encode_hcc(r.org, r.dir, b.lo[top], b.hi[top], 8)
    assert np.array_equal(k >> np.uint64(16), h)
    met = np.nonzero(h)[0]
    assert met.size > 100
    for i in met[:200]:
        rep = 8 - int(h[i]).bit_length()  # first set bit from the MSB
        lk = oracle.encode_hcc(r.org[i:i + 1], r.dir[i:i + 1], b.lo[low[rep]], b.hi[low[rep]], 8)[0]
        assert (int(k[i]) >> 8) & 0xFF == int(lk)
        assert int(k[i]) & 0xFF == 0
    assert np.all(k[h == 0] == 0)


# ------------------------------------------------------------- regular grid

def test_grid_cells_hand_computed():
    # cube: halve x, y, z, x, y -> 4 x 4 x 2 for 32 cells; 24 cells -> 16
    lo, hi, dims = oracle.grid_cells([0, 0, 0], [1, 1, 1], 32)
    assert dims.tolist() == [4, 4, 2] and lo.shape == (32, 3)
    assert oracle.grid_cells([0, 0, 0], [1, 1, 1], 24)[2].tolist() == [4, 2, 2]
    # the 10 x 3 x 8 room: x (5, 3, 8) -> z (5, 3, 4) -> x (2.5, 3, 4) -> z (2.5, 3, 2) -> y
    lo, hi, dims = oracle.grid_cells([0, 0, 0], [10, 3, 8], 32)
    assert dims.tolist() == [4, 2, 4]
    # cell (i, j, l) = number (i gy + j) gz + l
    r = (1 * 2 + 1) * 4 + 2
    assert lo[r].tolist() == [2.5, 1.5, 4.0] and hi[r].tolist() == [5.0, 3.0, 6.0]
    assert oracle.grid_cells([0, 0, 0], [1, 1, 1], 1)[2].tolist() == [1, 1, 1]


@pytest.mark.parametrize("cells", [1, 7, 32, 64])
def test_grid_cells_partition_the_box(cells):
    slo = np.array([-0.37, 1.1, -5.0], np.float32)
    shi = np.array([2.9, 1.35, 7.25], np.float32)
    lo, hi, dims = oracle.grid_cells(slo, shi, cells)
    m = lo.shape[0]
    assert m == int(np.prod(dims)) and m <= cells and 2 * m > cells
    assert np.all(lo <= hi)
    vol = np.prod(hi.astype(np.float64) - lo.astype(np.float64), axis=1).sum()
    assert np.isclose(vol, np.prod(shi.astype(np.float64) - slo.astype(np.float64)), rtol=1e-6)
    assert np.array_equal(lo.min(0), slo) and np.array_equal(hi.max(0), shi)
    # neighbours share their face exactly; interiors do not overlap
    g = dims.tolist()
    grid_lo = lo.reshape(g + [3])
    grid_hi = hi.reshape(g + [3])
    assert np.array_equal(grid_hi[:-1, :, :, 0], grid_lo[1:, :, :, 0])
    assert np.array_equal(grid_hi[:, :-1, :, 1], grid_lo[:, 1:, :, 1])
    assert np.array_equal(grid_hi[:, :, :-1, 2], grid_lo[:, :, 1:, 2])


def test_grid_key_closed_form():
    lo, hi, dims = oracle.grid_cells([0, 0, 0], [4, 4, 2], 32)  # 4 x 4 x 2 unit cells
    assert dims.tolist() == [4, 4, 2]
    # a ray along +x through the centre of row (j, l) meets the four cells of that row
    for j in range(4):
        for l in range(2):
            org = np.array([[-1.0, j + 0.5, l + 0.5, 0.0]], np.float32)
            dir_ = np.array([[1.0, 0.0, 0.0, np.inf]], np.float32)
            key = int(oracle.encode_hcc(org, dir_, lo, hi, 32)[0])
            expect = sum(1 << (31 - ((i * 4 + j) * 2 + l)) for i in range(4))
            assert key == expect


# -------------------------------------------------------------- prefix path

def _ppc_tree():
    """Pre-order tree: R=0 [0,4]^2, A=1 left half with leaves A1=2 (top strip)
    and A2=3 (bottom strip), B=4 right half with leaves B1=5 (upper) and B2=6 (lower)."""
    lo = np.array([[0, 0, 0], [0, 0, 0], [0, 3, 0], [0, 0, 0], [2, 0, 0], [2, 2, 0], [2, 0, 0]], np.float32)
    hi = np.array([[4, 4, 1], [2, 4, 1], [2, 4, 1], [2, 1, 1], [4, 4, 1], [4, 4, 1], [4, 2, 1]], np.float32)
    left = np.array([1, 2, -1, -1, 5, -1, -1], np.int32)
    right = np.array([4, 3, -1, -1, 6, -1, -1], np.int32)
    count = np.array([0, 0, 1, 1, 0, 1, 1], np.uint32)
    return HandTree(lo, hi, left, right, count)


def test_ppc_example_of_the_figure():
    # Sec. 4.1 figure: the first four results true, true, false, false give 1100.
    # The segment (0.5, 2) -> (3.5, 2.5) meets R and A, passes between A1 and A2,
    # then meets B and B1 (y >= 2.25 for x >= 2) but not B2.
    t = _ppc_tree()
    org = np.array([[0.5, 2.0, 0.5, 0.0]], np.float32)
    dir_ = np.array([[3.0, 0.5, 0.0, 1.0]], np.float32)
    assert format(int(oracle.encode_ppc(org, dir_, t, 4)[0]), "04b") == "1100"
    assert format(int(oracle.encode_ppc(org, dir_, t, 8)[0]), "08b") == "11001100"  # 7 tests, then 0
    assert int(oracle.encode_ppc(org, dir_, t, 1)[0]) == 1
    miss = np.array([[9.0, 9.0, 9.0, 0.0]], np.float32)
    assert int(oracle.encode_ppc(miss, dir_, t, 8)[0]) == 0  # root missed: one test, result 0


def test_ppc_equals_preorder_walk_of_node_hits():
    """PPC rebuilt from per-node box results (HCC bits with every node as a cut
    node) by walking node ids in pre-order and jumping over missed subtrees."""
    w = gen.tiny_workload(0, ntris=1500, nrays=300)
    b = w.bvh
    n = b.num_nodes
    size = np.ones(n, np.int64)
    for k in range(n - 1, -1, -1):  # pre-order: children after parents
        if b.left[k] >= 0:
            size[k] = 1 + size[b.left[k]] + size[b.right[k]]
    assert size[0] == n
    for kb in (16, 64):
        ppc = oracle.encode_ppc(w.rays.org, w.rays.dir, b, kb)
        for i in range(0, w.rays.n, 7):
            met = np.zeros(n, bool)
            for c in range(0, n, 64):
                ids = np.arange(c, min(c + 64, n))
                h = int(oracle.encode_hcc(w.rays.org[i:i + 1], w.rays.dir[i:i + 1], b.lo[ids], b.hi[ids], 64)[0])
                met[ids] = [(h >> (63 - r)) & 1 for r in range(ids.size)]
            key, m, k = 0, 0, 0
            while k < n and m < kb:
                if met[k]:
                    key |= 1 << (kb - 1 - m)
                    k += 1
                else:
                    k += size[k]
                m += 1
            assert int(ppc[i]) == key, i
