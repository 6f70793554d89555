"""Pins of the oracle's geometry against counts the paper states and brute-force enumeration."""
import os

import numpy as np
import pytest

from oracle import geometry as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_surface_counts_match_closed_form():
    for p, n in _golden_rows("surface_counts.txt"):
        assert G.n_surface(int(p)) == int(n)


@pytest.mark.parametrize("p", [2, 3, 4, 7])
def test_surface_points_lie_on_the_cube(p):
    w, alpha = 0.25, 1.05
    c = np.array([0.3, -0.2, 0.7])
    pts = G.surface_points(p, c, w, alpha)
    d = np.abs(pts - c)
    half = alpha * w / 2
    # every point on the boundary of the cube of half-side alpha*w/2, none outside it
    assert np.allclose(np.max(d, axis=1), half)
    assert np.all(d <= half + 1e-15)
    # lattice spacing alpha*w/(p-1) along each axis and all points distinct
    steps = (pts - (c - half)) / (alpha * w / (p - 1))
    assert np.allclose(steps, np.round(steps))
    assert len(np.unique(np.round(steps).astype(int), axis=0)) == len(pts)
    # every face carries a full p x p lattice
    for axis in range(3):
        for side in (-1, 1):
            on = np.isclose(pts[:, axis] - c[axis], side * half)
            assert on.sum() == p * p


def test_morton_roundtrip_and_order():
    level = 4
    keys = np.arange(8 ** level)
    idx = G.morton_decode(keys, level)
    assert np.array_equal(G.morton_encode(idx, level), keys)
    # x is the lowest bit of each triple
    assert tuple(G.morton_decode(np.array(1), level)) == (1, 0, 0)
    assert tuple(G.morton_decode(np.array(2), level)) == (0, 1, 0)
    assert tuple(G.morton_decode(np.array(4), level)) == (0, 0, 1)
    assert tuple(G.morton_decode(np.array(8), level)) == (2, 0, 0)


def test_paper_counts():
    gold = {r[0]: int(r[1]) for r in _golden_rows("paper_counts.txt")}
    assert len(G.transfer_vectors()) == gold["transfer_vectors"]
    sizes = [len(G.interaction_list(tau, 3)) for tau in G.all_boxes(3)]
    assert max(sizes) == gold["max_interaction_list"] == gold["far_field_of_target"]
    # union of transfer vectors met over a deep level is the full set
    seen = set()
    for tau in G.all_boxes(3):
        for s in G.interaction_list(tau, 3):
            seen.add(tuple(np.subtract(s, tau)))
    assert len(seen) == gold["transfer_vectors"]
    # App. A.1 cluster view: 26 source clusters x 64 pairs, of which 8 x 189 are far pairs
    n_far = 0
    for d in np.ndindex(3, 3, 3):
        d = np.array(d) - 1
        if not d.any():
            continue
        for ct in np.ndindex(2, 2, 2):
            for cs in np.ndindex(2, 2, 2):
                t = 2 * d + np.array(cs) - np.array(ct)
                n_far += int(np.max(np.abs(t)) >= 2)
    assert n_far == 8 * gold["max_interaction_list"]
    assert 26 * 64 == gold["source_clusters"] * gold["cluster_pairs"]


def test_interaction_list_brute_force_level3():
    """Independent statement of I_tau: all pairs at the level, filtered by the two conditions."""
    level = 3
    boxes = G.all_boxes(level)
    for ti in range(0, len(boxes), 7):
        tau = boxes[ti]
        expect = []
        for s in boxes:
            parents_near = np.max(np.abs(s // 2 - tau // 2)) <= 1
            far = np.max(np.abs(s - tau)) >= 2
            if parents_near and far:
                expect.append(tuple(s))
        got = G.interaction_list(tau, level)
        assert sorted(got) == sorted(expect)


@pytest.mark.parametrize("level", [2, 3, 4])
def test_pair_counts_two_ways(level):
    from oracle import m2l as M
    assert M.pair_count(level) == G.pair_count_closed_form(level)


def test_pair_counts_values():
    # levels 2..6 of a full non-periodic tree (closed form); levels 2..3 for the 8k-point tree,
    # 2..5 for the 1M-point tree and 2..6 for the 8M-point tree of the workloads
    vals = [G.pair_count_closed_form(l) for l in range(2, 7)]
    assert vals == [3096, 53352, 584136, 5398920, 46298376]


def test_vectorised_lists_match_loop_lists_sparse():
    level = 3
    rng = np.random.default_rng(3)
    keys = np.sort(rng.choice(8 ** level, size=200, replace=False))
    occ = {tuple(v) for v in G.morton_decode(keys, level)}
    from oracle import m2l as M
    rows, boxes, offsets, src, srow = M.interaction_csr(level, keys)
    for i in range(len(keys)):
        tau = boxes[i]
        expect = G.interaction_list(tau, level, occ)
        got = [tuple(v) for v in src[offsets[i]:offsets[i + 1]]]
        assert got == expect
        assert np.array_equal(keys[srow[offsets[i]:offsets[i + 1]]],
                              G.morton_encode(np.array(expect).reshape(-1, 3), level))


def test_occupied_boxes_parent_closure():
    rng = np.random.default_rng(5)
    pts = rng.random((500, 3))
    k4 = G.occupied_boxes(pts, 4, (0, 0, 0), 1.0)
    k3 = G.occupied_boxes(pts, 3, (0, 0, 0), 1.0)
    assert np.array_equal(np.unique(k4 >> 3), k3)
