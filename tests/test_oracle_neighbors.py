"""Pins of the neighbour predicate (reading X10) against counts fixed by geometry."""
import itertools

import numpy as np
import pytest

import scenes
from oracle import neighbors


def _lattice_offsets(radius):
    # integer offsets strictly inside the support radius (in units of dx)
    r = int(np.ceil(radius))
    out = []
    for v in itertools.product(range(-r, r + 1), repeat=3):
        if v != (0, 0, 0) and v[0] ** 2 + v[1] ** 2 + v[2] ** 2 < radius ** 2:
            out.append(v)
    return out


def test_lattice_count_is_80():
    # h = 1.3 dx, support 2.6 dx: the paper gives about 80 neighbours; the exact lattice count is 80
    assert len(_lattice_offsets(2.6)) == 80
    s = scenes.periodic_lattice(8)
    off, idx = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    counts = np.diff(off)
    assert np.all(counts == 80)


def test_gaussian_lattice_count_is_250():
    # truncated Gaussian, support 3h = 3.9 dx: the paper gives about 250 neighbours; the exact
    # lattice count is 250, and brute force and the k-d tree find it on every particle
    assert len(_lattice_offsets(3.9)) == 250
    s = scenes.periodic_lattice(12, kernel=scenes.KERNEL_GAUSSIAN)
    for method in ("bruteforce", "kdtree"):
        off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h, method, kernel_id=s.kernel)
        assert np.all(np.diff(off) == 250)


def test_gaussian_sets_contain_the_wendland_sets():
    s = scenes.random_box(8, nf=1600)
    sg = s.copy()
    sg.kernel = scenes.KERNEL_GAUSSIAN
    ow, iw = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    og, ig = neighbors.bruteforce(sg.pos, sg.lo, sg.hi, sg.periodic, sg.h, kernel_id=sg.kernel)
    ok, ik = neighbors.kdtree(sg.pos, sg.lo, sg.hi, sg.periodic, sg.h, kernel_id=sg.kernel)
    assert np.array_equal(og, ok) and np.array_equal(ig, ik)
    for b in range(s.n):
        assert set(iw[ow[b]:ow[b + 1]]) <= set(ig[og[b]:og[b + 1]])


def test_dummy_wall_layers_see_30_9_0():
    # wall layers at (k + 1/2) dx below the fluid: fluid neighbours 30, 9 and 0
    s = scenes.couette(0)
    off, idx = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    y = s.pos[:, 1].astype(np.float64)
    dx = s.dx
    for k, expect in enumerate((30, 9, 0)):
        rows = np.flatnonzero((s.ptype == scenes.WALL) & np.isclose(y, -(k + 0.5) * dx))
        assert rows.size == 200
        for b in rows:
            nb = idx[off[b]:off[b + 1]]
            assert np.count_nonzero(s.ptype[nb] == scenes.FLUID) == expect


@pytest.mark.parametrize("seed,periodic", [(0, (1, 0, 1)), (1, (0, 0, 0)), (2, (1, 1, 1)), (3, (0, 1, 0))])
def test_kdtree_equals_bruteforce(seed, periodic):
    s = scenes.random_box(seed, nf=300, periodic=periodic)
    a = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    b = neighbors.kdtree(s.pos, s.lo, s.hi, s.periodic, s.h)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_kdtree_equals_bruteforce_jittered_box():
    s = scenes.lava_box(0, n=10)
    a = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    b = neighbors.kdtree(s.pos, s.lo, s.hi, s.periodic, s.h)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_relation_is_symmetric_and_sorted():
    s = scenes.random_box(5, nf=250)
    off, idx = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    pairs = set()
    for b in range(s.n):
        row = idx[off[b]:off[b + 1]]
        assert np.all(np.diff(row) > 0) and b not in row
        pairs.update((int(b), int(a)) for a in row)
    assert all((a, b) in pairs for (b, a) in pairs)


def test_minimum_image_and_strict_edge():
    # two particles across a periodic face are neighbours; a pair just outside
    # the support is not; a pair at exactly float distance below it is
    h = np.float32(0.01)
    lo, hi = np.zeros(3), np.array([0.1, 0.1, 0.1])
    pos = np.zeros((4, 4), np.float32)
    pos[0, :3] = (0.002, 0.05, 0.05)
    pos[1, :3] = (0.098, 0.05, 0.05)   # 0.004 away through the x face
    pos[2, :3] = (0.05, 0.05, 0.05)
    pos[3, :3] = (0.05, 0.05 + 0.0200001, 0.05)  # just beyond 2h = 0.02
    off, idx = neighbors.bruteforce(pos, lo, hi, (1, 0, 0), h)
    assert list(idx[off[0]:off[1]]) == [1]
    assert list(idx[off[2]:off[3]]) == []
    off2, idx2 = neighbors.bruteforce(pos, lo, hi, (0, 0, 0), h)
    assert list(idx2[off2[0]:off2[1]]) == []


def test_rows_for_matches_full_build():
    s = scenes.random_box(7, nf=200)
    off, idx = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    rows = [0, 17, s.n - 1]
    for b, nb in zip(rows, neighbors.rows_for(s, rows)):
        np.testing.assert_array_equal(nb, idx[off[b]:off[b + 1]])
