"""The oracle against values the paper prints: the point counts of its
benchmark stencils (Table I, tests/golden/table1_points.txt).  The count is
read off the oracle's impulse response with every weight nonzero, so a
dropped or doubled offset in the oracle's star or box changes it; the 2D
kernels are the 3D oracle with its z weights zeroed (the centre kept)."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    rows = []
    for line in open(os.path.join(HERE, "golden", "table1_points.txt")):
        line = line.split("#")[0].split()
        if line:
            name, dims, shape, r, pts = line
            rows.append((name, int(dims), shape, int(r), int(pts)))
    return rows


def impulse_points(shape, r, dims, seed):
    g = np.random.default_rng(seed)
    w = 2 * r + 1
    if shape == "star":
        c = g.uniform(0.5, 1.5, (3, w)) * g.choice([-1.0, 1.0], (3, w))
        if dims == 2:
            c[2, :] = 0.0
            c[2, r] = 0.25            # the z axis keeps only a centre weight
    else:
        c = g.uniform(0.5, 1.5, (w, w, w)) * g.choice([-1.0, 1.0], (w, w, w))
        if dims == 2:
            keep = c[r].copy()
            c[:] = 0.0
            c[r] = keep               # only the plane dz = 0
    n = 2 * w + 1                     # interior big enough to hold the whole response
    grid = np.zeros((n + 2 * r,) * 3)
    grid[r + n // 2, r + n // 2, r + n // 2] = 1.0
    out = oracle.stencil(shape, r, c, grid)
    return int(np.count_nonzero(out))


@pytest.mark.parametrize("row", table1(), ids=lambda row: row[0])
def test_table1_point_counts(row):
    name, dims, shape, r, pts = row
    assert impulse_points(shape, r, dims, seed=r * 10 + dims) == pts
    if dims == 3:
        assert oracle.n_points(shape, r) == pts
    else:
        # the oracle's own planar stencil touches the same number of points
        shape2 = shape + "2d"
        assert oracle.n_points(shape2, r) == pts
        g = np.random.default_rng(r)
        c = g.uniform(0.5, 1.5, oracle.n_coeffs(shape2, r)) * g.choice([-1.0, 1.0], oracle.n_coeffs(shape2, r))
        n = 4 * r + 3
        grid = np.zeros((1, n + 2 * r, n + 2 * r))
        grid[0, r + n // 2, r + n // 2] = 1.0
        assert np.count_nonzero(oracle.stencil2d(shape2, r, c, grid)) == pts
