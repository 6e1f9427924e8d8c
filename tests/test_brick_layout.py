"""The voxel-brick order of CSR(D^T)'s columns (build option vox_grid), on the host.

The layout the header defines: bricks of 4 x 4 x 2 voxels (the 32 floats of one
128-byte line of g), bricks in x-fastest order over the grid padded up to whole
bricks, x fastest inside a brick, then y, then z.  These tests check that this
numbering is a one-to-one map of the voxels into the padded positions, and the
reason for it: on the 128x128x96 head-and-neck geometry, the 32 consecutive
entries of a beamlet row that a warp gathers at once touch about half as many
128-byte lines of g as in the grid's own voxel order.
"""
import numpy as np

import synth


def brick_pos(v, nx, ny, nz):
    nbx, nby = (nx + 3) // 4, (ny + 3) // 4
    x = v % nx
    y = (v // nx) % ny
    z = v // (nx * ny)
    brick = ((z // 2) * nby + y // 4) * nbx + x // 4
    return brick * 32 + (z % 2) * 16 + (y % 4) * 4 + x % 4


def n_positions(nx, ny, nz):
    return ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 1) // 2) * 32


def test_brick_order_is_one_to_one():
    for nx, ny, nz in ((8, 8, 8), (13, 11, 9), (1, 1, 1), (5, 3, 1), (128, 128, 96), (30, 35, 20)):
        v = np.arange(nx * ny * nz, dtype=np.int64)
        p = brick_pos(v, nx, ny, nz)
        assert p.min() >= 0 and p.max() < n_positions(nx, ny, nz)
        assert len(np.unique(p)) == len(p)
    # whole bricks: every position is a voxel, and the 32 voxels of a brick are one line
    nx, ny, nz = 16, 8, 4
    p = brick_pos(np.arange(nx * ny * nz), nx, ny, nz)
    assert np.array_equal(np.sort(p), np.arange(nx * ny * nz))
    x, y, z = np.meshgrid(np.arange(4), np.arange(4, 8), np.arange(2, 4), indexing="ij")
    line = np.unique(brick_pos(((z * ny + y) * nx + x).ravel(), nx, ny, nz) // 32)
    assert len(line) == 1


def _lines_per_chunk(col, blt):
    """Mean number of distinct 128-byte lines (32 floats) touched by 32 consecutive
    entries of a row, rows sorted by column and cut into chunks from each row start."""
    order = np.lexsort((col, blt))
    c, b = col[order], blt[order]
    start = np.r_[0, np.flatnonzero(b[1:] != b[:-1]) + 1]
    row_start = np.repeat(start, np.diff(np.r_[start, len(b)]))
    chunk = b.astype(np.int64) * 4096 + (np.arange(len(b)) - row_start) // 32  # rows < 131,072 entries
    pairs = np.unique(chunk * (1 << 26) + c // 32)                                 # lines < 2^26
    return len(pairs) / len(np.unique(chunk))


def test_brick_order_halves_the_lines_a_warp_gathers():
    geom = synth.GEOMETRIES["cfg2"]
    vox, blt, _ = synth.generate_coo_cps(geom, [0, 23, 45])  # beams along x, obliquely, along y
    assert len(blt) < 1 << 26 and np.bincount(blt).max() < 1 << 17
    voxel_order = _lines_per_chunk(vox.astype(np.int64), blt)
    brick_order = _lines_per_chunk(brick_pos(vox.astype(np.int64), geom.nx, geom.ny, geom.nz), blt)
    assert voxel_order > 5.0
    assert brick_order < 0.6 * voxel_order
