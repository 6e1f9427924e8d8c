"""Pins of the seeded input generator: entries recomputed from the pencil-beam
formula with an independent enumeration over every voxel."""
import math

import numpy as np

import synth


def formula_entries(geom, j):
    """Voxels and values of beamlet j by scanning the whole grid."""
    per_cp = geom.n_rows * geom.n_cols
    k, rem = divmod(j, per_cp)
    r, c = divmod(rem, geom.n_cols)
    arc, kk = divmod(k, geom.n_cp)
    th = math.radians(kk * 360.0 / geom.n_cp + arc * geom.arc_offset_deg)
    b = np.array([math.cos(th), math.sin(th), 0.0])
    u = np.array([-math.sin(th), math.cos(th), 0.0])
    iso = np.array([(geom.nx - 1) / 2, (geom.ny - 1) / 2, (geom.nz - 1) / 2])
    p0 = iso + (c - (geom.n_cols - 1) / 2) * geom.pitch_vox * u + np.array([0, 0, (r - (geom.n_rows - 1) / 2) * geom.pitch_vox])
    # entry parameter of the axis into the box [-0.5, n - 0.5]^3
    lo = np.array([-0.5] * 3)
    hi = np.array([geom.nx, geom.ny, geom.nz]) - 0.5
    ts = []
    for a in range(2):
        if abs(b[a]) > 1e-12:
            ts.append(min((lo[a] - p0[a]) / b[a], (hi[a] - p0[a]) / b[a]))
    t_entry = max(ts)
    qmax = math.log(1 / geom.cutoff)
    out = {}
    for z in range(geom.nz):
        for y in range(geom.ny):
            for x in range(geom.nx):
                w = np.array([x, y, z]) - p0
                t = float(w @ b)
                rho2 = float(np.sum((w - t * b) ** 2))
                q = geom.mu_per_vox * (t - t_entry) + rho2 / (2 * geom.sigma_vox ** 2)
                if t >= t_entry and q <= qmax:
                    out[(z * geom.ny + y) * geom.nx + x] = math.exp(-q)
    return out


def test_entries_match_formula():
    geom = synth.GEOMETRIES["ragged"]
    vox, blt, val = synth.generate_coo(geom)
    for j in (0, 11, 52, geom.J - 1):
        m = blt == j
        got = dict(zip(vox[m].tolist(), val[m].tolist()))
        want = formula_entries(geom, j)
        assert set(got) == set(want)
        for i, v in want.items():
            assert abs(got[i] - v) <= 1e-6 * v


def test_layout_sorted_and_deterministic():
    geom = synth.GEOMETRIES["tiny"]
    v1, b1, a1 = synth.generate_coo(geom)
    v2, b2, a2 = synth.generate_coo(geom)
    assert np.array_equal(v1, v2) and np.array_equal(b1, b2) and np.array_equal(a1, a2)
    key = b1.astype(np.int64) * geom.V + v1
    assert np.all(np.diff(key) > 0)
    assert np.all((a1 > 0.0099) & (a1 <= 1.0))


def test_structures_seeded():
    geom = synth.GEOMETRIES["cfg1"]
    s1 = synth.make_structures("cfg1", geom, 3)
    s2 = synth.make_structures("cfg1", geom, 3)
    assert np.array_equal(s1.struct_id, s2.struct_id)
    assert s1.names == ["tissue", "oar0", "oar1", "ptv0"]
    assert (s1.struct_id == 3).sum() > 1500      # sphere r=8: ~2145 voxels


def test_truncated_ddc_is_a_subset_of_the_full_one():
    """The truncated matrix (the paper's S1: entries outside a radius about each
    beamlet axis dropped) keeps exactly the full matrix's entries near the axis."""
    g = synth.GEOMETRIES["ragged"]
    full = synth.generate_coo(g)
    import dataclasses
    for radius, expect_all in ((1.25, False), (2.0, False), (3.1, True)):
        tr = synth.generate_coo(dataclasses.replace(g, trunc_vox=radius))
        key_full = {(int(v), int(b)): float(x) for v, b, x in zip(*full)}
        assert all(key_full[(int(v), int(b))] == float(x) for v, b, x in zip(*tr))
        assert (len(tr[2]) == len(full[2])) == expect_all
        # dropped entries are off-axis: their values are at most exp(-radius^2 / 2) of the peak
        kept = {(int(v), int(b)) for v, b in zip(tr[0], tr[1])}
        dropped = [x for (v, b), x in key_full.items() if (v, b) not in kept]
        if dropped:
            assert max(dropped) <= np.exp(-radius ** 2 / 2) * (1 + 1e-6)
