"""Pins of the oracle's sparse products (Section 2.1 z = D x; Eq. 3 pi = D^T g).

The oracle uses scipy's CSR product; these tests check it against a dense
matrix built entry by entry with explicit loops, the adjoint identity, and
single columns read straight from the COO arrays.
"""
import numpy as np

import oracle
import synth
from conftest import dense_from_coo


def test_dense_brute_force_tiny(tiny_case):
    c = tiny_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    Dd = dense_from_coo(c.V, c.J, c.vox, c.blt, c.val)
    x = synth.random_vector(c.J, 1, 0.0, 1.0).astype(np.float64)
    g = synth.random_vector(c.V, 2).astype(np.float64)
    z_loop = np.array([sum(Dd[i, j] * x[j] for j in range(c.J)) for i in range(c.V)])
    p_loop = np.array([sum(Dd[i, j] * g[i] for i in range(c.V)) for j in range(c.J)])
    np.testing.assert_allclose(oracle.dose_forward(D, x), z_loop, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.beamlet_price(D, g), p_loop, rtol=1e-13, atol=1e-13)


def test_adjoint_identity_cfg1(cfg1_case):
    c = cfg1_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    x = synth.random_vector(c.J, 3).astype(np.float64)
    g = synth.random_vector(c.V, 4).astype(np.float64)
    lhs = float(oracle.dose_forward(D, x) @ g)
    rhs = float(x @ oracle.beamlet_price(D, g))
    scale = float(np.abs(oracle.dose_forward(D, np.abs(x))) @ np.abs(g))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_unit_column_is_coo_column(ragged_case):
    c = ragged_case
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    for j in (0, 7, c.J // 2, c.J - 1):
        e = np.zeros(c.J)
        e[j] = 1.0
        col = np.zeros(c.V)
        m = c.blt == j
        col[c.vox[m]] = c.val[m]
        np.testing.assert_array_equal(oracle.dose_forward(D, e), col)


def test_duplicates_are_summed():
    vox = np.array([0, 1, 1, 2], np.int32)
    blt = np.array([0, 1, 1, 0], np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0], np.float32)
    D = oracle.ddc_matrix(3, 2, vox, blt, val)
    np.testing.assert_array_equal(D.toarray(), [[1, 0], [0, 5], [4, 0]])


def test_shuffled_coo_same_matrix(ragged_case):
    c = ragged_case
    v2, b2, a2 = synth.shuffled_coo(c.vox, c.blt, c.val, 5)
    D1 = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    D2 = oracle.ddc_matrix(c.V, c.J, v2, b2, a2)
    assert (D1 != D2).nnz == 0
