"""Differentiation form: dose(y) = D (A y) as a torch.autograd.Function whose
backward is A^T D^T g (libvmat kernels), on the 40^3 / 36-CP / 20x20 DDC with
60 seeded random apertures (rows open over 4-40 columns) and y ~ U(0, 1).

Checked against central finite differences (h = 1e-3, float64, through the
oracle) and the oracle's gradient -A^T D^T g; then the gradient drives a
projected BB solve of the master problem whose objective must reach the
oracle's optimum.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, host, make_ddc, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    require_cuda()
    import __graft_entry__
    __graft_entry__.build()
    from paper_1503_01721_gb300 import api
    c = synth.make_case("cfg1", seed=0)
    ddc = make_ddc(c)
    D = oracle.ddc_matrix(c.V, c.J, c.vox, c.blt, c.val)
    cps, leaves, y = synth.random_apertures(c.mlc, 60, 0)
    vox = api.VoxelParams.from_numpy(c.structs)
    return c, ddc, D, cps, leaves, y, vox


def oracle_F_and_grad(c, D, cps, leaves, y):
    s = c.structs
    z = D @ oracle.aperture_fluence(c.mlc, cps, leaves, y)
    F, g = oracle.objective_grad(z, s.struct_id, s.T, s.w_over, s.w_under)
    grad = -oracle.aperture_grad(c.mlc, cps, leaves, oracle.beamlet_price(D, g))
    return z, F, grad


def test_forward_and_backward(setup):
    from paper_1503_01721_gb300.autograd import ApertureDose, objective
    c, ddc, D, cps, leaves, y, vox = setup
    dose = ApertureDose(ddc, c.mlc, dev(cps, torch.int32), dev(leaves, torch.int16))
    yt = dev(y, torch.float32).requires_grad_(True)
    z = dose(yt)
    F = objective(z, vox)
    F.backward()
    z_ref, F_ref, grad_ref = oracle_F_and_grad(c, D, cps, leaves, y.astype(np.float64))
    assert np.max(np.abs(host(z) - z_ref)) <= 1e-5 * np.max(np.abs(z_ref))
    assert abs(F.item() - F_ref) <= 1e-5 * F_ref
    gy = host(yt.grad).astype(np.float64)
    scale = np.max(np.abs(grad_ref))
    assert np.max(np.abs(gy - grad_ref)) <= 1e-4 * scale
    # central finite differences in float64 (exact for the quadratic pieces)
    h = 1e-3
    y64 = y.astype(np.float64)
    for k in range(0, 60, 5):
        e = np.zeros(60)
        e[k] = h
        Fp = oracle_F_and_grad(c, D, cps, leaves, y64 + e)[1]
        Fm = oracle_F_and_grad(c, D, cps, leaves, y64 - e)[1]
        assert abs((Fp - Fm) / (2 * h) - gy[k]) <= 1e-4 * scale


def test_gradient_drives_master_problem(setup):
    """Projected BB steps (Eq. 7-10) on the autograd gradient reach the MP optimum."""
    from paper_1503_01721_gb300.autograd import ApertureDose, objective
    c, ddc, D, cps, leaves, y0, vox = setup
    n = 20
    cps, leaves = cps[:n], leaves[:n]
    dose = ApertureDose(ddc, c.mlc, dev(cps, torch.int32), dev(leaves, torch.int16))

    def F_and_grad(y):
        yt = y.clone().requires_grad_(True)
        F = objective(dose(yt), vox)
        F.backward()
        return F.item(), yt.grad.double()

    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    F, G = F_and_grad(y.float())
    # first step: exact minimiser along -G of the local quadratic (one extra evaluation)
    t = 1e-3
    F2, _ = F_and_grad((y - t * G).clamp_min(0).float())
    lin = float(G @ G)
    curv = 2 * (F2 - F + t * lin) / t ** 2
    delta = lin / curv if curv > 0 else t
    y_prev, G_prev = y.clone(), G.clone()
    y = (y - delta * G).clamp_min(0)
    for it in range(1, 400):
        F, G = F_and_grad(y.float())
        G = torch.where((y <= 0) & (G > 0), torch.zeros_like(G), G)
        s, r = y - y_prev, G - G_prev
        sr = float(s @ r)
        delta = (float(s @ s) / sr if it % 2 == 0 else sr / float(r @ r)) if sr > 0 else delta
        y_prev, G_prev = y.clone(), G.clone()
        y = (y - delta * G).clamp_min(0)
    DA = np.stack([oracle.aperture_dose(D, c.mlc, int(k), lv) for k, lv in zip(cps, leaves)], 1)
    tight = oracle.BBOptions(max_iter=20000, rel_tol5=1e-15, step_tol=1e-16)
    s = c.structs
    F_opt = oracle.mp_bb_solve(DA, s.struct_id, s.T, s.w_over, s.w_under, np.zeros(n), opts=tight)[2]
    assert F <= F_opt * (1 + 1e-3)
