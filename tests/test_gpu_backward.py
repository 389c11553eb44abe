"""GPU tests of hom_solve_backward (adjoint derivative of the fixed point and of the filter rules)
against the FP64 oracle: central finite differences (relative step 1e-4) of the oracle's filter
build + solve, the energy identity dC_ij/dc(x) = eps^(i)(x) eps^(j)(x) / N_v, and finite
differences of the oracle's homogenisation rules for the volume-fraction derivative."""
import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")
from gpu_helpers import dense_ctilde, unpack  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


TOL = 1e-12


def _packed(M, nc):
    """[..., nc, nc] symmetric -> [..., ns] upper triangle row by row."""
    idx = [(i, j) for i in range(nc) for j in range(i, nc)]
    return np.stack([M[..., i, j] for (i, j) in idx], axis=-1)


def _loss_oracle(cell, phases, c0, G, S):
    fb = O.filter_build(cell, phases)
    nc = O.nc_of(cell.dim)
    r = O.solve(fb["ctilde"], cell.dim, cell.n, c0[0], c0[1], np.eye(nc), tol=TOL, max_iter=5000)
    C = O.effective_stiffness(r["mean_sigma"], np.eye(nc))
    return float(np.sum(G * C) + np.sum(S * r["sigma"])), fb, r


def _gpu_forward_backward(cell, phases, c0, G, S, precision=hom.HOM_FP64):
    nc = O.nc_of(cell.dim)
    mat = hom.hom_filter_build([cell], phases)
    crit = hom.HOM_CRIT_E if precision == hom.HOM_FP64 else hom.HOM_CRIT_EN
    tol = TOL if precision == hom.HOM_FP64 else 1e-6
    fwd = hom.hom_solve(mat, np.eye(nc), c0, precision=precision, criterion=crit, tol=tol, max_iter=5000)
    dt = torch.float64 if precision == hom.HOM_FP64 else torch.float32
    Sd = None if S is None else torch.tensor(S.ravel(), dtype=dt, device="cuda")
    b = hom.hom_solve_backward(mat, fwd, c0, dL_dC=None if G is None else G[None], dL_dsigma=Sd,
                               precision=precision, criterion=crit, tol=tol, max_iter=5000)
    return mat, fwd, b


CASES = [
    ("disk27-2layer", lambda: H.centred_disk_cell(27, rule=H.RULE_TWO_LAYER), 10.0),
    ("disk21-reuss", lambda: H.centred_disk_cell(21, rule=H.RULE_REUSS), 0.1),
    ("disk15-voigt", lambda: H.centred_disk_cell(15, rule=H.RULE_VOIGT, radius_px=0.55), 5.0),
    ("sph9-2layer", lambda: H.rsa_spheres_cell(9, seed=9, vf=0.12, rmin=0.12, rmax=0.16, subgrid=4,
                                               gap_voxels=0.5), 10.0),
]


@pytest.mark.parametrize("name,make,contrast", CASES, ids=[c[0] for c in CASES])
def test_phase_gradient_matches_oracle_finite_differences(name, make, contrast):
    cell = make()
    phases = H.two_phases(contrast)
    c0 = H.mean_lame(phases)
    nc = O.nc_of(cell.dim)
    rng = np.random.default_rng(7)
    G = rng.standard_normal((nc, nc))
    S = 0.1 * rng.standard_normal((nc, nc) + (cell.n,) * cell.dim) / cell.n ** cell.dim
    mat, fwd, b = _gpu_forward_backward(cell, phases, c0, G, S)
    assert (b["adjoint_status"] == 0).all()
    for p in range(2):
        for k in range(2):
            h = 1e-4 * phases[p][k]
            vals = []
            for sgn in (+1, -1):
                ph = [list(q) for q in phases]
                ph[p][k] += sgn * h
                vals.append(_loss_oracle(cell, [tuple(q) for q in ph], c0, G, S)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            got = b["dphase"][p, k]
            assert abs(got - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(b["dphase"]).max()), (p, k, got, fd)


def test_ctilde_gradient_directional_and_energy_identity():
    cell = H.centred_disk_cell(27, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    nc = 3
    rng = np.random.default_rng(11)
    G = rng.standard_normal((nc, nc))
    S = 0.1 * rng.standard_normal((nc, nc, cell.n, cell.n)) / cell.n ** 2
    mat, fwd, b = _gpu_forward_backward(cell, phases, c0, G, S)
    g = b["dctilde"].cpu().numpy().reshape(-1, 6)
    L0, fb, r = _loss_oracle(cell, phases, c0, G, S)
    # directional derivative along a random symmetric perturbation field of c~
    D = rng.standard_normal((cell.n, cell.n, nc, nc))
    D = 0.5 * (D + np.swapaxes(D, -1, -2))
    h = 1e-5
    lp = lm = None
    for sgn in (+1, -1):
        ct = fb["ctilde"] + sgn * h * D
        rr = O.solve(ct, 2, cell.n, c0[0], c0[1], np.eye(nc), tol=TOL, max_iter=5000)
        C = O.effective_stiffness(rr["mean_sigma"], np.eye(nc))
        val = float(np.sum(G * C) + np.sum(S * rr["sigma"]))
        if sgn > 0:
            lp = val
        else:
            lm = val
    fd = (lp - lm) / (2 * h)
    got = float(np.sum(g * _packed(D.reshape(-1, nc, nc), nc)))
    assert abs(got - fd) <= 1e-4 * abs(fd), (got, fd)
    # energy identity: with only dL/dC = e_i e_j^T the gradient is eps^(i) (x) eps^(j) / N_v
    for (i, j) in [(0, 0), (0, 1), (2, 2), (1, 2)]:
        Gij = np.zeros((nc, nc))
        Gij[i, j] = 1.0
        b2 = hom.hom_solve_backward(mat, fwd, c0, dL_dC=Gij[None], precision=hom.HOM_FP64)
        got = b2["dctilde"].cpu().numpy().reshape(-1, 6)
        ei = r["eps"][i].reshape(nc, -1).T
        ej = r["eps"][j].reshape(nc, -1).T
        A = ei[:, :, None] * ej[:, None, :] / cell.n ** 2
        expect = _packed(A + np.swapaxes(A, -1, -2), nc)
        expect[:, [0, 3, 5]] *= 0.5  # diagonal entries count once
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-9 * np.abs(expect).max())


def test_fraction_gradient_matches_rule_finite_differences():
    cell = H.centred_disk_cell(27, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    rng = np.random.default_rng(5)
    G = rng.standard_normal((3, 3))
    mat, fwd, b = _gpu_forward_backward(cell, phases, c0, G, None)
    g = b["dctilde"].cpu().numpy().reshape(-1, 6)
    vox = mat.mixed_voxel[:mat.mixed_count].cpu().numpy()
    frac = mat.mixed_frac[:mat.mixed_count].cpu().numpy()
    nrm = mat.mixed_normal[:3 * mat.mixed_count].cpu().numpy().reshape(-1, 3)
    dfrac = b["dfrac"].cpu().numpy()
    Cs = [O.isotropic_mandel(*p, 2) for p in phases]
    for m in range(0, mat.mixed_count, max(1, mat.mixed_count // 12)):
        f, h = frac[m], 1e-6
        dC = (O.hr_two_layer(Cs[0], Cs[1], 1 - f - h, f + h, nrm[m, :2], 2)
              - O.hr_two_layer(Cs[0], Cs[1], 1 - f + h, f - h, nrm[m, :2], 2)) / (2 * h)
        expect = float(np.sum(g[vox[m]] * _packed(dC, 3)))
        assert abs(dfrac[m] - expect) <= 1e-6 * max(abs(expect), 1e-8), (m, dfrac[m], expect)


def test_fp32_backward_matches_fp64():
    cell = H.centred_disk_cell(45, rule=H.RULE_VOIGT)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, 3))
    S = 0.1 * rng.standard_normal((3, 3, cell.n, cell.n)) / cell.n ** 2
    _, _, b64 = _gpu_forward_backward(cell, phases, c0, G, S, hom.HOM_FP64)
    _, _, b32 = _gpu_forward_backward(cell, phases, c0, G, S, hom.HOM_FP32)
    np.testing.assert_allclose(b32["dphase"], b64["dphase"], rtol=1e-4, atol=1e-4 * np.abs(b64["dphase"]).max())


def test_autograd_function_matches_direct_call():
    cell = H.centred_disk_cell(21, rule=H.RULE_TWO_LAYER)
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    lame = torch.tensor(phases, dtype=torch.float64, requires_grad=True)
    settings = dict(precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=TOL, max_iter=5000)
    C, sigma = hom.HomSolve.apply(lame, [cell], c0, settings)
    target = C.detach() * (1.0 + 0.1 * torch.ones_like(C))
    loss = ((C - target) ** 2).sum() / (target ** 2).sum() + 0.5 * (sigma.double() ** 2).mean().cpu()
    loss.backward()
    Cn = C.detach().numpy()
    G = (2 * (Cn - target.numpy()) / (target.numpy() ** 2).sum())[0]
    mat, fwd, b = _gpu_forward_backward(cell, phases, c0, G, (sigma.detach().cpu().numpy() / sigma.numel()).reshape(
        (3, 3, cell.n, cell.n)))
    np.testing.assert_allclose(lame.grad.numpy(), b["dphase"], rtol=1e-7, atol=1e-12)
