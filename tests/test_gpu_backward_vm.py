"""Differentiation of the loss of the differentiation workload (a 3D random-sphere cell, 2-layer
filter, contrast 20): L = sum_ij (C_ij - T_ij)^2 / |T|^2 + w <sigma_vm^2> / <sigma_vm^2>_0, the von
Mises term taken on the first load case (xx), sigma_vm^2 = (3/2) s : s with s the deviatoric stress.
Its stress sensitivity dL/dsigma(x) = 3 w s(x) / (N_v <sigma_vm^2>_0) drives the adjoint solve.

* At 9^3 (generic FP64 passes): hom_solve_backward's phase-Lame gradient against central finite
  differences (relative step 1e-4) of the FP64 oracle's loss.
* The specialised FP32 passes run the adjoint solve too: against the generic passes at 45^2 and 27^3.
* At 135^3 (the workload's size, FP32 forward and adjoint on the specialised passes): the gradient
  against central finite differences of the loss computed by the FP64 GPU path (which matches the
  oracle to 1e-10 on fields), to 1e-4 of the gradient's largest component."""
import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


W_VM = 1.0


def _deviatoric(sig):
    """[6, ...] Mandel stress -> deviatoric part (the Mandel inner product is the tensor one)."""
    s = np.array(sig, dtype=np.float64, copy=True)
    tr = (s[0] + s[1] + s[2]) / 3.0
    for k in range(3):
        s[k] -= tr
    return s


def _vm2_mean(sig0):
    s = _deviatoric(sig0)
    return float(1.5 * np.mean(np.sum(s * s, axis=0)))


def _target(C0, seed):
    rng = np.random.default_rng(seed)
    T = C0 * (1.0 + 0.1 * rng.standard_normal(C0.shape))
    return 0.5 * (T + T.T)


def _loss(C, sig0, T, vm0):
    return float(np.sum((C - T) ** 2) / np.sum(T ** 2) + W_VM * _vm2_mean(sig0) / vm0)


def _loss_grads(C, sig, T, vm0, nv, dtype):
    """dL/dC [1, 6, 6] and dL/dsigma (device, the solver's field layout [load][comp][voxels])."""
    G = 2.0 * (C - T) / np.sum(T ** 2)
    S = np.zeros((6, 6, nv))
    S[0] = W_VM * 3.0 * _deviatoric(sig[0]) / (nv * vm0)
    return G[None], torch.tensor(S.ravel(), dtype=dtype, device="cuda")


def _sphere_cell(n, seed, gap):
    return H.rsa_spheres_cell(n, seed=seed, vf=0.25, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER, radius_px=1.0,
                              subgrid=8, gap_voxels=gap)


def test_von_mises_loss_gradient_matches_oracle_fd_9():
    cell = H.rsa_spheres_cell(9, seed=9, vf=0.12, rmin=0.12, rmax=0.16, subgrid=4, gap_voxels=0.5)
    phases = H.two_phases(20.0)
    c0 = H.mean_lame(phases)
    tol = 1e-12

    def oracle_eval(ph):
        fb = O.filter_build(cell, ph)
        r = O.solve(fb["ctilde"], 3, 9, c0[0], c0[1], np.eye(6), tol=tol, max_iter=5000)
        return O.effective_stiffness(r["mean_sigma"], np.eye(6)), r["sigma"][0].reshape(6, -1)

    C0, s0 = oracle_eval(phases)
    T = _target(C0, 3016)
    vm0 = _vm2_mean(s0)
    mat = hom.hom_filter_build([cell], phases)
    fwd = hom.hom_solve(mat, np.eye(6), c0, precision=hom.HOM_FP64, tol=tol, max_iter=5000)
    C = hom.hom_effective_stiffness(np.eye(6), fwd["mean_sigma"], 3)[0]
    sig = fwd["sigma"].cpu().numpy().reshape(6, 6, -1)
    G, S = _loss_grads(C, sig, T, vm0, 9 ** 3, torch.float64)
    b = hom.hom_solve_backward(mat, fwd, c0, dL_dC=G, dL_dsigma=S, precision=hom.HOM_FP64, tol=tol, max_iter=5000)
    assert (b["adjoint_status"] == 0).all()
    for p in range(2):
        for k in range(2):
            h = 1e-4 * phases[p][k]
            vals = []
            for sgn in (+1, -1):
                ph = [list(q) for q in phases]
                ph[p][k] += sgn * h
                Cp, sp = oracle_eval([tuple(q) for q in ph])
                vals.append(_loss(Cp, sp, T, vm0))
            fd = (vals[0] - vals[1]) / (2 * h)
            got = b["dphase"][p, k]
            assert abs(got - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(b["dphase"]).max()), (p, k, got, fd)


@pytest.mark.parametrize("case", ["disk45", "sph27"])
def test_fast_adjoint_matches_generic(case):
    """FP32 adjoint solve on the specialised passes (source term in their row pass) against the generic
    passes: the phase gradients and the c~ gradient field agree to FP32 accuracy."""
    if case == "disk45":
        cell, nc = H.centred_disk_cell(45, rule=H.RULE_TWO_LAYER), 3
    else:
        cell, nc = H.rsa_spheres_cell(27, seed=27, vf=0.2, rmin=0.1, rmax=0.15, subgrid=4, gap_voxels=1.0), 6
    phases = H.two_phases(10.0)
    c0 = H.mean_lame(phases)
    mat = hom.hom_filter_build([cell], phases)
    fwd = hom.hom_solve(mat, np.eye(nc), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6,
                        max_iter=3000)
    assert (fwd["status"] == 0).all()
    rng = np.random.default_rng(17)
    G = rng.standard_normal((1, nc, nc))
    S = torch.tensor(rng.standard_normal(fwd["sigma"].numel()) / cell.n ** cell.dim, dtype=torch.float32, device="cuda")
    out = {}
    for passes in (hom.HOM_PASSES_AUTO, hom.HOM_PASSES_GENERIC):
        out[passes] = hom.hom_solve_backward(mat, fwd, c0, dL_dC=G, dL_dsigma=S, precision=hom.HOM_FP32,
                                             criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=3000, passes=passes)
        assert (out[passes]["adjoint_status"] == 0).all()
    a, g = out[hom.HOM_PASSES_AUTO], out[hom.HOM_PASSES_GENERIC]
    np.testing.assert_allclose(a["dphase"], g["dphase"], rtol=0, atol=2e-5 * np.abs(g["dphase"]).max())
    da, dg = a["dctilde"].double(), g["dctilde"].double()
    assert float((da - dg).pow(2).mean().sqrt() / dg.pow(2).mean().sqrt()) < 2e-5


def test_backward_135_fp32_matches_fp64_fd():
    """The differentiation workload at 135^3: FP32 forward (6 loads) and FP32 adjoint on the
    specialised 3D passes; the phase-Lame gradient against central finite differences of the loss
    evaluated with FP64 forward solves (generic passes, e < 1e-11)."""
    n = 135
    cell = _sphere_cell(n, 3000, n / 243.0)
    phases = H.two_phases(20.0)
    c0 = H.mean_lame(phases)

    def fp64_eval(ph):
        m = hom.hom_filter_build([cell], ph)
        r = hom.hom_solve(m, np.eye(6), c0, precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-11, max_iter=5000)
        assert (r["status"] == 0).all()
        C = hom.hom_effective_stiffness(np.eye(6), r["mean_sigma"], 3)[0]
        return C, r["sigma"].view(6, 6, -1)[0].cpu().numpy()

    C0, s0 = fp64_eval(phases)
    T = _target(C0, 3001)
    vm0 = _vm2_mean(s0)
    mat = hom.hom_filter_build([cell], phases)
    # FP32 at contrast 20: e_n bottoms out near contrast x 6e-8 (about 1.2e-6), so stop at 4e-6
    fwd = hom.hom_solve(mat, np.eye(6), c0, precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=4e-6, max_iter=5000)
    assert (fwd["status"] == 0).all()
    C = hom.hom_effective_stiffness(np.eye(6), fwd["mean_sigma"], 3)[0]
    G, S = _loss_grads(C, fwd["sigma"].view(6, 6, -1).cpu().numpy().astype(np.float64), T, vm0, n ** 3, torch.float32)
    b = hom.hom_solve_backward(mat, fwd, c0, dL_dC=G, dL_dsigma=S, precision=hom.HOM_FP32,
                               criterion=hom.HOM_CRIT_EN, tol=4e-6, max_iter=5000)
    assert (b["adjoint_status"] == 0).all()
    big = np.abs(b["dphase"]).max()
    for p in range(2):
        for k in range(2):
            h = 1e-4 * phases[p][k]
            vals = []
            for sgn in (+1, -1):
                ph = [list(q) for q in phases]
                ph[p][k] += sgn * h
                Cp, sp = fp64_eval([tuple(q) for q in ph])
                vals.append(_loss(Cp, sp, T, vm0))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(b["dphase"][p, k] - fd) <= 1e-4 * big, (p, k, b["dphase"][p, k], fd)
