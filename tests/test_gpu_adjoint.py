"""GPU adjoint (inflow-parameter assimilation) against the oracle's
tangent-linear model and against FP64 central finite differences.

Tolerances: gradient relative error <= 1e-3 per component (the accuracy
target for the adjoint); the FP32 loss within 1e-4 relative of FP64; the
gradient independent of the checkpoint count (recomputation is exact; the
FP64 atomic accumulation order is not, hence 1e-12 relative).
"""
import math

import numpy as np
import pytest

from helpers import oracle_domain
from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()
    return torch.device("cuda")


def small_case():
    return dict(
        name="adjoint_small",
        domains=[dict(nx=18, ny=10, nz=8, boxes=[[5, 3, 0, 8, 7, 4]], bc=W.URBAN_BC, quad_level=1)],
        tau0=0.6, c_smag=0.0, u_ref=0.05, alpha=0.25, angle_deg=0.0, H_ref=0.0,
        inputs=[W.SPEED], lo=[-0.1], hi=[0.1], quad_rule=W.GL, ramp_steps=0,
        precision=W.FP32_SHIFT, gpc_degree=-1)


def test_adjoint_matches_oracle_tangent(O, cuda):
    wl = small_case()
    steps = 80
    p, flags = oracle_domain(O, wl)
    probes = O.probe_points(18, 10, 8, 7, flags, 6)
    # target: the oracle forward at (0.055, 0.28)
    uin_t = O.inflow(8, 0.055, 0.0, 0.28, 8, 0.0)
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin_t, f, 0, steps)
    _, u = O.macros(p, flags, f)
    target = np.array([u[:, x + 18 * (y + 10 * z)] for x, y, z in probes])
    # oracle tangent at (0.05, 0.25)
    uin = O.inflow(8, 0.05, 0.0, 0.25, 8, 0.0)
    hh = (np.arange(8) + 0.5) / 8
    duin = np.stack([uin / 0.05, uin * np.log(hh)[:, None]])
    f = O.init_equilibrium(p, flags)
    J, dJ, _ = O.tangent_run(p, flags, uin, duin, f, steps, probes, target)
    ens = S.Ensemble(S.make_config(wl))
    assim = S.Assimilation(ens, probes, target, steps, n_snapshots=0)
    Jg, gg, up = assim.loss_and_grad(0.05, 0.25)
    assert abs(Jg - J) <= 1e-4 * J
    for k in range(2):
        assert abs(gg[k] - dJ[k]) <= 1e-3 * abs(dJ[k]), (gg, dJ)
    # every checkpoint count gives the same gradient (exact recomputation)
    for K in (1, 5, 9, 80):
        a2 = S.Assimilation(ens, probes, target, steps, n_snapshots=K)
        J2, g2, _ = a2.loss_and_grad(0.05, 0.25)
        assert J2 == Jg and np.allclose(g2, gg, rtol=1e-12, atol=0)
    ens.close()


def test_adjoint_unsupported_with_smagorinsky(cuda):
    wl = dict(small_case(), c_smag=0.14)
    ens = S.Ensemble(S.make_config(wl))
    with pytest.raises(S.ScError) as ei:
        S.Assimilation(ens, [[9, 5, 3]], [[0.0, 0.0, 0.0]], 10).loss_and_grad(0.05, 0.25)
    assert ei.value.code == S.SC_ERR_UNSUPPORTED
    ens.close()


def test_adjoint_unsupported_with_regularized_collision(cuda):
    wl = dict(small_case(), collision=W.RR)
    ens = S.Ensemble(S.make_config(wl))
    with pytest.raises(S.ScError) as ei:
        S.Assimilation(ens, [[9, 5, 3]], [[0.0, 0.0, 0.0]], 10).loss_and_grad(0.05, 0.25)
    assert ei.value.code == S.SC_ERR_UNSUPPORTED
    ens.close()


def _fp64_probe_velocity(wl, u_ref, alpha, steps, probes):
    cfg = S.make_config(dict(wl, precision=W.FP64_PLAIN, u_ref=u_ref, alpha=alpha))
    ens = S.Ensemble(cfg)
    ens.step(steps)
    f = ens.populations(0, 0).cpu().numpy()
    D = wl["domains"][0]
    cx = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0], float)
    cy = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1], float)
    cz = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1], float)
    out = []
    for x, y, z in probes:
        fc = f[:, x + D["nx"] * (y + D["ny"] * z)]
        rho = fc.sum()
        out.append([cx @ fc / rho, cy @ fc / rho, cz @ fc / rho])
    ens.close()
    return np.array(out)


def test_adjoint_full_size_matches_fp64_finite_differences(cuda):
    """128x64x48 urban domain, 2000 steps, 16 probes: FP32 adjoint gradient
    against FP64 central differences (h = 1e-6) of the FP64 GPU path."""
    wl = W.URBAN_ADJOINT
    steps = wl["steps"]
    cfg = S.make_config(wl)
    probes = S.sc_lbm_probe_points(cfg, 0, wl["n_probes"])
    target = _fp64_probe_velocity(wl, *wl["truth"], steps, probes)

    def J64(u_ref, alpha):
        u = _fp64_probe_velocity(wl, u_ref, alpha, steps, probes)
        return float(((u - target) ** 2).sum())

    h = 1e-6
    u0, a0 = wl["guess"]
    fd = [(J64(u0 + h, a0) - J64(u0 - h, a0)) / (2 * h), (J64(u0, a0 + h) - J64(u0, a0 - h)) / (2 * h)]
    ens = S.Ensemble(cfg)
    assim = S.Assimilation(ens, probes, target, steps)
    J, g, _ = assim.loss_and_grad(u0, a0)
    assert abs(J - J64(u0, a0)) <= 1e-4 * J
    for k in range(2):
        assert abs(g[k] - fd[k]) <= 1e-3 * abs(fd[k]), (g, fd)
    ens.close()


def test_gradient_descent_assimilation(cuda):
    """20 gradient-descent iterations (Barzilai-Borwein trial steps under an
    Armijo backtracking condition) move (u_ref, alpha) from (0.05, 0.25)
    toward the truth (0.055, 0.28) with a monotone loss."""
    wl = W.URBAN_ADJOINT
    steps = wl["steps"]
    cfg = S.make_config(wl)
    probes = S.sc_lbm_probe_points(cfg, 0, wl["n_probes"])
    ens = S.Ensemble(cfg)
    S.sc_lbm_set_inflow(ens.h, *wl["truth"], 0.0)
    ens.step(steps)
    u = ens.velocity(0, 0).double().cpu().numpy()
    D = wl["domains"][0]
    target = np.array([u[:, x + D["nx"] * (y + D["ny"] * z)] for x, y, z in probes])
    assim = S.Assimilation(ens, probes, target, steps)
    hist = S.assimilate(assim, wl["guess"], iters=wl["gd_iters"])
    Js = [h[1] for h in hist]
    print("assimilation history:", [(list(h[0]), h[1]) for h in hist])
    assert all(b <= a for a, b in zip(Js, Js[1:]))
    assert Js[-1] < 1e-3 * Js[0]
    err0 = np.abs(np.array(wl["guess"]) - wl["truth"]) / np.array(wl["truth"])
    err1 = np.abs(hist[-1][0] - wl["truth"]) / np.array(wl["truth"])
    assert np.all(err1 < 0.1 * err0), (hist[-1], err0, err1)
    # the autograd wrapper returns the same gradient
    F = S.InflowLoss()
    theta = torch.tensor(wl["guess"], dtype=torch.float64, requires_grad=True)
    loss = F.apply(theta, assim)
    loss.backward()
    _, g, _ = assim.loss_and_grad(*wl["guess"])
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)
    ens.close()
