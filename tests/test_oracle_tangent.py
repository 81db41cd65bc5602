"""Pin for the oracle's tangent-linear model: the dual-number derivative of the
probe-misfit loss with respect to (u_ref, alpha) must match FP64 central
finite differences (h = 1e-6) of the plain solver."""
import math

import numpy as np

VEL, OUT, BB, FS = 0, 1, 2, 3


def _setup(O):
    nx, ny, nz = 18, 10, 8
    flags = O.geometry(nx, ny, nz, boxes=[[5, 3, 0, 8, 7, 4]])
    p = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 0.6, 0.0)
    probes = O.probe_points(nx, ny, nz, 7, flags, 6)
    return p, flags, probes


def _loss(O, p, flags, probes, u_ref, alpha, target, steps):
    uin = O.inflow(p.nz, u_ref, 0.0, alpha, p.nz, 0.0)
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin, f, 0, steps)
    _, u = O.macros(p, flags, f)
    J = 0.0
    for q, (x, y, z) in enumerate(probes):
        c = x + p.nx * (y + p.ny * z)
        J += float(np.sum((u[:, c] - target[q]) ** 2))
    return J


def test_tangent_matches_central_differences(O):
    p, flags, probes = _setup(O)
    steps = 80
    target = np.zeros((len(probes), 3))
    # synthetic truth at (0.055, 0.28)
    uin_t = O.inflow(p.nz, 0.055, 0.0, 0.28, p.nz, 0.0)
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin_t, f, 0, steps)
    _, u = O.macros(p, flags, f)
    for q, (x, y, z) in enumerate(probes):
        target[q] = u[:, x + p.nx * (y + p.ny * z)]
    u_ref, alpha = 0.05, 0.25
    uin = O.inflow(p.nz, u_ref, 0.0, alpha, p.nz, 0.0)
    h = (np.arange(p.nz) + 0.5) / p.nz
    duin = np.stack([uin / u_ref, uin * np.log(h)[:, None]])
    f = O.init_equilibrium(p, flags)
    J, dJ, up = O.tangent_run(p, flags, uin, duin, f, steps, probes, target)
    assert abs(J - _loss(O, p, flags, probes, u_ref, alpha, target, steps)) < 1e-18
    hh = 1e-6
    fd = [(_loss(O, p, flags, probes, u_ref + hh, alpha, target, steps)
           - _loss(O, p, flags, probes, u_ref - hh, alpha, target, steps)) / (2 * hh),
          (_loss(O, p, flags, probes, u_ref, alpha + hh, target, steps)
           - _loss(O, p, flags, probes, u_ref, alpha - hh, target, steps)) / (2 * hh)]
    assert J > 0 and abs(dJ[0]) > 0 and abs(dJ[1]) > 0
    for k in range(2):
        assert abs(dJ[k] - fd[k]) <= 1e-6 * abs(fd[k]), (dJ, fd)
