"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Small ragged domains (several tiles plus a ragged tail in x, y and z) cover
every boundary kind on both parities of the AA pattern, FP64 plain and FP32
shifted storage; full-size checks run in the launch shape the benchmark
times.  Tolerances (relative L2 over fluid cells and all components, per the
accuracy targets of the method): FP32 laminar velocity <= 1e-5 after 1000
steps, LES <= 1e-3 after 100 steps, ensemble mean / std <= 1e-3; FP64 plain
<= 1e-12; one FP32 step from an exported state <= 2e-6 max abs.
"""
import math

import numpy as np
import pytest

from helpers import oracle_domain, oracle_nodes, oracle_run_node, oracle_uin, rel_l2
from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VEL, OUT, BB, FS, PER = W.VEL, W.OUT, W.BB, W.FS, W.PER

# A ragged domain (37 x 19 x 13) with blocks touching the outlet, the lid and a
# side face, so that every link rule (including two-face edges) is exercised.
RAGGED_BOXES = [[6, 3, 0, 10, 8, 5], [14, 0, 0, 17, 4, 13], [33, 9, 0, 37, 13, 6],
                [24, 14, 0, 28, 19, 9], [20, 7, 3, 23, 11, 7]]

BC_SETS = {
    "urban": [VEL, OUT, VEL, VEL, BB, FS],
    "channel": [VEL, OUT, BB, BB, BB, BB],
    "periodic_y_freeslip": [VEL, OUT, PER, PER, FS, FS],
    "closed_box": [BB, BB, BB, BB, BB, FS],
    "velocity_both_x": [VEL, VEL, FS, FS, BB, FS],
    "periodic_all": [PER, PER, PER, PER, PER, PER],
}


def ragged(bc, precision=W.FP32_SHIFT, c_smag=0.14, tau0=0.56, ramp=8, nx=37, ny=19, nz=13,
           angle=12.0, quad_level=3, boxes=RAGGED_BOXES, collision=W.BGK):
    return dict(
        name="ragged", domains=[dict(nx=nx, ny=ny, nz=nz, boxes=boxes, bc=bc, quad_level=quad_level)],
        tau0=tau0, c_smag=c_smag, u_ref=0.05, alpha=0.25, angle_deg=angle, H_ref=0.0,
        inputs=[W.SPEED], lo=[-0.1], hi=[0.1], quad_rule=W.GL, ramp_steps=ramp,
        precision=precision, gpc_degree=2, collision=collision)


def fluid_mask(flags):
    return np.asarray(flags) == 0


def gpu_state(ens, d, j):
    return ens.populations(d, j).cpu().numpy()


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()
    return torch.device("cuda")


@pytest.mark.parametrize("collision", [W.BGK, W.RR], ids=["bgk", "rr"])
@pytest.mark.parametrize("bcname", list(BC_SETS))
@pytest.mark.parametrize("precision,tol,nx,variant", [(W.FP32_SHIFT, 2e-6, 37, 0), (W.FP32_SHIFT, 2e-6, 40, 1),
                                                      (W.FP32_SHIFT, 2e-6, 38, 3), (W.FP64_PLAIN, 1e-13, 37, 0)])
def test_ragged_domain_all_boundaries(O, cuda, bcname, precision, tol, nx, variant, collision):
    """Populations after 1..6 and 31 steps (both AA parities) at every fluid
    cell and node, max abs difference, for both collision forms.  Variant 1
    (nx = 40) runs the TMA-staged kernels (partial last run of 256 cells),
    variant 3 (nx = 38) the per-thread odd kernel with the larger register
    budget, variant 0 (nx = 37) the default per-thread ones."""
    wl = ragged(BC_SETS[bcname], precision=precision, nx=nx, collision=collision)
    ens = S.Ensemble(S.make_config(wl))
    if variant == 1:
        S.sc_lbm_set_tuning(ens.h, 128, 2, 1, variant=1)
    elif variant == 3:
        S.sc_lbm_set_tuning(ens.h, 32, 2, 3, variant=3)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    fl = fluid_mask(flags)
    fo = [O.init_equilibrium(p, flags) for _ in range(len(a))]
    done = 0
    for target in (1, 2, 3, 4, 5, 6, 31):
        ens.step(target - done)
        for j in range(len(a)):
            O.run(p, flags, oracle_uin(O, wl, 0, Z[j]), fo[j], done, target - done)
        done = target
        for j in range(len(a)):
            fg = gpu_state(ens, 0, j)
            err = np.max(np.abs(fg[:, fl] - fo[j][:, fl]))
            assert err < tol, (bcname, target, j, err)
    ens.sync()
    ens.close()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("precision", [W.BF16_STORE, W.FP16_STORE])
def test_reduced_storage_tracks_oracle(O, cuda, precision, variant):
    """BF16 / FP16 storage of the shifted populations: error report against
    FP64 after 40 steps (bounded, not bit-level); nx = 40 runs the TMA-staged
    kernels (variant 1) or the per-thread ones (variant 0) with 2-byte
    elements."""
    wl = ragged(BC_SETS["urban"], precision=precision, nx=40)
    ens = S.Ensemble(S.make_config(wl))
    S.sc_lbm_set_tuning(ens.h, 128 if variant == 1 else 32, 2, 1 if variant == 1 else 4, variant=variant)
    ens.step(40)
    p, flags, f = oracle_run_node(O, wl, 0, 1, 40)
    _, uo = O.macros(p, flags, f)
    ug = ens.velocity(0, 1).cpu().numpy()
    fl = fluid_mask(flags)
    err = rel_l2(ug[:, fl], uo[:, fl])
    bound = 5e-2 if precision == W.BF16_STORE else 5e-3
    assert err < bound, err
    ens.close()


@pytest.mark.parametrize("series", [False, True], ids=["steady", "series"])
@pytest.mark.parametrize("precision,unit", [(W.BF16_STORE, 2.0 ** -8), (W.FP16_STORE, 2.0 ** -11)],
                         ids=["bf16", "fp16"])
def test_two_cell_even_level_matches_one_cell_form(cuda, precision, unit, series):
    """16-bit storage, even nx: the even level with two x-adjacent cells per
    thread (variants 0 and 3: 32-bit population words, the collision on
    packed FP32x2 operations, pairs with one bulk cell next to a solid or
    listed cell) against the one-cell form (variant 2) after 9 even and 9 odd
    levels.  The two collisions round differently in FP32, which can move a
    stored value by one unit of the 16-bit format now and then; unit is the
    format's unit roundoff (BF16 8, FP16 11 significant bits) and g = f - w
    the stored deviation.  With an inflow series (a 10-degree offset from
    level 0) the odd levels take the kernels that turn the inflow."""
    wl = ragged(BC_SETS["urban"], precision=precision, nx=40)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]
    states = {}
    for variant in (2, 0, 3):
        ens = S.Ensemble(S.make_config(wl))
        S.sc_lbm_set_tuning(ens.h, 32, 2, 4, variant=variant)
        if series:
            ens.set_inflow_series(*SERIES)
        ens.step(18)
        states[variant] = [gpu_state(ens, 0, j) for j in range(ens.n_nodes[0])]
        ens.sync()
        ens.close()
    flags = S.sc_lbm_geometry(S.make_config(wl), 0).reshape(-1)
    fl = fluid_mask(flags)
    for variant in (0, 3):
        for j, (a, b) in enumerate(zip(states[variant], states[2])):
            ga, gb = a[:, fl] - w, b[:, fl] - w
            scale = np.max(np.abs(gb))
            assert scale > 1e-3, scale
            e_max = float(np.max(np.abs(ga - gb)) / scale)
            e_l2 = rel_l2(ga, gb)
            assert e_max <= 16 * unit, (variant, j, e_max)
            assert e_l2 <= unit, (variant, j, e_l2)


def test_laminar_channel_1000_steps(O, cuda):
    """Cube in a channel, BGK tau = 0.6, FP32 shifted vs FP64: velocity relative
    L2 <= 1e-5 after 1000 steps (first and last collocation nodes)."""
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    ens = S.Ensemble(S.make_config(wl))
    ens.step(1000)
    for j in (0, 4):
        p, flags, f = oracle_run_node(O, wl, 0, j, 1000)
        _, uo = O.macros(p, flags, f)
        ug = ens.velocity(0, j).cpu().numpy()
        fl = fluid_mask(flags)
        assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-5
    ens.close()


@pytest.mark.parametrize("precision,tol", [(W.FP64_PLAIN, 1e-11), (W.FP32_SHIFT, 1e-5)])
def test_channel_ensemble_statistics(O, cuda, precision, tol):
    """Five Gauss-Legendre nodes, 300 steps: mean / std of |u| (Eq.
    quad_moments), the profile band behind the cube and the gPC coefficients
    (Eq. coef_discrete) against the oracle's two-pass reduction."""
    wl = dict(W.CHANNEL_CUBE, precision=precision)
    ens = S.Ensemble(S.make_config(wl))
    ens.step(wl["steps"])
    out = ens.moments(0, probes=wl["columns"], nodes_profiles=True, gpc=True)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    Qv = O.ensemble(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, wl["steps"])
    mean, std, _ = O.moments_two_pass(a, Qv)
    fl = fluid_mask(flags)
    assert rel_l2(out["mean"].cpu().numpy()[fl], mean[fl]) <= tol
    assert rel_l2(out["std"].cpu().numpy()[fl], std[fl]) <= tol * 10
    prof, pn = O.profiles(a, Qv, p.nx, p.ny, p.nz, wl["columns"])
    assert rel_l2(out["prof"].cpu().numpy(), prof) <= tol * 10
    assert rel_l2(out["prof_nodes"].cpu().numpy(), pn) <= 1e-6
    s = O.legendre_s(Z, wl["lo"], wl["hi"])
    coef = O.gpc_project(a, Qv, O.gpc_basis(1, wl["gpc_degree"], s))
    cg = out["coef"].cpu().numpy()
    assert rel_l2(cg[0][fl], coef[0][fl]) <= tol
    assert rel_l2(cg[1][fl], coef[1][fl]) <= tol * 10
    # gPC mean equals the quadrature mean (Eq. gPC with orthonormal basis)
    assert np.max(np.abs(cg[0] - out["mean"].cpu().numpy())) < 1e-12
    ens.close()


@pytest.mark.parametrize("precision,tol", [(W.FP64_PLAIN, 1e-11), (W.FP32_SHIFT, 1e-5)])
def test_gaussian_inputs_ensemble_statistics(O, cuda, precision, tol):
    """The paper's input model on the cube channel: speed factor and wind
    direction normal (std 0.1 and 6 degrees) on a 3 x 3 Gauss-Hermite rule,
    logarithmic profile, recursive regularized collision; mean / std / profile
    band and the Hermite gPC coefficients against the oracle."""
    wl = dict(W.CHANNEL_CUBE, precision=precision, inputs=[W.SPEED, W.ANGLE], lo=[0.0, 0.0],
              hi=[0.1, 6.0], quad_rule=W.GH, profile=W.PROFILE_LOG, z0=0.1, collision=W.RR,
              gpc_degree=2, domains=[dict(W.CHANNEL_CUBE["domains"][0], quad_level=3)])
    ens = S.Ensemble(S.make_config(wl))
    ens.step(wl["steps"])
    out = ens.moments(0, probes=wl["columns"], nodes_profiles=True, gpc=True)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    assert Z.shape == (9, 2)
    Qv = O.ensemble(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, wl["steps"],
                    z0=wl["z0"])
    mean, std, _ = O.moments_two_pass(a, Qv)
    fl = fluid_mask(flags)
    assert rel_l2(out["mean"].cpu().numpy()[fl], mean[fl]) <= tol
    assert rel_l2(out["std"].cpu().numpy()[fl], std[fl]) <= tol * 10
    prof, _ = O.profiles(a, Qv, p.nx, p.ny, p.nz, wl["columns"])
    assert rel_l2(out["prof"].cpu().numpy(), prof) <= tol * 10
    coef = O.gpc_project(a, Qv, O.gpc_basis_family(2, 2, O.HERMITE, O.normal_s(Z, wl["lo"], wl["hi"])))
    cg = out["coef"].cpu().numpy()
    for k in range(coef.shape[0]):
        assert rel_l2(cg[k][fl], coef[k][fl]) <= tol * 10, k
    ens.close()


SERIES = ([1.0, 1.3, 0.8, 1.1], [10.0, -15.0, 30.0, 355.0], 24, 10)


@pytest.mark.parametrize("precision,tol", [(W.FP64_PLAIN, 1e-12), (W.FP32_SHIFT, 1e-5)])
@pytest.mark.parametrize("steps", [79, 120])
def test_inflow_series_parity(O, cuda, precision, tol, steps):
    """Hourly inflow targets (speed and direction, the last across 0 degrees)
    joined by 10-level interpolation intervals, on the cube channel with the
    paper's Gaussian inputs (3 x 3 Gauss-Hermite) and log profile: each node's
    velocity against the oracle, which builds every level's profile from the
    reference speed and direction of that level.  Level 79 lies inside an
    interval (an odd level: the exported velocity uses its factor), level 120
    after the last target.  FP64: populations, max abs error; FP32: velocity,
    relative L2."""
    wl = dict(W.CHANNEL_CUBE, precision=precision, inputs=[W.SPEED, W.ANGLE], lo=[0.0, 0.0],
              hi=[0.1, 6.0], quad_rule=W.GH, profile=W.PROFILE_LOG, z0=0.1, ramp_steps=12,
              domains=[dict(W.CHANNEL_CUBE["domains"][0], quad_level=3)])
    ens = S.Ensemble(S.make_config(wl))
    ens.set_inflow_series(*SERIES)
    ens.step(steps)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    U, F = O.ensemble_series(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, steps, SERIES,
                             z0=wl["z0"], keep_f=True)
    fl = fluid_mask(flags)
    for j in range(len(a)):
        if precision == W.FP64_PLAIN:
            err = np.max(np.abs(gpu_state(ens, 0, j)[:, fl] - F[j][:, fl]))
            assert err <= tol, (j, err)
        else:
            ug = ens.velocity(0, j).cpu().numpy()
            assert rel_l2(ug[:, fl], U[j][:, fl]) <= tol, j
    # the steady inflow gives another flow
    Us = O.ensemble(p, flags, Z[:1], wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, steps, keep_u=True,
                    z0=wl["z0"])[1][0]
    assert rel_l2(Us[:, fl], U[0][:, fl]) > 1e-2
    ens.close()


@pytest.mark.parametrize("precision,tol", [(W.FP64_PLAIN, 1e-12), (W.FP32_SHIFT, 1e-5)])
@pytest.mark.parametrize("collision,c_smag", [(W.BGK, 0.14), (W.RR, 0.25)])
def test_circular_domain_parity(O, cuda, precision, tol, collision, c_smag):
    """The paper's cylinder at small size: velocity mantle (links into the
    columns beyond the radius take the moving-wall rule), two blocks near
    the axis, 3 x 3 Gauss-Hermite nodes on speed and direction, log profile;
    every node against the oracle after 60 steps (FP64: populations, max
    abs error; FP32: velocity, relative L2)."""
    wl = dict(W.DISK_SMALL, precision=precision, collision=collision, c_smag=c_smag)
    steps = 60
    ens = S.Ensemble(S.make_config(wl))
    ens.step(steps)
    p, flags = oracle_domain(O, wl)
    assert (flags == 2).sum() > 0
    Z, a = oracle_nodes(O, wl)
    fl = fluid_mask(flags)
    D = wl["domains"][0]
    for j in range(len(a)):
        xi, al, th = O.node_inflow_params(Z[j], wl["inputs"], wl["u_ref"], wl["alpha"], wl["angle_deg"])
        uin = O.inflow_log(D["nz"], wl["u_ref"], xi, wl["z0"], D["nz"], th)
        f = O.init_equilibrium(p, flags)
        O.run(p, flags, uin, f, 0, steps)
        if precision == W.FP64_PLAIN:
            err = np.max(np.abs(gpu_state(ens, 0, j)[:, fl] - f[:, fl]))
            assert err <= tol, (j, err)
        else:
            ug = ens.velocity(0, j).cpu().numpy()
            assert rel_l2(ug[:, fl], O.macros(p, flags, f)[1][:, fl]) <= tol, j
    ens.close()


def test_circular_domain_with_series(O, cuda):
    """The paper's full input pipeline at small size: cylinder, Gaussian
    speed and direction on 3 x 3 Gauss-Hermite nodes, log profile, the
    recursive regularized collision with C_S = 0.25 and an hourly series
    whose direction swings by 60 degrees; FP32 velocity of every node
    against the oracle, level 71 (inside an interpolation interval)."""
    wl = dict(W.DISK_SMALL, collision=W.RR, c_smag=0.25)
    series = ([1.0, 1.2, 0.9], [0.0, 60.0, 10.0], 25, 12)
    steps = 71
    ens = S.Ensemble(S.make_config(wl))
    ens.set_inflow_series(*series)
    ens.step(steps)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    U = O.ensemble_series(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], wl["angle_deg"], p.nz, steps,
                          series, z0=wl["z0"])
    fl = fluid_mask(flags)
    for j in range(len(a)):
        assert rel_l2(ens.velocity(0, j).cpu().numpy()[:, fl], U[j][:, fl]) <= 1e-5, j
    ens.close()


def test_paper_case_full_size(O, cuda):
    """The paper's configuration at full size on one GPU (disk of radius 270
    and height 40, 121 Gauss-Hermite nodes, regularized collision, C_S =
    0.25, Re = 1.8e6; 107 GB of populations) in the launch configuration
    bench.py times it in: the first, middle and last nodes (the two extremes
    of the rule and its centre) at levels 20 and 100 against the oracle
    (relative L2 of u <= 1e-3, the LES bound), and no non-finite or
    non-positive density.  The velocities are small early in the start-up
    ramp (about 1e-6 at level 20); the observables are summed on the shifted
    populations, so FP32 rounding of the O(1) density does not enter them."""
    wl = W.URBAN_DISK_PAPER
    ens = S.Ensemble(S.make_config(wl))      # the default launch configuration, as bench.py's leg
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    assert len(a) == 121
    D = wl["domains"][0]
    fl = fluid_mask(flags)
    nodes = (0, 60, 120)
    fo = {j: O.init_equilibrium(p, flags) for j in nodes}
    uins = {}
    for j in nodes:
        xi, al, th = O.node_inflow_params(Z[j], wl["inputs"], wl["u_ref"], wl["alpha"], wl["angle_deg"])
        uins[j] = O.inflow_log(D["nz"], wl["u_ref"], xi, wl["z0"], D["nz"], th)
    done = 0
    for level in (20, 100):
        ens.step(level - done)
        assert S.sc_lbm_check(ens.h) == (S.SC_OK, 0)
        for j in nodes:
            O.run(p, flags, uins[j], fo[j], done, level - done)
            uo = O.macros(p, flags, fo[j])[1]
            ug = ens.velocity(0, j).cpu().numpy()
            err = rel_l2(ug[:, fl], uo[:, fl])
            print("paper case level %d node %d: relative L2 of u %.2e" % (level, j, err))
            assert err <= 1e-3, (level, j, err)
        done = level
    ens.close()


def test_les_full_size_ensemble_fields_100_steps(O, cuda):
    """The 13-node urban LES ensemble at full size (256x128x64, BGK +
    Smagorinsky) in the benchmark's launch shape: mean, std and the profile
    bands of |u| after 100 steps against the oracle's own 13 runs and its
    two-pass reduction (relative L2 over fluid cells <= 1e-3, the ensemble
    bound)."""
    wl = W.URBAN_LES
    ens = S.Ensemble(S.make_config(wl))
    S.sc_lbm_autotune(ens.h, None)
    ens.step(100)
    cfg = S.make_config(wl)
    cols = S.sc_lbm_probe_columns(cfg, 0, wl["n_columns"])
    out = ens.moments(0, probes=cols, gpc=True)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    Qv = O.ensemble(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, 100)
    mean, std, _ = O.moments_two_pass(a, Qv)
    prof, _ = O.profiles(a, Qv, p.nx, p.ny, p.nz, cols)
    fl = fluid_mask(flags)
    errs = (rel_l2(out["mean"].cpu().numpy()[fl], mean[fl]), rel_l2(out["std"].cpu().numpy()[fl], std[fl]),
            rel_l2(out["prof"].cpu().numpy(), prof))
    print("LES 13-node fields after 100 steps: mean %.2e std %.2e band %.2e" % errs)
    assert errs[0] <= 1e-3 and errs[1] <= 1e-3 and errs[2] <= 1e-3, errs
    coef = O.gpc_project(a, Qv, O.gpc_basis(2, wl["gpc_degree"], O.legendre_s(Z, wl["lo"], wl["hi"])))
    cg = out["coef"].cpu().numpy()
    assert rel_l2(cg[0][fl], coef[0][fl]) <= 1e-3
    ens.close()


@pytest.mark.parametrize("family", ["legendre", "hermite"])
def test_gpc_quantile_bounds(O, cuda, family):
    """Confidence bounds of the profile behind the cube from the gPC
    surrogate (2.5 / 50 / 97.5 %, 3000 samples): the GPU's quantiles against
    the oracle's on the same coefficients (evaluation, sort and selection,
    to rounding), and the whole chain against the oracle's own ensemble and
    projection."""
    rng = np.random.default_rng(5)
    if family == "legendre":
        wl = dict(W.CHANNEL_CUBE)
        samples = rng.uniform(-1.0, 1.0, (3000, 1))
        fam = O.LEGENDRE
    else:
        wl = dict(W.CHANNEL_CUBE, inputs=[W.SPEED, W.ANGLE], lo=[0.0, 0.0], hi=[0.1, 6.0], quad_rule=W.GH,
                  profile=W.PROFILE_LOG, z0=0.1, gpc_degree=2,
                  domains=[dict(W.CHANNEL_CUBE["domains"][0], quad_level=3)])
        samples = rng.standard_normal((3000, 2))
        fam = O.HERMITE
    steps = 120
    ens = S.Ensemble(S.make_config(wl))
    ens.step(steps)
    coef = ens.moments(0, gpc=True)["coef"]
    D = wl["domains"][0]
    x, y = wl["columns"][0]
    cells = [x + D["nx"] * (y + D["ny"] * z) for z in range(D["nz"])]
    q = [0.025, 0.5, 0.975]
    got = ens.gpc_quantiles(0, coef, cells, samples, q).cpu().numpy()
    d = len(wl["inputs"])
    phi = O.gpc_basis_family(d, wl["gpc_degree"], fam, samples)
    cg = coef.cpu().numpy()
    np.testing.assert_allclose(got, O.gpc_quantiles(cg[:, cells], phi, q), rtol=0, atol=1e-14)
    assert (got[0] <= got[1]).all() and (got[1] <= got[2]).all()
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    Qv = O.ensemble(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, steps, z0=wl.get("z0"))
    s_nodes = O.legendre_s(Z, wl["lo"], wl["hi"]) if fam == O.LEGENDRE else O.normal_s(Z, wl["lo"], wl["hi"])
    co = O.gpc_project(a, Qv, O.gpc_basis_family(d, wl["gpc_degree"], fam, s_nodes))
    assert rel_l2(got, O.gpc_quantiles(co[:, cells], phi, q)) <= 1e-10
    for bad in (dict(q=[1.5]), dict(cells=[D["nx"] * D["ny"] * D["nz"]]),
                dict(samples=np.zeros((S.SC_QUANTILE_MAX_SAMPLES + 1, d)))):
        args = dict(cells=cells, samples=samples, q=q)
        args.update(bad)
        with pytest.raises(S.ScError) as ei:
            ens.gpc_quantiles(0, coef, args["cells"], args["samples"], args["q"])
        assert ei.value.code == S.SC_ERR_ARG
    ens.close()


def test_inflow_series_modes_are_bitwise_identical(cuda):
    """Under a series (ramp, three interpolation intervals, holds between)
    the graph mode, which replays graphs captured per hold, matches plain
    launches bit for bit; the persistent mode matches to rounding.  Removing
    the series mid-run gives the steady inflow back in every mode."""
    wl = ragged(BC_SETS["urban"])
    series = ([1.0, 1.2, 0.9, 1.05], [0.0, 40.0, -30.0, 185.0], 12, 5)
    got = {}
    for mode in (S.SC_EXEC_LAUNCH, S.SC_EXEC_GRAPH, S.SC_EXEC_PERSISTENT):
        ens = S.Ensemble(S.make_config(wl))
        S.sc_lbm_set_tuning(ens.h, 64, 1, 1, exec_mode=mode, graph_steps=4, variant=0)
        ens.set_inflow_series(*series)
        ens.step(45)
        ens.set_inflow_series([], [], 1, 0)
        ens.step(8)
        got[mode] = _states(ens)
        ens.close()
    for a, b in zip(got[S.SC_EXEC_LAUNCH], got[S.SC_EXEC_GRAPH]):
        assert np.array_equal(a, b)
    for a, b in zip(got[S.SC_EXEC_LAUNCH], got[S.SC_EXEC_PERSISTENT]):
        assert np.max(np.abs(a - b)) < 1e-6


def test_inflow_series_rejected_by_the_adjoint(cuda):
    wl = dict(W.CHANNEL_CUBE, precision=W.FP32_SHIFT)
    ens = S.Ensemble(S.make_config(wl))
    ens.set_inflow_series([1.0, 1.1], [0.0, 5.0], 10, 2)
    ws = torch.empty(S.sc_lbm_adjoint_workspace_size(ens.h, 0, 10, 0, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_adjoint(ens.h, 0, 0, np.array([[30, 12, 18]], np.int32), np.zeros((1, 3)), 10, 0,
                         ws.data_ptr(), ws.numel())
    assert ei.value.code == S.SC_ERR_UNSUPPORTED
    ens.close()


@pytest.mark.parametrize("precision,tol", [(W.FP64_PLAIN, 1e-11), (W.FP32_SHIFT, 1e-5)])
def test_time_averaged_fields(O, cuda, precision, tol):
    """Time-averaged |u| per node (5 samples, 15 steps apart, after 150
    steps) and its quadrature statistics against the oracle."""
    wl = dict(W.CHANNEL_CUBE, precision=precision, time_average=1)
    ens = S.Ensemble(S.make_config(wl))
    with pytest.raises(S.ScError):
        ens.average_field(0, 0)          # no sample yet
    ens.step(150)
    S.sc_lbm_average_add(ens.h)          # discarded by the reset below
    S.sc_lbm_average_reset(ens.h)
    for k in range(5):
        if k:
            ens.step(15)
        S.sc_lbm_average_add(ens.h)
    assert S.sc_lbm_average_samples(ens.h) == 5
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    A = O.ensemble_time_average(p, flags, Z, wl["inputs"], wl["u_ref"], wl["alpha"], 0.0, p.nz, 150, 5, 15)
    fl = fluid_mask(flags)
    for j in (0, len(a) - 1):
        assert rel_l2(ens.average_field(0, j).cpu().numpy()[fl], A[j][fl]) <= tol
    out = ens.average_moments(0, probes=wl["columns"], gpc=True)
    mean, std, _ = O.moments_two_pass(a, A)
    assert rel_l2(out["mean"].cpu().numpy()[fl], mean[fl]) <= tol
    assert rel_l2(out["std"].cpu().numpy()[fl], std[fl]) <= tol * 10
    prof, _ = O.profiles(a, A, p.nx, p.ny, p.nz, wl["columns"])
    assert rel_l2(out["prof"].cpu().numpy(), prof) <= tol * 10
    ens.close()
    # configurations without accumulators reject the calls
    plain = S.Ensemble(S.make_config(W.CHANNEL_CUBE))
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_average_add(plain.h)
    assert ei.value.code == S.SC_ERR_STATE
    plain.close()


def test_qcriterion(O, cuda):
    """Q of an exported velocity field of the ragged urban case (solid blocks,
    velocity, outflow and free-slip faces) against the oracle's stencil, and
    the closed form Omega^2 of a solid-body rotation around the blocks."""
    wl = ragged(BC_SETS["urban"])
    ens = S.Ensemble(S.make_config(wl))
    ens.step(20)
    u = ens.velocity(0, 1)
    q = ens.qcriterion(0, u).cpu().numpy()
    p, flags = oracle_domain(O, wl)
    bc = wl["domains"][0]["bc"]
    qo = O.qcriterion(u.cpu().numpy(), flags, p.nx, p.ny, p.nz, bc)
    assert np.max(np.abs(q - qo)) <= 1e-6 * max(np.max(np.abs(qo)), 1e-30)
    nx, ny, nz = p.nx, p.ny, p.nz
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Wr = 0.01
    ur = np.stack([-Wr * yy.reshape(-1), Wr * xx.reshape(-1), 0.0 * xx.reshape(-1)]).astype(np.float32)
    qr = ens.qcriterion(0, torch.from_numpy(ur).cuda()).cpu().numpy()
    fl = fluid_mask(flags)
    # every fluid cell of this domain has a fluid neighbour along each axis
    np.testing.assert_allclose(qr[fl], Wr * Wr, rtol=1e-5)
    assert np.all(qr[~fl] == 0)
    ens.close()


@pytest.mark.parametrize("nx2", [29, 32])
def test_batched_uneven_domains_match_oracle(O, cuda, nx2):
    """Three domains of different sizes and node counts advance in one launch;
    each matches its own oracle run (nx2 = 32: all domains take the TMA-staged
    kernels; 29: the per-thread ones)."""
    doms = [dict(nx=40, ny=18, nz=12, seed=1, n_buildings=2, fp=(4, 6), h=(3, 7), bc=W.URBAN_BC, quad_level=2),
            dict(nx=nx2, ny=23, nz=14, seed=2, n_buildings=3, fp=(3, 5), h=(3, 9), bc=W.URBAN_BC, quad_level=3),
            dict(nx=52, ny=11, nz=9, seed=3, n_buildings=1, fp=(3, 4), h=(2, 4), bc=W.URBAN_BC, quad_level=1)]
    wl = dict(W.URBAN_BATCHED, domains=doms, ramp_steps=5, tau0=0.56)
    ens = S.Ensemble(S.make_config(wl))
    ens.step(27)
    for d in range(3):
        Z, a = oracle_nodes(O, wl, d)
        assert len(a) == ens.n_nodes[d]
        for j in sorted({0, len(a) - 1}):
            p, flags, f = oracle_run_node(O, wl, d, j, 27)
            fg = gpu_state(ens, d, j)
            fl = fluid_mask(flags)
            assert np.max(np.abs(fg[:, fl] - f[:, fl])) < 2e-6
    ens.close()


def _states(ens):
    return [gpu_state(ens, d, j) for d in range(len(ens.n_nodes)) for j in range(ens.n_nodes[d])]


@pytest.mark.parametrize("shape", [(32, 1, 1, 0), (64, 4, 2, 1), (128, 2, 4, 0), (256, 1, 3, 1)])
def test_launch_shapes_and_modes_are_bitwise_identical(cuda, shape):
    """Every launch shape, tile order, execution mode (launch, graph,
    persistent) and kernel form (per-thread with either register budget,
    TMA-staged) gives the same bits."""
    wl = ragged(BC_SETS["urban"], nx=40)
    want = {}
    variants = (0, 1, 2, 3)
    for variant in variants:
        ref = S.Ensemble(S.make_config(wl))
        S.sc_lbm_set_tuning(ref.h, 64, 1, 1, variant=variant)
        ref.step(17)
        want[variant] = _states(ref)
        ref.close()
    # the kernel forms are compiled separately (rounding may differ in the
    # last bit); within a form every shape and mode is bitwise identical
    for v in variants[1:]:
        for a, b in zip(want[0], want[v]):
            assert np.max(np.abs(a - b)) < 1e-6
    for mode in (S.SC_EXEC_LAUNCH, S.SC_EXEC_GRAPH, S.SC_EXEC_PERSISTENT):
        for variant in variants:
            ens = S.Ensemble(S.make_config(wl))
            S.sc_lbm_set_tuning(ens.h, *shape, exec_mode=mode, graph_steps=4, variant=variant)
            ens.step(17)
            got = _states(ens)
            if mode == S.SC_EXEC_PERSISTENT:
                # one kernel for both levels, compiled on its own: same
                # arithmetic, rounding may differ in the last bit
                for a, b in zip(got, want[0]):
                    assert np.max(np.abs(a - b)) < 1e-6, (shape, mode, variant)
            else:
                for a, b in zip(got, want[variant]):
                    assert np.array_equal(a, b), (shape, mode, variant)
            ens.sync()
            ens.close()


def test_les_full_size_100_steps(O, cuda):
    """Synthetic urban LES at full size (256x128x64, BGK + Smagorinsky): the
    first and last node after 100 steps, relative L2 of u <= 1e-3."""
    wl = W.URBAN_LES
    ens = S.Ensemble(S.make_config(wl))
    S.sc_lbm_autotune(ens.h, None)
    ens.step(100)
    for j in (0, ens.n_nodes[0] - 1):
        p, flags, f = oracle_run_node(O, wl, 0, j, 100)
        _, uo = O.macros(p, flags, f)
        ug = ens.velocity(0, j).cpu().numpy()
        fl = fluid_mask(flags)
        assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-3
    ens.close()


def test_les_full_size_100_steps_regularized(O, cuda):
    """The urban LES ensemble with the paper's collision (recursive
    regularized, third-order equilibrium, C_S = 0.25) at full size: first and
    last node after 100 steps, relative L2 of u <= 1e-3."""
    wl = W.URBAN_LES_RR
    ens = S.Ensemble(S.make_config(wl))
    ens.step(100)
    for j in (0, ens.n_nodes[0] - 1):
        p, flags, f = oracle_run_node(O, wl, 0, j, 100)
        _, uo = O.macros(p, flags, f)
        ug = ens.velocity(0, j).cpu().numpy()
        fl = fluid_mask(flags)
        assert rel_l2(ug[:, fl], uo[:, fl]) <= 1e-3
    ens.close()


def test_full_size_single_step_from_exported_state(O, cuda):
    """At full size and in the benchmark's launch shape, one GPU step from any
    state equals one oracle step from the exported populations (both parities,
    after the ramp has started so that every boundary carries flow)."""
    wl = W.URBAN_LES
    ens = S.Ensemble(S.make_config(wl))
    S.sc_lbm_autotune(ens.h, None)
    p, flags = oracle_domain(O, wl)
    Z, a = oracle_nodes(O, wl)
    fl = fluid_mask(flags)
    ens.step(300)
    for n in (300, 301):
        j = n % len(a)
        f0 = gpu_state(ens, 0, j)
        ens.step(1)
        f1 = gpu_state(ens, 0, j)
        O.run(p, flags, oracle_uin(O, wl, 0, Z[j]), f0, n, 1)
        assert np.max(np.abs(f1[:, fl] - f0[:, fl])) < 2e-6
    ens.close()


@pytest.mark.parametrize("name", ["urban_batched_3domains", "urban_large_512x256x128_cc4"])
def test_other_full_size_workloads_single_step(O, cuda, name):
    """The batched ensemble (128x64x48 / 192x96x64 / 320x160x64 with 13 / 29 /
    5 nodes in one launch) and the large one (512x256x128, 69 nodes, 89.7 GB):
    one GPU step from the exported state of a sampled node of every domain
    equals one oracle step, at both parities during the ramp."""
    wl = {w["name"]: w for w in W.ALL}[name]
    ens = S.Ensemble(S.make_config(wl))
    ens.step(300)
    doms = range(len(wl["domains"]))
    oracle = [oracle_domain(O, wl, d) for d in doms]
    nodes = [oracle_nodes(O, wl, d) for d in doms]
    for n in (300, 301):
        pick = [(n + 7 * d) % len(nodes[d][1]) for d in doms]
        f0 = [gpu_state(ens, d, pick[d]) for d in doms]
        ens.step(1)
        for d in doms:
            p, flags = oracle[d]
            fl = fluid_mask(flags)
            f1 = gpu_state(ens, d, pick[d])
            O.run(p, flags, oracle_uin(O, wl, d, nodes[d][0][pick[d]]), f0[d], n, 1)
            assert np.max(np.abs(f1[:, fl] - f0[d][:, fl])) < 2e-6, (name, d, n)
            del f1
        del f0
    ens.close()


@pytest.mark.parametrize("gpc_degree", [2, 3, 5], ids=["P6", "P10", "P21"])
def test_ensemble_moments_match_exported_fields(O, cuda, gpc_degree):
    """Property at full size: the on-device FP64 reduction equals the oracle's
    two-pass moments of the per-node |u| fields the GPU exports, and the gPC
    sums (compensated FP32 pairs, bases of 6, 10 and 21 terms) equal the FP64
    projection of the same fields."""
    wl = dict(W.URBAN_LES, gpc_degree=gpc_degree)
    ens = S.Ensemble(S.make_config(wl))
    ens.step(60)
    cfg = S.make_config(wl)
    Z, a = S.sc_lbm_quadrature(cfg, 0)
    flags = S.sc_lbm_geometry(cfg, 0)
    # |u| as the library forms it from its FP32 velocity: (ux^2 + uy^2) + uz^2
    # and the square root, each rounded once in FP32
    us = [ens.velocity(0, j).cpu().numpy() for j in range(len(a))]
    Qv = np.stack([np.sqrt((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]).astype(np.float64) for u in us])
    Qv[:, flags != 0] = 0.0
    mean, std, _ = O.moments_two_pass(a, Qv)
    cols = S.sc_lbm_probe_columns(cfg, 0, 4)
    out = ens.moments(0, probes=cols, gpc=True)
    assert np.max(np.abs(out["mean"].cpu().numpy() - mean)) < 1e-12
    assert np.max(np.abs(out["std"].cpu().numpy() - std)) < 1e-9
    prof, _ = O.profiles(a, Qv, 256, 128, 64, cols)
    assert np.max(np.abs(out["prof"].cpu().numpy() - prof)) < 1e-9
    # gPC sums: compensated FP32 pairs against the FP64 projection of the
    # same fields, within 1e-12 of sum_j |a_j Phi_alpha(Z_j) Q_j| per cell
    phi = O.gpc_basis(2, wl["gpc_degree"], O.legendre_s(Z, wl["lo"], wl["hi"]))
    coef = O.gpc_project(a, Qv, phi)
    bound = (np.abs(a[:, None] * phi)).T @ np.abs(Qv)
    assert np.all(np.abs(out["coef"].cpu().numpy() - coef) <= 1e-12 * bound)
    ens.close()


def test_host_outputs_match_device_outputs(cuda):
    wl = ragged(BC_SETS["urban"])
    ens = S.Ensemble(S.make_config(wl))
    ens.step(9)
    dev = ens.moments(0, probes=[[30, 4]], nodes_profiles=True, gpc=True)
    n = 37 * 19 * 13
    mean, std = np.zeros(n), np.zeros(n)
    prof, pn = np.zeros((1, 13, 4)), np.zeros((1, 3, 13), np.float32)
    coef = np.zeros((3, n))
    S.sc_lbm_moments(ens.h, 0, mean, std, [[30, 4]], prof, pn, coef, out_host=True)
    assert np.array_equal(mean, dev["mean"].cpu().numpy())
    assert np.array_equal(std, dev["std"].cpu().numpy())
    assert np.array_equal(prof, dev["prof"].cpu().numpy())
    assert np.array_equal(pn, dev["prof_nodes"].cpu().numpy())
    assert np.array_equal(coef, dev["coef"].cpu().numpy())
    ens.close()


def test_bounded_barrier_wait_times_out_and_recovers(cuda):
    """A grid-barrier arrival that never comes: the wait gives up after its
    poll limit, the call reports SC_ERR_TIMEOUT and the device stays usable.
    No start-up ramp: levels inside it are launched one by one, outside the
    persistent kernel."""
    wl = ragged(BC_SETS["urban"], ramp=0)
    ens = S.Ensemble(S.make_config(wl))
    S.sc_lbm_set_tuning(ens.h, 64, 2, 1, exec_mode=S.SC_EXEC_PERSISTENT)
    S.sc_lbm_debug_barrier(ens.h, 1, 20000)
    ens.step(3)
    with pytest.raises(S.ScError) as ei:
        ens.sync()
    assert ei.value.code == S.SC_ERR_TIMEOUT
    S.sc_lbm_debug_barrier(ens.h, 0, 1 << 26)
    S.sc_lbm_reset(ens.h)
    ens.step(5)
    ens.sync()
    ref = S.Ensemble(S.make_config(wl))
    ref.step(5)
    assert np.max(np.abs(gpu_state(ens, 0, 0) - gpu_state(ref, 0, 0))) < 1e-6
    ens.close()
    ref.close()


def test_non_finite_state_is_detected(cuda):
    """Host-side fault injection: a NaN written into one population is
    reported by sc_lbm_check and by the moments reduction."""
    wl = ragged(BC_SETS["urban"])
    ens = S.Ensemble(S.make_config(wl))
    ens.step(4)
    rc, nbad = S.sc_lbm_check(ens.h)
    assert rc == S.SC_OK and nbad == 0
    S.sc_lbm_step(ens.h, 1)
    torch.cuda.synchronize()
    # inject through a snapshot: save, corrupt one value (population 0 of
    # node 1 at fluid cell 1234; rows are padded to a multiple of 256 cells), load
    buf = np.zeros(S.sc_lbm_state_size(ens.h), np.uint8)
    S.sc_lbm_save(ens.h, buf)
    hdr = 48
    pitch = (37 * 19 * 13 + 255) // 256 * 256
    vals = buf[hdr:].view(np.float32)
    vals[19 * pitch + 1234] = np.nan
    with pytest.raises(S.ScError):      # checksum catches the corrupted snapshot
        S.sc_lbm_load(ens.h, buf)
    # a consistent snapshot with a NaN: recompute the payload checksum (FNV-1a)
    payload = buf[hdr:].tobytes()
    h = 1469598103934665603
    for byte in payload:
        h ^= byte
        h = (h * 1099511628211) & ((1 << 64) - 1)
    buf[24:32] = np.frombuffer(np.uint64(h).tobytes(), np.uint8)
    S.sc_lbm_load(ens.h, buf)
    rc, nbad = S.sc_lbm_check(ens.h)
    assert rc == S.SC_ERR_DIVERGED and nbad >= 1
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_moments(ens.h, 0, np.zeros(37 * 19 * 13), np.zeros(37 * 19 * 13), out_host=True)
    assert ei.value.code == S.SC_ERR_DIVERGED
    ens.close()


def test_save_load_resume(cuda):
    wl = ragged(BC_SETS["urban"])
    a = S.Ensemble(S.make_config(wl))
    a.step(7)
    buf = np.zeros(S.sc_lbm_state_size(a.h), np.uint8)
    S.sc_lbm_save(a.h, buf)
    a.step(6)
    want = _states(a)
    b = S.Ensemble(S.make_config(wl))
    S.sc_lbm_load(b.h, buf)
    assert S.sc_lbm_counters(b.h)[0] == 7
    b.step(6)
    for x, y in zip(_states(b), want):
        assert np.array_equal(x, y)
    a.close()
    b.close()
