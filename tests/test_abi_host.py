"""CPU tests of the C ABI: the library loads, exports every function that
include/*.h declares, and its host-only calls (quadrature, geometry, probes,
validation) agree bit for bit with the oracle.  No GPU is touched."""
import glob
import math
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2508_18202_gb300 import sclbm as S
from paper_2508_18202_gb300 import workloads as W


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = S.lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header():
    names = _declared()
    assert names <= set(S.SIGNATURES), sorted(names - set(S.SIGNATURES))


def _oracle_rule(O, cfg, d):
    c = cfg.c
    lo = [c.lo[k] for k in range(c.n_inputs)]
    hi = [c.hi[k] for k in range(c.n_inputs)]
    return O.quadrature(c.quad_rule, c.n_inputs, cfg.domains[d]["quad_level"], lo, hi)


@pytest.mark.parametrize("wl", W.ALL, ids=lambda w: w["name"])
def test_quadrature_bit_exact_with_oracle(O, wl):
    """Gauss-Legendre and Clenshaw-Curtis Smolyak rules are a bit-exact
    contract; Gauss-Hermite nodes come from an eigenproblem in the library and
    from bisection in the oracle, so they agree to rounding."""
    cfg = S.make_config(wl)
    for d in range(len(wl["domains"])):
        Z, w = S.sc_lbm_quadrature(cfg, d)
        Zo, wo = _oracle_rule(O, cfg, d)
        assert Z.shape == Zo.shape
        if wl["quad_rule"] == W.GH:
            scale = np.abs(np.asarray(wl["hi"]))[None, :]
            assert np.max(np.abs(Z - Zo) / scale) < 1e-13
            assert np.max(np.abs(w - wo) / wo) < 1e-12
        else:
            assert Z.tobytes() == Zo.tobytes()
            assert w.tobytes() == wo.tobytes()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 11, 16, 25, 40])
def test_gauss_hermite_library_rule(O, n):
    """The library's Golub-Welsch rule against the oracle's bisection rule."""
    cfg = S.make_config(dict(W.URBAN_GH121, domains=[dict(W.URBAN_GH121["domains"][0], quad_level=n)],
                             inputs=[W.SPEED], lo=[0.0], hi=[1.0], gpc_degree=-1))
    Z, w = S.sc_lbm_quadrature(cfg, 0)
    Zo, wo = O.quadrature(W.GH, 1, n, [0.0], [1.0])
    assert np.max(np.abs(Z - Zo)) < 1e-13
    assert np.max(np.abs(w - wo) / wo) < 1e-12
    assert np.all(Z[:, 0] == -Z[::-1, 0]) and np.all(w == w[::-1])


@pytest.mark.parametrize("rule,d,level", [(0, 1, n) for n in range(1, 6)] + [(0, 2, 3), (0, 3, 2)]
                         + [(1, d, L) for d in (1, 2, 3) for L in (1, 2, 3, 4, 5)])
def test_quadrature_rules_bit_exact(O, rule, d, level):
    lo = [-0.15, 0.15, -10.0][:d]
    hi = [0.15, 0.35, 10.0][:d]
    dom = dict(nx=8, ny=8, nz=8, bc=[2] * 6, quad_level=level)
    inputs = [W.SPEED, W.ALPHA, W.ANGLE][:d]
    cfg = S.Config([dom], 0.6, 0.0, 0.05, 0.25, inputs, lo, hi, rule, W.FP32_SHIFT)
    Z, w = S.sc_lbm_quadrature(cfg, 0)
    Zo, wo = O.quadrature(rule, d, level, lo, hi)
    assert Z.tobytes() == Zo.tobytes() and w.tobytes() == wo.tobytes()


@pytest.mark.parametrize("wl", W.ALL, ids=lambda w: w["name"])
def test_geometry_and_probes_bit_exact_with_oracle(O, wl):
    cfg = S.make_config(wl)
    for d, D in enumerate(wl["domains"]):
        flags = S.sc_lbm_geometry(cfg, d)
        fo = O.geometry(D["nx"], D["ny"], D["nz"], D.get("seed", 0), D.get("n_buildings", 0),
                        *D.get("fp", (1, 1)), *D.get("h", (1, 1)), boxes=D.get("boxes"),
                        disk_radius=D.get("disk_radius", 0.0))
        assert flags.tobytes() == fo.tobytes()
        if D.get("boxes") is None:
            xy = S.sc_lbm_probe_columns(cfg, d, 4)
            assert np.array_equal(xy, O.probe_columns(D["nx"], D["ny"], D["nz"], D["seed"], fo, 4))
            pts = S.sc_lbm_probe_points(cfg, d, 16)
            assert np.array_equal(pts, O.probe_points(D["nx"], D["ny"], D["nz"], D["seed"], fo, 16))


def test_workspace_size_scales_with_precision():
    b32 = S.sc_lbm_workspace_size(S.make_config(W.URBAN_LES))
    b16 = S.sc_lbm_workspace_size(S.make_config(W.URBAN_LES, precision=W.BF16_STORE))
    b64 = S.sc_lbm_workspace_size(S.make_config(W.URBAN_LES, precision=W.FP64_PLAIN))
    pops = 13 * 19 * 256 * 128 * 64
    assert b32 > 4 * pops and b16 > 2 * pops and b64 > 16 * pops
    assert b16 < b32 < b64


@pytest.mark.parametrize("bad,code", [
    (dict(tau0=0.5), S.SC_ERR_ARG),
    (dict(tau0=0.45), S.SC_ERR_ARG),
    (dict(c_smag=-0.1), S.SC_ERR_ARG),
    (dict(lo=[0.1, 0.15], hi=[-0.1, 0.35]), S.SC_ERR_ARG),
    (dict(quad_rule=7), S.SC_ERR_ARG),
    (dict(precision=9), S.SC_ERR_ARG),
    (dict(gpc_degree=7), S.SC_ERR_UNSUPPORTED),
    (dict(collision=3), S.SC_ERR_ARG),
    (dict(profile=5), S.SC_ERR_ARG),
    (dict(profile=W.PROFILE_LOG, z0=0.0), S.SC_ERR_ARG),
    (dict(quad_rule=W.GH, lo=[0.0, 0.0], hi=[0.1, 0.0]), S.SC_ERR_ARG),
    (dict(domain_over=dict(bc=[W.OUT, W.VEL, W.VEL, W.VEL, W.BB, W.FS])), S.SC_ERR_UNSUPPORTED),
    (dict(domain_over=dict(bc=[W.PER, W.OUT, W.VEL, W.VEL, W.BB, W.FS])), S.SC_ERR_ARG),
    (dict(domain_over=dict(nx=0)), S.SC_ERR_ARG),
    (dict(domain_over=dict(disk_radius=-1.0)), S.SC_ERR_ARG),
    (dict(domain_over=dict(disk_radius=float("nan"))), S.SC_ERR_ARG),
    (dict(domain_over=dict(disk_radius=60.0)), S.SC_ERR_UNSUPPORTED),   # URBAN_BC has an outflow face
])
def test_invalid_configurations_rejected(bad, code):
    wl = W.variant(W.URBAN_LES, **bad)
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_workspace_size(S.make_config(wl))
    assert ei.value.code == code


def test_device_calls_reject_null_handles():
    L = S.lib()
    assert L.sc_lbm_step(None, 1) == S.SC_ERR_ARG
    assert L.sc_lbm_sync(None) == S.SC_ERR_ARG
    assert L.sc_lbm_destroy(None) == S.SC_ERR_ARG
    assert L.sc_lbm_last_error(None) == b"null handle"


def test_init_rejects_missing_workspace():
    cfg = S.make_config(W.CHANNEL_CUBE)
    import ctypes as C
    h = C.c_void_p()
    rc = S.lib().sc_lbm_init(cfg.ref, None, 0, None, None, C.byref(h))
    assert rc == S.SC_ERR_WORKSPACE
    rc = S.lib().sc_lbm_init(cfg.ref, C.c_void_p(0x1000), 16, None, None, C.byref(h))
    assert rc == S.SC_ERR_WORKSPACE


SERIES = ([1.0, 1.35, 0.6, 0.9], [350.0, 20.0, 200.0, -170.0])


@pytest.mark.parametrize("ramp,per,interp", [(0, 10, 4), (7, 10, 4), (25, 10, 10), (3, 6, 0), (0, 1, 1)])
def test_inflow_factor_matches_oracle_schedule(O, ramp, per, interp):
    """The library's factor of every level (ramp, interpolation intervals,
    shorter-arc turns, the hold after the last target) against the oracle's
    schedule: (a, b, m) = r s (cos delta, sin delta, 1)."""
    speed, dirs = SERIES
    for m in list(range(0, 5 * per + ramp + 3)) + [10 ** 7]:
        s, d = O.series_at(speed, dirs, per, interp, m)
        r = O.ramp(ramp, m)
        want = r * s * np.array([math.cos(math.radians(d)), math.sin(math.radians(d)), 1.0])
        got = S.sc_lbm_inflow_factor(ramp, speed, dirs, per, interp, m)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14, err_msg=str(m))


def test_inflow_factor_without_series_is_the_ramp(O):
    for m in (0, 1, 5, 9, 10, 1000):
        np.testing.assert_array_equal(S.sc_lbm_inflow_factor(10, [], [], 1, 0, m),
                                      [O.ramp(10, m), 0.0, O.ramp(10, m)])


@pytest.mark.parametrize("args", [
    dict(speed=[1.0, 1.0], dirs=[0.0, 0.0], per=10, interp=11),   # interval longer than a target
    dict(speed=[1.0, 1.0], dirs=[0.0, 0.0], per=0, interp=0),
    dict(speed=[1.0, 1.0], dirs=[0.0, 0.0], per=(1 << 40) + 1, interp=0),
    dict(speed=[1.0, -0.1], dirs=[0.0, 0.0], per=10, interp=2),   # negative speed factor
    dict(speed=[1.0, 1.0], dirs=[0.0, float("nan")], per=10, interp=2),
    dict(speed=[1.0, float("inf")], dirs=[0.0, 0.0], per=10, interp=2),
    dict(speed=[1.0], dirs=[0.0], per=10, interp=-1),
    dict(speed=[1.0], dirs=[0.0], per=10, interp=2, level=-1),
    dict(speed=[1.0], dirs=[0.0], per=10, interp=2, ramp=-1),
])
def test_inflow_series_rejects_invalid_arguments(args):
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_inflow_factor(args.get("ramp", 0), args["speed"], args["dirs"], args["per"], args["interp"],
                               args.get("level", 0))
    assert ei.value.code == S.SC_ERR_ARG


def test_inflow_series_rejects_too_many_targets():
    n = S.SC_SERIES_MAX_TARGETS + 1
    with pytest.raises(S.ScError) as ei:
        S.sc_lbm_inflow_factor(0, np.ones(n), np.zeros(n), 1, 0, 0)
    assert ei.value.code == S.SC_ERR_ARG


@pytest.mark.parametrize("ramp,per,interp", [(0, 10, 4), (7, 10, 4), (25, 10, 10), (3, 6, 0), (0, 1, 1),
                                             (12, 5, 5)])
def test_inflow_stretches_never_miss_a_change(ramp, per, interp):
    """The execution stretches of sc_lbm_step: from every level m the factor
    stays exactly W(m) up to the reported next change, so graph replays and
    persistent launches that bake W(m) into a stretch use the right inflow;
    and the stretches are long where nothing changes (holds, after the
    last target)."""
    speed, dirs = SERIES
    end = 5 * per + ramp + 3
    for m in range(end):
        nxt = S.sc_lbm_inflow_next_change(ramp, speed, dirs, per, interp, m)
        assert nxt > m
        w = S.sc_lbm_inflow_factor(ramp, speed, dirs, per, interp, m)
        for k in range(m, min(nxt, end + per)):
            assert np.array_equal(S.sc_lbm_inflow_factor(ramp, speed, dirs, per, interp, k), w), (m, k, nxt)
    last = (len(speed) - 1) * per + max(interp, 0) + ramp
    assert S.sc_lbm_inflow_next_change(ramp, speed, dirs, per, interp, last + 1) > 2 ** 62
    if interp < per and ramp < per:
        # inside the hold of target 1 the next change is the start of the move to target 2
        m = per + interp + 1
        assert S.sc_lbm_inflow_next_change(ramp, speed, dirs, per, interp, m) == 2 * per + (1 if interp else 0)
    # without a series only the ramp changes the factor
    assert S.sc_lbm_inflow_next_change(ramp, [], [], 1, 0, ramp) > 2 ** 62
    if ramp:
        assert S.sc_lbm_inflow_next_change(ramp, [], [], 1, 0, 0) == 1
