"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg import this module.  It never touches the CUDA library.

Array conventions follow sclbm_oracle.h: cell index c = x + nx*(y + ny*z),
populations f[19][ncell] (unshifted FP64, natural layout), u[3][ncell].
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

VELOCITY, OUTFLOW, BOUNCE_BACK, FREE_SLIP, PERIODIC = 0, 1, 2, 3, 4
IN_SPEED_REL, IN_ALPHA, IN_ANGLE_DEG = 0, 1, 2
Q_GL, Q_CC_SMOLYAK = 0, 1
Z95 = 1.959963984540054


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("bc", C.c_int * 6), ("tau0", C.c_double), ("csmag", C.c_double),
                ("ramp_steps", C.c_int), ("force", C.c_double * 3), ("collision", C.c_int)]


BGK, RR = 0, 1  # collision: BGK, or recursive regularized with the third-order equilibrium


def params(nx, ny, nz, bc, tau0, csmag=0.0, ramp_steps=0, force=(0.0, 0.0, 0.0), collision=BGK):
    p = Params()
    p.nx, p.ny, p.nz = nx, ny, nz
    for k in range(6):
        p.bc[k] = int(bc[k])
    p.tau0, p.csmag, p.ramp_steps = float(tau0), float(csmag), int(ramp_steps)
    for a in range(3):
        p.force[a] = float(force[a])
    p.collision = int(collision)
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
        i32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        ip = C.POINTER(C.c_int)
        pp = C.POINTER(Params)
        L.oc_lattice.argtypes = [ip, ip, ip, C.POINTER(C.c_double), ip]
        L.oc_equilibrium.argtypes = [C.c_double, dp, dp]
        L.oc_equilibrium3.argtypes = [C.c_double, dp, dp]
        L.oc_collide_cell.argtypes = [pp, dp, dp, C.POINTER(C.c_double)]
        L.oc_ramp.argtypes = [C.c_int, C.c_longlong]
        L.oc_ramp.restype = C.c_double
        L.oc_set_threads.argtypes = [C.c_int]
        L.oc_init_equilibrium.argtypes = [pp, u8, C.c_void_p, C.c_void_p, dp]
        L.oc_run.argtypes = [pp, u8, dp, dp, C.c_longlong, C.c_int]
        L.oc_macros.argtypes = [pp, u8, dp, dp, dp]
        L.oc_splitmix64.argtypes = [C.c_uint64, C.c_int, np.ctypeslib.ndpointer(dtype=np.uint64)]
        L.oc_geometry.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_int,
                                  C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, u8]
        L.oc_mark_mantle.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, u8]
        L.oc_probe_columns.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, u8, C.c_int, i32]
        L.oc_probe_points.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, u8, C.c_int, i32]
        L.oc_inflow.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_double, dp]
        L.oc_quadrature.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, ip, C.c_void_p,
                                    C.c_void_p, C.c_int]
        L.oc_moments_two_pass.argtypes = [C.c_int, C.c_longlong, dp, dp, dp, dp,
                                          C.POINTER(C.c_longlong)]
        L.oc_profiles.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, i32, dp,
                                  C.c_void_p]
        L.oc_gpc_basis_family.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
        L.oc_inflow_log.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double, dp]
        L.oc_gpc_basis_size.argtypes = [C.c_int, C.c_int]
        L.oc_gpc_basis.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        L.oc_gpc_project.argtypes = [C.c_int, C.c_int, C.c_longlong, dp, dp, dp, dp]
        L.oc_tangent_run.argtypes = [pp, u8, dp, dp, dp, C.c_int, C.c_int, i32, dp,
                                     C.POINTER(C.c_double), dp, dp]
        _lib = L
    return _lib


def _chk(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (%d)" % (what, rc))


def set_threads(n):
    return lib().oc_set_threads(int(n))


def lattice():
    cx, cy, cz, opp = (np.zeros(19, np.int32) for _ in range(4))
    w = np.zeros(19, np.float64)
    ip = C.POINTER(C.c_int)
    lib().oc_lattice(cx.ctypes.data_as(ip), cy.ctypes.data_as(ip), cz.ctypes.data_as(ip),
                     w.ctypes.data_as(C.POINTER(C.c_double)), opp.ctypes.data_as(ip))
    return cx, cy, cz, w, opp


def equilibrium(rho, u):
    feq = np.zeros(19)
    lib().oc_equilibrium(float(rho), np.ascontiguousarray(u, np.float64), feq)
    return feq


def equilibrium3(rho, u):
    """Third-order D3Q19 equilibrium of the recursive regularized model."""
    feq = np.zeros(19)
    lib().oc_equilibrium3(float(rho), np.ascontiguousarray(u, np.float64), feq)
    return feq


def collide_cell(p, f):
    fpost = np.zeros(19)
    tau = C.c_double(0.0)
    _chk(lib().oc_collide_cell(C.byref(p), np.ascontiguousarray(f, np.float64), fpost,
                               C.byref(tau)), "collide")
    return fpost, tau.value


def ramp(ramp_steps, m):
    return lib().oc_ramp(int(ramp_steps), int(m))


def init_equilibrium(p, flags, rho=None, u=None):
    n = p.nx * p.ny * p.nz
    f = np.zeros((19, n))
    r = None if rho is None else np.ascontiguousarray(rho, np.float64)
    uu = None if u is None else np.ascontiguousarray(u, np.float64)
    _chk(lib().oc_init_equilibrium(C.byref(p), np.ascontiguousarray(flags, np.uint8),
                                   None if r is None else r.ctypes.data,
                                   None if uu is None else uu.ctypes.data, f), "init")
    return f


def run(p, flags, uin, f, n0=0, n_steps=1):
    """Advance f (shape [19, ncell], modified in place) by n_steps from time n0."""
    assert f.dtype == np.float64 and f.flags.c_contiguous
    _chk(lib().oc_run(C.byref(p), np.ascontiguousarray(flags, np.uint8),
                      np.ascontiguousarray(uin, np.float64).reshape(-1), f, int(n0),
                      int(n_steps)), "run")
    return f


def macros(p, flags, f):
    n = p.nx * p.ny * p.nz
    rho = np.zeros(n)
    u = np.zeros((3, n))
    _chk(lib().oc_macros(C.byref(p), np.ascontiguousarray(flags, np.uint8), f, rho, u),
         "macros")
    return rho, u


def splitmix64(seed, n):
    out = np.zeros(n, np.uint64)
    lib().oc_splitmix64(C.c_uint64(seed), n, out)
    return out


def geometry(nx, ny, nz, seed=0, n_buildings=0, fp_min=1, fp_max=1, h_min=1, h_max=1,
             boxes=None, disk_radius=0.0):
    """Solid flags (1) of the buildings; with disk_radius > 0 the cells beyond
    the circular mantle get flag 2 (Sec. 2.2 circular domain)."""
    flags = np.zeros(nx * ny * nz, np.uint8)
    nb = 0
    bptr = None
    if boxes is not None and len(boxes):
        b = np.ascontiguousarray(np.asarray(boxes, np.int32).reshape(-1, 6))
        nb = b.shape[0]
        bptr = b.ctypes.data
    _chk(lib().oc_geometry(nx, ny, nz, C.c_uint64(seed), n_buildings, fp_min, fp_max, h_min,
                           h_max, bptr, nb, flags), "geometry")
    if disk_radius > 0:
        _chk(lib().oc_mark_mantle(nx, ny, nz, float(disk_radius), flags), "mark_mantle")
    return flags


def probe_columns(nx, ny, nz, seed, flags, n):
    xy = np.zeros(2 * n, np.int32)
    _chk(lib().oc_probe_columns(nx, ny, nz, C.c_uint64(seed), flags, n, xy), "probe_columns")
    return xy.reshape(n, 2)


def probe_points(nx, ny, nz, seed, flags, n):
    xyz = np.zeros(3 * n, np.int32)
    _chk(lib().oc_probe_points(nx, ny, nz, C.c_uint64(seed), flags, n, xyz), "probe_points")
    return xyz.reshape(n, 3)


def inflow(nz, u_ref, xi, alpha, H, theta_deg=0.0):
    uin = np.zeros((nz, 3))
    _chk(lib().oc_inflow(nz, u_ref, xi, alpha, H, theta_deg, uin.reshape(-1)), "inflow")
    return uin


GL, CC_SMOLYAK, GH = 0, 1, 2


def quadrature(rule, d, level, lo, hi):
    """Nodes Z[n][d] and probability weights w[n].  GL / CC_SMOLYAK: uniform
    inputs on [lo, hi]; GH: normal inputs, mean lo and standard deviation hi."""
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    n = C.c_int(0)
    _chk(lib().oc_quadrature(rule, d, level, lo, hi, C.byref(n), None, None, 0), "quadrature")
    Z = np.zeros((n.value, d))
    w = np.zeros(n.value)
    _chk(lib().oc_quadrature(rule, d, level, lo, hi, C.byref(n), Z.ctypes.data, w.ctypes.data,
                             n.value), "quadrature")
    return Z, w


def moments_two_pass(a, Qv):
    a = np.ascontiguousarray(a, np.float64)
    Qv = np.ascontiguousarray(Qv, np.float64)
    nq, n = Qv.shape
    mean, std = np.zeros(n), np.zeros(n)
    ncl = C.c_longlong(0)
    _chk(lib().oc_moments_two_pass(nq, n, a, Qv, mean, std, C.byref(ncl)), "moments")
    return mean, std, ncl.value


def profiles(a, Qv, nx, ny, nz, xy):
    a = np.ascontiguousarray(a, np.float64)
    Qv = np.ascontiguousarray(Qv, np.float64)
    xy = np.ascontiguousarray(np.asarray(xy, np.int32).reshape(-1))
    n_p = xy.size // 2
    nq = Qv.shape[0]
    prof = np.zeros((n_p, nz, 4))
    pn = np.zeros((n_p, nq, nz))
    _chk(lib().oc_profiles(nq, nx, ny, nz, a, Qv, n_p, xy, prof, pn.ctypes.data), "profiles")
    return prof, pn


def gpc_basis(d, degree, s):
    s = np.ascontiguousarray(s, np.float64).reshape(-1, d)
    P = lib().oc_gpc_basis_size(d, degree)
    phi = np.zeros((s.shape[0], P))
    _chk(lib().oc_gpc_basis(d, degree, s.shape[0], s, phi), "gpc_basis")
    return phi


LEGENDRE, HERMITE = 0, 1


def gpc_basis_family(d, degree, family, s):
    """Orthonormal basis values: Legendre on [-1,1] (family 0) or
    probabilists' Hermite He_n / sqrt(n!) of standard-normal coordinates
    (family 1)."""
    s = np.ascontiguousarray(s, np.float64).reshape(-1, d)
    P = lib().oc_gpc_basis_size(d, degree)
    phi = np.zeros((s.shape[0], P))
    _chk(lib().oc_gpc_basis_family(d, degree, family, s.shape[0], s, phi), "gpc_basis_family")
    return phi


def inflow_log(nz, u_ref, xi, z0, H, theta_deg=0.0):
    uin = np.zeros((nz, 3))
    _chk(lib().oc_inflow_log(nz, u_ref, xi, z0, H, theta_deg, uin.reshape(-1)), "inflow_log")
    return uin


def gpc_project(a, Qv, phi):
    a = np.ascontiguousarray(a, np.float64)
    Qv = np.ascontiguousarray(Qv, np.float64)
    phi = np.ascontiguousarray(phi, np.float64)
    nq, n = Qv.shape
    P = phi.shape[1]
    coef = np.zeros((P, n))
    _chk(lib().oc_gpc_project(nq, P, n, a, Qv, phi, coef), "gpc_project")
    return coef


def tangent_run(p, flags, uin, duin, f, n_steps, probes, u_target):
    """Dual-number run; returns (loss, dloss[2], u_probe[n,3]); f is advanced in place."""
    probes = np.ascontiguousarray(np.asarray(probes, np.int32).reshape(-1))
    ut = np.ascontiguousarray(u_target, np.float64).reshape(-1)
    npb = probes.size // 3
    loss = C.c_double(0.0)
    dl = np.zeros(2)
    up = np.zeros(3 * npb)
    _chk(lib().oc_tangent_run(C.byref(p), np.ascontiguousarray(flags, np.uint8),
                              np.ascontiguousarray(uin, np.float64).reshape(-1),
                              np.ascontiguousarray(duin, np.float64).reshape(-1), f,
                              int(n_steps), npb, probes, ut, C.byref(loss), dl, up),
         "tangent_run")
    return loss.value, dl, up.reshape(npb, 3)


# ------------------------------------------------------------------ pipeline
def node_inflow_params(Zj, inputs, u_ref, alpha, theta_deg):
    """Map one collocation node to (xi, alpha, theta) (Sec. 2.1 noise model in
    the configuration's uniform form): speed error multiplies u_ref by (1+xi),
    the exponent and the angle are used as drawn."""
    xi, al, th = 0.0, alpha, theta_deg
    for t, kind in enumerate(inputs):
        if kind == IN_SPEED_REL:
            xi = Zj[t]
        elif kind == IN_ALPHA:
            al = Zj[t]
        elif kind == IN_ANGLE_DEG:
            th = Zj[t]
        else:
            raise ValueError(kind)
    return xi, al, th


def velocity_magnitude(u, flags):
    q = np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    q[np.asarray(flags) != 0] = 0.0
    return q


def ensemble(p, flags, Z, inputs, u_ref, alpha, theta_deg, H, n_steps, keep_u=False, z0=None):
    """Run the deterministic solver at every collocation node (Sec. 2.4 steps
    4-6) and return |u| per node, Q[nq][ncell] (and u per node if asked).
    z0: None for the power-law profile, else the roughness length of the
    logarithmic profile (Sec. 3)."""
    n = p.nx * p.ny * p.nz
    nq = Z.shape[0]
    Qv = np.zeros((nq, n))
    us = []
    for j in range(nq):
        xi, al, th = node_inflow_params(Z[j], inputs, u_ref, alpha, theta_deg)
        if z0 is None:
            uin = inflow(p.nz, u_ref, xi, al, H, th)
        else:
            uin = inflow_log(p.nz, u_ref, xi, z0, H, th)
        f = init_equilibrium(p, flags)
        run(p, flags, uin, f, 0, n_steps)
        _, u = macros(p, flags, f)
        Qv[j] = velocity_magnitude(u, flags)
        if keep_u:
            us.append(u)
    return (Qv, us) if keep_u else Qv


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def normal_s(Z, mean, std):
    """Normal nodes mapped to standard-normal coordinates: (Z - mean) / std."""
    return (np.asarray(Z, np.float64) - np.asarray(mean, np.float64)) / np.asarray(std, np.float64)


def legendre_s(Z, lo, hi):
    """Nodes mapped to [-1, 1]: s = (2 Z - lo - hi) / (hi - lo)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return (2.0 * Z - lo - hi) / (hi - lo)


PI = math.pi


def qcriterion(u, flags, nx, ny, nz, bc):
    """Q-criterion of a velocity field u[3][ncell] (cell index x + nx (y + ny z)):
    Q = (|Omega|^2 - |S|^2) / 2 with S, Omega the symmetric and antisymmetric
    parts of grad u.  Per axis: central difference where both neighbours are
    fluid cells, one-sided where only one is, zero where none is; axes whose
    faces are periodic (bc[2a] == 4) wrap.  Solid cells give 0."""
    U = np.asarray(u, np.float64).reshape(3, nz, ny, nx)
    fluid = (np.asarray(flags).reshape(nz, ny, nx) == 0)
    J = np.zeros((3, 3, nz, ny, nx))
    for a in range(3):
        ax = 2 - a                      # array axis of x, y, z
        periodic = bc[2 * a] == 4
        n = U.shape[1 + ax]
        idx = np.arange(n)
        shape = [1, 1, 1]
        shape[ax] = n
        inside_p = (idx + 1 < n).reshape(shape) | periodic
        inside_m = (idx - 1 >= 0).reshape(shape) | periodic
        ok_p = inside_p & np.roll(fluid, -1, axis=ax)
        ok_m = inside_m & np.roll(fluid, 1, axis=ax)
        for i in range(3):
            up = np.roll(U[i], -1, axis=ax)
            um = np.roll(U[i], 1, axis=ax)
            d = np.where(ok_p & ok_m, 0.5 * (up - um),
                         np.where(ok_p, up - U[i], np.where(ok_m, U[i] - um, 0.0)))
            J[i, a] = d
    S = 0.5 * (J + J.transpose(1, 0, 2, 3, 4))
    Wm = 0.5 * (J - J.transpose(1, 0, 2, 3, 4))
    Q = 0.5 * ((Wm ** 2).sum((0, 1)) - (S ** 2).sum((0, 1)))
    Q[~fluid] = 0.0
    return Q.reshape(-1)


def ensemble_time_average(p, flags, Z, inputs, u_ref, alpha, theta_deg, H, n_warm, n_samples, every,
                          z0=None):
    """Per-node time average of |u| (Sec. 2.4 step 6): after n_warm steps,
    n_samples samples of |u|, the first at level n_warm, then every `every`
    steps.  Returns A[nq][ncell]."""
    n = p.nx * p.ny * p.nz
    A = np.zeros((Z.shape[0], n))
    for j in range(Z.shape[0]):
        xi, al, th = node_inflow_params(Z[j], inputs, u_ref, alpha, theta_deg)
        uin = inflow(p.nz, u_ref, xi, al, H, th) if z0 is None else inflow_log(p.nz, u_ref, xi, z0, H, th)
        f = init_equilibrium(p, flags)
        run(p, flags, uin, f, 0, n_warm)
        t = n_warm
        for s in range(n_samples):
            if s:
                run(p, flags, uin, f, t, every)
                t += every
            _, u = macros(p, flags, f)
            A[j] += velocity_magnitude(u, flags)
        A[j] /= n_samples
    return A


def unwrap_directions(dir_deg):
    """Directions of a series of targets made continuous: each step from one
    target to the next is taken along the shorter arc, in (-180, 180] read
    as [-180, 180) (a half turn goes clockwise, negative)."""
    d = [float(dir_deg[0])]
    for k in range(1, len(dir_deg)):
        step = (float(dir_deg[k]) - float(dir_deg[k - 1]) + 180.0) % 360.0 - 180.0
        d.append(d[-1] + step)
    return d


def series_at(speed, dir_deg, steps_per_target, interp_steps, m):
    """Wind speed factor s(m) and direction offset delta(m) (degrees) of the
    inflow at time level m under a series of targets (Sec. 2.2: the boundary
    velocity is moved from one target magnitude and direction to the next
    over an interpolation interval; Sec. 2.4 step 1 and Sec. 3: one target
    per hour of measurements).

    Target 0 holds from level 0.  Target k >= 1 takes over at level
    k * steps_per_target: over the following interp_steps levels magnitude
    and direction move linearly from target k - 1 to target k, lam =
    min(o, interp_steps) / interp_steps at offset o into the interval (lam =
    1 at once when interp_steps = 0); then target k holds until the next one
    takes over.  After the last target the series holds it."""
    K = len(speed)
    D = unwrap_directions(dir_deg)
    k = m // steps_per_target
    if k <= 0:
        return float(speed[0]), D[0]
    if k >= K:
        return float(speed[K - 1]), D[K - 1]
    o = m - k * steps_per_target
    lam = 1.0 if interp_steps == 0 else min(o, interp_steps) / interp_steps
    return (float(speed[k - 1]) + lam * (float(speed[k]) - float(speed[k - 1])),
            D[k - 1] + lam * (D[k] - D[k - 1]))


def run_series(p, flags, f, n0, n_steps, inflow_at):
    """Advance f by n_steps from level n0 with an inflow that changes from
    level to level: inflow_at(m) is uin[nz][3] of arrival level m, start-up
    ramp included (the stepping itself is run() with no ramp)."""
    q = params(p.nx, p.ny, p.nz, list(p.bc), p.tau0, p.csmag, 0, tuple(p.force), p.collision)
    for s in range(n_steps):
        m = n0 + s + 1
        run(q, flags, inflow_at(m), f, m - 1, 1)
    return f


def ensemble_series(p, flags, Z, inputs, u_ref, alpha, theta_deg, H, n_steps, series, z0=None,
                    keep_f=False):
    """The ensemble of ensemble() under a time-varying inflow (Sec. 3): at
    node j and arrival level m the profile is that of reference speed
    u_ref * s(m) and direction theta + delta(m) with the node's perturbations
    (speed factor 1 + xi, direction offset) applied on top, times the ramp
    r(m).  series = (speed, dir_deg, steps_per_target, interp_steps).
    Returns u[nq][3][ncell] (and f[nq][19][ncell] with keep_f)."""
    speed, dirs, per, interp = series
    out, fs = [], []
    for j in range(Z.shape[0]):
        xi, al, th = node_inflow_params(Z[j], inputs, u_ref, alpha, theta_deg)

        def inflow_at(m, xi=xi, al=al, th=th):
            s, d = series_at(speed, dirs, per, interp, m)
            if z0 is None:
                prof = inflow(p.nz, u_ref * s, xi, al, H, th + d)
            else:
                prof = inflow_log(p.nz, u_ref * s, xi, z0, H, th + d)
            return ramp(p.ramp_steps, m) * np.asarray(prof)

        f = init_equilibrium(p, flags)
        run_series(p, flags, f, 0, n_steps, inflow_at)
        out.append(macros(p, flags, f)[1])
        if keep_f:
            fs.append(f)
    return (np.array(out), np.array(fs)) if keep_f else np.array(out)


def gpc_quantiles(coef, phi_samples, q):
    """Empirical quantiles of the gPC surrogate at every cell (Sec. 2.4 step
    7: confidence intervals from the expansion coefficients).  The surrogate
    sum_a c_a(x) Phi_a(s_m) is evaluated at M given input samples s_m
    (phi_samples[m][a] = Phi_a(s_m)); the q-quantile is its k-th smallest
    value, k = ceil(q M) in double arithmetic, clamped to [1, M].
    coef [P][ncell] -> [n_q][ncell]."""
    Y = np.asarray(phi_samples, np.float64) @ np.asarray(coef, np.float64)   # [M][ncell]
    Y = np.sort(Y, axis=0)
    M = Y.shape[0]
    out = []
    for qq in q:
        k = min(M, max(1, int(math.ceil(float(qq) * M))))
        out.append(Y[k - 1])
    return np.array(out)
