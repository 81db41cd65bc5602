"""Test helpers: map a workload description onto the oracle's inputs and
compare GPU outputs with oracle outputs."""
import numpy as np


def oracle_domain(O, wl, d=0):
    D = wl["domains"][d]
    p = O.params(D["nx"], D["ny"], D["nz"], D["bc"], wl["tau0"], wl["c_smag"], wl["ramp_steps"],
                 collision=wl.get("collision", 0))
    flags = O.geometry(D["nx"], D["ny"], D["nz"], D.get("seed", 0), D.get("n_buildings", 0),
                       *D.get("fp", (1, 1)), *D.get("h", (1, 1)), boxes=D.get("boxes"),
                       disk_radius=D.get("disk_radius", 0.0))
    return p, flags


def oracle_nodes(O, wl, d=0):
    return O.quadrature(wl["quad_rule"], len(wl["inputs"]), wl["domains"][d]["quad_level"],
                        wl["lo"], wl["hi"])


def oracle_uin(O, wl, d, Zj):
    D = wl["domains"][d]
    xi, al, th = O.node_inflow_params(Zj, wl["inputs"], wl["u_ref"], wl["alpha"], wl.get("angle_deg", 0.0))
    H = wl.get("H_ref", 0.0) or D["nz"]
    return O.inflow(D["nz"], wl["u_ref"], xi, al, H, th)


def oracle_run_node(O, wl, d, j, steps, f=None, n0=0):
    p, flags = oracle_domain(O, wl, d)
    Z, a = oracle_nodes(O, wl, d)
    uin = oracle_uin(O, wl, d, Z[j])
    if f is None:
        f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin, f, n0, steps)
    return p, flags, f


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
