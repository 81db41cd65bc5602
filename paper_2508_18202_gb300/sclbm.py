"""Thin Python binding of libsclbm (include/sclbm.h).

Argument marshalling only: every step of the stochastic-collocation LBM path
runs in the library's CUDA kernels.  PyTorch supplies device memory (the
workspace and output tensors) and the CUDA stream.  The functions carry the
C names; each raises ScError on a non-zero status.  If the shared library is
missing it is built in-tree; if it cannot be built or loaded, import of the
calls fails loudly (there is no fallback implementation).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

SC_OK = 0
SC_ERR_ARG, SC_ERR_WORKSPACE, SC_ERR_CUDA = -1, -2, -3
SC_ERR_DIVERGED, SC_ERR_TIMEOUT, SC_ERR_UNSUPPORTED, SC_ERR_STATE = -4, -5, -6, -7
SC_ERR_SCRATCH = -8
SC_NOALLOC_MAX_NODES = 1024
SC_SERIES_MAX_TARGETS = 100000
SC_QUANTILE_MAX_SAMPLES, SC_QUANTILE_MAX_CELLS, SC_QUANTILE_MAX_Q = 8192, 65536, 16
SC_BC_VELOCITY, SC_BC_OUTFLOW, SC_BC_BOUNCE_BACK, SC_BC_FREE_SLIP, SC_BC_PERIODIC = 0, 1, 2, 3, 4
SC_IN_SPEED_REL, SC_IN_ALPHA, SC_IN_ANGLE_DEG = 0, 1, 2
SC_Q_GL, SC_Q_CC_SMOLYAK, SC_Q_GH = 0, 1, 2
SC_PROFILE_POWER, SC_PROFILE_LOG = 0, 1
SC_P_FP64_PLAIN, SC_P_FP32_SHIFT, SC_P_BF16_STORE, SC_P_FP16_STORE = 0, 1, 2, 3
SC_EXEC_LAUNCH, SC_EXEC_GRAPH, SC_EXEC_PERSISTENT = 0, 1, 2
SC_COLL_BGK, SC_COLL_RR = 0, 1

_NAMES = {SC_ERR_ARG: "SC_ERR_ARG", SC_ERR_WORKSPACE: "SC_ERR_WORKSPACE", SC_ERR_CUDA: "SC_ERR_CUDA",
          SC_ERR_DIVERGED: "SC_ERR_DIVERGED", SC_ERR_TIMEOUT: "SC_ERR_TIMEOUT",
          SC_ERR_UNSUPPORTED: "SC_ERR_UNSUPPORTED", SC_ERR_STATE: "SC_ERR_STATE",
          SC_ERR_SCRATCH: "SC_ERR_SCRATCH"}


class ScError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__("%s returned %s%s" % (where, _NAMES.get(code, code),
                                                (": " + detail) if detail else ""))


class sc_domain_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("geom_seed", C.c_uint64),
                ("n_buildings", C.c_int), ("fp_min", C.c_int), ("fp_max", C.c_int),
                ("h_min", C.c_int), ("h_max", C.c_int), ("boxes", C.POINTER(C.c_int32)),
                ("n_boxes", C.c_int), ("bc", C.c_int * 6), ("quad_level", C.c_int),
                ("disk_radius", C.c_double)]


class sc_lbm_config(C.Structure):
    _fields_ = [("n_domains", C.c_int), ("domains", C.POINTER(sc_domain_desc)),
                ("tau0", C.c_double), ("c_smag", C.c_double), ("u_ref", C.c_double),
                ("alpha", C.c_double), ("angle_deg", C.c_double), ("H_ref", C.c_double),
                ("n_inputs", C.c_int), ("inputs", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("quad_rule", C.c_int), ("ramp_steps", C.c_int),
                ("precision", C.c_int), ("gpc_degree", C.c_int), ("collision", C.c_int),
                ("profile", C.c_int), ("z0", C.c_double), ("time_average", C.c_int),
                ("node_begin", C.c_int), ("node_count", C.c_int)]


class sc_lbm_tuning(C.Structure):
    _fields_ = [("block_x", C.c_int), ("block_y", C.c_int), ("slab_z", C.c_int),
                ("tile_order", C.c_int), ("exec_mode", C.c_int), ("graph_steps", C.c_int),
                ("variant", C.c_int)]


# Every exported symbol of include/sclbm.h with its ctypes signature.
_H = C.c_void_p
_P = C.c_void_p
SIGNATURES = {
    "sc_lbm_workspace_size": (C.c_int, [C.POINTER(sc_lbm_config), C.POINTER(C.c_size_t)]),
    "sc_lbm_quadrature": (C.c_int, [C.POINTER(sc_lbm_config), C.c_int, C.POINTER(C.c_int), _P, _P,
                                    C.c_int]),
    "sc_lbm_geometry": (C.c_int, [C.POINTER(sc_lbm_config), C.c_int, _P]),
    "sc_lbm_probe_columns": (C.c_int, [C.POINTER(sc_lbm_config), C.c_int, C.c_int, _P]),
    "sc_lbm_probe_points": (C.c_int, [C.POINTER(sc_lbm_config), C.c_int, C.c_int, _P]),
    "sc_lbm_init": (C.c_int, [C.POINTER(sc_lbm_config), _P, C.c_size_t, _P, _P, C.POINTER(_H)]),
    "sc_lbm_reset": (C.c_int, [_H]),
    "sc_lbm_step": (C.c_int, [_H, C.c_int]),
    "sc_lbm_moments": (C.c_int, [_H, C.c_int, _P, _P, _P, C.c_int, _P, _P, _P, C.c_int]),
    "sc_lbm_velocity": (C.c_int, [_H, C.c_int, C.c_int, _P]),
    "sc_lbm_moment_sums": (C.c_int, [_H, C.c_int, _P, _P, _P, C.c_int]),
    "sc_lbm_weight_sum": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double)]),
    "sc_lbm_rule_weight_sum": (C.c_int, [C.POINTER(sc_lbm_config), C.c_int, C.POINTER(C.c_double)]),
    "sc_lbm_moments_from_sums": (C.c_int, [_H, C.c_int, _P, _P, C.c_double, _P, _P]),
    "sc_lbm_average_reset": (C.c_int, [_H]),
    "sc_lbm_average_add": (C.c_int, [_H]),
    "sc_lbm_average_samples": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "sc_lbm_average_moments": (C.c_int, [_H, C.c_int, _P, _P, _P, C.c_int, _P, _P, _P, C.c_int]),
    "sc_lbm_average_field": (C.c_int, [_H, C.c_int, C.c_int, _P]),
    "sc_lbm_qcriterion": (C.c_int, [_H, C.c_int, _P, _P]),
    "sc_lbm_gpc_quantiles": (C.c_int, [_H, C.c_int, _P, C.c_int, _P, C.c_int, _P, C.c_int, _P, _P]),
    "sc_lbm_populations": (C.c_int, [_H, C.c_int, C.c_int, _P]),
    "sc_lbm_autotune": (C.c_int, [_H, C.c_char_p]),
    "sc_lbm_set_tuning": (C.c_int, [_H, C.POINTER(sc_lbm_tuning)]),
    "sc_lbm_get_tuning": (C.c_int, [_H, C.POINTER(sc_lbm_tuning)]),
    "sc_lbm_counters": (C.c_int, [_H, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "sc_lbm_sync": (C.c_int, [_H]),
    "sc_lbm_check": (C.c_int, [_H, C.POINTER(C.c_longlong)]),
    "sc_lbm_debug_barrier": (C.c_int, [_H, C.c_int, C.c_longlong]),
    "sc_lbm_state_size": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "sc_lbm_save": (C.c_int, [_H, _P, C.c_size_t]),
    "sc_lbm_load": (C.c_int, [_H, _P, C.c_size_t]),
    "sc_lbm_set_inflow": (C.c_int, [_H, C.c_double, C.c_double, C.c_double]),
    "sc_lbm_set_inflow_series": (C.c_int, [_H, C.c_int, _P, _P, C.c_longlong, C.c_longlong]),
    "sc_lbm_inflow_factor": (C.c_int, [C.c_int, C.c_int, _P, _P, C.c_longlong, C.c_longlong, C.c_longlong,
                                       _P]),
    "sc_lbm_inflow_next_change": (C.c_int, [C.c_int, C.c_int, _P, _P, C.c_longlong, C.c_longlong,
                                            C.c_longlong, C.POINTER(C.c_longlong)]),
    "sc_lbm_adjoint_workspace_size": (C.c_int, [_H, C.c_int, C.c_int, C.c_int, C.c_int,
                                                C.POINTER(C.c_size_t)]),
    "sc_lbm_adjoint": (C.c_int, [_H, C.c_int, C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, _P, C.c_size_t,
                                 C.POINTER(C.c_double), _P, _P]),
    "sc_lbm_last_error": (C.c_char_p, [_H]),
    "sc_lbm_destroy": (C.c_int, [_H]),
    "sc_lbm_quad_moments_noalloc": (C.c_int, [_P, C.c_int, C.c_longlong, _P, _P, _P, _P, _P, C.c_char_p,
                                              C.c_size_t]),
}

_lib = None


def lib():
    """Load libsclbm (building it in-tree first if it is absent)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _call(name, *args, handle=None):
    rc = getattr(lib(), name)(*args)
    if rc != SC_OK:
        detail = ""
        if handle:
            msg = lib().sc_lbm_last_error(handle)
            detail = msg.decode() if msg else ""
        raise ScError(rc, name, detail)
    return rc


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# ------------------------------------------------------------------ config
class Config:
    """Owns an sc_lbm_config and the arrays it points to."""

    def __init__(self, domains, tau0, c_smag, u_ref, alpha, inputs, lo, hi, quad_rule,
                 precision, ramp_steps=0, angle_deg=0.0, H_ref=0.0, gpc_degree=-1, collision=SC_COLL_BGK,
                 profile=SC_PROFILE_POWER, z0=0.1, time_average=0, node_begin=0, node_count=0):
        self._doms = (sc_domain_desc * len(domains))()
        self._boxes = []
        for k, d in enumerate(domains):
            D = self._doms[k]
            D.nx, D.ny, D.nz = d["nx"], d["ny"], d["nz"]
            D.geom_seed = d.get("seed", 0)
            D.n_buildings = d.get("n_buildings", 0)
            D.fp_min, D.fp_max = d.get("fp", (1, 1))
            D.h_min, D.h_max = d.get("h", (1, 1))
            boxes = d.get("boxes")
            if boxes:
                arr = np.ascontiguousarray(np.asarray(boxes, np.int32).reshape(-1))
                self._boxes.append(arr)
                D.boxes = arr.ctypes.data_as(C.POINTER(C.c_int32))
                D.n_boxes = arr.size // 6
            for f in range(6):
                D.bc[f] = int(d["bc"][f])
            D.quad_level = d["quad_level"]
            D.disk_radius = float(d.get("disk_radius", 0.0))
        c = sc_lbm_config()
        c.n_domains = len(domains)
        c.domains = C.cast(self._doms, C.POINTER(sc_domain_desc))
        c.tau0, c.c_smag, c.u_ref, c.alpha = tau0, c_smag, u_ref, alpha
        c.angle_deg, c.H_ref = angle_deg, H_ref
        c.n_inputs = len(inputs)
        for k in range(len(inputs)):
            c.inputs[k], c.lo[k], c.hi[k] = inputs[k], lo[k], hi[k]
        c.quad_rule, c.ramp_steps, c.precision, c.gpc_degree = quad_rule, ramp_steps, precision, gpc_degree
        c.collision = collision
        c.profile, c.z0 = profile, z0
        c.time_average = time_average
        c.node_begin, c.node_count = node_begin, node_count
        self.c = c
        self.domains = [dict(d) for d in domains]

    @property
    def ref(self):
        return C.byref(self.c)


# ------------------------------------------------------------------ host-only calls
def sc_lbm_workspace_size(cfg):
    n = C.c_size_t(0)
    _call("sc_lbm_workspace_size", cfg.ref, C.byref(n))
    return n.value


def sc_lbm_quadrature(cfg, domain):
    n = C.c_int(0)
    _call("sc_lbm_quadrature", cfg.ref, domain, C.byref(n), None, None, 0)
    Z = np.zeros((n.value, cfg.c.n_inputs))
    w = np.zeros(n.value)
    _call("sc_lbm_quadrature", cfg.ref, domain, C.byref(n), Z.ctypes.data, w.ctypes.data, n.value)
    return Z, w


def sc_lbm_geometry(cfg, domain):
    d = cfg.domains[domain]
    flags = np.zeros(d["nx"] * d["ny"] * d["nz"], np.uint8)
    _call("sc_lbm_geometry", cfg.ref, domain, flags.ctypes.data)
    return flags


def sc_lbm_probe_columns(cfg, domain, n):
    xy = np.zeros((n, 2), np.int32)
    _call("sc_lbm_probe_columns", cfg.ref, domain, n, xy.ctypes.data)
    return xy


def sc_lbm_probe_points(cfg, domain, n):
    xyz = np.zeros((n, 3), np.int32)
    _call("sc_lbm_probe_points", cfg.ref, domain, n, xyz.ctypes.data)
    return xyz


# ------------------------------------------------------------------ device calls
def sc_lbm_init(cfg, ws_ptr, nbytes, stream_ptr, flags_host=None):
    h = C.c_void_p()
    keep = None
    fh = None
    if flags_host is not None:
        arrs = [None if f is None else np.ascontiguousarray(f, np.uint8) for f in flags_host]
        keep = arrs
        fh = (C.c_void_p * len(arrs))(*[None if a is None else a.ctypes.data for a in arrs])
    _call("sc_lbm_init", cfg.ref, C.c_void_p(ws_ptr), nbytes, C.c_void_p(stream_ptr), fh, C.byref(h))
    del keep
    return h


def sc_lbm_reset(h):
    _call("sc_lbm_reset", h, handle=h)


def sc_lbm_step(h, n):
    _call("sc_lbm_step", h, int(n), handle=h)


def sc_lbm_moments(h, domain, mean, std, probes=None, prof=None, prof_nodes=None, coef=None,
                   out_host=False):
    n_p = 0
    pp = None
    if probes is not None:
        probes = np.ascontiguousarray(np.asarray(probes, np.int32).reshape(-1, 2))
        n_p = probes.shape[0]
        pp = probes.ctypes.data
    _call("sc_lbm_moments", h, domain, _ptr(mean), _ptr(std), pp, n_p, _ptr(prof), _ptr(prof_nodes),
          _ptr(coef), 1 if out_host else 0, handle=h)


def sc_lbm_velocity(h, domain, node, u):
    _call("sc_lbm_velocity", h, domain, node, _ptr(u), handle=h)


def sc_lbm_moment_sums(h, domain, s1, s2, gpc_sums=None, accumulate=False):
    _call("sc_lbm_moment_sums", h, domain, _ptr(s1), _ptr(s2), _ptr(gpc_sums), int(bool(accumulate)),
          handle=h)


def sc_lbm_weight_sum(h, domain):
    w = C.c_double(0.0)
    _call("sc_lbm_weight_sum", h, domain, C.byref(w), handle=h)
    return w.value


def sc_lbm_rule_weight_sum(cfg, domain):
    w = C.c_double(0.0)
    _call("sc_lbm_rule_weight_sum", cfg.ref, domain, C.byref(w))
    return w.value


def sc_lbm_moments_from_sums(h, domain, s1, s2, wsum, mean, std):
    _call("sc_lbm_moments_from_sums", h, domain, _ptr(s1), _ptr(s2), float(wsum), _ptr(mean), _ptr(std),
          handle=h)


def shard_nodes(n_nodes, world, rank):
    """Contiguous, balanced node range (begin, count) of `rank` among `world`
    shards of an n_nodes rule (the first n_nodes % world shards take one
    more node)."""
    if not (0 <= rank < world) or n_nodes < world:
        raise ValueError("need 0 <= rank < world <= n_nodes")
    base, extra = divmod(n_nodes, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def run_in_waves(workload, n_steps, nodes_per_wave, domain=0, gpc=False, prepare=None):
    """An ensemble whose nodes do not fit on the device at once, run in waves:
    the collocation nodes are taken nodes_per_wave at a time, each wave a
    handle over its node range (the runs are independent, Sec. 2.4 step 5)
    that is stepped n_steps and reduces its nodes into the same FP64 sum
    arrays (sc_lbm_moment_sums: the first wave overwrites, the later ones
    accumulate, so the sums carry the bits of one reduction over the whole
    rule); each handle is released before the next is made, so one wave's
    workspace is held at a time.  The last wave's handle finishes mean and
    std with the rule's weight sum.  Single-domain workloads.  prepare(ens),
    if given, is called on every wave's ensemble before it steps (for
    instance to set an inflow series).  Returns dict(mean, std, coef (None
    without gpc), waves)."""
    import torch
    from math import comb
    if len(workload["domains"]) != 1:
        raise ValueError("waves run single-domain workloads")
    if nodes_per_wave < 1:
        raise ValueError("nodes_per_wave must be >= 1")
    cfg = make_config(workload)
    _, a_full = sc_lbm_quadrature(cfg, 0)
    n_total = len(a_full)
    wsum = sc_lbm_rule_weight_sum(cfg, domain)
    ranges = [(b, min(nodes_per_wave, n_total - b)) for b in range(0, n_total, nodes_per_wave)]
    s1 = s2 = gs = mean = std = None
    for i, (b, c) in enumerate(ranges):
        ens = Ensemble(make_config(workload, node_begin=b, node_count=c))
        try:
            if prepare is not None:
                prepare(ens)
            ens.step(n_steps)
            if s1 is None:
                n = ens.ncell(domain)
                s1, s2 = ens._out(n), ens._out(n)
                if gpc:
                    gs = ens._out(comb(ens.cfg.c.gpc_degree + ens.cfg.c.n_inputs, ens.cfg.c.n_inputs), n)
            else:
                # the sums were written on the previous wave's stream
                ens.stream.wait_stream(torch.cuda.current_stream(ens.device))
            sc_lbm_moment_sums(ens.h, domain, s1, s2, gs, accumulate=i > 0)
            if i == len(ranges) - 1:
                mean, std = ens._out(s1.shape[0]), ens._out(s1.shape[0])
                sc_lbm_moments_from_sums(ens.h, domain, s1, s2, wsum, mean, std)
            ens._hand_over(s1, s2, gs, mean, std)
            ens.sync()
        finally:
            ens.close()
    return dict(mean=mean, std=std, coef=gs, waves=len(ranges))


def sc_lbm_average_reset(h):
    _call("sc_lbm_average_reset", h, handle=h)


def sc_lbm_average_add(h):
    _call("sc_lbm_average_add", h, handle=h)


def sc_lbm_average_samples(h):
    n = C.c_longlong(0)
    _call("sc_lbm_average_samples", h, C.byref(n), handle=h)
    return n.value


def sc_lbm_average_moments(h, domain, mean, std, probes=None, prof=None, prof_nodes=None, coef=None,
                           out_host=False):
    n_p = 0
    pp = None
    if probes is not None:
        probes = np.ascontiguousarray(np.asarray(probes, np.int32).reshape(-1, 2))
        n_p = probes.shape[0]
        pp = probes.ctypes.data
    _call("sc_lbm_average_moments", h, domain, _ptr(mean), _ptr(std), pp, n_p, _ptr(prof), _ptr(prof_nodes),
          _ptr(coef), 1 if out_host else 0, handle=h)


def sc_lbm_average_field(h, domain, node, q):
    _call("sc_lbm_average_field", h, domain, node, _ptr(q), handle=h)


def sc_lbm_qcriterion(h, domain, u, q):
    _call("sc_lbm_qcriterion", h, domain, _ptr(u), _ptr(q), handle=h)


def sc_lbm_populations(h, domain, node, f):
    _call("sc_lbm_populations", h, domain, node, _ptr(f), handle=h)


def sc_lbm_autotune(h, cache_path=None):
    _call("sc_lbm_autotune", h, cache_path.encode() if cache_path else None, handle=h)


def sc_lbm_set_tuning(h, block_x, block_y, slab_z, tile_order=0, exec_mode=SC_EXEC_LAUNCH,
                      graph_steps=50, variant=0):
    t = sc_lbm_tuning(block_x, block_y, slab_z, tile_order, exec_mode, graph_steps, variant)
    _call("sc_lbm_set_tuning", h, C.byref(t), handle=h)


def sc_lbm_get_tuning(h):
    t = sc_lbm_tuning()
    _call("sc_lbm_get_tuning", h, C.byref(t), handle=h)
    return dict(block_x=t.block_x, block_y=t.block_y, slab_z=t.slab_z, tile_order=t.tile_order,
                exec_mode=t.exec_mode, graph_steps=t.graph_steps, variant=t.variant)


def sc_lbm_counters(h):
    s, k = C.c_longlong(0), C.c_longlong(0)
    _call("sc_lbm_counters", h, C.byref(s), C.byref(k), handle=h)
    return s.value, k.value


def sc_lbm_sync(h):
    _call("sc_lbm_sync", h, handle=h)


def sc_lbm_check(h):
    n = C.c_longlong(0)
    rc = lib().sc_lbm_check(h, C.byref(n))
    return rc, n.value


def sc_lbm_debug_barrier(h, never_arrive, spin_limit):
    _call("sc_lbm_debug_barrier", h, int(never_arrive), int(spin_limit), handle=h)


def sc_lbm_state_size(h):
    n = C.c_size_t(0)
    _call("sc_lbm_state_size", h, C.byref(n), handle=h)
    return n.value


def sc_lbm_save(h, buf):
    _call("sc_lbm_save", h, _ptr(buf), buf.nbytes if hasattr(buf, "nbytes") else len(buf), handle=h)


def sc_lbm_load(h, buf):
    _call("sc_lbm_load", h, _ptr(buf), buf.nbytes, handle=h)


def sc_lbm_set_inflow(h, u_ref, alpha, angle_deg=0.0):
    _call("sc_lbm_set_inflow", h, float(u_ref), float(alpha), float(angle_deg), handle=h)


def sc_lbm_gpc_quantiles(h, domain, coef, cells, samples, q, out):
    """q-quantiles of the gPC surrogate at the given cells: coef device
    double [P][ncell], samples host [M][n_inputs] in the basis's standard
    coordinates, out device double [n_q][n_cells]."""
    cells = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1))
    samples = np.ascontiguousarray(np.asarray(samples, np.float64))
    n_s = samples.shape[0]
    q = np.ascontiguousarray(np.asarray(q, np.float64).reshape(-1))
    _call("sc_lbm_gpc_quantiles", h, domain, _ptr(coef), cells.size, cells.ctypes.data if cells.size else None,
          n_s, samples.ctypes.data, q.size, q.ctypes.data, _ptr(out), handle=h)


def _series_arrays(speed, dir_deg):
    sp = np.ascontiguousarray(speed, np.float64).reshape(-1)
    dd = np.ascontiguousarray(dir_deg, np.float64).reshape(-1)
    if sp.shape != dd.shape:
        raise ValueError("speed and dir_deg need one entry per target")
    return sp, dd


def sc_lbm_set_inflow_series(h, speed, dir_deg, steps_per_target, interp_steps):
    """Hourly targets of the inflow: speed factors relative to u_ref and
    direction offsets in degrees (empty arrays: steady inflow again)."""
    sp, dd = _series_arrays(speed, dir_deg)
    _call("sc_lbm_set_inflow_series", h, int(sp.size), _ptr(sp) if sp.size else None,
          _ptr(dd) if dd.size else None, int(steps_per_target), int(interp_steps), handle=h)


def sc_lbm_inflow_factor(ramp_steps, speed, dir_deg, steps_per_target, interp_steps, level):
    """(a, b, m) of time level `level` (host only)."""
    sp, dd = _series_arrays(speed, dir_deg)
    out = np.zeros(3)
    _call("sc_lbm_inflow_factor", int(ramp_steps), int(sp.size), _ptr(sp) if sp.size else None,
          _ptr(dd) if dd.size else None, int(steps_per_target), int(interp_steps), int(level), _ptr(out))
    return out


def sc_lbm_inflow_next_change(ramp_steps, speed, dir_deg, steps_per_target, interp_steps, level):
    """First level after `level` at which the inflow factor may change (host only)."""
    sp, dd = _series_arrays(speed, dir_deg)
    out = C.c_longlong(0)
    _call("sc_lbm_inflow_next_change", int(ramp_steps), int(sp.size), _ptr(sp) if sp.size else None,
          _ptr(dd) if dd.size else None, int(steps_per_target), int(interp_steps), int(level), C.byref(out))
    return out.value


def sc_lbm_adjoint_workspace_size(h, domain, n_steps, n_snapshots, n_probes):
    n = C.c_size_t(0)
    _call("sc_lbm_adjoint_workspace_size", h, domain, n_steps, n_snapshots, n_probes, C.byref(n), handle=h)
    return n.value


def sc_lbm_adjoint(h, domain, node, probes, u_target, n_steps, n_snapshots, ws_ptr, ws_bytes):
    """Returns (loss, grad[2], u_probe[n][3])."""
    probes = np.ascontiguousarray(np.asarray(probes, np.int32).reshape(-1, 3))
    ut = np.ascontiguousarray(np.asarray(u_target, np.float64).reshape(-1, 3))
    loss = C.c_double(0.0)
    grad = np.zeros(2)
    up = np.zeros((probes.shape[0], 3))
    _call("sc_lbm_adjoint", h, domain, node, probes.ctypes.data, probes.shape[0], ut.ctypes.data,
          int(n_steps), int(n_snapshots), C.c_void_p(ws_ptr), ws_bytes, C.byref(loss), grad.ctypes.data,
          up.ctypes.data, handle=h)
    return loss.value, grad, up


def sc_lbm_last_error(h):
    m = lib().sc_lbm_last_error(h)
    return m.decode() if m else ""


def sc_lbm_destroy(h):
    _call("sc_lbm_destroy", h)


def sc_lbm_quad_moments_noalloc(field, weights, mean, std, nonfinite=None, stream=0):
    """Quadrature mean / std of a caller-held per-node field without device
    allocation (no handle, no workspace; scratch is the library's fixed
    device array).  field: device double [n_nodes][n_cells]; weights: host
    doubles; mean, std: device double [n_cells]; nonfinite: device uint64[1]
    or None; stream: raw CUDA stream handle (0 = legacy default stream)."""
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    n_nodes = int(w.shape[0])
    n_cells = int(field.shape[-1]) if n_nodes else 0
    err = C.create_string_buffer(256)
    rc = lib().sc_lbm_quad_moments_noalloc(_ptr(field), n_nodes, n_cells, w.ctypes.data, _ptr(mean),
                                          _ptr(std), _ptr(nonfinite), stream, err, len(err))
    if rc != SC_OK:
        raise ScError(rc, "sc_lbm_quad_moments_noalloc", err.value.decode())


# ------------------------------------------------------------------ convenience
class Ensemble:
    """One library handle with a torch-allocated workspace and its own stream.

    All outputs are torch tensors allocated on the handle's stream; the
    caller's current stream is made to wait for them before they are
    returned."""

    def __init__(self, cfg, flags_host=None, device="cuda"):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(device=self.device)
        self.nbytes = sc_lbm_workspace_size(cfg)
        with torch.cuda.stream(self.stream):
            self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.h = sc_lbm_init(cfg, self.ws.data_ptr(), self.nbytes, self.stream.cuda_stream, flags_host)
        # nodes this handle runs (its node range of every domain's rule)
        full = [sc_lbm_quadrature(cfg, d)[1].size for d in range(cfg.c.n_domains)]
        b, c = cfg.c.node_begin, cfg.c.node_count
        self.n_nodes = [c if c > 0 else n - b for n in full]

    def _out(self, *shape, dtype=None):
        with self.torch.cuda.stream(self.stream):
            return self.torch.empty(*shape, dtype=dtype or self.torch.float64, device=self.device)

    def _hand_over(self, *tensors):
        """Make the caller's current stream wait for the handle's stream and
        mark the outputs as used there, so that the caching allocator does
        not hand their memory to a later output of the handle's stream while
        the caller's stream still reads them."""
        cur = self.torch.cuda.current_stream(self.device)
        cur.wait_stream(self.stream)
        for t in tensors:
            if t is not None:
                t.record_stream(cur)

    def ncell(self, d):
        D = self.cfg.domains[d]
        return D["nx"] * D["ny"] * D["nz"]

    def step(self, n):
        sc_lbm_step(self.h, n)

    def set_inflow_series(self, speed, dir_deg, steps_per_target, interp_steps):
        sc_lbm_set_inflow_series(self.h, speed, dir_deg, steps_per_target, interp_steps)

    def moments(self, domain=0, probes=None, nodes_profiles=False, gpc=False, _reader=None):
        t = self.torch
        n = self.ncell(domain)
        nz = self.cfg.domains[domain]["nz"]
        mean, std = self._out(n), self._out(n)
        prof = pn = coef = None
        if probes is not None:
            probes = np.asarray(probes, np.int32).reshape(-1, 2)
            prof = self._out(probes.shape[0], nz, 4)
            if nodes_profiles:
                pn = self._out(probes.shape[0], self.n_nodes[domain], nz, dtype=t.float32)
        if gpc:
            from math import comb
            P = comb(self.cfg.c.gpc_degree + self.cfg.c.n_inputs, self.cfg.c.n_inputs)
            coef = self._out(P, n)
        (_reader or sc_lbm_moments)(self.h, domain, mean, std, probes, prof, pn, coef)
        self._hand_over(mean, std, prof, pn, coef)
        return dict(mean=mean, std=std, prof=prof, prof_nodes=pn, coef=coef)

    def velocity(self, domain, node):
        u = self._out(3, self.ncell(domain), dtype=self.torch.float32)
        sc_lbm_velocity(self.h, domain, node, u)
        self._hand_over(u)
        return u

    def sharded_moments(self, domain=0, group=None, gpc=False):
        """Quadrature mean / std (and gPC coefficients) of an ensemble whose
        nodes are sharded over the processes of a torch.distributed group:
        this handle's moment sums and weight sum are all-reduced (sum), then
        finished by the library."""
        t = self.torch
        import torch.distributed as dist
        n = self.ncell(domain)
        s1, s2 = self._out(n), self._out(n)
        gs = None
        if gpc:
            from math import comb
            gs = self._out(comb(self.cfg.c.gpc_degree + self.cfg.c.n_inputs, self.cfg.c.n_inputs), n)
        sc_lbm_moment_sums(self.h, domain, s1, s2, gs)
        self._hand_over(s1, s2, gs)
        w = t.tensor([sc_lbm_weight_sum(self.h, domain)], dtype=t.float64, device=s1.device)
        for x in (s1, s2, gs, w):
            if x is not None:
                dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
        mean, std = self._out(n), self._out(n)
        self.stream.wait_stream(t.cuda.current_stream(self.device))
        sc_lbm_moments_from_sums(self.h, domain, s1, s2, float(w.item()), mean, std)
        self._hand_over(mean, std)
        return dict(mean=mean, std=std, coef=gs)

    def average_moments(self, domain=0, probes=None, nodes_profiles=False, gpc=False):
        """moments() of the time-averaged |u| fields (configurations with
        time_average = 1)."""
        return self.moments(domain, probes, nodes_profiles, gpc, _reader=sc_lbm_average_moments)

    def average_field(self, domain, node):
        q = self._out(self.ncell(domain))
        sc_lbm_average_field(self.h, domain, node, q)
        self._hand_over(q)
        return q

    def gpc_quantiles(self, domain, coef, cells, samples, q):
        """Quantiles [n_q][n_cells] of the gPC surrogate of coefficients coef
        (from moments(..., gpc=True)["coef"]) at the M input samples
        (standard coordinates, [M][n_inputs])."""
        d = self.cfg.c.n_inputs
        samples = np.asarray(samples, np.float64).reshape(-1, d)
        out = self._out(len(q), len(cells))
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        sc_lbm_gpc_quantiles(self.h, domain, coef, cells, samples, q, out)
        self._hand_over(out)
        return out

    def qcriterion(self, domain, u):
        """Q-criterion of a velocity field u[3][ncell] (device float)."""
        q = self._out(self.ncell(domain), dtype=self.torch.float32)
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        sc_lbm_qcriterion(self.h, domain, u, q)
        self._hand_over(q)
        return q

    def populations(self, domain, node):
        f = self._out(19, self.ncell(domain))
        sc_lbm_populations(self.h, domain, node, f)
        self._hand_over(f)
        return f

    def sync(self):
        sc_lbm_sync(self.h)

    def close(self):
        if self.h:
            sc_lbm_destroy(self.h)
            self.h = None
        # sc_lbm_destroy has waited for the handle's stream, so the library is
        # done with the workspace: release it now, not when this object goes,
        # so that the next ensemble (the next wave of run_in_waves) can have
        # the memory while a reference to this one is still alive
        self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_config(workload, **over):
    """sc_lbm_config for a workload dict (see workloads.py); keyword arguments
    replace top-level fields (e.g. precision=SC_P_BF16_STORE)."""
    w = dict(workload)
    w.update(over)
    return Config(w["domains"], w["tau0"], w["c_smag"], w["u_ref"], w["alpha"], w["inputs"], w["lo"],
                  w["hi"], w["quad_rule"], w["precision"], ramp_steps=w["ramp_steps"],
                  angle_deg=w.get("angle_deg", 0.0), H_ref=w.get("H_ref", 0.0),
                  gpc_degree=w.get("gpc_degree", -1), collision=w.get("collision", SC_COLL_BGK),
                  profile=w.get("profile", SC_PROFILE_POWER), z0=w.get("z0", 0.1),
                  time_average=w.get("time_average", 0), node_begin=w.get("node_begin", 0),
                  node_count=w.get("node_count", 0))


# ------------------------------------------------------------------ assimilation
class Assimilation:
    """Probe-misfit loss of one collocation node and its adjoint gradient with
    respect to the inflow parameters (u_ref, alpha)."""

    def __init__(self, ens, probes, u_target, n_steps, n_snapshots=0, domain=0, node=0):
        import torch
        self.ens, self.domain, self.node = ens, domain, node
        self.probes = np.asarray(probes, np.int32).reshape(-1, 3)
        self.u_target = np.asarray(u_target, np.float64).reshape(-1, 3)
        self.n_steps, self.n_snapshots = int(n_steps), int(n_snapshots)
        self.nbytes = sc_lbm_adjoint_workspace_size(ens.h, domain, self.n_steps, self.n_snapshots,
                                                    self.probes.shape[0])
        with torch.cuda.stream(ens.stream):
            self.ws = torch.empty(self.nbytes, dtype=torch.uint8, device=ens.device)

    def loss_and_grad(self, u_ref, alpha):
        c = self.ens.cfg.c
        sc_lbm_set_inflow(self.ens.h, u_ref, alpha, c.angle_deg)
        return sc_lbm_adjoint(self.ens.h, self.domain, self.node, self.probes, self.u_target, self.n_steps,
                              self.n_snapshots, self.ws.data_ptr(), self.nbytes)


def _inflow_loss_function():
    import torch

    class InflowLoss(torch.autograd.Function):
        """J(theta) for theta = (u_ref, alpha); the backward pass returns the
        adjoint gradient computed alongside the forward run."""

        @staticmethod
        def forward(ctx, theta, assim):
            t = theta.detach().cpu().double().numpy()
            loss, grad, _ = assim.loss_and_grad(float(t[0]), float(t[1]))
            ctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(loss, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad, None

    return InflowLoss


def InflowLoss():
    """torch.autograd.Function class computing the assimilation loss."""
    return _inflow_loss_function()


def assimilate(assim, theta0, iters=20, scale=(0.05, 0.25), c1=1e-4, step0=0.1):
    """Gradient descent on the inflow parameters scaled to O(1): the trial step
    length is the Barzilai-Borwein one (s.s / s.y), accepted under a
    backtracking Armijo condition, so the loss decreases monotonically.
    Returns the history of (theta, J)."""
    scale = np.asarray(scale, np.float64)
    x = np.asarray(theta0, np.float64) / scale
    J, g, _ = assim.loss_and_grad(*(x * scale))
    gx = g * scale
    hist = [(x * scale, J)]
    t0 = step0 / max(np.linalg.norm(gx), 1e-300)
    for _ in range(iters):
        if not np.any(gx):
            break
        t = t0
        while True:
            xn = x - t * gx
            Jn, gn, _ = assim.loss_and_grad(*(xn * scale))
            if Jn <= J - c1 * t * float(gx @ gx) or t < 1e-14:
                break
            t *= 0.5
        gnx = gn * scale
        s, y = xn - x, gnx - gx
        sy = float(s @ y)
        t0 = float(s @ s) / sy if sy > 0 else 2.0 * t
        x, J, gx = xn, Jn, gnx
        hist.append((x * scale, J))
    return hist
