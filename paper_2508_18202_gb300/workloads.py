"""Named synthetic workloads of the SC-LBM path (sizes, seeds, boundary kinds,
uncertain inputs).  Shared by tests, bench.py and smoke(): this module only
describes inputs; it holds none of the method's arithmetic.

Every workload is synthetic: the paper's real Reutlingen scene and its
measured inflow series are not available, so seeded rectangular buildings
and a power-law inflow stand in for them.
"""
import copy

VEL, OUT, BB, FS, PER = 0, 1, 2, 3, 4
SPEED, ALPHA, ANGLE = 0, 1, 2
GL, CC_SMOLYAK, GH = 0, 1, 2
PROFILE_POWER, PROFILE_LOG = 0, 1
FP64_PLAIN, FP32_SHIFT, BF16_STORE, FP16_STORE = 0, 1, 2, 3
BGK, RR = 0, 1   # collision: BGK, or the recursive regularized form with the third-order equilibrium

URBAN_BC = [VEL, OUT, VEL, VEL, BB, FS]     # inlet, outlet, wind on the sides, ground, sky
CHANNEL_BC = [VEL, OUT, BB, BB, BB, BB]


def tau_for_reynolds(u_ref, length, reynolds):
    """tau0 = 3 nu + 1/2 with nu = u_ref * length / Re (lattice units)."""
    return 0.5 + 3.0 * u_ref * length / reynolds


# D3Q19 channel 48x24x24 with one 8x8x12 cube on the floor; BGK tau = 0.6; one
# uncertain input (relative speed error) on 5 Gauss-Legendre nodes; 300 steps.
CHANNEL_CUBE = dict(
    name="channel_cube_48x24x24_gl5",
    domains=[dict(nx=48, ny=24, nz=24, boxes=[[12, 8, 0, 20, 16, 12]], bc=CHANNEL_BC, quad_level=5)],
    tau0=0.6, c_smag=0.0, u_ref=0.05, alpha=0.25, angle_deg=0.0, H_ref=0.0,
    inputs=[SPEED], lo=[-0.1], hi=[0.1], quad_rule=GL, ramp_steps=0,
    precision=FP64_PLAIN, gpc_degree=4, steps=300, columns=[[28, 12]],
)

# Synthetic urban block, 256x128x64, 24 seeded buildings (footprints 8..24,
# heights 10..40), BGK + Smagorinsky C_S = 0.14 at Re ~ 1e4 on the domain
# height; two inputs (speed error, power-law exponent) on the level-3
# Clenshaw-Curtis Smolyak grid (13 nodes); 5000 steps with a 1000-step ramp.
URBAN_LES = dict(
    name="urban_les_256x128x64_cc3",
    domains=[dict(nx=256, ny=128, nz=64, seed=2025, n_buildings=24, fp=(8, 24), h=(10, 40),
                  bc=URBAN_BC, quad_level=3)],
    tau0=tau_for_reynolds(0.05, 64, 1.0e4), c_smag=0.14, u_ref=0.05, alpha=0.25, angle_deg=0.0,
    H_ref=0.0, inputs=[SPEED, ALPHA], lo=[-0.15, 0.15], hi=[0.15, 0.35], quad_rule=CC_SMOLYAK,
    ramp_steps=1000, precision=FP32_SHIFT, gpc_degree=2, steps=5000, n_columns=4,
)

# Three uneven urban domains advanced together: 128x64x48 (13 nodes),
# 192x96x64 (29 nodes), 320x160x64 (5 nodes).
URBAN_BATCHED = dict(
    name="urban_batched_3domains",
    domains=[
        dict(nx=128, ny=64, nz=48, seed=1, n_buildings=6, fp=(8, 24), h=(10, 40), bc=URBAN_BC, quad_level=3),
        dict(nx=192, ny=96, nz=64, seed=2, n_buildings=14, fp=(8, 24), h=(10, 40), bc=URBAN_BC, quad_level=4),
        dict(nx=320, ny=160, nz=64, seed=3, n_buildings=38, fp=(8, 24), h=(10, 40), bc=URBAN_BC, quad_level=2),
    ],
    tau0=tau_for_reynolds(0.05, 64, 1.0e4), c_smag=0.14, u_ref=0.05, alpha=0.25, angle_deg=0.0,
    H_ref=0.0, inputs=[SPEED, ALPHA], lo=[-0.15, 0.15], hi=[0.15, 0.35], quad_rule=CC_SMOLYAK,
    ramp_steps=1000, precision=FP32_SHIFT, gpc_degree=2, steps=2000, n_columns=4,
)

# Inflow-parameter assimilation: 128x64x48 urban domain, laminar BGK tau = 0.6,
# 2000 steps, misfit of u at 16 seeded probe points against a truth run at
# (u_ref, alpha) = (0.055, 0.28), starting from (0.05, 0.25).
URBAN_ADJOINT = dict(
    name="urban_adjoint_128x64x48",
    domains=[dict(nx=128, ny=64, nz=48, seed=7, n_buildings=6, fp=(8, 24), h=(10, 40), bc=URBAN_BC,
                  quad_level=1)],
    tau0=0.6, c_smag=0.0, u_ref=0.05, alpha=0.25, angle_deg=0.0, H_ref=0.0,
    inputs=[SPEED], lo=[-0.1], hi=[0.1], quad_rule=GL, ramp_steps=0, precision=FP32_SHIFT,
    gpc_degree=-1, steps=2000, n_probes=16, truth=(0.055, 0.28), guess=(0.05, 0.25), gd_iters=20,
)

# Large ensemble: 512x256x128 (16.8M cells), 96 buildings, three inputs
# (speed error, exponent, wind angle in degrees), level-4 Smolyak (69 nodes).
URBAN_LARGE = dict(
    name="urban_large_512x256x128_cc4",
    domains=[dict(nx=512, ny=256, nz=128, seed=11, n_buildings=96, fp=(8, 24), h=(10, 40),
                  bc=URBAN_BC, quad_level=4)],
    tau0=tau_for_reynolds(0.05, 128, 1.0e4), c_smag=0.14, u_ref=0.05, alpha=0.25, angle_deg=0.0,
    H_ref=0.0, inputs=[SPEED, ALPHA, ANGLE], lo=[-0.15, 0.15, -10.0], hi=[0.15, 0.35, 10.0],
    quad_rule=CC_SMOLYAK, ramp_steps=1000, precision=FP32_SHIFT, gpc_degree=2, steps=10000,
    n_columns=4,
)

# The urban LES ensemble with the paper's collision: recursive regularized,
# third-order equilibrium, Smagorinsky C_S = 0.25.
URBAN_LES_RR = dict(URBAN_LES, name="urban_les_rr_256x128x64_cc3", collision=RR, c_smag=0.25)

# The paper's uncertainty setup on the synthetic urban block (Sec. 2.1, Sec. 3,
# Sec. 2.4): Gaussian speed factor zeta_1 ~ N(1, 0.1^2) (speed error mean 0,
# std 0.1) and direction perturbation zeta_2 ~ N(0, 6^2) degrees on the dense
# 11 x 11 Gauss-Hermite rule (121 nodes), logarithmic profile with roughness
# length 0.1 cells, Hermite gPC of total degree 5, the recursive regularized
# collision with C_S = 0.25.
URBAN_GH121 = dict(
    URBAN_LES, name="urban_gh121_256x128x64_rr",
    domains=[dict(URBAN_LES["domains"][0], quad_level=11)],
    inputs=[SPEED, ANGLE], lo=[0.0, 0.0], hi=[0.1, 6.0], quad_rule=GH, collision=RR, c_smag=0.25,
    profile=PROFILE_LOG, z0=0.1, gpc_degree=5, n_columns=4,
)

# The paper's case (Sec. 3 and its table of parameters) on one GPU: a disk of
# radius 270 cells (270 m at dx = 1 m) and height 40 whose mantle carries the
# velocity boundary, two buildings at the centre (stand-ins for the Reutlingen
# pair), bounce-back ground, free-slip sky; Ma = 0.0346 (u = 0.02) and
# Re = 1.8e6 on the domain height; the 121-node Gauss-Hermite rule on the
# speed factor and direction, logarithmic profile z0 = 0.1, recursive
# regularized collision with C_S = 0.25, Hermite gPC of degree 5.
DISK_BC = [VEL, VEL, VEL, VEL, BB, FS]
URBAN_DISK_PAPER = dict(
    name="urban_disk_540x540x40_gh121",
    domains=[dict(nx=540, ny=540, nz=40, boxes=[[240, 248, 0, 266, 288, 26], [272, 236, 0, 300, 270, 33]],
                  bc=DISK_BC, quad_level=11, disk_radius=270.0)],
    tau0=tau_for_reynolds(0.02, 40, 1.8e6), c_smag=0.25, u_ref=0.02, alpha=0.25, angle_deg=0.0, H_ref=0.0,
    inputs=[SPEED, ANGLE], lo=[0.0, 0.0], hi=[0.1, 6.0], quad_rule=GH, collision=RR, profile=PROFILE_LOG,
    z0=0.1, ramp_steps=1000, precision=FP32_SHIFT, gpc_degree=5, steps=2000, n_columns=4,
)

# A small circular domain for parity tests: 48 x 48 x 14, radius 23, two blocks
# near the axis, 3 x 3 Gauss-Hermite nodes (wind from 20 +- 6 degrees), log profile.
DISK_SMALL = dict(
    name="disk_small_48x48x14_gh9",
    domains=[dict(nx=48, ny=48, nz=14, boxes=[[20, 18, 0, 26, 28, 8], [28, 20, 0, 32, 26, 10]], bc=DISK_BC,
                  quad_level=3, disk_radius=23.0)],
    tau0=0.56, c_smag=0.14, u_ref=0.05, alpha=0.25, angle_deg=0.0, H_ref=0.0,
    inputs=[SPEED, ANGLE], lo=[0.0, 20.0], hi=[0.1, 6.0], quad_rule=GH, profile=PROFILE_LOG, z0=0.1,
    ramp_steps=10, precision=FP32_SHIFT, gpc_degree=2, steps=100, n_columns=2,
)

ALL = [CHANNEL_CUBE, URBAN_LES, URBAN_BATCHED, URBAN_ADJOINT, URBAN_LARGE, URBAN_LES_RR, URBAN_GH121,
       URBAN_DISK_PAPER, DISK_SMALL]


def variant(workload, **over):
    """A copy of a workload with fields replaced; `domain_over` (dict or list
    of dicts) replaces fields of the domains."""
    w = copy.deepcopy(workload)
    dom_over = over.pop("domain_over", None)
    w.update(over)
    if dom_over is not None:
        if isinstance(dom_over, dict):
            dom_over = [dom_over] * len(w["domains"])
        for d, o in zip(w["domains"], dom_over):
            d.update(o)
    return w
