"""Seeded synthetic inputs for the coupled thermal LBM step.

This module holds the input recipe only: parameter sets, boundary specs,
initial density / velocity / temperature fields and a counter-based noise
generator.  It contains none of the method's arithmetic and imports neither
the CUDA binding nor the CPU oracle, so both can be fed identical arrays.

The paper's experiments (Section 4) are setups, not datasets; the shapes
below follow them:

* droplet in open space (Section 4.1): a centred droplet at saturation
  temperature, hotter surrounding vapour, Dirichlet temperature edges;
* droplet on a heated surface (Section 4.2): a sessile droplet centred on a
  bottom wall, tanh initial profile (Eqs. 57-58);
* nucleate boiling (Section 4.3): a liquid pool on a wall with a heater
  segment, vapour layer at the top, buoyancy.
"""
from __future__ import annotations

import os

import numpy as np

PERIODIC, WALL, OPEN = 0, 1, 2
T_PERIODIC, T_DIRICHLET, T_ADIABATIC = 0, 1, 2

# Peng-Robinson constants (Section 2) and the parameter readings used
# throughout: nu = 0.1 and c_v = 5 (the printed pair "5.0, 0.1" read swapped,
# since rho c_v < 1/2 in the vapour makes the weighted streaming unstable),
# w_dot = 2/3, every non-physical relaxation rate 1.0 (Section 4), and the
# Li forcing parameter sigma = 1.25, calibrated on a flat interface against
# the Maxwell coexistence densities (oracle/calibrate_sigma.py).
BASE_PARAMS = dict(
    a=3.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0, sigma=1.25,
    nu=0.1, s0=1.0, s_e=1.0, s_eps=1.0, s_j=1.0, s_q=1.0,
    lambda_=1.0 / 3.0, cv=5.0, w_dot=2.0 / 3.0, vs0=1.0, vs3=1.0, vs4=1.0,
    gravity=0.0, frozen_flow=0, frozen_thermal=0,
)

# T_c of the EOS above: a/b = (0.45724 / 0.0778) R T_c.
TC = 0.0778 * BASE_PARAMS["a"] / (0.45724 * BASE_PARAMS["b"] * BASE_PARAMS["R"])

# Flat-interface coexistence densities (rho_g, rho_l) by Maxwell's equal-area
# construction on the EOS above, keyed by T / T_c.  Written by
# tests/golden/make_coexistence.py, which calls the CPU oracle only; a test
# re-derives them.  They are inputs (initial densities and the interface level
# of the diagnostics), not expected results.
COEXISTENCE = {
    0.80: (0.19712190648103, 7.20385167137751),
    0.86: (0.37967899939970, 6.49894576328788),
    0.90: (0.58009862036263, 5.90789904550754),
    0.95: (1.01316189867770, 4.92815724813840),
}


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood 2014) of (seed, index) -> uint64."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15)
             + (index.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, np.arange(n, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64)
    return lo + (hi - lo) * u * (1.0 / 9007199254740992.0)


def noise(seed: int, shape, amp: float) -> np.ndarray:
    """Additive noise uniform in [-amp, amp), one draw per node."""
    n = int(np.prod(shape))
    return uniform(seed, n, -amp, amp).reshape(shape)


def bc_spec(flow, therm, T_edge=(0.0, 0.0, 0.0, 0.0), theta_deg=90.0,
            heater=(0, 0), T_heater=0.0) -> dict:
    """Boundary spec, edges ordered west, east, south, north."""
    return dict(flow=list(flow), therm=list(therm), T_edge=list(T_edge),
                theta_deg=float(theta_deg), heater_x0=int(heater[0]),
                heater_x1=int(heater[1]), T_heater=float(T_heater))


def periodic_bc() -> dict:
    return bc_spec([PERIODIC] * 4, [T_PERIODIC] * 4)


def tanh_disc(nx, ny, x0, y0, R, w, inside, outside):
    """(inside+outside)/2 - (inside-outside)/2 tanh((|x-x0| - R) / (w/2))
    (Eq. 57); nodes sit at integer coordinates."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 * (inside + outside) - 0.5 * (inside - outside) * np.tanh((d - R) / (0.5 * w))


def tanh_layer(nx, ny, y_if, w, below, above):
    """Flat layer: `below` for y << y_if, `above` for y >> y_if."""
    y = np.mgrid[0:ny, 0:nx][0].astype(np.float64)
    return 0.5 * (below + above) - 0.5 * (below - above) * np.tanh((y - y_if) / (0.5 * w))


class Case:
    """A fully specified simulation input: sizes, params, bc and fields."""

    def __init__(self, name, nx, ny, params, bc, rho, ux, uy, T, steps,
                 rho_l, rho_g, sessile=False):
        self.name, self.nx, self.ny = name, nx, ny
        self.params, self.bc = params, bc
        self.rho, self.ux, self.uy, self.T = rho, ux, uy, T
        self.steps, self.rho_l, self.rho_g, self.sessile = steps, rho_l, rho_g, sessile

    def fields(self):
        return self.rho, self.ux, self.uy, self.T


def params(**over) -> dict:
    p = dict(BASE_PARAMS)
    p.update(over)
    return p


def static_droplet(nx=64, ny=64, R=16.0, w=4.0, Tr=0.86, amp=1e-4, seed=1, steps=1000,
                   p=None) -> Case:
    """Static droplet in a periodic box at uniform T (the 64x64 parity case)."""
    rg, rl = COEXISTENCE[Tr]
    rho = tanh_disc(nx, ny, 0.5 * (nx - 1), 0.5 * (ny - 1), R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    z = np.zeros((ny, nx))
    T = np.full((ny, nx), Tr * TC)
    return Case("static_droplet_%dx%d" % (nx, ny), nx, ny, p or params(), periodic_bc(),
                rho, z, z.copy(), T, steps, rl, rg)


def open_evaporation(nx=256, ny=256, R=40.0, w=4.0, T_sat=0.86, T_edge=0.95, amp=1e-4,
                     seed=2, steps=20000, p=None) -> Case:
    """Droplet evaporating in open space (Section 4.1 shape): droplet at T_sat,
    hotter vapour, Dirichlet T on all four edges, open outflow."""
    rg, rl = COEXISTENCE[T_sat]
    cx, cy = 0.5 * (nx - 1), 0.5 * (ny - 1)
    rho = tanh_disc(nx, ny, cx, cy, R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    T = tanh_disc(nx, ny, cx, cy, R, w, T_sat * TC, T_edge * TC)
    z = np.zeros((ny, nx))
    bc = bc_spec([OPEN] * 4, [T_DIRICHLET] * 4, T_edge=[T_edge * TC] * 4)
    return Case("open_evaporation_%dx%d" % (nx, ny), nx, ny, p or params(), bc,
                rho, z, z.copy(), T, steps, rl, rg)


def d2_droplet(n=200, D0=60.0, w=4.0, T_sat=0.86, T_g=1.0, amp=0.0, seed=2, steps=20000,
               p=None) -> Case:
    """The D^2-law test of Section 4.1 as the paper states it: an n x n box,
    a centred droplet of diameter D0 at T_sat in vapour at T_g, the flow
    populations streamed periodically at the edges and T = T_g held on all
    four edges (halfway anti-bounce-back)."""
    rg, rl = COEXISTENCE[T_sat]
    c0 = 0.5 * (n - 1)
    rho = tanh_disc(n, n, c0, c0, 0.5 * D0, w, rl, rg)
    if amp:
        rho = rho + noise(seed, (n, n), amp)
    T = tanh_disc(n, n, c0, c0, 0.5 * D0, w, T_sat * TC, T_g * TC)
    z = np.zeros((n, n))
    bc = bc_spec([PERIODIC] * 4, [T_DIRICHLET] * 4, T_edge=[T_g * TC] * 4)
    return Case("d2_droplet_%d" % n, n, n, p or params(), bc, rho, z, z.copy(), T, steps, rl, rg)


def heated_surface(nx=400, ny=200, R=50.0, w=5.0, T_sat=0.86, T_wall=0.95, theta=90.0,
                   amp=0.0, seed=3, steps=30000, p=None) -> Case:
    """Sessile droplet on a heated wall (Section 4.2 shape): wall at the
    bottom held at T_wall, open top at T_sat, periodic in x."""
    rg, rl = COEXISTENCE[T_sat]
    rho = tanh_disc(nx, ny, 0.5 * nx, 0.0, R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    T = np.full((ny, nx), T_sat * TC)
    z = np.zeros((ny, nx))
    bc = bc_spec([PERIODIC, PERIODIC, WALL, OPEN],
                 [T_PERIODIC, T_PERIODIC, T_DIRICHLET, T_DIRICHLET],
                 T_edge=[0.0, 0.0, T_wall * TC, T_sat * TC], theta_deg=theta)
    return Case("heated_surface_%dx%d" % (nx, ny), nx, ny, p or params(lambda_=0.08), bc,
                rho, z, z.copy(), T, steps, rl, rg, sessile=True)


def nucleate_boiling(nx=300, ny=600, gravity=2e-5, heater_w=20, T_sat=0.86, T_h=1.1,
                     theta=75.0, amp=1e-3, seed=4, steps=60000, p=None,
                     vapour_layer=True) -> Case:
    """Pool boiling (Section 4.3 shape): liquid pool on a wall with a central
    heater segment, buoyancy (rho-rho_ave)g, open top.  With vapour_layer the
    top sixth starts as vapour (the benchmark configuration's pool); without
    it the enclosure starts filled with saturated liquid, as Section 4.3
    states."""
    rg, rl = COEXISTENCE[T_sat]
    if vapour_layer:
        rho = tanh_layer(nx, ny, 5.0 * ny / 6.0, 4.0, rl, rg)
    else:
        rho = np.full((ny, nx), rl)
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    T = np.full((ny, nx), T_sat * TC)
    z = np.zeros((ny, nx))
    x0 = nx // 2 - heater_w // 2
    bc = bc_spec([PERIODIC, PERIODIC, WALL, OPEN],
                 [T_PERIODIC, T_PERIODIC, T_DIRICHLET, T_DIRICHLET],
                 T_edge=[0.0, 0.0, T_sat * TC, T_sat * TC], theta_deg=theta,
                 heater=(x0, x0 + heater_w), T_heater=T_h * TC)
    return Case("nucleate_boiling_%dx%d_g%g%s" % (nx, ny, gravity, "" if vapour_layer else "_liquid"),
                nx, ny,
                p or params(lambda_=2.0 / 3.0, gravity=gravity), bc, rho, z, z.copy(), T,
                steps, rl, rg)


def sessile_cap(nx=160, ny=80, R=30.0, theta=90.0, w=4.0, Tr=0.86, x0=None, amp=0.0,
                seed=6, top=OPEN, steps=0, p=None) -> Case:
    """Sessile droplet whose initial shape is a circular cap meeting the south
    wall line y = -1/2 at the angle `theta` (inside the liquid): the circle of
    radius R is centred at (x0, -1/2 - R cos(theta)), with the tanh profile of
    Eq. 57 across its boundary.  Isothermal at Tr T_c; periodic in x; the wall
    and the top are held at that temperature."""
    rg, rl = COEXISTENCE[Tr]
    x0 = 0.5 * (nx - 1) if x0 is None else x0
    yc = -0.5 - R * np.cos(np.radians(theta))
    rho = tanh_disc(nx, ny, x0, yc, R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    T = np.full((ny, nx), Tr * TC)
    z = np.zeros((ny, nx))
    bc = bc_spec([PERIODIC, PERIODIC, WALL, top],
                 [T_PERIODIC, T_PERIODIC, T_DIRICHLET, T_DIRICHLET],
                 T_edge=[0.0, 0.0, Tr * TC, Tr * TC], theta_deg=theta)
    return Case("sessile_cap_%dx%d_%g" % (nx, ny, theta), nx, ny, p or params(), bc,
                rho, z, z.copy(), T, steps, rl, rg, sessile=True)


def bubble_field(nx, ny, bubbles, w=4.0, Tr=0.86, periodic_x=False, periodic_y=False,
                 amp=0.0, seed=7):
    """Liquid at rest with vapour bubbles: `bubbles` lists (x0, y0, R); each
    bubble is a tanh disc (Eq. 57) around its centre, distances taken across
    the seams of periodic axes.  Returns (rho, T) at Tr T_c."""
    rg, rl = COEXISTENCE[Tr]
    vap = np.zeros((ny, nx))
    for (x0, y0, R) in bubbles:
        # the profile is evaluated within R + 10 w of the centre; beyond it
        # the tanh tail is below 1e-17
        h = int(np.ceil(R + 10.0 * w))

        def axis(c, n, per):
            idx = np.arange(int(np.floor(c)) - h, int(np.floor(c)) + h + 2)
            if per:
                dist = np.abs(idx - c)
                idx = idx % n
                dist = np.minimum(dist, n - dist)
                keep = np.unique(idx, return_index=True)[1]
                return idx[keep], dist[keep]
            idx = idx[(idx >= 0) & (idx < n)]
            return idx, np.abs(idx - c)

        xi, dx = axis(x0, nx, periodic_x)
        yi, dy = axis(y0, ny, periodic_y)
        d = np.sqrt(dx[None, :] ** 2 + dy[:, None] ** 2)
        win = np.ix_(yi, xi)
        vap[win] = np.maximum(vap[win], 0.5 - 0.5 * np.tanh((d - R) / (0.5 * w)))
    rho = rl - (rl - rg) * vap
    if amp:
        rho = rho + noise(seed, (ny, nx), amp)
    return rho, np.full((ny, nx), Tr * TC)


def batch_instances(n=512, seed=5, side_lo=64, side_hi=512, steps=5000):
    """The batched / served population: open-space evaporating droplets with
    square sides uniform in [side_lo, side_hi], radii 0.2-0.3 of the side and
    edge temperatures uniform in [0.90, 0.98] T_c."""
    u = uniform(seed, 3 * n).reshape(n, 3)
    out = []
    for k in range(n):
        side = int(side_lo + np.floor(u[k, 0] * (side_hi - side_lo + 1)))
        R = (0.2 + 0.1 * u[k, 1]) * side
        Te = 0.90 + 0.08 * u[k, 2]
        c = open_evaporation(side, side, R=R, T_edge=Te, seed=seed * 100003 + k, steps=steps)
        c.name = "batch%03d_%d" % (k, side)
        out.append(c)
    return out


# ---- three-dimensional form ------------------------------------------------

def periodic_bc3() -> dict:
    return dict(flow_z=PERIODIC, therm=[T_PERIODIC, T_PERIODIC], T_edge=[0.0, 0.0],
                theta_deg=90.0)


def wall_bc3(T_bottom, T_top, theta_deg=90.0, adiabatic=(False, False)) -> dict:
    """Walls at both z ends, Dirichlet at the given temperatures (or adiabatic)."""
    th = [T_ADIABATIC if a else T_DIRICHLET for a in adiabatic]
    return dict(flow_z=WALL, therm=th, T_edge=[float(T_bottom), float(T_top)],
                theta_deg=float(theta_deg))


class Case3:
    """A 3-D simulation input: sizes, params, bc and fields [nz][ny][nx]."""

    def __init__(self, name, nx, ny, nz, params, bc, rho, T, steps, rho_l, rho_g,
                 sessile=False):
        self.name, self.nx, self.ny, self.nz = name, nx, ny, nz
        self.params, self.bc = params, bc
        self.rho, self.T = rho, T
        z = np.zeros_like(rho)
        self.ux, self.uy, self.uz = z, z.copy(), z.copy()
        self.steps, self.rho_l, self.rho_g, self.sessile = steps, rho_l, rho_g, sessile

    def fields(self):
        return self.rho, self.ux, self.uy, self.uz, self.T


def tanh_ball(nx, ny, nz, x0, y0, z0, R, w, inside, outside):
    """Eq. 57 around a sphere; nodes at integer coordinates."""
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    d = np.sqrt((x - x0) ** 2 + (y - y0) ** 2 + (z - z0) ** 2)
    return 0.5 * (inside + outside) - 0.5 * (inside - outside) * np.tanh((d - R) / (0.5 * w))


def droplet3d(nx=32, ny=32, nz=32, R=8.0, w=4.0, Tr=0.86, amp=1e-4, seed=8, steps=1000,
              p=None) -> Case3:
    """Static droplet in a periodic box at uniform T."""
    rg, rl = COEXISTENCE[Tr]
    rho = tanh_ball(nx, ny, nz, 0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * (nz - 1), R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, rho.shape, amp)
    T = np.full(rho.shape, Tr * TC)
    return Case3("droplet3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, p or params(),
                 periodic_bc3(), rho, T, steps, rl, rg)


def heated_droplet3d(nx=64, ny=64, nz=64, R=16.0, w=4.0, T_sat=0.86, T_wall=0.95, amp=1e-4,
                     seed=9, steps=1000, p=None) -> Case3:
    """Droplet at T_sat between two walls at T_wall (z ends), periodic in x
    and y: it evaporates as heat conducts in from the walls."""
    rg, rl = COEXISTENCE[T_sat]
    c = (0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * (nz - 1))
    rho = tanh_ball(nx, ny, nz, *c, R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, rho.shape, amp)
    T = tanh_ball(nx, ny, nz, *c, R, w, T_sat * TC, T_wall * TC)
    return Case3("heated_droplet3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, p or params(),
                 wall_bc3(T_wall * TC, T_wall * TC), rho, T, steps, rl, rg)


def sessile3d(nx=48, ny=48, nz=32, R=12.0, theta=90.0, w=4.0, Tr=0.86, amp=1e-4, seed=10,
              steps=0, p=None) -> Case3:
    """Spherical cap meeting the bottom wall line z = -1/2 at `theta`, walls at
    both z ends held at Tr T_c."""
    rg, rl = COEXISTENCE[Tr]
    zc = -0.5 - R * np.cos(np.radians(theta))
    rho = tanh_ball(nx, ny, nz, 0.5 * (nx - 1), 0.5 * (ny - 1), zc, R, w, rl, rg)
    if amp:
        rho = rho + noise(seed, rho.shape, amp)
    T = np.full(rho.shape, Tr * TC)
    bc = wall_bc3(Tr * TC, Tr * TC, theta_deg=theta)
    return Case3("sessile3d_%g" % theta, nx, ny, nz, p or params(), bc, rho, T, steps, rl, rg,
                 sessile=True)


def droplet_cloud3d(n=256, cells=4, R=None, w=4.0, Tr=0.86, amp=1e-4, seed=11, steps=1000,
                    p=None) -> Case3:
    """A periodic n^3 box tiled by cells^3 sub-cubes, each holding one droplet
    at its centre (an evaporating spray's droplet cloud at T_sat).  R
    defaults to a quarter of the sub-cube side."""
    rg, rl = COEXISTENCE[Tr]
    s = n // cells
    R = 0.25 * s if R is None else R
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    # distance to the centre of the node's own sub-cube
    c = 0.5 * (s - 1)
    d = np.sqrt((np.mod(x, s) - c) ** 2 + (np.mod(y, s) - c) ** 2 + (np.mod(z, s) - c) ** 2)
    rho = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh((d - R) / (0.5 * w))
    if amp:
        rho = rho + noise(seed, rho.shape, amp)
    T = np.full(rho.shape, Tr * TC)
    return Case3("droplet_cloud3d_%d_%dx%dx%d" % (n, cells, cells, cells), n, n, n,
                 p or params(), periodic_bc3(), rho, T, steps, rl, rg)


# ---- named configurations (configs/*.json) -----------------------------------

CONFIG_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "configs")


def load_config(name_or_path: str) -> dict:
    """A named configuration: {"name", "about", "case", "args", "precisions",
    "steps", ...}.  `name_or_path` is a file or a name under configs/."""
    import json
    path = name_or_path if os.path.exists(name_or_path) else os.path.join(
        CONFIG_DIR, name_or_path + ".json")
    with open(path) as fh:
        return json.load(fh)


def config_case(cfg: dict, **override):
    """Builds the configuration's input (a Case, Case3, or a list of Cases)."""
    fn = globals()[cfg["case"]]
    args = dict(cfg.get("args", {}))
    args.update(override)
    return fn(**args)
