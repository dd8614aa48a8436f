"""Pins of the CPU oracle's time step against invariants, special cases and
analytic solutions that the paper and the mathematics fix (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

CX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CX5 = np.array([0, 1, 0, -1, 0])
CY5 = np.array([0, 0, 1, 0, -1])
TC = W.TC


def run_case(case, steps=None):
    s = O.Sim(case.nx, case.ny, case.params, case.bc)
    s.init(*case.fields())
    if steps:
        s.step(steps)
    return s


# ---------------------------------------------------------------------------
# exact invariants of the periodic box

def test_mass_conserved_to_roundoff():
    c = W.static_droplet(48, 40, R=11)
    s = run_case(c)
    m0 = s.diagnostics(c.rho_l, c.rho_g)["mass"]
    s.step(300)
    m1 = s.diagnostics(c.rho_l, c.rho_g)["mass"]
    assert abs(m1 - m0) <= 1e-12 * m0


@pytest.mark.parametrize("gravity", [0.0, 3e-5])
def test_total_momentum_stays_zero(gravity):
    """sum_x F_m = 0 by the pair antisymmetry of Eq. 9 on a periodic box and
    sum_x (rho - rho_ave) g = 0 because mass is conserved, so the population
    momentum sum_i c_i f_i summed over the box stays at its initial 0."""
    c = W.static_droplet(40, 40, R=10, p=W.params(gravity=gravity))
    s = run_case(c, 200)
    f = s.populations()[0]
    jx = np.einsum("i,iyx->", CX9, f)
    jy = np.einsum("i,iyx->", CY9, f)
    assert abs(jx) < 1e-11 and abs(jy) < 1e-11


@pytest.mark.parametrize("bc", ["periodic", "open_dirichlet", "wall_open"])
def test_uniform_state_is_a_fixed_point(bc):
    nx, ny = 12, 10
    Tr = 0.9
    rg, _ = W.COEXISTENCE[Tr]
    T = Tr * TC
    if bc == "periodic":
        spec = W.periodic_bc()
    elif bc == "open_dirichlet":
        spec = W.bc_spec([W.OPEN] * 4, [W.T_DIRICHLET] * 4, T_edge=[T] * 4)
    else:
        spec = W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.OPEN],
                         [W.T_PERIODIC, W.T_PERIODIC, W.T_ADIABATIC, W.T_DIRICHLET],
                         T_edge=[0, 0, T, T], theta_deg=90.0)
    rho = np.full((ny, nx), rg)
    z = np.zeros((ny, nx))
    s = O.Sim(nx, ny, W.params(), spec)
    s.init(rho, z, z, np.full((ny, nx), T))
    s.step(50)
    r, ux, uy, TT = s.fields()
    assert np.abs(r - rg).max() < 1e-14
    assert np.abs(ux).max() < 1e-15 and np.abs(uy).max() < 1e-15
    assert np.abs(TT - T).max() < 1e-16


def test_centred_droplet_keeps_eightfold_symmetry():
    c = W.static_droplet(32, 32, R=8, amp=0.0)
    s = run_case(c, 200)
    r, ux, uy, T = s.fields()
    assert np.abs(r - r[:, ::-1]).max() < 1e-12
    assert np.abs(r - r[::-1, :]).max() < 1e-12
    assert np.abs(r - r.T).max() < 1e-12
    assert np.abs(ux + ux[:, ::-1]).max() < 1e-12
    assert np.abs(T - T.T).max() < 1e-14


def test_energy_conserved_by_the_weighted_streaming():
    """With the flow frozen (u = 0, so Q = S = 0) the rho c_v-weighted
    streaming of Eq. 39 conserves sum_x rho c_v T exactly on a periodic box
    even where rho c_v varies -- the property that lets the scheme avoid
    grad(rho c_v)."""
    nx, ny = 24, 20
    rho = 0.4 + 5.0 * W.uniform(11, nx * ny).reshape(ny, nx)
    T = 0.09 + 0.01 * W.uniform(12, nx * ny).reshape(ny, nx)
    z = np.zeros((ny, nx))
    p = W.params(frozen_flow=1)
    s = O.Sim(nx, ny, p, W.periodic_bc())
    s.init(rho, z, z, T)
    e0 = (rho * p["cv"] * T).sum()
    s.step(200)
    T1 = s.fields()[3]
    e1 = (rho * p["cv"] * T1).sum()
    assert abs(e1 - e0) < 1e-13 * e0
    assert np.abs(T1 - T).max() > 1e-4     # it did diffuse


# ---------------------------------------------------------------------------
# special cases that reduce to textbook schemes

def d2q5_collision_operator(p):
    """K with g* = K g for the source-free MRT collision of Eq. 39, built
    from Eq. 40 and Eq. 47 in moment space."""
    Mh = O.matrices()[2]
    wd = p["w_dot"]
    vs = 1.0 / (p["lambda_"] / (wd / 2) + 0.5)
    Lam = np.diag([p["vs0"], vs, vs, p["vs3"], p["vs4"]])
    E = np.zeros((5, 5))
    E[0, 0] = 1.0
    E[3, 0] = wd
    return np.linalg.inv(Mh) @ (np.eye(5) - Lam @ (np.eye(5) - E)) @ Mh


def test_reduces_to_textbook_d2q5_mrt_diffusion_when_rho_cv_is_one():
    """rho c_v = 1 removes the blend: g_i(x + c_i, t+1) = g*_i(x, t)."""
    nx, ny = 16, 12
    p = W.params(frozen_flow=1, cv=4.0, vs3=1.3, vs4=0.7)
    rho = np.full((ny, nx), 0.25)
    T = 0.09 + 0.01 * W.uniform(21, nx * ny).reshape(ny, nx)
    z = np.zeros((ny, nx))
    s = O.Sim(nx, ny, p, W.periodic_bc())
    s.init(rho, z, z, T)
    K = d2q5_collision_operator(p)
    g = O.geq(p, 1.0)[:, None, None] * T[None]
    for _ in range(40):
        gs = np.einsum("ij,jyx->iyx", K, g)
        g = np.stack([np.roll(np.roll(gs[i], CY5[i], 0), CX5[i], 1) for i in range(5)])
    s.step(40)
    assert np.abs(s.populations()[1] - g).max() < 1e-15


def test_mrt_with_equal_rates_is_the_bgk_scheme_of_eq21():
    """Eq. 39 with all varsigma = 1/tau_g is Eq. 21 (BGK), here with a
    spatially varying rho c_v."""
    nx, ny = 14, 10
    lam = 0.2
    wd = 2.0 / 3.0
    tau = lam / (wd / 2) + 0.5
    p = W.params(frozen_flow=1, lambda_=lam, vs0=1 / tau, vs3=1 / tau, vs4=1 / tau)
    rho = 0.5 + 4.0 * W.uniform(31, nx * ny).reshape(ny, nx)
    T = 0.09 + 0.01 * W.uniform(32, nx * ny).reshape(ny, nx)
    z = np.zeros((ny, nx))
    s = O.Sim(nx, ny, p, W.periodic_bc())
    s.init(rho, z, z, T)
    s.step(30)
    w = O.geq(p, 1.0)
    C = rho * p["cv"]
    g = w[:, None, None] * T[None]
    for _ in range(30):
        Tn = g.sum(0)
        rhs = g - (g - w[:, None, None] * Tn[None]) / tau
        # rho c_v g_i(x + c_i, t+1) = g_i(x,t) + (rho c_v - 1) g_i(x + c_i, t) - ...
        # rewritten for the destination y = x + c_i
        sh = np.stack([np.roll(np.roll(rhs[i], CY5[i], 0), CX5[i], 1) for i in range(5)])
        g = (sh + (C[None] - 1.0) * g) / C[None]
    assert np.abs(s.populations()[1] - g).max() < 1e-15


# ---------------------------------------------------------------------------
# the exact Fourier amplification of the weighted streaming, and its limit

def amplification(p, C, k):
    K = d2q5_collision_operator(p)
    D = np.diag(np.exp(-1j * k * CX5))
    return (1 - 1 / C) * np.eye(5) + (1 / C) * D @ K


@pytest.mark.parametrize("C", [2.0, 5.0])
@pytest.mark.parametrize("m", [1, 4])
def test_fourier_mode_matches_exact_amplification(C, m):
    """Frozen flow, uniform rho c_v = C: each Fourier mode of g evolves by the
    5x5 matrix (1 - 1/C) I + (1/C) diag(e^{-i k c_x}) K exactly."""
    nx, ny = 128, 2
    p = W.params(frozen_flow=1, cv=C / 0.5)
    rho = np.full((ny, nx), 0.5)
    k = 2 * np.pi * m / nx
    A = 1e-3
    T = 0.09 + A * np.cos(k * np.arange(nx))[None, :] * np.ones((ny, 1))
    s = O.Sim(nx, ny, p, W.periodic_bc())
    z = np.zeros((ny, nx))
    s.init(rho, z, z, T)
    n = 150
    s.step(n)
    g = s.populations()[1]
    gh = 2 * np.fft.fft(g[:, 0, :], axis=1)[:, m] / nx
    pred = np.linalg.matrix_power(amplification(p, C, k), n) @ (O.geq(p, 1.0) * A)
    assert np.abs(gh - pred).max() < 1e-12 * A


@pytest.mark.parametrize("C", [2.0, 5.0])
def test_decay_rate_approaches_lambda_k2_over_rho_cv(C):
    """Eq. 54: rho c_v d_t T = div(lambda grad T) with lambda = (1/vs1 - 1/2)
    cs2h, so a long-wave mode decays at rate lambda k^2 / (rho c_v) + O(k^4)."""
    p = W.params(frozen_flow=1, cv=C / 0.5)
    errs = []
    for m in (1, 2, 4):
        nx, ny = 128, 2
        k = 2 * np.pi * m / nx
        rho = np.full((ny, nx), 0.5)
        T = 0.09 + 1e-3 * np.cos(k * np.arange(nx))[None, :] * np.ones((ny, 1))
        s = O.Sim(nx, ny, p, W.periodic_bc())
        z = np.zeros((ny, nx))
        s.init(rho, z, z, T)
        s.step(200)
        a1 = abs(np.fft.fft(s.fields()[3][0])[m])
        s.step(100)
        a2 = abs(np.fft.fft(s.fields()[3][0])[m])
        rate = -math.log(a2 / a1) / 100
        errs.append(abs(rate / (p["lambda_"] * k * k / C) - 1))
        assert errs[-1] < 0.1 * k * k
    assert errs[0] <= errs[1] <= errs[2]


# ---------------------------------------------------------------------------
# conduction with Dirichlet walls (halfway anti-bounce-back)

def conduction_setup(ny, T1, T2, cv):
    nx = 4
    spec = W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                     [W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET],
                     T_edge=[0, 0, T1, T2])
    p = W.params(frozen_flow=1, cv=cv)
    s = O.Sim(nx, ny, p, spec)
    return s, p, nx


def test_steady_conduction_is_linear_across_two_phases():
    """Steady state of rho c_v d_t T = div(lambda grad T) with uniform lambda
    is linear whatever rho c_v is; the walls sit half a spacing outside."""
    ny, T1, T2 = 16, 0.08, 0.11
    s, p, nx = conduction_setup(ny, T1, T2, 2.0)
    rho = np.where(np.arange(ny)[:, None] < ny // 2, 0.5, 3.0) * np.ones((1, nx))
    z = np.zeros((ny, nx))
    s.init(rho, z, z, np.full((ny, nx), 0.5 * (T1 + T2)))
    s.step(40000)
    T = s.fields()[3][:, 0]
    exact = T1 + (T2 - T1) * (np.arange(ny) + 0.5) / ny
    assert np.abs(T - exact).max() < 1e-11


def test_transient_conduction_matches_fourier_series():
    """T(y, 0) = T1 between walls held at T2: the series solution of
    C d_t T = lambda d_yy T on a slab of width L = ny (walls at -1/2, ny-1/2)."""
    ny, T1, T2, cv, rho0 = 40, 0.08, 0.1, 2.0, 1.5
    s, p, nx = conduction_setup(ny, T2, T2, cv)
    rho = np.full((ny, nx), rho0)
    z = np.zeros((ny, nx))
    s.init(rho, z, z, np.full((ny, nx), T1))
    t = 1500
    s.step(t)
    T = s.fields()[3][:, 0]
    D = p["lambda_"] / (rho0 * cv)
    L = float(ny)
    yy = np.arange(ny) + 0.5
    series = np.zeros(ny)
    for n in range(1, 400, 2):
        series += 4 / (n * np.pi) * np.sin(n * np.pi * yy / L) * np.exp(-D * (n * np.pi / L) ** 2 * t)
    exact = T2 + (T1 - T2) * series
    assert np.abs(T - exact).max() < 2e-3 * abs(T1 - T2)


# ---------------------------------------------------------------------------
# the flow lattice against thermodynamics

@pytest.mark.slow
@pytest.mark.parametrize("Tr", [0.86, 0.95])
def test_flat_interface_coexistence_matches_maxwell(Tr):
    """Isothermal liquid slab: the bulk densities must reach the Maxwell
    equal-area coexistence densities of the Peng-Robinson EOS (sigma = 1.25
    calibrated at 0.86 T_c)."""
    rg, rl = W.COEXISTENCE[Tr]
    nx, ny = 2, 160
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    rho = rg + (rl - rg) * 0.5 * (np.tanh((y - ny / 4) / 2) - np.tanh((y - 3 * ny / 4) / 2))
    z = np.zeros((ny, nx))
    s = O.Sim(nx, ny, W.params(frozen_thermal=1), W.periodic_bc())
    s.init(rho, z, z, np.full((ny, nx), Tr * TC))
    s.step(15000)
    r = s.fields()[0][:, 0]
    assert abs(r[ny // 2] - rl) < 0.01 * rl
    assert abs(r[0] - rg) < 0.03 * rg


@pytest.mark.slow
def test_laplace_law():
    """Isothermal droplets: p_in - p_out is linear in 1/R (Young-Laplace),
    with an intercept small against the smallest pressure jump (the radius is
    taken at the interface level, not at the surface of tension, and the
    interface is ~4 nodes wide, so the intercept is not zero)."""
    P = W.params(frozen_thermal=1)
    inv_r, dp = [], []
    for R in (10, 12, 14, 16, 18):
        c = W.static_droplet(64, 64, R=R, amp=0.0, p=P)
        s = run_case(c, 4000)
        r = s.fields()[0]
        T = 0.86 * TC
        d = O.p_eos(P, r[32, 32], T) - O.p_eos(P, r[0, 0], T)
        # radius from the area inside the interface level
        area = (r > 0.5 * (c.rho_l + c.rho_g)).sum()
        inv_r.append(1.0 / math.sqrt(area / math.pi))
        dp.append(d)
    inv_r, dp = np.array(inv_r), np.array(dp)
    A = np.vstack([inv_r, np.ones_like(inv_r)]).T
    (slope, icpt), res, *_ = np.linalg.lstsq(A, dp, rcond=None)
    r2 = 1 - res[0] / ((dp - dp.mean()) ** 2).sum()
    assert slope > 0
    assert r2 > 0.99
    assert abs(icpt) < 0.15 * dp.min()


def test_literal_cv_reading_is_unstable():
    """Section 4.1 prints (lambda, nu, c_v) = (1/3, 5.0, 0.1).  With c_v = 0.1,
    rho c_v < 1/2 in the vapour and the weighted streaming multiplies the
    non-equilibrium moments by (1 - varsigma/(rho c_v)) < -1 per step; the
    run must break down within a few hundred steps."""
    c = W.static_droplet(48, 48, R=12, p=W.params(nu=5.0, cv=0.1))
    s = run_case(c)
    rc = s.step(400, check=False)
    assert rc in (-3, -4)      # non-finite fields or a negative psi^2


def test_periodic_flow_with_dirichlet_temperature_edges():
    """Section 4.1 streams the flow populations periodically and holds T = T_g
    on the edges by halfway anti-bounce-back.  (a) Mass is conserved to
    round-off (periodic flow) while the thermal edges exchange heat;
    (b) with the flow frozen the thermal lattice sees only the two Dirichlet
    edges, so the transient equals the one between flow walls bit for bit,
    and its steady state is exactly linear across a two-phase rho c_v."""
    c = W.d2_droplet(40, D0=16.0, T_g=0.95)
    s = run_case(c)
    d0 = s.diagnostics(c.rho_l, c.rho_g)
    s.step(300)
    d1 = s.diagnostics(c.rho_l, c.rho_g)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-12 * d0["mass"]
    ny, T1, T2 = 16, 0.08, 0.11
    rho = np.where(np.arange(ny)[:, None] < ny // 2, 0.5, 3.0) * np.ones((1, 4))
    z = np.zeros((ny, 4))
    th = [W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET]
    out = {}
    for name, fl in (("periodic", [W.PERIODIC] * 4),
                     ("walls", [W.PERIODIC, W.PERIODIC, W.WALL, W.WALL])):
        sm = O.Sim(4, ny, W.params(frozen_flow=1, cv=2.0), W.bc_spec(fl, th, T_edge=[0, 0, T1, T2]))
        sm.init(rho, z, z, np.full((ny, 4), 0.5 * (T1 + T2)))
        sm.step(300)
        out[name] = sm.fields()[3].copy()
        sm.step(40000)
        out[name + "_steady"] = sm.fields()[3][:, 0].copy()
    assert np.array_equal(out["periodic"], out["walls"])
    exact = T1 + (T2 - T1) * (np.arange(ny) + 0.5) / ny
    assert np.abs(out["periodic_steady"] - exact).max() < 1e-11


def test_thermal_periodic_without_flow_periodic_is_refused():
    spec = W.bc_spec([W.OPEN] * 4, [W.T_PERIODIC] * 4)
    with pytest.raises(Exception):
        O.Sim(8, 8, W.params(), spec)
