"""Pins of the three-dimensional oracle (D3Q19 MRT flow lattice + D3Q7
temperature lattice with the rho c_v-weighted streaming) against published
moment equilibria, invariants, exact linear analysis, a textbook scheme and
the two-dimensional oracle (no GPU)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

TC = W.TC


def run3(case, steps=0, params=None):
    s = O.Sim3(case.nx, case.ny, case.nz, params or case.params, case.bc)
    s.init(*case.fields())
    if steps:
        s.step(steps)
    return s


# ---------------------------------------------------------------------------
# lattice and moment basis

def test_velocity_set_isotropy():
    """D3Q19 weights give the isotropic moments of a c_s^2 = 1/3 lattice up
    to fourth order; the set is closed under c -> -c."""
    cx, cy, cz, w = O.velocities3()
    c = np.stack([cx, cy, cz], axis=1).astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-15)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) +
            np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    rows = {tuple(v) for v in c.astype(int)}
    assert all(tuple(-np.array(v)) in rows for v in rows) and len(rows) == 19


def test_moment_matrices_orthogonal_and_inverted():
    M, Mi, Mh, Mhi = O.matrices3()
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() == 0       # orthogonal rows
    assert np.abs(Mi @ M - np.eye(19)).max() < 1e-13
    assert np.abs(Mhi @ Mh - np.eye(7)).max() < 1e-14


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.05, -0.03, 0.02), (-0.1, 0.07, 0.11)])
def test_equilibrium_moments_are_dhumieres(u):
    """M f^eq equals the published D3Q19 equilibria of d'Humieres et al.
    (2002) with w_eps = 3, w_epsj = -11/2, w_xx = -1/2: e = -11 rho + 19 rho u^2,
    eps = 3 rho - 11/2 rho u^2, q = -2/3 j, 3p_xx = rho (3ux^2 - u^2),
    3pi_xx = -1/2 3p_xx, p_ww = rho (uy^2 - uz^2), pi_ww = -1/2 p_ww,
    p_ab = rho u_a u_b, m = 0."""
    M = O.matrices3()[0]
    rho = 1.7
    ux, uy, uz = u
    uu = ux * ux + uy * uy + uz * uz
    m = M @ O.feq3(rho, ux, uy, uz)
    ref = [rho, -11 * rho + 19 * rho * uu, 3 * rho - 5.5 * rho * uu,
           rho * ux, -2 / 3 * rho * ux, rho * uy, -2 / 3 * rho * uy, rho * uz, -2 / 3 * rho * uz,
           rho * (3 * ux * ux - uu), -0.5 * rho * (3 * ux * ux - uu),
           rho * (uy * uy - uz * uz), -0.5 * rho * (uy * uy - uz * uz),
           rho * ux * uy, rho * uy * uz, rho * ux * uz, 0.0, 0.0, 0.0]
    assert np.allclose(m, ref, rtol=0, atol=1e-13)


def test_forcing_moments():
    """M of the discrete force term is the published D3Q19 MRT forcing
    vector: e: 38 u.F, eps: -11 u.F, j: F, q: -2/3 F, 3p_xx: 2(2uxFx - uyFy -
    uzFz), 3pi_xx: -(2uxFx - uyFy - uzFz), p_ww: 2(uyFy - uzFz), pi_ww:
    -(uyFy - uzFz), p_ab: u_a F_b + u_b F_a, m: 0."""
    M = O.matrices3()[0]
    u = np.array([0.03, -0.05, 0.08])
    F = np.array([1e-3, 2e-3, -1.5e-3])
    m = M @ O.force_term3(*u, *F)
    uF = u @ F
    a = 2 * u[0] * F[0] - u[1] * F[1] - u[2] * F[2]
    b = u[1] * F[1] - u[2] * F[2]
    ref = [0, 38 * uF, -11 * uF, F[0], -2 / 3 * F[0], F[1], -2 / 3 * F[1], F[2], -2 / 3 * F[2],
           2 * a, -a, 2 * b, -b, u[0] * F[1] + u[1] * F[0], u[1] * F[2] + u[2] * F[1],
           u[0] * F[2] + u[2] * F[0], 0, 0, 0]
    assert np.allclose(m, ref, rtol=0, atol=1e-16)


# ---------------------------------------------------------------------------
# invariants

@pytest.mark.parametrize("walls", [False, True])
def test_mass_conserved(walls):
    c = W.droplet3d(14, 12, 16, R=4.5)
    if walls:
        c.bc = W.wall_bc3(0.9 * TC, 0.9 * TC, theta_deg=70.0)
    s = run3(c)
    m0 = s.diagnostics(c.rho_l, c.rho_g)["mass"]
    s.step(60)
    m1 = s.diagnostics(c.rho_l, c.rho_g)["mass"]
    assert abs(m1 - m0) <= 1e-12 * m0


@pytest.mark.parametrize("gravity", [0.0, 3e-5])
def test_total_momentum_stays_zero(gravity):
    """Pair antisymmetry of F_m and mass conservation keep sum_i c_i f_i at
    its initial zero on a periodic box."""
    c = W.droplet3d(14, 12, 16, R=4.5, p=W.params(gravity=gravity))
    s = run3(c, 60)
    f = s.populations()[0]
    cx, cy, cz, _ = O.velocities3()
    for comp in (cx, cy, cz):
        assert abs(np.einsum("i,izyx->", comp, f)) < 1e-11


@pytest.mark.parametrize("walls", [False, True])
def test_uniform_state_is_a_fixed_point(walls):
    T = 0.9 * TC
    rg, _ = W.COEXISTENCE[0.90]
    shape = (6, 5, 4)
    rho = np.full(shape, rg)
    z = np.zeros(shape)
    bc = W.wall_bc3(T, T) if walls else W.periodic_bc3()
    s = O.Sim3(4, 5, 6, W.params(), bc)
    s.init(rho, z, z, z, np.full(shape, T))
    f0, g0, _ = s.populations()
    s.step(20)
    f1, g1, _ = s.populations()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-14


def test_droplet_keeps_cubic_symmetry():
    """A noise-free droplet centred on a node of a cube stays invariant under
    the 48 symmetries of the cube (axis permutations and reflections)."""
    c = W.droplet3d(15, 15, 15, R=4.0, amp=0.0)
    s = run3(c, 40)
    r = s.fields()[0]
    for perm in itertools.permutations(range(3)):
        rp = np.transpose(r, perm)
        assert np.abs(rp - r).max() < 1e-12
    for ax in range(3):
        assert np.abs(np.flip(r, ax) - r).max() < 1e-12


# ---------------------------------------------------------------------------
# the thermal lattice

def _frozen_box(nx, ny, nz, rho, T, params):
    s = O.Sim3(nx, ny, nz, params, W.periodic_bc3())
    z = np.zeros((nz, ny, nx))
    s.init(np.full((nz, ny, nx), rho), z, z, z, T)
    return s


@pytest.mark.parametrize("k", [(1, 0, 0), (1, 1, 0), (1, 2, 1)])
def test_fourier_amplification_exact(k):
    """Frozen flow, uniform rho c_v = C: each Fourier mode of g evolves by
    A = (1 - 1/C) I + (1/C) diag(e^{-i k.c_i}) Mh^-1 ((I - L) Mh + L E Mh),
    E the map to m^eq = [T, 0, 0, 0, w_dot T, 0, 0]; the oracle's mode matches
    A^n g^ to 1e-12."""
    nx, ny, nz = 8, 6, 4
    P = W.params(frozen_flow=1, lambda_=0.2)
    rho = 0.8                                   # C = 4
    C = rho * P["cv"]
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    kv = 2 * np.pi * np.array([k[0] / nx, k[1] / ny, k[2] / nz])
    ph = kv[0] * x + kv[1] * y + kv[2] * z
    T = 0.9 * TC + 1e-3 * TC * np.cos(ph)
    s = _frozen_box(nx, ny, nz, rho, T, P)
    g0 = s.populations()[1]
    n = 7
    s.step(n)
    g1 = s.populations()[1]
    M, _, Mh, Mhi = O.matrices3()
    wd = P["w_dot"]
    cs2 = wd / 3
    vs = 1 / (P["lambda_"] / cs2 + 0.5)
    L = np.diag([1, vs, vs, vs, 1, 1, 1])
    E = np.zeros((7, 7))
    E[0, 0] = 1
    E[4, 0] = wd
    K = Mhi @ ((np.eye(7) - L) @ Mh + L @ E @ Mh)
    hx = np.array([0, 1, -1, 0, 0, 0, 0])
    hy = np.array([0, 0, 0, 1, -1, 0, 0])
    hz = np.array([0, 0, 0, 0, 0, 1, -1])
    D = np.diag(np.exp(-1j * (kv[0] * hx + kv[1] * hy + kv[2] * hz)))
    A = (1 - 1 / C) * np.eye(7) + (1 / C) * D @ K
    e = np.exp(1j * ph)
    norm = e.size
    ghat0 = np.array([(g0[i] * np.conj(e)).sum() / norm for i in range(7)])
    ghat1 = np.array([(g1[i] * np.conj(e)).sum() / norm for i in range(7)])
    pred = np.linalg.matrix_power(A, n) @ ghat0
    assert np.abs(ghat1 - pred).max() < 1e-12 * np.abs(ghat0).max() + 1e-18


def test_continuum_decay_rate():
    """The long-wave decay rate of T is lambda k^2 / (rho c_v): the paper's
    macroscopic equation rho c_v d_t T = div(lambda grad T) with
    c^_s^2 = w_dot / 3 and lambda = c^_s^2 (1/varsigma - 1/2)."""
    nx = 64
    P = W.params(frozen_flow=1, lambda_=1 / 3)
    rho = 0.6
    C = rho * P["cv"]
    x = np.arange(nx)[None, None, :] * np.ones((1, 1, 1))
    k = 2 * np.pi / nx
    T = 0.9 * TC + 1e-3 * TC * np.cos(k * x)
    s = _frozen_box(nx, 1, 1, rho, T, P)
    s.step(200)
    a0 = np.abs((s.fields()[4][0, 0] * np.exp(-1j * k * np.arange(nx))).sum())
    s.step(400)
    a1 = np.abs((s.fields()[4][0, 0] * np.exp(-1j * k * np.arange(nx))).sum())
    rate = -np.log(a1 / a0) / 400
    exact = P["lambda_"] * k * k / C
    assert abs(rate / exact - 1) < 0.01


def test_reduces_to_textbook_d3q7_bgk():
    """rho c_v = 1, all relaxation rates equal, frozen flow: one step is the
    textbook D3Q7 BGK scheme g_i(x + c_i) = g_i - vs (g_i - w^_i T)."""
    nx, ny, nz = 5, 4, 3
    vs = 1.3
    wd = 2 / 3
    cs2 = wd / 3
    lam = cs2 * (1 / vs - 0.5)
    P = W.params(frozen_flow=1, cv=1.0, lambda_=lam, vs0=vs, vs3=vs, vs4=vs)
    s = O.Sim3(nx, ny, nz, P, W.periodic_bc3())
    z = np.zeros((nz, ny, nx))
    s.init(np.ones((nz, ny, nx)), z, z, z, np.full((nz, ny, nx), 0.09))
    g = 0.01 + 0.02 * W.uniform(3, 7 * nx * ny * nz).reshape(7, nz, ny, nx)
    f = s.populations()[0]
    s.set_populations(f, g, np.zeros((nz, ny, nx)), 5, 1.0)
    s.step(1)
    g1 = s.populations()[1]
    w = np.array([1 - wd] + [wd / 6] * 6)
    T = g.sum(axis=0)
    shifts = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    for i, (dx, dy, dz) in enumerate(shifts):
        post = g[i] - vs * (g[i] - w[i] * T)
        ref = np.roll(post, (dz, dy, dx), axis=(0, 1, 2))
        assert np.abs(g1[i] - ref).max() < 1e-15


def test_steady_conduction_between_walls_is_linear():
    """Frozen flow, Dirichlet walls (anti-bounce-back at z = -1/2 and
    nz - 1/2) and a two-phase rho c_v: the steady T is exactly linear."""
    nz = 8
    P = W.params(frozen_flow=1, lambda_=0.3)
    T1, T2 = 0.86 * TC, 0.95 * TC
    s = O.Sim3(1, 1, nz, P, W.wall_bc3(T1, T2))
    rho = np.where(np.arange(nz) < 4, 6.0, 0.5).reshape(nz, 1, 1)
    z = np.zeros((nz, 1, 1))
    s.init(rho, z, z, z, np.full((nz, 1, 1), 0.9 * TC))
    s.step(20000)
    T = s.fields()[4][:, 0, 0]
    exact = T1 + (T2 - T1) * (np.arange(nz) + 0.5) / nz
    assert np.abs(T - exact).max() < 1e-12


# ---------------------------------------------------------------------------
# the flow lattice against thermodynamics and the 2-D model

@pytest.mark.slow
@pytest.mark.parametrize("Tr", [0.86, 0.95])
def test_flat_interface_matches_maxwell_and_2d(Tr):
    """A liquid slab varying along z: the bulk densities reach the Maxwell
    coexistence densities (1% / 3%) and equal those of the 2-D oracle's slab
    to 3e-4 (rho_g) and 1e-5 (rho_l): the 3-D force stencil, forcing moments
    and sigma term give the 2-D pressure tensor on a planar interface."""
    rg, rl = W.COEXISTENCE[Tr]
    n = 96
    zz = np.arange(n, dtype=float)
    prof = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh((np.abs(zz - 47.5) - 24) / 2.0)
    P = W.params(frozen_thermal=1)
    rho3 = np.broadcast_to(prof[:, None, None], (n, 2, 2)).copy()
    z3 = np.zeros_like(rho3)
    s3 = O.Sim3(2, 2, n, P, W.periodic_bc3())
    s3.init(rho3, z3, z3, z3, np.full_like(rho3, Tr * TC))
    rho2 = np.broadcast_to(prof[:, None], (n, 2)).copy()
    z2 = np.zeros_like(rho2)
    s2 = O.Sim(2, n, P, W.periodic_bc())
    s2.init(rho2, z2, z2, np.full_like(rho2, Tr * TC))
    s3.step(15000)
    s2.step(15000)
    r3 = s3.fields()[0][:, 0, 0]
    r2 = s2.fields()[0][:, 0]
    assert abs(r3.max() / rl - 1) < 0.01 and abs(r3.min() / rg - 1) < 0.03
    assert abs(r3.min() / r2.min() - 1) < 3e-4
    assert abs(r3.max() / r2.max() - 1) < 1e-5
