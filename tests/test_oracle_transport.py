"""Pins of the oracle's flow lattice: viscosity and the relaxation rate s_p
(Eq. 5 and Section 4's "relaxation times related to physical parameters"),
the halfway bounce-back no-slip wall, the forcing vector of Eq. 8 and the
Ding-Spelt wetting ghost layer of Section 3.3 (no GPU).

Expectations come from outside the oracle: decay rates of the Navier-Stokes
shear modes, Guo et al.'s velocity-space forcing term (the form Eq. 8 is the
moment-space image of), exact momentum balance, and the contact angle the
wetting condition prescribes.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

TC = W.TC
CX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
RHO0, T0 = 0.3, 0.95 * TC


# ---------------------------------------------------------------------------
# viscosity and the no-slip wall

@pytest.mark.parametrize("nu", [0.1, 0.03])
def test_shear_wave_decays_at_nu_k2(nu):
    """u_x = U sin(ky) on a uniform state is a pure shear mode: div u = 0 and
    grad T = 0, so the thermal lattice stays at rest and the flow obeys
    d_t u_x = nu d_yy u_x.  The amplitude decays as exp(-nu k^2 t), with
    nu = c_s^2 (1/s_p - 1/2) the viscosity that fixes s_p.  A wrong s_p
    mapping (or s_p on the wrong moments) changes the rate."""
    p = W.params(nu=nu)
    ny = 64
    k = 2 * math.pi / ny
    y = np.arange(ny)
    s = O.Sim(1, ny, p, W.periodic_bc())
    z = np.zeros((ny, 1))
    s.init(np.full((ny, 1), RHO0), (1e-3 * np.sin(k * y))[:, None], z, np.full((ny, 1), T0))
    amp = []
    for _ in range(400):
        s.step(1)
        amp.append(s.fields()[1][:, 0] @ np.sin(k * y))
    t = np.arange(1, 401)
    rate = -np.polyfit(t[50:], np.log(np.abs(amp[50:])), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 2e-3, rate / (nu * k * k)
    assert np.abs(s.fields()[3] - T0).max() < 1e-9 * T0     # O(U^2) at most


def test_no_slip_walls_sit_halfway():
    """Between halfway bounce-back walls at y = -1/2 and y = H - 1/2 the
    slowest shear mode is u_x = U sin(pi (y + 1/2) / H), decaying at
    nu (pi/H)^2 with its shape unchanged.  A wall placed on the boundary
    nodes instead (channel width H - 1) decays 6.6 % faster at H = 32; a wall
    that does not stop the fluid does not keep the shape."""
    nu, H = 0.1, 32
    p = W.params(nu=nu)
    bc = W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                   [W.T_PERIODIC, W.T_PERIODIC, W.T_ADIABATIC, W.T_ADIABATIC], theta_deg=90.0)
    yy = np.arange(H)
    prof = np.sin(math.pi * (yy + 0.5) / H)
    s = O.Sim(1, H, p, bc)
    z = np.zeros((H, 1))
    s.init(np.full((H, 1), RHO0), (1e-3 * prof)[:, None], z, np.full((H, 1), T0))
    a = []
    for _ in range(1500):
        s.step(1)
        a.append(s.fields()[1][:, 0] @ prof / (prof @ prof))
    t = np.arange(1, 1501)
    rate = -np.polyfit(t[300:], np.log(np.abs(a[300:])), 1)[0]
    assert abs(rate / (nu * (math.pi / H) ** 2) - 1) < 3e-3
    ux = s.fields()[1][:, 0]
    assert np.abs(ux / ux.max() - prof / prof.max()).max() < 1e-6


# ---------------------------------------------------------------------------
# the forcing vector of Eq. 8

def guo_force_term(ux, uy, Fx, Fy):
    """Guo, Zheng & Shi (2002): F_i = w_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F."""
    cu = CX9 * ux + CY9 * uy
    return W9 * (3.0 * ((CX9 - ux) * Fx + (CY9 - uy) * Fy) + 9.0 * cu * (CX9 * Fx + CY9 * Fy))


def test_eq8_is_the_moment_image_of_guos_force_term():
    """Eq. 8 without its sigma part equals M times Guo's velocity-space force
    term (the printed M of Eq. 4 with the Lallemand-Luo third row)."""
    M = O.matrices()[0]
    rng = np.random.default_rng(3)
    for _ in range(5):
        ux, uy, Fx, Fy = rng.uniform(-0.1, 0.1, 4)
        m = M @ guo_force_term(ux, uy, Fx, Fy)
        uF = ux * Fx + uy * Fy
        ref = [0, 6 * uF, -6 * uF, Fx, -Fx, Fy, -Fy, 2 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx]
        assert np.allclose(m, ref, rtol=0, atol=1e-16)


def droplet_step(rates):
    """One coupled step of a moving droplet with buoyancy (so u . F != 0 at
    the interface); returns (pre-collision f, the Sim after the step)."""
    p = W.params(gravity=3e-5, **rates)
    c = W.static_droplet(24, 20, R=6.0, amp=1e-3, p=p)
    s = O.Sim(c.nx, c.ny, p, c.bc)
    rho, _, _, T = c.fields()
    s.init(rho, np.full_like(rho, 0.03), np.full_like(rho, -0.02), T)
    s.step(3)
    f = s.populations()[0]
    s.step(1)
    return p, f, s


@pytest.mark.parametrize("rates", [{}, dict(s_e=0.8, s_eps=1.1, s_j=0.9, s_q=1.2)])
def test_collision_applies_guos_force_term(rates):
    """The oracle's D2Q9 collision (Eq. 5) must add (I - S/2) F with F the
    moment image of Guo's velocity-space term plus Li's sigma part on rows 1
    and 2 (Eq. 8): M f* = m - S (m - m_eq) + (I - S/2) F at every node, with
    u and F_n as the step computed them.  Any wrong row of the forcing vector
    (the 6 u.F of rows 1-2, the j rows, the stress rows 7-8) fails it."""
    p, f, s = droplet_step(rates)
    M = O.matrices()[0]
    sp = 1.0 / (3.0 * p["nu"] + 0.5)
    S = np.array([p["s0"], p["s_e"], p["s_eps"], p["s_j"], p["s_q"], p["s_j"], p["s_q"], sp, sp])
    rho, ux, uy = s.work("rho"), s.work("ux"), s.work("uy")
    Fx, Fy, Fmx, Fmy, psi = (s.work(n) for n in ("Fx", "Fy", "Fmx", "Fmy", "psi"))
    fstar = s.work("fstar")
    worst = 0.0
    for y in range(f.shape[1]):
        for x in range(f.shape[2]):
            m = M @ f[:, y, x]
            r, u, v = rho[y, x], ux[y, x], uy[y, x]
            meq = r * np.array([1, -2 + 3 * (u * u + v * v), 1 - 3 * (u * u + v * v),
                                u, -u, v, -v, u * u - v * v, u * v])
            F = M @ guo_force_term(u, v, Fx[y, x], Fy[y, x])
            sig = p["sigma"] * (Fmx[y, x] ** 2 + Fmy[y, x] ** 2) / psi[y, x] ** 2
            F[1] += sig / (1 / S[1] - 0.5)
            F[2] -= sig / (1 / S[2] - 0.5)
            expect = m - S * (m - meq) + (1 - 0.5 * S) * F
            worst = max(worst, np.abs(M @ fstar[:, y, x] - expect).max())
    assert worst < 1e-13, worst
    assert np.abs(Fx * ux + Fy * uy).max() > 1e-5


@pytest.mark.parametrize("s_j", [1.0, 0.8])
def test_post_collision_momentum_gains_the_full_force(s_j):
    """With u = (sum c f + F/2)/rho (Eq. 11) the collision adds exactly F_n to
    the momentum of every node, whatever s_j is: sum_i c_i f*_i =
    sum_i c_i f_i + F_n."""
    p, f, s = droplet_step(dict(s_j=s_j))
    fs = s.work("fstar")
    jx, jy = np.einsum("i,iyx->yx", CX9, f), np.einsum("i,iyx->yx", CY9, f)
    jsx, jsy = np.einsum("i,iyx->yx", CX9, fs), np.einsum("i,iyx->yx", CY9, fs)
    assert np.abs(jsx - jx - s.work("Fx")).max() < 1e-14
    assert np.abs(jsy - jy - s.work("Fy")).max() < 1e-14
    assert np.abs(s.work("Fy")).max() > 1e-3


# ---------------------------------------------------------------------------
# Ding-Spelt wetting ghost layer (Section 3.3)

@pytest.mark.slow
@pytest.mark.parametrize("theta_w", [60.0, 120.0])
def test_wetting_ghost_layer_relaxes_a_droplet_to_its_angle(theta_w):
    """A droplet started as a half disc (90 degrees) on a wall whose ghost
    layer prescribes theta_w (closed 120 x 60 box, isothermal) spreads or
    beads up to within a few degrees of theta_w, measured by the circle fit
    of the interface (pinned separately against exact circles).  A sign error
    in the tan(pi/2 - theta) term, or the layers of the formula swapped,
    sends it the wrong way or nowhere."""
    c = W.sessile_cap(120, 60, R=18.0, theta=90.0, amp=1e-4, top=W.WALL)
    bc = dict(c.bc, theta_deg=theta_w)
    s = O.Sim(c.nx, c.ny, dict(c.params, frozen_thermal=1), bc)
    s.init(*c.fields())
    hist = []
    for _ in range(6):
        s.step(2000)
        hist.append(O.contact_angle(s.fields()[0], c.rho_l, c.rho_g)["theta_deg"])
    assert abs(hist[-1] - theta_w) < 7.0, hist
    assert (hist[-1] - 90.0) * (theta_w - 90.0) > 0 and abs(hist[-1] - 90.0) > 20.0, hist
    assert abs(hist[-1] - hist[-2]) < 1.0, hist
