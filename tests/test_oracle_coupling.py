"""Pins of the oracle's coupling between the flow and the temperature lattice
(no GPU): the source Q of Eq. 20 with its convective and compression terms,
the divergence of u (reading R7), the local temperature gradient of
Eqs. 49-50 and the history term S of Eq. 24 (reading R8).

Each test compares the oracle with something it does not contain: the
linearised continuum equations the paper's Chapman-Enskog analysis recovers
(Eqs. 20, 34, 54), thermodynamic identities of the Peng-Robinson EOS with
derivatives taken by finite differences of p_EOS, and spectral derivatives of
the oracle's own fields.  The setups are single Fourier modes on a uniform
vapour-like state (rho = 0.3 at 0.95 T_c, where psi^2 > 0 and the state is
mechanically stable), so every expectation is a closed form.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

TC = W.TC
RHO0, T0 = 0.3, 0.95 * TC


def thermo(p):
    """(dp/drho)_T, (dp/dT)_rho by central differences of p_EOS (Eq. 10), and
    the adiabatic slope kappa = (dT/drho)_s = T (dp/dT)_rho / (rho^2 c_v), the
    adiabatic sound speed and c_p = c_v + T (dp/dT)^2 / (rho^2 (dp/drho))."""
    hT, hr = 1e-6 * T0, 1e-6 * RHO0
    dpdT = (O.p_eos(p, RHO0, T0 + hT) - O.p_eos(p, RHO0, T0 - hT)) / (2 * hT)
    dpdr = (O.p_eos(p, RHO0 + hr, T0) - O.p_eos(p, RHO0 - hr, T0)) / (2 * hr)
    cv = p["cv"]
    kappa = T0 * dpdT / (RHO0 ** 2 * cv)
    c_ad = math.sqrt(dpdr + T0 * dpdT ** 2 / (RHO0 ** 2 * cv))
    cp = cv + T0 * dpdT ** 2 / (RHO0 ** 2 * dpdr)
    return dict(dpdT=dpdT, dpdr=dpdr, kappa=kappa, c_ad=c_ad, c_T=math.sqrt(dpdr), cp=cp)


def mode_amp(field_row, k):
    """complex amplitude a of a + conj(a) over a row: field = Re(a e^{ikx}) * 2/2"""
    nx = field_row.size
    return (field_row - field_row.mean()) @ np.exp(-1j * k * np.arange(nx)) * 2.0 / nx


def sim_1d(nx, p, rho, ux, T):
    s = O.Sim(nx, 1, p, W.periodic_bc())
    z = np.zeros((1, nx))
    s.init(np.asarray(rho, float).reshape(1, nx), np.asarray(ux, float).reshape(1, nx), z,
           np.asarray(T, float).reshape(1, nx))
    return s


# ---------------------------------------------------------------------------
# compression term of Q and the divergence stencil

@pytest.mark.parametrize("nx", [64, 128])
def test_compression_heating_in_one_step(nx):
    """Uniform rho and T with u_x = U sin(kx): psi is uniform, so F = 0 and u
    is exactly the prescribed field.  The first step has S = 0, dT/dx = 0 and
    Q = -T (dp/dT)_rho div u, so Eq. 20 gives T(t+1) - T(t) = -T (dp/dT)_rho
    U k cos(kx) / (rho c_v), up to the O(k^2) error of the discrete div u and
    of the streaming average.  A dropped or sign-flipped compression term, a
    wrong stencil factor or a missing 1/(rho c_v) fails this."""
    p = W.params()
    th = thermo(p)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    U = 1e-3
    s = sim_1d(nx, p, np.full(nx, RHO0), U * np.sin(k * x), np.full(nx, T0))
    s.step(1)
    dT = s.fields()[3][0] - T0
    pred = -T0 * th["dpdT"] * U * k * np.cos(k * x) / (RHO0 * p["cv"])
    err = np.abs(dT - pred).max() / np.abs(pred).max()
    assert err < 0.5 * k * k, err
    # the divergence itself is (1/c_s^2) sum_i w_i c_i . u(x + c_i) -> U k cos(kx)
    divu = s.work("divu")[0]
    assert np.abs(divu - U * k * np.cos(k * x)).max() < 0.25 * k * k * U * k


def test_sound_wave_is_adiabatic():
    """A standing sound wave (u_x = U sin(kx) on a uniform state) compresses the
    fluid.  With Q's compression term the temperature follows the density
    along the adiabat: T' / rho' = T (dp/dT)_rho / (rho^2 c_v), and the wave
    oscillates at the adiabatic sound speed sqrt((dp/drho)_T + T (dp/dT)^2 /
    (rho^2 c_v)) instead of the isothermal one (18 % slower here).  Both are
    thermodynamic identities of the EOS, independent of the lattice."""
    p = W.params()
    th = thermo(p)
    nx = 256
    k = 2 * math.pi / nx
    x = np.arange(nx)
    U = 1e-4
    s = sim_1d(nx, p, np.full(nx, RHO0), U * np.sin(k * x), np.full(nx, T0))
    period = 2 * math.pi / (th["c_ad"] * k)
    ratios, u_im = [], []
    for t in range(1, int(0.35 * period)):
        s.step(1)
        r, ux, _, T = s.fields()
        rh, Th = mode_amp(r[0], k), mode_amp(T[0], k)
        if t <= 50:
            ratios.append((Th / rh).real)
        u_im.append(mode_amp(ux[0], k).imag)
    ratios = np.array(ratios)
    assert np.abs(ratios / th["kappa"] - 1).max() < 5e-3, ratios[[0, -1]] / th["kappa"]
    # first zero of the velocity: a quarter period
    u_im = np.array(u_im)
    t_q = 1 + np.argmax(u_im[:-1] * u_im[1:] <= 0)
    assert abs(t_q / (0.25 * period) - 1) < 0.02, (t_q, 0.25 * period)
    assert abs(t_q / (0.25 * 2 * math.pi / (th["c_T"] * k)) - 1) > 0.1


def test_history_source_keeps_the_sound_wave_adiabatic():
    """Eq. 24's S_i = w_i rho c_v (dt/2) d_t^2 T, with d_t^2 T read as
    P^n - P^{n-1} (P = Q / (rho c_v), R8), turns the source's time integration
    into T^{n+1} - T^n = (3/2) P^n - (1/2) P^{n-1}, a half-step-centred rule.
    The density of the flow lattice advances with the half-step momentum
    (j + F/2), so with S the temperature increments of a sound wave stay on the
    adiabat at every phase of the wave.  Without S they lag the density by half
    a step: the increment ratio drifts by (omega/2) tan(omega t), 4 % by
    omega t = 1 here (omega = 0.063); a sign error drifts the other way.
    Small lambda keeps diffusion out of the ratio."""
    p = W.params(lambda_=0.01)
    th = thermo(p)
    nx = 32
    k = 2 * math.pi / nx
    x = np.arange(nx)
    s = sim_1d(nx, p, np.full(nx, RHO0), 1e-4 * np.sin(k * x), np.full(nx, T0))
    om = th["c_ad"] * k
    prev = (0.0, 0.0)
    incr = {}
    for t in range(1, int(1.05 / om) + 2):
        s.step(1)
        r, _, _, T = s.fields()
        rh, Th = mode_amp(r[0], k).real, mode_amp(T[0], k).real
        if t > 1:
            incr[t] = (Th - prev[1]) / (rh - prev[0]) / th["kappa"]
        prev = (rh, Th)
    early = incr[int(round(0.2 / om))]
    late = incr[int(round(1.0 / om))]
    assert abs(early - 1) < 0.02 and abs(late - 1) < 0.03, (early, late)
    assert abs(late / early - 1) < 0.015, (early, late)


# ---------------------------------------------------------------------------
# the entropy mode: convective term, local gradient, compression term together

def entropy_mode(nx, u0, steps, p=None):
    """An isobaric temperature wave (rho' = -(dp/dT)/(dp/drho) T', so p' = 0)
    on a uniform stream u0; returns (k, thermo, complex T amplitudes per step,
    the Sim)."""
    p = p or W.params()
    th = thermo(p)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    A = 1e-5 * T0
    T = T0 + A * np.cos(k * x)
    rho = RHO0 - th["dpdT"] / th["dpdr"] * A * np.cos(k * x)
    s = sim_1d(nx, p, rho, np.full(nx, u0), T)
    amps = []
    for _ in range(steps):
        s.step(1)
        amps.append(mode_amp(s.fields()[3][0], k))
    return k, th, np.array(amps), s


def fit_rates(amps, start):
    t = np.arange(1, len(amps) + 1)[start:]
    decay = -np.polyfit(t, np.log(np.abs(amps[start:])), 1)[0]
    phase = np.polyfit(t, np.unwrap(np.angle(amps))[start:], 1)[0]
    return decay, phase


def test_entropy_mode_decays_at_lambda_k2_over_rho_cp():
    """At constant pressure a temperature wave diffuses with lambda / (rho c_p),
    not lambda / (rho c_v): the compression term T (dp/dT)_rho div u of Eq. 20
    does the work of the thermal expansion.  Linearised continuum (Eqs. 20 and
    54 with mass and momentum balance) gives the decay rate lambda k^2 /
    (rho c_p) + O(k^4); c_p / c_v = 1.38 here, so a dropped or mis-scaled
    compression term (or div u stencil) is far outside the 1 % bound."""
    nx, steps = 64, 2400
    k, th, amps, _ = entropy_mode(nx, 0.0, steps)
    decay, _ = fit_rates(amps, steps // 3)
    rate_cp = W.params()["lambda_"] * k * k / (RHO0 * th["cp"])
    assert abs(decay / rate_cp - 1) < 0.01, decay / rate_cp


@pytest.mark.parametrize("u0", [0.05, -0.04])
def test_entropy_mode_is_advected_at_the_flow_speed(u0):
    """On a uniform stream u0 the same wave travels at u0 (Galilean invariance
    of Eq. 20: the convective term -rho c_v u . grad T, with grad T from the
    local moments of Eqs. 49-50, is the only thing that moves it).  A sign
    error in the convective term reverses the motion; a wrong varsigma /
    c_s^2 factor in Eqs. 49-50 scales the speed.  The decay rate stays
    lambda k^2 / (rho c_p) up to the O(u0^2) lag of the local gradient."""
    nx, steps = 64, 2400
    k, th, amps, _ = entropy_mode(nx, u0, steps)
    decay, phase = fit_rates(amps, steps // 3)
    assert abs(-phase / k / u0 - 1) < 5e-3, -phase / k / u0
    rate_cp = W.params()["lambda_"] * k * k / (RHO0 * th["cp"])
    assert abs(decay / rate_cp - 1) < 0.02, decay / rate_cp


def test_local_gradient_matches_the_field_gradient():
    """Eqs. 49-50 read grad T from the first moments of the non-equilibrium
    thermal populations.  On the diffusing entropy mode the oracle's dT/dx must
    equal the spectral derivative of its own temperature field (to the
    scheme's O(k^2)), with the paper's sign."""
    nx = 64
    k, _, _, s = entropy_mode(nx, 0.0, 600)
    dTx = s.work("dTx")[0]
    Tw = s.work("T")[0]
    spec = np.fft.ifft(2j * math.pi * np.fft.fftfreq(nx) * np.fft.fft(Tw)).real
    assert np.abs(dTx - spec).max() < 0.02 * np.abs(spec).max()
    assert np.abs(s.work("dTy")).max() < 1e-20


@pytest.mark.parametrize("cv", [2.0, 4.0])
def test_local_gradient_is_exact_in_steady_conduction(cv):
    """Between two Dirichlet walls (frozen flow, piecewise rho c_v) the steady
    temperature is linear; for a linear profile the non-equilibrium first
    moment is exactly -c_s^2 dT/dy / varsigma_1, so Eqs. 49-50 recover the
    slope to round-off at every node, whatever rho c_v is."""
    nx, ny = 4, 16
    Tb, Tt = 0.08, 0.11
    bc = W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                   [W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET],
                   T_edge=[0, 0, Tb, Tt])
    rho = np.where(np.arange(ny) < ny // 2, 0.5, 3.0)[:, None] * np.ones((1, nx))
    z = np.zeros((ny, nx))
    s = O.Sim(nx, ny, W.params(frozen_flow=1, cv=cv), bc)
    s.init(rho, z, z, np.full((ny, nx), 0.5 * (Tb + Tt)))
    s.step(40000)
    slope = (Tt - Tb) / ny            # walls half a spacing outside rows 0 and ny-1
    T = s.fields()[3]
    assert np.abs(np.diff(T[:, 0]) - slope).max() < 1e-12
    s.step(1)
    assert np.abs(s.work("dTy") - slope).max() < 1e-9 * slope
    assert np.abs(s.work("dTx")).max() < 1e-15


# ---------------------------------------------------------------------------
# the source moments (Eq. 33) on the oracle's own collision

def test_source_moments_of_the_thermal_collision():
    """Eq. 33: sum_i G_i = Q, sum_i c_i G_i = 0, sum_i S_i = rho c_v (dt/2)
    d_t^2 T, sum_i c_i S_i = 0.  On a coupled droplet step the post-collision
    moments differ from the source-free MRT relaxation of Eqs. 39, 40 and 47
    by exactly M_hat (G + S) = (Q + S, 0, 0, w_dot (Q + S), 0)."""
    c = W.static_droplet(24, 20, R=6.0, amp=1e-3, p=W.params(gravity=2e-5))
    s = O.Sim(c.nx, c.ny, c.params, c.bc)
    s.init(*c.fields())
    s.step(5)
    g = s.populations()[1]
    s.step(1)
    Mh = O.matrices()[2]
    wd = c.params["w_dot"]
    vs = 1.0 / (c.params["lambda_"] / (wd / 2) + 0.5)
    Lam = np.array([1.0, vs, vs, 1.0, 1.0])
    m = np.einsum("ki,iyx->kyx", Mh, g)
    T = m[0]
    meq = np.stack([T, 0 * T, 0 * T, wd * T, 0 * T])
    relaxed = m - Lam[:, None, None] * (m - meq)
    src = np.einsum("ki,iyx->kyx", Mh, s.work("gstar")) - relaxed
    QS = s.work("Q") + s.work("S")
    assert np.abs(QS).max() > 1e-6
    scale = np.abs(QS).max()
    assert np.abs(src[0] - QS).max() < 1e-12 * max(scale, 1.0)
    assert np.abs(src[1]).max() < 1e-14 and np.abs(src[2]).max() < 1e-14
    assert np.abs(src[3] - wd * QS).max() < 1e-12 * max(scale, 1.0)
    assert np.abs(src[4]).max() < 1e-14
