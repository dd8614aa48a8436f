"""Pins of the 3-D oracle's thermal coupling and transport (no GPU): the same
closed forms as for the 2-D oracle (test_oracle_coupling.py), on single
Fourier modes of a uniform vapour-like state in periodic boxes, along x, along
z and along a diagonal, so that every direction of the D3Q19 divergence
stencil and of the D3Q7 local gradient is exercised: one-step compression
heating, the adiabatic slope of a sound wave, the decay of an isobaric
temperature wave at lambda k^2 / (rho c_p) and its advection at the flow
speed, and shear waves at nu k^2 (s_p on the stress moments, reading R33)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

TC = W.TC
RHO0, T0 = 0.3, 0.95 * TC


def thermo(p):
    hT, hr = 1e-6 * T0, 1e-6 * RHO0
    dpdT = (O.p_eos(p, RHO0, T0 + hT) - O.p_eos(p, RHO0, T0 - hT)) / (2 * hT)
    dpdr = (O.p_eos(p, RHO0 + hr, T0) - O.p_eos(p, RHO0 - hr, T0)) / (2 * hr)
    cv = p["cv"]
    return dict(dpdT=dpdT, dpdr=dpdr, kappa=T0 * dpdT / (RHO0 ** 2 * cv),
                c_ad=math.sqrt(dpdr + T0 * dpdT ** 2 / (RHO0 ** 2 * cv)),
                cp=cv + T0 * dpdT ** 2 / (RHO0 ** 2 * dpdr))


# box shapes (nx, ny, nz) and wave vectors in lattice units: along x, along z,
# and along the (1, 1, 1) diagonal of a cube
MODES = {
    "x": ((32, 1, 1), (1, 0, 0)),
    "z": ((1, 1, 32), (0, 0, 1)),
    "diag": ((12, 12, 12), (1, 1, 1)),
}


def grid(shape, m):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = (2 * math.pi * mi / ni for mi, ni in zip(m, (nx, ny, nz)))
    phase = kx * x + ky * y + kz * z
    k = math.sqrt(kx * kx + ky * ky + kz * kz)
    return phase, np.array([kx, ky, kz]) / k, k


def amp(field, phase):
    return (field - field.mean()).ravel() @ np.exp(-1j * phase.ravel()) * 2.0 / field.size


def sim(shape, p, rho, u, T):
    s = O.Sim3(*shape, p, W.periodic_bc3())
    s.init(rho, u[0], u[1], u[2], T)
    return s


@pytest.mark.parametrize("mode", list(MODES))
def test_compression_heating_in_one_step(mode):
    """u = U khat sin(k.x) on a uniform state: after one step T changes by
    -T (dp/dT)_rho U k cos(k.x) / (rho c_v) to O(k^2) (Eq. 20)."""
    shape, m = MODES[mode]
    p = W.params()
    th = thermo(p)
    ph, kh, k = grid(shape, m)
    U = 1e-3
    u = [kh[i] * U * np.sin(ph) for i in range(3)]
    s = sim(shape, p, np.full(ph.shape, RHO0), u, np.full(ph.shape, T0))
    s.step(1)
    dT = s.fields()[4] - T0
    pred = -T0 * th["dpdT"] * U * k * np.cos(ph) / (RHO0 * p["cv"])
    err = np.abs(dT - pred).max() / np.abs(pred).max()
    assert err < 0.5 * k * k, err


@pytest.mark.parametrize("shape,m", [((128, 1, 1), (1, 0, 0)), ((48, 48, 48), (1, 1, 1))])
def test_sound_wave_is_adiabatic(shape, m):
    """T' / rho' = T (dp/dT)_rho / (rho^2 c_v) along a standing sound wave,
    to the O(k^2) of the discrete stencils (k = 0.049 along x, 0.23 along the
    diagonal; small lambda keeps diffusion, lambda k^2 / (rho c_v) per step, out
    of the ratio)."""
    p = W.params(lambda_=0.01)
    th = thermo(p)
    ph, kh, k = grid(shape, m)
    U = 1e-4
    u = [kh[i] * U * np.sin(ph) for i in range(3)]
    s = sim(shape, p, np.full(ph.shape, RHO0), u, np.full(ph.shape, T0))
    for t in range(1, 9):
        s.step(1)
        r, _, _, _, T = s.fields()
        ratio = (amp(T, ph) / amp(r, ph)).real / th["kappa"]
        assert abs(ratio - 1) < max(5e-3, 0.4 * k * k), (t, ratio)


def entropy_run(mode, u0, steps):
    shape, m = MODES[mode]
    p = W.params()
    th = thermo(p)
    ph, kh, k = grid(shape, m)
    A = 1e-5 * T0
    T = T0 + A * np.cos(ph)
    rho = RHO0 - th["dpdT"] / th["dpdr"] * A * np.cos(ph)
    u = [np.full(ph.shape, kh[i] * u0) for i in range(3)]
    s = sim(shape, p, rho, u, T)
    a = []
    for _ in range(steps):
        s.step(1)
        a.append(amp(s.fields()[4], ph))
    a = np.array(a)
    t = np.arange(1, steps + 1)[steps // 3:]
    decay = -np.polyfit(t, np.log(np.abs(a[steps // 3:])), 1)[0]
    phase = np.polyfit(t, np.unwrap(np.angle(a))[steps // 3:], 1)[0]
    return decay / (p["lambda_"] * k * k / (RHO0 * th["cp"])), -phase / k


@pytest.mark.parametrize("mode", ["x", "z"])
def test_entropy_mode_decays_at_lambda_k2_over_rho_cp(mode):
    decay, _ = entropy_run(mode, 0.0, 2400)
    assert abs(decay - 1) < 0.01, decay


@pytest.mark.parametrize("mode,u0", [("x", 0.05), ("z", -0.04)])
def test_entropy_mode_is_advected_at_the_flow_speed(mode, u0):
    decay, speed = entropy_run(mode, u0, 2400)
    assert abs(speed / u0 - 1) < 5e-3, speed / u0
    assert abs(decay - 1) < 0.02, decay


@pytest.mark.parametrize("shape,comp,axis", [((1, 1, 48), 0, 2), ((48, 1, 1), 1, 0),
                                             ((1, 48, 1), 2, 1)])
@pytest.mark.parametrize("nu", [0.1, 0.04])
def test_shear_wave_decays_at_nu_k2(shape, comp, axis, nu):
    """u_comp = U sin(k x_axis) with comp != axis is a pure shear mode decaying
    at nu k^2, nu = c_s^2 (1/s_p - 1/2): pins s_p on the stress moments."""
    p = W.params(nu=nu)
    n = shape[axis]
    k = 2 * math.pi / n
    z, y, x = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                          indexing="ij")
    coord = (x, y, z)[axis]
    u = [np.zeros(x.shape) for _ in range(3)]
    u[comp] = 1e-3 * np.sin(k * coord)
    s = sim(shape, p, np.full(x.shape, RHO0), u, np.full(x.shape, T0))
    a = []
    for _ in range(300):
        s.step(1)
        a.append(s.fields()[1 + comp].ravel() @ np.sin(k * coord).ravel())
    t = np.arange(1, 301)[50:]
    rate = -np.polyfit(t, np.log(np.abs(a[50:])), 1)[0]
    assert abs(rate / (nu * k * k) - 1) < 3e-3, rate / (nu * k * k)


@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_rotated_shear_wave_decays_at_nu_k2(plane):
    """A shear wave whose wave vector and velocity lie along the diagonals of
    a coordinate plane (k ~ (1, 1), u ~ (1, -1)) strains the normal stresses
    p_aa - p_bb: it decays at nu k^2 only if s_p also relaxes the diagonal
    stress moments 3p_xx and p_ww (reading R33)."""
    nu, n = 0.08, 32
    p = W.params(nu=nu)
    a, b = {"xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}[plane]
    shape = [1, 1, 1]
    shape[a] = shape[b] = n
    z, y, x = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                          indexing="ij")
    c = (x, y, z)
    kk = 2 * math.pi / n
    phase = kk * (c[a] + c[b])
    u = [np.zeros(x.shape) for _ in range(3)]
    u[a] = 1e-3 * np.sin(phase) / math.sqrt(2)
    u[b] = -1e-3 * np.sin(phase) / math.sqrt(2)
    s = sim(tuple(shape), p, np.full(x.shape, RHO0), u, np.full(x.shape, T0))
    amp_ = []
    for _ in range(300):
        s.step(1)
        f = s.fields()
        amp_.append((f[1 + a] - f[1 + b]).ravel() @ np.sin(phase).ravel())
    t = np.arange(1, 301)[50:]
    rate = -np.polyfit(t, np.log(np.abs(amp_[50:])), 1)[0]
    assert abs(rate / (nu * 2 * kk * kk) - 1) < 5e-3, rate / (nu * 2 * kk * kk)
