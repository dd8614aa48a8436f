"""Pins of the oracle's diagnostics (mass, energy, liquid area and the
equivalent diameter used for the D^2 law of Section 4.1 and the sessile
droplet of Section 4.2) against direct sums and the geometry of the initial
droplet (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W


@pytest.mark.parametrize("R", [10.0, 17.5])
def test_free_droplet_diagnostics(R):
    c = W.static_droplet(64, 56, R=R, amp=1e-3)
    s = O.Sim(c.nx, c.ny, c.params, c.bc)
    s.init(*c.fields())
    rho, ux, uy, T = s.fields()
    d = s.diagnostics(c.rho_l, c.rho_g)
    mid = 0.5 * (c.rho_l + c.rho_g)
    assert d["mass"] == pytest.approx(rho.sum(), rel=1e-14)
    assert d["energy"] == pytest.approx((rho * c.params["cv"] * T).sum(), rel=1e-14)
    liquid = rho > mid
    assert d["liquid_area"] == liquid.sum()
    assert d["liquid_mass"] == pytest.approx(rho[liquid].sum(), rel=1e-14)
    phi = np.clip((rho - c.rho_g) / (c.rho_l - c.rho_g), 0, 1)
    assert d["liquid_area_smooth"] == pytest.approx(phi.sum(), rel=1e-13)
    assert d["max_u"] == pytest.approx(np.hypot(ux, uy).max(), rel=1e-13)
    assert d["nonfinite"] == 0 and d["step"] == 0
    # the tanh disc is centred on its level set rho_mid at radius R: the
    # equivalent diameter of the area above rho_mid is 2R to the lattice's
    # resolution of the circle
    assert abs(d["diameter"] - 2 * R) < 0.4
    assert abs(d["diameter_smooth"] - 2 * R) < 0.4


def test_sessile_droplet_uses_the_half_disc():
    c = W.sessile_cap(160, 80, R=30.0, theta=90.0)
    s = O.Sim(c.nx, c.ny, c.params, c.bc)
    s.init(*c.fields())
    d = s.diagnostics(c.rho_l, c.rho_g, sessile=True)
    # half a disc of radius 30 whose centre sits on the wall line y = -1/2
    assert abs(d["diameter"] - 60.0) < 0.6
    assert d["diameter"] == pytest.approx(math.sqrt(8 * d["liquid_area"] / math.pi), rel=1e-14)
