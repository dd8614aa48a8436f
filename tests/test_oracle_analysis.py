"""Pins of the oracle's interface analyses (contact angle, connected regions)
and of its between-step reconfiguration, against geometry, a library
labelling routine and exact restarts (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W


# ---------------------------------------------------------------------------
# circle fit and interface points

@pytest.mark.parametrize("arc", [2 * math.pi, math.pi, 2 * math.pi / 3])
def test_circle_fit_recovers_exact_circles(arc):
    """Points on a circle (full circle, half circle, 120-degree arc) give the
    circle back to round-off: the algebraic fit is exact on exact data."""
    t = np.linspace(0.3, 0.3 + arc, 77, endpoint=arc < 2 * math.pi)
    xc, yc, R = 123.25, -17.5, 41.0
    out = O.circle_fit(xc + R * np.cos(t), yc + R * np.sin(t))
    assert np.allclose(out, (xc, yc, R), rtol=0, atol=1e-9)


def test_interface_points_on_a_linear_field_are_exact():
    """Linear interpolation on a link is exact for a linear field: rho = a +
    b x + c y crosses rho_mid on the horizontal link of row y at
    x = (rho_mid - a - c y) / b."""
    ny, nx = 7, 9
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    a, b, c = 1.0, 0.7, 0.05
    rho = a + b * x + c * y
    mid = 4.3
    px, py = O.interface_points(rho, mid, 0)
    for X, Y in zip(px, py):
        assert abs(a + b * X + c * Y - mid) < 1e-12
    # one crossing per row on horizontal links, plus the vertical links where
    # the small y slope carries a node across the level
    horiz = [(X, Y) for X, Y in zip(px, py) if Y == int(Y) and X != int(X)]
    assert len(horiz) == ny
    assert len(O.interface_points(rho, mid, 3)[0]) < len(px)


@pytest.mark.parametrize("theta", [45.0, 60.0, 90.0, 120.0, 135.0])
def test_contact_angle_of_synthetic_caps(theta):
    """A tanh profile (Eq. 57) around a circle that meets the wall line
    y = -1/2 at angle theta: the measured angle, radius and base chord are the
    construction's to within 0.1 degree / 0.05 lattice spacing (a wall line
    misplaced by half a spacing moves the angle by about 1 degree)."""
    R = 30.0
    c = W.sessile_cap(160, 90, R=R, theta=theta)
    m = O.contact_angle(c.rho, c.rho_l, c.rho_g, skip_rows=3)
    assert abs(m["theta_deg"] - theta) < 0.1, m
    assert abs(m["radius"] - R) < 0.05
    assert abs(m["xc"] - 79.5) < 1e-6        # mirror symmetry about the centre column
    assert abs(m["base_width"] - 2 * R * math.sin(math.radians(theta))) < 0.05
    assert abs(m["height"] - R * (1 - math.cos(math.radians(theta)))) < 0.05


def test_contact_angle_mirror_and_shift():
    """The angle does not depend on where the droplet sits or on a mirror
    image; the centre moves with the droplet."""
    c1 = W.sessile_cap(160, 80, R=25.0, theta=70.0, x0=60.0)
    c2 = W.sessile_cap(160, 80, R=25.0, theta=70.0, x0=97.0)
    m1 = O.contact_angle(c1.rho, c1.rho_l, c1.rho_g)
    m2 = O.contact_angle(c2.rho, c2.rho_l, c2.rho_g)
    m3 = O.contact_angle(c1.rho[:, ::-1], c1.rho_l, c1.rho_g)
    assert abs(m1["theta_deg"] - m2["theta_deg"]) < 1e-9
    assert abs(m2["xc"] - m1["xc"] - 37.0) < 1e-9
    assert abs(m1["theta_deg"] - m3["theta_deg"]) < 1e-9
    assert abs(m3["xc"] - (159 - m1["xc"])) < 1e-9


# ---------------------------------------------------------------------------
# connected regions

def _scipy_label(mask):
    import scipy.ndimage as ndi
    lab, n = ndi.label(mask, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    return lab, n


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_components_match_scipy_labelling(seed):
    """Non-periodic 4-connected regions agree with scipy.ndimage.label as a
    partition; each label is the region's smallest node index; the per-region
    area, row range and edge contacts agree with direct counts."""
    ny, nx = 37, 53
    rho = W.uniform(seed, nx * ny, 0.0, 1.0).reshape(ny, nx)
    for below in (True, False):
        labels, comps = O.components(rho, 0.45, below=below)
        mask = rho < 0.45 if below else rho > 0.45
        ref, n = _scipy_label(mask)
        assert len(comps) == n
        assert np.array_equal(labels < 0, ~mask)
        idx = np.arange(nx * ny).reshape(ny, nx)
        by_label = {c["label"]: c for c in comps}
        for k in range(1, n + 1):
            sel = ref == k
            labs = np.unique(labels[sel])
            assert len(labs) == 1 and labs[0] == idx[sel].min()
            c = by_label[int(labs[0])]
            ys = np.nonzero(sel)[0]
            xs = np.nonzero(sel)[1]
            assert c["area"] == sel.sum() and c["sum_y"] == ys.sum()
            assert c["y_min"] == ys.min() and c["y_max"] == ys.max()
            assert c["touches_w"] == int((xs == 0).any()) and c["touches_e"] == int((xs == nx - 1).any())
            assert c["touches_s"] == int((ys == 0).any()) and c["touches_n"] == int((ys == ny - 1).any())
        assert [c["label"] for c in comps] == sorted(by_label)


def test_components_across_periodic_seams():
    """A bubble cut by the x seam is one region when x is periodic and two
    when it is not; a column of vapour through the y seam joins likewise."""
    nx, ny = 64, 48
    rho, _ = W.bubble_field(nx, ny, [(1.0, 20.0, 6.0), (40.0, 30.0, 5.0)], periodic_x=True)
    thr = 0.5 * sum(W.COEXISTENCE[0.86])
    _, c_per = O.components(rho, thr, periodic_x=True)
    _, c_open = O.components(rho, thr, periodic_x=False)
    assert len(c_per) == 2 and len(c_open) == 3
    seam = [c for c in c_per if c["touches_w"] and c["touches_e"]]
    pieces = [c for c in c_open if c["touches_w"] or c["touches_e"]]
    assert len(seam) == 1 and len(pieces) == 2
    assert seam[0]["area"] == sum(c["area"] for c in pieces)
    # vapour rows at the bottom and top of a y-periodic box: one region
    rho2 = np.full((ny, nx), 6.0)
    rho2[:3, 10:20] = 0.4
    rho2[-2:, 12:15] = 0.4
    _, a = O.components(rho2, thr, periodic_y=True)
    _, b = O.components(rho2, thr, periodic_y=False)
    assert len(a) == 1 and len(b) == 2 and a[0]["area"] == 30 + 6


def test_component_area_gives_departure_diameter():
    """A detached bubble (no node on row 0) and an attached one on the wall:
    the detached one is identified and its equivalent diameter 2 sqrt(A/pi)
    is that of its disc to within the lattice resolution."""
    nx, ny = 120, 120
    R = 12.0
    rho, _ = W.bubble_field(nx, ny, [(60.0, 0.0, 10.0), (60.0, 70.0, R)])
    thr = 0.5 * sum(W.COEXISTENCE[0.86])
    _, comps = O.components(rho, thr, below=True)
    assert len(comps) == 2
    att = [c for c in comps if c["touches_s"]]
    det = [c for c in comps if not c["touches_s"]]
    assert len(att) == 1 and len(det) == 1
    D = 2 * math.sqrt(det[0]["area"] / math.pi)
    assert abs(D - 2 * R) < 1.0
    assert abs(det[0]["sum_y"] / det[0]["area"] - 70.0) < 0.05


# ---------------------------------------------------------------------------
# reconfiguration between steps

def test_reconfigure_equals_a_fresh_start():
    """Relax isothermally (frozen thermal lattice), then switch on heating by
    changing the wall temperature and unfreezing: the continued run equals a
    fresh simulation started from the relaxed populations with the heated
    configuration."""
    c = W.sessile_cap(40, 30, R=10.0, theta=60.0)
    iso = dict(c.params, frozen_thermal=1)
    s = O.Sim(c.nx, c.ny, iso, c.bc)
    s.init(*c.fields())
    g0 = s.populations()[1].copy()
    s.step(15)
    f1, g1, P1 = s.populations()
    assert np.array_equal(g1, g0)           # thermal lattice frozen
    heated = dict(c.bc, T_edge=[0.0, 0.0, 0.95 * W.TC, 0.86 * W.TC])
    s.reconfigure(c.params, heated)
    s.step(10)
    ref = O.Sim(c.nx, c.ny, c.params, heated)
    ref.init(*c.fields())
    ref.set_populations(f1, g1, P1, 15, float(c.rho.mean()))
    ref.step(10)
    for a, b in zip(s.populations(), ref.populations()):
        assert np.array_equal(a, b)


def test_reconfigure_rejects_geometry_changes():
    c = W.sessile_cap(40, 30, R=10.0, theta=60.0)
    s = O.Sim(c.nx, c.ny, c.params, c.bc)
    s.init(*c.fields())
    bad = dict(c.bc, flow=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL])
    with pytest.raises(O.OracleError):
        s.reconfigure(c.params, bad)
    with pytest.raises(O.OracleError):
        s.reconfigure(dict(c.params, w_dot=0.5), c.bc)
