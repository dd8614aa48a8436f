"""Host logic of the wall-experiment protocols (relax to the contact angle,
watch for bubble departure, Fritz sweep) against scripted fake domains; no
GPU."""
import math

import pytest

from paper_2205_00686_gb300 import protocols as PR


class FakeDomain:
    """Scripted stand-in for Domain: angle(step) and regions(step)."""

    def __init__(self, angle=None, regions=None, fail_at=None):
        self.step_count = 0
        self._angle = angle
        self._regions = regions
        self._fail_at = fail_at
        self.reconfigured = None
        self.closed = False

    def step(self, n):
        self.step_count += n
        if self._fail_at is not None and self.step_count >= self._fail_at:
            raise RuntimeError("lbm error -4")

    def contact_angle(self, rho_l, rho_g, skip_rows=3):
        return {"theta_deg": self._angle(self.step_count), "radius": 10.0, "base_width": 1.0,
                "height": 1.0, "xc": 0.0, "yc": 0.0, "n_points": 100}

    def regions(self, thr, below=True):
        return self._regions(self.step_count)

    def reconfigure(self, p, bc):
        self.reconfigured = (p, bc)

    def close(self):
        self.closed = True


def reg(label, area, touches_s, sum_y=None):
    return {"label": label, "area": area, "sum_y": sum_y if sum_y is not None else 10 * area,
            "y_min": 0, "y_max": 5, "touches_w": 0, "touches_e": 0, "touches_s": touches_s,
            "touches_n": 0}


def test_relax_wetting_stops_when_settled():
    d = FakeDomain(angle=lambda s: 60.0 + 30.0 * math.exp(-s / 2000.0))
    h = PR.relax_wetting(d, 6.5, 0.38, check_every=1000, tol_deg=0.05, window=3)
    thetas = [x["theta_deg"] for x in h]
    assert max(thetas[-4:]) - min(thetas[-4:]) < 0.05
    assert max(thetas[-5:]) - min(thetas[-5:]) >= 0.05     # not earlier
    assert h[-1]["step"] == d.step_count == 1000 * len(h)


def test_relax_wetting_respects_max_steps():
    d = FakeDomain(angle=lambda s: 60.0 + math.sin(s))
    h = PR.relax_wetting(d, 6.5, 0.38, check_every=500, max_steps=3000)
    assert d.step_count == 3000 and len(h) == 6


def test_start_heating_unfreezes():
    d = FakeDomain()
    PR.start_heating(d, {"frozen_thermal": 1, "cv": 5.0}, {"flow": [0] * 4})
    assert d.reconfigured[0]["frozen_thermal"] == 0 and d.reconfigured[0]["cv"] == 5.0


def test_watch_departure_finds_first_detached_bubble():
    # a vapour layer at the top (touching the north edge, ignored), a bubble
    # growing on the wall that leaves it at step 1200
    def regions(s):
        top = dict(reg(5000, 900, 0), touches_n=1)
        if s < 1200:
            return [reg(40, 30 + s // 10, 1), top]
        return [reg(40, 3, 1), reg(700, 154, 0, sum_y=154 * 22), top]
    d = FakeDomain(regions=regions)
    res = PR.watch_departure(d, 6.5, 0.38, check_every=200, min_area=8)
    assert res["step"] == 1200
    assert abs(res["diameter"] - 2 * math.sqrt(154 / math.pi)) < 1e-12
    assert res["centroid_y"] == 22.0


def test_watch_departure_min_area_and_timeout():
    d = FakeDomain(regions=lambda s: [reg(40, 50, 1), reg(900, 4, 0) if s >= 400 else reg(41, 1, 1)])
    assert PR.watch_departure(d, 6.5, 0.38, check_every=200, max_steps=2000, min_area=8) is None
    assert d.step_count == 2000


def test_loglog_slope_of_power_law():
    gs = [1e-5, 2e-5, 4e-5, 8e-5]
    assert abs(PR.loglog_slope(gs, [3.0 * g ** -0.5 for g in gs]) + 0.5) < 1e-12
    with pytest.raises(ValueError):
        PR.loglog_slope([1.0], [2.0])


def test_fritz_sweep_collects_departures_and_failures():
    made = []

    def make(g):
        area = int(round(math.pi * (0.05 / math.sqrt(g)) ** 2 / 4))
        if g > 5e-5:
            d = FakeDomain(regions=lambda s: [reg(1, 10, 1)], fail_at=400)
        else:
            d = FakeDomain(regions=lambda s, a=area: [reg(1, 10, 1)] if s < 600 else
                           [reg(1, 2, 1), reg(9, a, 0)])
        made.append(d)
        return d
    out = PR.fritz_sweep(make, [1e-5, 2e-5, 4e-5, 8e-5], 6.5, 0.38, check_every=200,
                         max_steps=2000)
    assert [r["error"] is None for r in out["runs"]] == [True, True, True, False]
    assert all(d.closed for d in made)
    assert abs(out["slope"] + 0.5) < 0.02
