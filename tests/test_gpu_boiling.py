"""Section 4.3 on the GPU: nucleate boiling and bubble departure.  A
300 x 600 pool (periodic sides, no-slip wall at the bottom with a 20-node
heater at 1.1 T_c, the rest of the wall and the open top at T_sat = 0.86 T_c,
contact angle 75 degrees, lambda = 2/3) starts filled with saturated liquid,
as Section 4.3 states.  A bubble grows on the heater and departs; the
departure diameter follows Fritz's D_d ~ g^(-1/2).  The paper's figure is a
placeholder, so the pin is the scaling law: the log-log slope over
g = 1, 2, 4, 8 x 1e-5 lies within 0.15 of -1/2, and every departure is a
single bubble above the heater."""
import pytest

from paper_2205_00686_gb300 import protocols as PR
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def test_departure_diameter_follows_fritz():
    import paper_2205_00686_gb300 as lbm

    def make(g):
        c = W.nucleate_boiling(300, 600, gravity=g, vapour_layer=False)
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        return d

    rg, rl = W.COEXISTENCE[0.86]
    gs = [1e-5, 2e-5, 4e-5, 8e-5]
    out = PR.fritz_sweep(make, gs, rl, rg, check_every=200, max_steps=150000, min_area=8)
    rows = out["runs"]
    for r in rows:
        print("g %.0e: %s %s" % (r["g"], r["departure"], r["error"]))
    assert all(r["departure"] is not None and r["error"] is None for r in rows)
    d = [r["departure"]["diameter"] for r in rows]
    assert all(a > b for a, b in zip(d, d[1:]))           # larger g, smaller bubbles
    assert abs(out["slope"] + 0.5) < 0.15, out["slope"]
    for r in rows:
        reg = r["departure"]["region"]
        assert not reg["touches_s"] and not reg["touches_n"]
