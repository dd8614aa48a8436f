"""One domain split into slabs of rows on one GPU (halo rows exchanged by
device copies, density sums combined for the buoyancy mean): the split
gives the whole domain's result.  FP64 against the oracle of the whole
domain element by element; FP32 against one whole-domain context on the
same tile, bit for bit."""
import numpy as np
import pytest

import parity as P
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,n_slabs,ghost,gravity", [
    ("wall_open_heater", 2, 3, 3e-5),      # buoyancy: slabs step one at a time
    ("two_walls_adiabatic", 3, 3, 2e-5),
    ("periodic", 2, 6, 0.0),               # periodic y: the halos wrap; two steps per exchange
    ("open_dirichlet", 3, 9, 0.0),
    ("periodic_x_open_y", 4, 3, 0.0),
])
def test_slabs_match_the_oracle_fp64(name, n_slabs, ghost, gravity):
    from paper_2205_00686_gb300.slabs import SlabRunner
    c = P.droplet_case(90, 64, P.bc_variants()[name], seed=17, gravity=gravity)
    r = SlabRunner(c.nx, c.ny, c.params, c.bc, n_slabs, prec="fp64", ghost=ghost)
    r.init_fields(*c.fields())
    r.step(7)
    r.step(53)
    o = P.run_oracle(c, 60)
    fe = P.field_errors(r.get_rho_u_T(), o.fields())
    assert max(fe.values()) <= 1e-12, (name, fe)
    f, g, _ = r.populations()
    of, og, _ = o.populations()
    assert P.rel_err(f, of) <= 1e-12 and P.rel_err(g, og) <= 1e-12
    r.close()


def test_periodic_flow_with_held_temperature_is_refused():
    """Section 4.1's box (flow periodic in y, temperature held at the y
    edges) cannot be cut into y-slabs: the wrapped flow halo would have to
    carry the thermal edge inside a slab."""
    from paper_2205_00686_gb300.slabs import SlabRunner
    c = P.droplet_case(64, 64, P.bc_variants()["periodic_flow_fixed_T"])
    with pytest.raises(ValueError):
        SlabRunner(c.nx, c.ny, c.params, c.bc, 2)


def test_slabs_equal_the_whole_domain_fp32_bitwise():
    """Without buoyancy a node's arithmetic does not depend on which context
    computes it: on the same tile and load path the two slabs' own rows equal
    the whole domain's, bit for bit."""
    import paper_2205_00686_gb300 as lbm
    from paper_2205_00686_gb300.slabs import SlabRunner
    c = P.droplet_case(216, 120, P.bc_variants()["open_x_periodic_y"], seed=19)
    r = SlabRunner(c.nx, c.ny, c.params, c.bc, 2, prec="fp32", ghost=6)
    r.init_fields(*c.fields())
    r.set_tile(128, 32, staged=False)
    r.step(80)
    # the same storage references as the slabs
    p = dict(c.params, rho_ref=float(c.rho.mean()), T_ref=float(c.T.mean()))
    d = lbm.Domain(c.nx, c.ny, p, c.bc, prec="fp32")
    d.set_tile(128, 32)
    d.staged = False
    d.init_fields(*c.fields())
    d.step(80)
    for a, b in zip(r.populations(), d.populations()):
        assert np.array_equal(a, b)
    r.close()
    d.close()
