"""Three-dimensional form (D3Q19 MRT flow + D3Q7 thermal lattice) on the
GPU against the 3-D oracle: fields and populations element by element
(FP64 to 1e-10, FP32 to 2e-4 after 1000 steps), walls, buoyancy, frozen
lattices, chunked stepping through the CUDA graph, diagnostics, the sticky
EOS error, and invariants at 256^3."""
import numpy as np
import pytest

import oracle as O
import parity as P
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def with_T_bump(c, amp=0.02, seed=21):
    """Adds a smooth temperature bump and noise so Q, S and grad T act."""
    z, y, x = np.mgrid[0:c.nz, 0:c.ny, 0:c.nx].astype(float)
    bump = np.exp(-((x - 0.3 * c.nx) ** 2 + (y - 0.6 * c.ny) ** 2 + (z - 0.4 * c.nz) ** 2) / 20.0)
    c.T = c.T * (1.0 + amp * bump) + W.noise(seed, c.T.shape, 1e-4 * W.TC)
    return c


def run_both(c, steps, prec, chunks=None, fused=True, zseg=0):
    import paper_2205_00686_gb300 as lbm
    o = O.Sim3(c.nx, c.ny, c.nz, c.params, c.bc)
    o.init(*c.fields())
    o.step(steps)
    d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec=prec)
    d.set_path(fused, zseg)
    d.init_fields(*c.fields())
    for k in (chunks or [steps]):
        d.step(k)
    d.sync()
    return d, o


def fields_err(d, o):
    g = d.get_fields()
    r = o.fields()
    return {k: P.rel_err(a, b) for k, a, b in zip(("rho", "ux", "uy", "uz", "T"), g, r)}


def cases():
    Tc = W.TC
    out = {}
    out["periodic"] = with_T_bump(W.droplet3d(20, 18, 16, R=5.0, amp=1e-3))
    c = with_T_bump(W.droplet3d(16, 14, 20, R=4.5, amp=1e-3, p=W.params(gravity=2e-5)))
    c.bc = W.wall_bc3(0.95 * Tc, 0.88 * Tc, theta_deg=65.0)
    out["walls_dirichlet_gravity"] = c
    c = with_T_bump(W.sessile3d(18, 16, 14, R=6.0, theta=110.0, amp=1e-3))
    c.bc = W.wall_bc3(0.9 * Tc, 0.0, theta_deg=110.0, adiabatic=(False, True))
    out["sessile_adiabatic_top"] = c
    return out


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "three_kernels"])
@pytest.mark.parametrize("name", ["periodic", "walls_dirichlet_gravity", "sessile_adiabatic_top"])
def test_fp64_matches_oracle(name, fused):
    c = cases()[name]
    d, o = run_both(c, 200, "fp64", fused=fused, zseg=7 if fused else 0)
    fe = fields_err(d, o)
    assert max(fe.values()) <= 1e-10, (name, fe)
    gf, gg, gP = d.populations()
    of, og, oP = o.populations()
    assert P.rel_err(gf, of) <= 1e-12 and P.rel_err(gg, og) <= 1e-12, name
    assert np.abs(gP - oP).max() <= 1e-10 * max(np.abs(oP).max(), 1e-30)
    d.close()


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "three_kernels"])
def test_fp32_matches_oracle_after_1000_steps(fused):
    c = with_T_bump(W.droplet3d(14, 14, 20, R=4.5, amp=1e-3, p=W.params(gravity=1e-5)))
    c.bc = W.wall_bc3(0.9 * W.TC, 0.86 * W.TC, theta_deg=80.0)
    d, o = run_both(c, 1000, "fp32", fused=fused)
    fe = fields_err(d, o)
    assert max(fe.values()) <= 2e-4, fe
    d.close()


def test_chunked_steps_equal_one_call():
    """7 + 45 + 1 steps (single launches, then the 32-step graph and the
    rest) give the bit-identical state of one 53-step call."""
    import paper_2205_00686_gb300 as lbm
    c = cases()["walls_dirichlet_gravity"]
    out = []
    for chunks in ([53], [7, 45, 1]):
        d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        for k in chunks:
            d.step(k)
        out.append(d.populations())
        assert d.step_count == 53
        d.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("frozen", ["frozen_flow", "frozen_thermal"])
def test_frozen_lattices_match_oracle(frozen):
    c = cases()["walls_dirichlet_gravity"]
    c.params = dict(c.params, **{frozen: 1})
    d, o = run_both(c, 60, "fp64")
    fe = fields_err(d, o)
    assert max(fe.values()) <= 1e-10, fe
    if frozen == "frozen_thermal":
        T = d.get_fields()[4]
        assert np.abs(T - c.T).max() < 1e-12
    d.close()


def test_diagnostics_match_oracle():
    c = cases()["sessile_adiabatic_top"]
    d, o = run_both(c, 50, "fp64")
    a = d.diagnostics(c.rho_l, c.rho_g, sessile=True)
    b = o.diagnostics(c.rho_l, c.rho_g, sessile=True)
    for k in ("mass", "energy", "liquid_mass", "liquid_area_smooth", "max_u", "diameter_smooth"):
        assert abs(a[k] - b[k]) <= 1e-10 * max(abs(b[k]), 1e-30), (k, a[k], b[k])
    assert a["liquid_area"] == b["liquid_area"] and a["step"] == 50
    d.close()


def test_psi_error_is_sticky_not_a_fault():
    import paper_2205_00686_gb300 as lbm
    c = W.droplet3d(12, 12, 12, R=3.0)
    rho = c.rho.copy()
    rho[6, 6, 6] = 9.7
    d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec="fp32")
    with pytest.raises(lbm.LbmError) as ei:
        d.init_fields(rho, c.ux, c.uy, c.uz, c.T)
    assert ei.value.code == lbm.LBM_EPSI
    d.init_fields(*c.fields())       # clears the error
    d.step(3)
    assert d.sync() == 0
    d.close()


def test_invariants_at_256_cubed():
    """FP32, 256^3: the benchmark's cloud of 64 droplets (thermal lattice
    running) and one isothermal droplet of radius 64.  After 200 steps the
    state is finite, mass is conserved to 1e-5 and the total momentum (zero by
    the pair antisymmetry of F_m) stays below 1e-4 of the summed momentum
    magnitude."""
    import paper_2205_00686_gb300 as lbm
    n = 256
    for c in (W.droplet_cloud3d(n),
              W.droplet3d(n, n, n, R=64.0, amp=1e-4, p=W.params(frozen_thermal=1))):
        d = lbm.Domain3(n, n, n, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        m0 = d.diagnostics(c.rho_l, c.rho_g)["mass"]
        d.step(200)
        dg = d.diagnostics(c.rho_l, c.rho_g)
        assert dg["nonfinite"] == 0, c.name
        assert abs(dg["mass"] - m0) <= 1e-5 * m0, c.name
        rho, ux, uy, uz, _ = d.get_fields()
        for u in (ux, uy, uz):
            assert abs((rho * u).sum()) <= 1e-4 * np.abs(rho * u).sum(), c.name
        d.close()


@pytest.mark.parametrize("zseg", [0, 16])
@pytest.mark.parametrize("walls", [False, True])
def test_multi_block_domain_matches_oracle(walls, zseg):
    """A domain of several tiles with ragged x and y edges (45 x 9: three 16 x
    16 tiles, the last 13 wide, all cut at y = 9) and 70 planes, periodic z
    and between walls, against the oracle in FP64 after 30 steps; zseg 16
    cuts z into segments of 16 planes and a ragged one of 6."""
    Tc = W.TC
    c = with_T_bump(W.droplet3d(45, 9, 70, R=6.0, amp=1e-3, p=W.params(gravity=2e-5)))
    if walls:
        c.bc = W.wall_bc3(0.95 * Tc, 0.88 * Tc, theta_deg=70.0)
    d, o = run_both(c, 30, "fp64", zseg=zseg)
    e = fields_err(d, o)
    assert max(e.values()) <= 1e-10, e
    gf, gg, gP = d.populations()
    of, og, oP = o.populations()
    assert P.rel_err(gf, of) <= 1e-12 and P.rel_err(gg, og) <= 1e-12
    d.close()


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("zseg", [1, 2, 3])
def test_domain_smaller_than_a_tile(walls, zseg):
    """5 x 3 x 7 nodes inside one 16 x 16 tile (the tile's halos wrap several
    times around x and y) with segments of 1, 2 and 3 planes, against the
    oracle in FP64 after 25 steps."""
    Tc = W.TC
    c = with_T_bump(W.droplet3d(5, 3, 7, R=1.5, amp=1e-3, p=W.params(gravity=2e-5)))
    if walls:
        c.bc = W.wall_bc3(0.93 * Tc, 0.9 * Tc, theta_deg=75.0, adiabatic=(True, False))
    d, o = run_both(c, 25, "fp64", zseg=zseg)
    e = fields_err(d, o)
    assert max(e.values()) <= 1e-10, e
    gf, gg, gP = d.populations()
    of, og, oP = o.populations()
    assert P.rel_err(gf, of) <= 1e-12 and P.rel_err(gg, og) <= 1e-12
    d.close()


def test_switching_paths_mid_run_matches_oracle():
    """Fused, three-kernel and fused steps again (12 + 9 + 14) continue one
    another: the per-node planes and the density ring are handed over."""
    import paper_2205_00686_gb300 as lbm
    c = cases()["walls_dirichlet_gravity"]
    o = O.Sim3(c.nx, c.ny, c.nz, c.params, c.bc)
    o.init(*c.fields())
    o.step(35)
    d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec="fp64")
    d.init_fields(*c.fields())
    for fused, n in ((True, 12), (False, 9), (True, 14)):
        d.set_path(fused, 5)
        assert d.path == (fused, 5)
        d.step(n)
    e = fields_err(d, o)
    assert max(e.values()) <= 1e-10, e
    d.close()


def test_fused_fp32_equals_itself_for_any_segment_length():
    """In FP32 the segment length changes only which CTA computes a node,
    never its arithmetic: without buoyancy (whose density sum is rounded per
    CTA) the populations are bitwise equal for zseg 5, 16 and the whole
    column, walls and wetting included."""
    import paper_2205_00686_gb300 as lbm
    c = cases()["sessile_adiabatic_top"]
    assert float(c.params.get("gravity", 0.0)) == 0.0
    out = []
    for zs in (5, 16, c.nz):
        d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec="fp32")
        d.set_path(True, zs)
        d.init_fields(*c.fields())
        d.step(40)
        out.append(d.populations())
        d.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "three_kernels"])
@pytest.mark.parametrize("shape", [(20, 1, 1), (1, 18, 1), (1, 1, 24), (12, 9, 1), (1, 7, 11)])
def test_thin_domains_match_oracle(shape, fused):
    """Domains one node thick along one or two axes (every neighbour along
    those axes is the node itself, and a 16 x 16 tile wraps many times onto
    the domain): a uniform vapour-like state with density and temperature
    noise and a small velocity, periodic, FP64 against the oracle after 20
    steps."""
    import paper_2205_00686_gb300 as lbm
    nx, ny, nz = shape
    p = W.params()
    sh = (nz, ny, nx)
    rho = 0.3 * (1.0 + W.noise(3, sh, 1e-3))
    T = 0.95 * W.TC * (1.0 + W.noise(4, sh, 1e-3))
    u = [W.noise(5 + i, sh, 1e-3) for i in range(3)]
    o = O.Sim3(nx, ny, nz, p, W.periodic_bc3())
    o.init(rho, *u, T)
    o.step(20)
    d = lbm.Domain3(nx, ny, nz, p, W.periodic_bc3(), prec="fp64")
    d.set_path(fused, 0)
    d.init_fields(rho, *u, T)
    d.step(20)
    e = fields_err(d, o)
    assert max(e.values()) <= 1e-10, e
    gf, gg, gP = d.populations()
    of, og, oP = o.populations()
    assert P.rel_err(gf, of) <= 1e-12 and P.rel_err(gg, og) <= 1e-12
    d.close()


def test_set_path_refuses_a_negative_segment():
    import paper_2205_00686_gb300 as lbm
    c = cases()["periodic"]
    d = lbm.Domain3(c.nx, c.ny, c.nz, c.params, c.bc, prec="fp32")
    with pytest.raises(lbm.LbmError):
        d.set_path(True, -1)
    d.set_path(True, 10 ** 6)            # clamped to the domain's planes
    assert d.path == (True, c.nz)
    d.close()


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "three_kernels"])
@pytest.mark.parametrize("walls", [False, True])
def test_two_planes_deep(walls, fused):
    """nz = 2: between walls both planes touch a wall (each node's +z and -z
    neighbours are the ghost layer or the other plane); periodic, each plane
    is the other's neighbour on both sides.  FP64 against the oracle after
    25 steps."""
    import paper_2205_00686_gb300 as lbm
    nx, ny, nz = 9, 7, 2
    Tc = W.TC
    sh = (nz, ny, nx)
    p = W.params(gravity=1e-5)
    rho = 0.3 * (1.0 + W.noise(6, sh, 1e-3))
    T = 0.92 * Tc * (1.0 + W.noise(7, sh, 1e-3))
    u = [W.noise(8 + i, sh, 1e-3) for i in range(3)]
    bc = W.wall_bc3(0.93 * Tc, 0.9 * Tc, theta_deg=70.0) if walls else W.periodic_bc3()
    o = O.Sim3(nx, ny, nz, p, bc)
    o.init(rho, *u, T)
    o.step(25)
    d = lbm.Domain3(nx, ny, nz, p, bc, prec="fp64")
    d.set_path(fused, 0)
    d.init_fields(rho, *u, T)
    d.step(25)
    e = fields_err(d, o)
    assert max(e.values()) <= 1e-10, e
    gf, gg, gP = d.populations()
    of, og, oP = o.populations()
    assert P.rel_err(gf, of) <= 1e-12 and P.rel_err(gg, og) <= 1e-12
    d.close()
