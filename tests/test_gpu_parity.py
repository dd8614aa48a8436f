"""GPU (sm_103a) parity of the fused step against the FP64 CPU oracle, through
the C ABI.  Tolerances: max relative field error <= 1e-10 for FP64 and
<= 2e-4 for FP32 after 1000 steps of the 64x64 droplet; the FP16-storage
variant's error is reported and bounded loosely (its storage rounding is
2^-11 of the deviation from the reference temperature)."""
import numpy as np
import pytest

import parity as P
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def test_static_droplet_64_fp64_1000_steps():
    c = W.static_droplet()
    fe, pe, g, o = P.compare(c, 1000, "fp64")
    print("fp64 64x64 1000 steps", fe, pe)
    assert max(fe.values()) <= TOL64
    assert max(pe.values()) <= TOL64


def test_static_droplet_64_fp32_1000_steps():
    c = W.static_droplet()
    fe, pe, g, o = P.compare(c, 1000, "fp32")
    print("fp32 64x64 1000 steps", fe, pe)
    assert max(fe.values()) <= TOL32


def test_static_droplet_64_g16_1000_steps():
    c = W.static_droplet()
    fe, pe, g, o = P.compare(c, 1000, "fp32_g16")
    print("fp32+fp16-g 64x64 1000 steps", fe, pe)
    assert fe["rho"] <= 1e-3 and fe["T"] <= 1e-3


@pytest.mark.parametrize("name", list(P.bc_variants()))
@pytest.mark.parametrize("size", [(8, 8), (17, 13)])
def test_tiny_domains_every_boundary_fp64(name, size):
    bc = P.bc_variants()[name]
    c = P.droplet_case(size[0], size[1], bc, gravity=2e-5)
    fe, pe, g, o = P.compare(c, 50, "fp64")
    assert max(fe.values()) <= 1e-12, (name, fe)
    assert max(pe.values()) <= 1e-12, (name, pe)


@pytest.mark.parametrize("name", ["periodic", "wall_open_heater", "open_x_walls_y",
                                  "periodic_flow_fixed_T"])
@pytest.mark.parametrize("tile", [(128, 16), (256, 7), (128, 75)])
def test_ragged_multi_tile_fp64(name, tile):
    """250 x 75 spans several strips and segments with ragged tails."""
    bc = P.bc_variants()[name]
    c = P.droplet_case(250, 75, bc, gravity=3e-5)
    fe, pe, g, o = P.compare(c, 120, "fp64", tile=tile, chunks=[1, 40, 79])
    assert max(fe.values()) <= 1e-11, (name, tile, fe)
    assert max(pe.values()) <= 1e-11, (name, tile, pe)


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-4), ("fp32_g16", 2e-3)])
@pytest.mark.parametrize("name", ["open_dirichlet", "wall_open_heater"])
@pytest.mark.parametrize("tile", [None, (256, 40)])
def test_ragged_multi_tile_reduced_precision(prec, tol, name, tile):
    c = P.droplet_case(600, 75, P.bc_variants()[name], gravity=3e-5)
    fe, pe, g, o = P.compare(c, 200, prec, tile=tile)
    print(prec, name, fe)
    assert fe["rho"] <= tol and fe["T"] <= tol


@pytest.mark.parametrize("case_fn,steps", [
    (lambda: W.open_evaporation(256, 256, steps=0), 200),
    (lambda: W.heated_surface(400, 200, steps=0), 100),
    (lambda: W.nucleate_boiling(300, 600, gravity=2e-5, steps=0), 60),
    (lambda: W.d2_droplet(200, steps=0), 200),
])
def test_workload_shapes_fp64(case_fn, steps):
    c = case_fn()
    fe, pe, g, o = P.compare(c, steps, "fp64")
    print(c.name, fe)
    assert max(fe.values()) <= TOL64


def test_graph_replay_matches_single_launches():
    """lbm_step(n >= 32) replays a captured CUDA graph; the result must be
    bitwise the same as n single launches."""
    import paper_2205_00686_gb300 as lbm
    c = P.droplet_case(130, 70, P.bc_variants()["wall_open_heater"], gravity=2e-5)
    a = P.run_gpu(c, 70, "fp32")
    b = P.run_gpu(c, 70, "fp32", chunks=[1] * 70)
    fa, ga, Pa = a.populations()
    fb, gb, Pb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    del lbm


def test_tiles_give_identical_results():
    """The segment height never changes the arithmetic of a node: results are
    bitwise equal for one kernel instantiation.  The 128- and 256-thread
    instantiations are compiled separately (the compiler may contract
    multiply-adds differently), so across them the results agree to FP32
    rounding."""
    c = P.droplet_case(300, 90, P.bc_variants()["open_dirichlet"])
    ref = {}
    for tile in [(128, 16), (128, 90), (128, 7), (256, 33), (256, 8), (256, 90)]:
        d = P.run_gpu(c, 40, "fp32", tile=tile)
        f, g, _ = d.populations()
        if tile[0] not in ref:
            ref[tile[0]] = (f, g)
        else:
            r = ref[tile[0]]
            assert np.array_equal(r[0], f) and np.array_equal(r[1], g), tile
    for th in (256,):
        assert P.rel_err(ref[128][0], ref[th][0]) < 1e-6
        assert P.rel_err(ref[128][1], ref[th][1]) < 1e-6


@pytest.mark.parametrize("prec", ["fp32", "fp32_g16"])
@pytest.mark.parametrize("name", ["periodic", "open_dirichlet", "wall_open_heater",
                                  "two_walls_adiabatic", "open_x_walls_y", "periodic_x_open_y",
                                  "open_x_periodic_y", "periodic_flow_fixed_T"])
@pytest.mark.parametrize("size", [(36, 20), (64, 48), (250, 75), (200, 40), (17, 13)])
def test_staged_rows_equal_register_rows(name, size, prec):
    """The step with its rows staged in shared memory by bulk copies does the
    same arithmetic as the register-prefetch form: in FP32 the populations
    are equal bit for bit (g*_0, which the staged form hands to stage D5 in a
    register, is an unfused product in both forms); with FP16 storage of g
    they agree to the FP16 rounding of a stored g.  This holds on single and
    multi-strip domains, ragged tails, windows that wrap several times around
    a periodic axis, and every boundary kind.  Sizes the staged form cannot
    take (periodic x with nx not a multiple of 4, or of 8 for FP16 g) are
    refused with LBM_EINVAL and keep the register form."""
    import paper_2205_00686_gb300 as lbm
    bc = P.bc_variants()[name]
    c = P.droplet_case(size[0], size[1], bc, gravity=2e-5)
    perx = bc["flow"][0] == W.PERIODIC
    if perx and size[0] % (8 if prec == "fp32_g16" else 4):
        d = P.run_gpu(c, 0, prec)
        assert not d.staged
        with pytest.raises(lbm.LbmError) as e:
            d.staged = True
        assert e.value.code == lbm.LBM_EINVAL
        return
    tol = 2e-3
    for tile in [None, (192, 10), (224, 13), (256, 11)]:
        a = P.run_gpu(c, 60, prec, tile=tile, staged=True, chunks=[1, 59])
        b = P.run_gpu(c, 60, prec, tile=tile, staged=False, chunks=[1, 59])
        assert a.staged and not b.staged
        fa, ga, Pa = a.populations()
        fb, gb, Pb = b.populations()
        assert np.isfinite(fa).all() and np.isfinite(ga).all()
        if prec == "fp32":
            assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (name, size, tile)
            assert np.array_equal(Pa, Pb), (name, size, tile)
        else:
            assert P.rel_err(fa, fb) < tol and P.rel_err(ga, gb) < tol, (name, size, tile)
            assert P.rel_err(Pa, Pb) < 10 * tol, (name, size, tile)


def test_staged_rows_match_oracle_g16_1000_steps():
    """The staged FP16-g path against the FP64 oracle on the 64 x 64 droplet
    (its FP16 storage error is bounded as for the register form)."""
    c = W.static_droplet()
    o = P.run_oracle(c, 1000)
    g = P.run_gpu(c, 1000, "fp32_g16", staged=True)
    assert g.staged
    fe = P.field_errors(g.get_rho_u_T(), o.fields())
    assert fe["rho"] <= 1e-3 and fe["T"] <= 1e-3, fe


def test_staged_rows_match_oracle_fp32_1000_steps():
    """The staged FP32 path against the FP64 oracle on the 64 x 64 droplet
    (periodic, nx a multiple of 4) and a 250 x 75 open-x case, 1000 steps."""
    c = W.static_droplet()
    o = P.run_oracle(c, 1000)
    g = P.run_gpu(c, 1000, "fp32", staged=True)
    assert g.staged
    fe = P.field_errors(g.get_rho_u_T(), o.fields())
    assert max(fe.values()) <= TOL32, fe
    c = P.droplet_case(250, 75, P.bc_variants()["open_dirichlet"], gravity=3e-5)
    o = P.run_oracle(c, 300)
    g = P.run_gpu(c, 300, "fp32", staged=True)
    assert g.staged
    fe = P.field_errors(g.get_rho_u_T(), o.fields())
    assert fe["rho"] <= TOL32 and fe["T"] <= TOL32, fe


def test_diagnostics_match_oracle():
    c = W.open_evaporation(96, 96, R=24)
    o = P.run_oracle(c, 100)
    g = P.run_gpu(c, 100, "fp64")
    do = o.diagnostics(c.rho_l, c.rho_g)
    dg = g.diagnostics(c.rho_l, c.rho_g)
    for k in ("mass", "energy", "liquid_mass", "liquid_area", "liquid_area_smooth",
              "diameter", "max_u"):
        assert abs(dg[k] - do[k]) <= 1e-10 * max(1.0, abs(do[k])), (k, dg[k], do[k])
    assert dg["nonfinite"] == 0 and dg["step"] == 100


def test_set_populations_roundtrip_and_continue():
    """State handed over mid-run from the oracle continues identically."""
    c = P.droplet_case(60, 40, P.bc_variants()["wall_open_heater"], gravity=2e-5)
    o = P.run_oracle(c, 30)
    f, g, Pp = o.populations()
    import paper_2205_00686_gb300 as lbm
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp64")
    # the buoyancy force of step 30 uses the mean density of step 29
    o2 = P.run_oracle(c, 29)
    rho_ave = o2.fields()[0].mean()
    d.set_populations(f, g, Pp, 30, rho_ave)
    gf, gg, gP = d.populations()
    assert P.rel_err(gf, f) < 1e-15 and P.rel_err(gg, g) < 1e-15
    d.step(20)
    o.step(20)
    fe = P.field_errors(d.get_rho_u_T(), o.fields())
    assert max(fe.values()) <= 1e-11, fe


def test_checkpoint_roundtrip_is_bitwise(tmp_path):
    c = P.droplet_case(70, 50, P.bc_variants()["wall_open_heater"], gravity=2e-5)
    a = P.run_gpu(c, 40, "fp32")
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(25)
    fa, ga, _ = a.populations()
    import paper_2205_00686_gb300 as lbm
    b = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    b.load(path)
    assert b.step_count == 40
    b.step(25)
    fb, gb, _ = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_psi_error_is_reported_not_faulted():
    """A density beyond the EOS range gives psi^2 < 0: the kernel flags it and
    the next synchronising call returns LBM_EPSI."""
    import paper_2205_00686_gb300 as lbm
    c = W.static_droplet(32, 32, R=8, amp=0.0)
    rho = c.rho.copy()
    rho[10, 10] = 9.6
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    d.init_fields(rho, c.ux, c.uy, c.T)
    d.step(1)
    with pytest.raises(lbm.LbmError) as ei:
        d.sync()
    assert ei.value.code == lbm.LBM_EPSI
    with pytest.raises(lbm.LbmError):
        d.step(1)
    d.init_fields(*c.fields())      # clears the sticky error
    d.step(2)
    assert d.sync() == 0


def test_invalid_arguments_rejected():
    import paper_2205_00686_gb300 as lbm
    bad = W.bc_spec([W.WALL, W.WALL, W.PERIODIC, W.PERIODIC], [1, 1, 0, 0])
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Domain(16, 16, W.params(), bad)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.Domain(0, 16, W.params(), W.periodic_bc())
    with pytest.raises(lbm.LbmError):
        lbm.Domain(16, 16, W.params(w_dot=1.5), W.periodic_bc())
    d = lbm.Domain(16, 16, W.params(), W.periodic_bc())
    with pytest.raises(lbm.LbmError) as ei:
        d.step(1)     # before init
    assert ei.value.code == lbm.LBM_ESTATE


def test_full_size_one_launch_matches_oracle():
    """4096 x 4096 in the benchmark's launch configuration: two steps against
    the oracle on every node."""
    c = W.open_evaporation(4096, 4096, R=640.0, steps=0)
    fe, pe, g, o = P.compare(c, 2, "fp32")
    print("4096^2 fp32 2 steps", fe, pe)
    assert max(fe.values()) <= 1e-5


def test_full_size_mass_conserved_fp32():
    """Periodic 4096 x 4096: sum rho is invariant (any size); FP32 storage
    keeps it to 1e-5 relative over 500 steps."""
    import paper_2205_00686_gb300 as lbm
    c = W.static_droplet(4096, 4096, R=1024.0, steps=0)
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    d.init_fields(*c.fields())
    m0 = d.diagnostics(c.rho_l, c.rho_g)["mass"]
    d.step(500)
    m1 = d.diagnostics(c.rho_l, c.rho_g)["mass"]
    assert abs(m1 - m0) <= 1e-5 * m0


def test_staged_wait_timeout_is_reported_not_hung():
    """Failure detection of the staged path without a GPU fault: with the test
    hook on, every CTA also waits on an mbarrier that nothing arms.  The wait
    is bounded (about a second), the launch ends, LBM_ETIMEOUT is reported
    through the sticky error word, the step's populations equal a normal
    step's (the row pipeline kept its own waits), and after lbm_init_fields
    the context steps normally again."""
    import time

    import paper_2205_00686_gb300 as lbm
    c = W.static_droplet()
    ref = P.run_gpu(c, 1, "fp32", staged=True)
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    d.staged = True
    d.init_fields(*c.fields())
    d.set_wait_probe(True)
    t0 = time.perf_counter()
    d.step(1)
    with pytest.raises(lbm.LbmError) as e:
        d.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the readback still copies the state, then reports the sticky error
    f = np.empty((9, c.ny, c.nx))
    g = np.empty((5, c.ny, c.nx))
    Pp = np.empty((c.ny, c.nx))
    rc = lbm.lib().lbm_get_populations(d.handle, *[lbm._ptr(a) for a in (f, g, Pp)])
    assert rc == lbm.LBM_ETIMEOUT
    for a, b in zip((f, g, Pp), ref.populations()):
        assert np.array_equal(a, b)
    d.set_wait_probe(False)
    d.init_fields(*c.fields())
    d.step(5)
    d.sync()
    assert d.step_count == 5


def test_autotune_keeps_state_and_picks_a_valid_tile():
    """lbm_autotune times load paths x threads x rows (powers of two and the
    heights that fill the grid in whole waves) on a scratch domain: the
    caller's state is untouched, the chosen tile is one of the candidates,
    and a fresh domain of the same size starts with the cached choice."""
    import paper_2205_00686_gb300 as lbm
    c = P.droplet_case(600, 130, P.bc_variants()["open_dirichlet"])
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    d.init_fields(*c.fields())
    d.step(7)
    before = d.populations()
    threads, rows = d.autotune(3)
    assert threads in (128, 192, 224, 256) and 1 <= rows <= c.ny
    for a, b in zip(d.populations(), before):
        assert np.array_equal(a, b)
    assert d.step_count == 7
    e = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    assert e.tile() == (threads, rows) and e.staged == d.staged
    d.step(5)
    d.sync()


def test_largest_accepted_domain_steps():
    """The largest square FP32 domain lbm_create accepts (15424^2: the nine f
    planes stay below 2^31 elements, 28 GB of state) steps in the default
    staged launch: a uniform state is a fixed point of the step (every unit
    of the persistent grid ran; nothing was read out of place), and the mass
    is unchanged."""
    import paper_2205_00686_gb300 as lbm
    n = 15424
    Tr = 0.86
    rg, rl = W.COEXISTENCE[Tr]
    d = lbm.Domain(n, n, W.params(), W.periodic_bc(), prec="fp32")
    assert d.staged
    rho = np.full((n, n), rg)
    z = np.zeros((n, n))
    d.init_fields(rho, z, z, np.full((n, n), Tr * W.TC))
    del rho
    m0 = d.diagnostics(rl, rg)["mass"]
    d.step(3)
    dg = d.diagnostics(rl, rg)
    assert dg["nonfinite"] == 0 and dg["max_u"] < 1e-6
    assert abs(dg["mass"] - m0) <= 1e-6 * m0
    d.close()
