"""Batched stepping (one persistent launch per step over a work list of
(domain, strip, segment) units from many domains): every domain's result must
be the one it gets alone."""
import numpy as np
import pytest

import parity as P
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def mixed_cases(gravity=0.0):
    v = P.bc_variants()
    specs = [(64, 64, "periodic"), (100, 80, "open_dirichlet"), (257, 129, "wall_open_heater"),
             (33, 47, "two_walls_adiabatic"), (512, 64, "periodic_x_open_y"),
             (130, 200, "open_x_walls_y"), (17, 13, "open_x_periodic_y")]
    return [P.droplet_case(nx, ny, v[name], seed=11 + i, gravity=gravity)
            for i, (nx, ny, name) in enumerate(specs)]


def solo(case, steps, prec):
    return P.run_gpu(case, steps, prec).populations()


def test_batch_matches_solo_bitwise():
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases()
    b = lbm.Batch()
    doms = []
    for c in cases:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    assert len(b) == len(cases)
    b.step(60)
    assert b.sync() == 0
    for c, d in zip(cases, doms):
        b.detach(d)
        f, g, Pp = d.populations()
        fs, gs, Ps = solo(c, 60, "fp32")
        assert np.array_equal(f, fs) and np.array_equal(g, gs) and np.array_equal(Pp, Ps), c.name
        assert d.step_count == 60
    b.close()


def test_attach_and_detach_mid_run():
    """Domains join and leave between launches; each keeps its own step
    counter, ping-pong parity and d_t^2 T history."""
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases()[:3]
    b = lbm.Batch()
    d = [lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32") for c in cases]
    for x, c in zip(d, cases):
        x.init_fields(*c.fields())
    b.attach(d[0])
    b.step(31)                  # d0 at 31 (odd parity)
    b.attach(d[1])
    b.step(20)                  # d0 51, d1 20
    b.detach(d[0])
    b.attach(d[2])
    b.step(45)                  # d1 65, d2 45 (graph replay path)
    b.detach(d[1])
    b.detach(d[2])
    d[0].step(9)                # continue alone: 60
    for x, c, n in zip(d, cases, (60, 65, 45)):
        f, g, _ = x.populations()
        fs, gs, _ = solo(c, n, "fp32")
        assert x.step_count == n
        assert np.array_equal(f, fs) and np.array_equal(g, gs), c.name
    b.close()


def test_batch_fp64_with_gravity_matches_oracle():
    """Each domain keeps its own buoyancy density history in the batch."""
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases(gravity=3e-5)[1:4]
    b = lbm.Batch()
    doms = []
    for c in cases:
        x = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp64")
        x.init_fields(*c.fields())
        b.attach(x)
        doms.append(x)
    b.step(40)
    assert b.sync() == 0
    for c, x in zip(cases, doms):
        o = P.run_oracle(c, 40)
        fe = P.field_errors(x.get_rho_u_T(), o.fields())
        assert max(fe.values()) <= 1e-12, (c.name, fe)
    b.close()


def test_poisoned_domain_fails_alone():
    """A domain that goes out of the EOS range flags only itself; after it
    is detached the others continue exactly as they would alone."""
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases()[:4]
    bad = 2
    b = lbm.Batch()
    doms = []
    for i, c in enumerate(cases):
        x = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        rho = c.rho.copy()
        if i == bad:
            rho[c.ny // 2, c.nx // 2] = 9.7       # psi^2 < 0 there
        x.init_fields(rho, c.ux, c.uy, c.T)
        b.attach(x)
        doms.append(x)
    b.step(3)
    assert b.sync() == lbm.LBM_EPSI
    with pytest.raises(lbm.LbmError) as ei:
        doms[bad].sync()
    assert ei.value.code == lbm.LBM_EPSI
    b.detach(doms[bad])
    b.step(27)
    assert b.sync() == 0
    for i, (c, x) in enumerate(zip(cases, doms)):
        if i == bad:
            continue
        assert x.sync() == 0
        f, g, _ = x.populations()
        fs, gs, _ = solo(c, 30, "fp32")
        assert np.array_equal(f, fs) and np.array_equal(g, gs), c.name
    b.close()


def test_batch_rejects_mixed_physics():
    import paper_2205_00686_gb300 as lbm
    c = mixed_cases()[0]
    b = lbm.Batch()
    x = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    x.init_fields(*c.fields())
    y = lbm.Domain(c.nx, c.ny, W.params(lambda_=0.2), c.bc, prec="fp32")
    y.init_fields(*c.fields())
    z = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp64")
    z.init_fields(*c.fields())
    b.attach(x)
    with pytest.raises(lbm.LbmError):
        b.attach(y)
    with pytest.raises(lbm.LbmError):
        b.attach(z)
    with pytest.raises(lbm.LbmError) as ei:
        x.step(1)                 # attached: the batch owns its stepping
    assert ei.value.code == lbm.LBM_ESTATE
    b.close()


def test_batched_population_sample_matches_oracle():
    """The batched population (512 open-evaporation domains, sides 64-512):
    a seeded sample of 16 of them advanced together in one FP64 batch for
    60 steps equals the oracle run of each, element by element."""
    import paper_2205_00686_gb300 as lbm
    pop = W.batch_instances()
    idx = sorted(int(i) for i in np.argsort(W.uniform(99, len(pop)))[:16])
    sample = [pop[i] for i in idx]
    b = lbm.Batch()
    doms = []
    for c in sample:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp64")
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    b.step(60)
    assert b.sync() == 0
    for c, d in zip(sample, doms):
        b.detach(d)
        o = P.run_oracle(c, 60)
        fe = P.field_errors(d.get_rho_u_T(), o.fields())
        assert max(fe.values()) <= 1e-12, (c.name, fe)
        d.close()
    b.close()


def test_batch_autotune_leaves_members_untouched():
    """lbm_batch_autotune times its candidates on a shadow batch: the members'
    populations and step counters are unchanged by it, the chosen tile is one
    of the candidates, and stepping on with it gives each domain its solo
    result (to FP32 rounding: the tile may select another kernel
    instantiation than the solo run's)."""
    import paper_2205_00686_gb300 as lbm
    v = P.bc_variants()
    cases = [P.droplet_case(nx, ny, v[name], seed=31 + i)
             for i, (nx, ny, name) in enumerate([(600, 90, "open_dirichlet"),
                                                 (256, 128, "periodic"),
                                                 (130, 70, "open_x_periodic_y")])]
    b = lbm.Batch()
    doms = []
    for c in cases:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    b.step(10)
    assert b.sync() == 0
    before = [d.populations() for d in doms]
    threads, rows, staged = b.autotune(2)
    assert threads in (128, 192, 224, 256) and rows in (16, 32, 64, 128, 256)
    for d, pb in zip(doms, before):
        assert d.step_count == 10
        for a, r in zip(d.populations(), pb):
            assert np.array_equal(a, r)
    b.step(30)
    assert b.sync() == 0
    for c, d in zip(cases, doms):
        f, g, Pp = d.populations()
        fs, gs, Ps = solo(c, 40, "fp32")
        assert P.rel_err(f, fs) < 1e-6 and P.rel_err(g, gs) < 1e-6, (c.name, threads, rows, staged)
        assert d.step_count == 40
    b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp32_g16"])
def test_staged_batch_matches_solo_bitwise(prec):
    """A batch whose members all take the bulk-copy staged load path (no
    walls; open x, or periodic x with nx a multiple of 8; widths that 216-column
    strips cover with no more thread columns than 120-column ones) runs the
    staged kernel over all members' work units in one launch per step. Each
    member's populations equal those of its solo run on the same tile and
    load path, bit for bit."""
    import paper_2205_00686_gb300 as lbm
    v = P.bc_variants()
    specs = [(648, 96, "open_dirichlet"), (432, 64, "periodic"), (864, 40, "open_x_periodic_y"),
             (216, 72, "periodic_flow_fixed_T")]
    cases = [P.droplet_case(nx, ny, v[name], seed=41 + i) for i, (nx, ny, name) in enumerate(specs)]
    b = lbm.Batch()
    doms = []
    for c in cases:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec=prec)
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    threads, rows, staged = b.tile()
    assert staged and threads == 224, (threads, rows, staged)
    b.step(45)
    assert b.sync() == 0
    for c, d in zip(cases, doms):
        b.detach(d)
        f, g, Pp = d.populations()
        s = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec=prec)
        s.set_tile(threads, rows)
        s.staged = True
        s.init_fields(*c.fields())
        s.step(45)
        fs, gs, Ps = s.populations()
        assert np.array_equal(f, fs) and np.array_equal(g, gs) and np.array_equal(Pp, Ps), c.name
        assert d.step_count == 45
        s.close()
    b.close()


@pytest.mark.parametrize("staged_set", [False, True])
def test_gravity_batch_matches_solo_bitwise(staged_set):
    """With buoyancy on, each step reads the mean density of the previous
    step (reading R16).  The CTAs add their block sums of it as fixed-point
    integers, so the sum does not depend on which CTA finishes first: a
    member of a batch gets, bit for bit, the populations of its solo run on
    the same tile, and a rerun repeats them exactly."""
    import paper_2205_00686_gb300 as lbm
    v = P.bc_variants()
    if staged_set:
        specs = [(648, 96, "open_dirichlet"), (432, 64, "periodic"), (864, 40, "open_x_periodic_y")]
    else:
        specs = [(100, 80, "open_dirichlet"), (257, 129, "wall_open_heater"),
                 (33, 47, "two_walls_adiabatic"), (130, 200, "open_x_walls_y")]
    cases = [P.droplet_case(nx, ny, v[name], seed=51 + i, gravity=3e-5)
             for i, (nx, ny, name) in enumerate(specs)]
    b = lbm.Batch()
    doms = []
    for c in cases:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    threads, rows, staged = b.tile()
    assert bool(staged) == staged_set, (threads, rows, staged)
    b.step(70)
    assert b.sync() == 0
    for c, d in zip(cases, doms):
        b.detach(d)
        got = d.populations()
        runs = []
        for _ in range(2):
            s = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
            s.set_tile(threads, rows)
            s.staged = bool(staged)
            s.init_fields(*c.fields())
            s.step(70)
            runs.append(s.populations())
            s.close()
        for a, r1, r2 in zip(got, runs[0], runs[1]):
            assert np.array_equal(r1, r2), c.name        # rerun: identical
            assert np.array_equal(a, r1), c.name         # batch member = solo
        d.close()
    b.close()


def test_reconfigure_switches_buoyancy_on_with_the_last_mean_density():
    """Gravity switched on between steps (lbm_reconfigure) takes the previous
    step's mean density at once, as the oracle does (FP64, 1e-12)."""
    import oracle
    import paper_2205_00686_gb300 as lbm
    c = P.droplet_case(90, 70, P.bc_variants()["wall_open_heater"], seed=61)
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp64")
    d.init_fields(*c.fields())
    o = oracle.Sim(c.nx, c.ny, c.params, c.bc)
    o.init(*c.fields())
    d.step(25)
    o.step(25)
    p2 = dict(c.params, gravity=4e-5)
    d.reconfigure(p2, c.bc)
    o.reconfigure(p2, c.bc)
    d.step(25)
    o.step(25)
    fe = P.field_errors(d.get_rho_u_T(), o.fields())
    assert max(fe.values()) <= 1e-12, fe
    d.close()


def test_error_words_arrive_without_waiting_for_later_chunks():
    """lbm_batch_errors_async queues a copy of each member's error word into
    pinned host memory: after the event of the chunk it follows, the word of
    the domain that left the EOS range is set and the others are clear, while
    a later chunk may still be queued (it is not waited for)."""
    import torch
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases()[:3]
    stream = torch.cuda.Stream()
    b = lbm.Batch(stream=stream.cuda_stream)
    doms = []
    for i, c in enumerate(cases):
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        rho = c.rho.copy()
        if i == 1:
            rho[c.ny // 2, c.nx // 2] = 9.7       # psi^2 < 0 there
        d.init_fields(rho, c.ux, c.uy, c.T)
        b.attach(d)
        doms.append(d)
    errs = torch.full((3,), -1, dtype=torch.int32).pin_memory()
    b.step(2)
    b.errors_async(errs.data_ptr())
    ev = torch.cuda.Event()
    ev.record(stream)
    b.step(40)                                   # queued behind, not waited for
    ev.synchronize()
    e = errs.tolist()
    assert e[0] == 0 and e[2] == 0 and e[1] & 1, e
    assert b.sync() == lbm.LBM_EPSI
    b.close()
    for d in doms:
        d.close()


def test_detached_domain_reads_back_after_its_last_batched_step():
    """A domain detached while a later chunk of the batch is still queued
    reads back the state its last batched step left (its own stream waits
    for the batch's steps queued before the detach, and no longer), and
    equals its solo run."""
    import torch
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases()[:3]
    bstream = torch.cuda.Stream()
    b = lbm.Batch(stream=bstream.cuda_stream)
    doms = []
    for c in cases:
        own = torch.cuda.Stream()
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32", stream=own.cuda_stream)
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append((d, own))
    b.step(30)
    b.detach(doms[0][0])
    b.step(400)                                  # the others go on
    f, g, _ = doms[0][0].populations()
    fs, gs, _ = solo(cases[0], 30, "fp32")
    assert np.array_equal(f, fs) and np.array_equal(g, gs)
    assert b.sync() == 0
    for (d, _), c in zip(doms[1:], cases[1:]):
        b.detach(d)
        f, g, _ = d.populations()
        fs, gs, _ = solo(c, 430, "fp32")
        assert np.array_equal(f, fs) and np.array_equal(g, gs), c.name
    b.close()


def test_domains_stop_at_their_own_targets_inside_shared_launches():
    """lbm_set_target: in a batch stepped 100 times, a domain with target 30
    and one with target 70 end exactly at those step counts with their solo
    states, buoyancy history included, while a third runs all 100; a solo
    domain stops the same way and continues once the target is lifted."""
    import paper_2205_00686_gb300 as lbm
    cases = mixed_cases(gravity=2e-5)[:3]
    b = lbm.Batch()
    doms = []
    for c, tgt in zip(cases, (30, 70, 0)):
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        d.set_target(tgt)
        b.attach(d)
        doms.append(d)
    threads, rows, staged = b.tile()
    b.step(100)
    assert b.sync() == 0
    for d, c, n in zip(doms, cases, (30, 70, 100)):
        b.detach(d)
        assert d.step_count == n
        s = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        s.set_tile(threads, rows)
        s.staged = staged
        s.init_fields(*c.fields())
        s.step(n)
        for a, r in zip(d.populations(), s.populations()):
            assert np.array_equal(a, r), (c.name, n)
        s.close()
    d = doms[0]
    d.set_target(0)
    d.step(5)
    assert d.step_count == 35
    b.close()
