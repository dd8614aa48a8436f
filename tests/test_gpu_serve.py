"""Continuous batching on the GPU: requests of different sizes arriving at
different times share launches, state lives in PyTorch-allocated memory
under a budget, and every result equals the same simulation run alone."""
import numpy as np
import pytest

from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(autouse=True, params=[1, 2], ids=["pipeline1", "pipeline2"])
def _pipeline(request, monkeypatch):
    """Every test runs with one and with two chunks queued ahead."""
    from paper_2205_00686_gb300.serve import Server
    init = Server.__init__

    def with_depth(self, *a, **k):
        k.setdefault("pipeline", request.param)
        init(self, *a, **k)
    monkeypatch.setattr(Server, "__init__", with_depth)


def requests():
    sides = [64, 96, 128, 80, 160, 112, 72]
    steps = [60, 45, 90, 30, 75, 50, 40]
    out = []
    for i, (s, n) in enumerate(zip(sides, steps)):
        c = W.open_evaporation(s, s, R=0.25 * s, T_edge=0.90 + 0.01 * i, seed=100 + i, steps=n)
        out.append((0.002 * i, c, n))
    return out


def solo(case, steps):
    import paper_2205_00686_gb300 as lbm
    d = lbm.Domain(case.nx, case.ny, case.params, case.bc, prec="fp32")
    d.init_fields(*case.fields())
    d.step(steps)
    return d.get_rho_u_T()


def test_served_results_equal_solo_results():
    import paper_2205_00686_gb300 as lbm
    from paper_2205_00686_gb300.serve import CudaBackend, Server
    be = CudaBackend("fp32")
    reqs = requests()
    # room for about three of the domains at a time
    budget = 3 * be.bytes_for(reqs[4][1])
    srv = Server(be, mem_budget=budget, chunk=16)
    st = srv.run(reqs)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert st["p50_s"] > 0 and st["p99_s"] >= st["p50_s"] and st["mlups"] > 0
    done = {r.case.name + str(r.steps): r for r in srv.finished}
    assert 2 <= st["max_active"] < len(reqs)      # shared launches, gated by memory
    for off, c, n in reqs:
        r = done[c.name + str(n)]
        ref = solo(c, n)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b), c.name
    del lbm


def test_bad_request_and_cancellation_leave_the_others_exact():
    """A request whose initial density is outside the EOS range fails alone
    at its first chunk (the step kernel reports psi^2 < 0 in the domain's
    sticky error word; lbm_init_fields does not evaluate the EOS), one running
    request is cancelled between chunks, and every other request still equals
    its solo run bit for bit."""
    import paper_2205_00686_gb300 as lbm
    from paper_2205_00686_gb300.serve import CANCELLED, CudaBackend, Server
    be = CudaBackend("fp32")
    base = [c for _, c, _ in requests()[:4]]
    bad = W.open_evaporation(64, 64, R=16.0, seed=7, steps=40)
    bad.rho = bad.rho.copy()
    bad.rho[32, 32] = 9.7
    srv = Server(be, mem_budget=4 * be.bytes_for(base[-1]), chunk=10)
    rs = [srv.submit(c, 40) for c in base[:2]]
    rb = srv.submit(bad, 40)
    rs += [srv.submit(c, 40) for c in base[2:]]
    srv.tick()
    victim = rs[1]
    assert victim.rid in srv.active and srv.cancel(victim.rid)
    while srv.tick():
        pass
    assert rb.error == lbm.LBM_EPSI and rb.result is None and rb.done_steps == 10
    assert victim.error == CANCELLED and victim.result is None
    for r, c in zip(rs, base):
        if r is victim:
            continue
        assert r.error == 0
        for a, b in zip(r.result, solo(c, 40)):
            assert np.array_equal(a, b), c.name
    assert srv.mem_used == 0
