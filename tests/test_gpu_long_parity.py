"""Parity after 1000 steps on every workload configuration, with the error
recorded at 250-step checkpoints so that its growth with run length is
visible.  Max relative field error (max |a - b| / max |b| per field) against
the FP64 oracle:

* FP64 <= 1e-10 on every field;
* FP32 <= 2e-4 on density and temperature.  The velocity fields are
  normalised by their own maximum, which in these nearly resting flows is
  1e-2 or less and falls as the start-up flow dies down; there the FP32
  storage of the populations (rounding ~1e-7 of each population per step)
  gives 7e-5 to 8e-4 after 1000 steps, largest at the corners of open edges
  and at the contact line, and the bound is 1e-3;
* FP32 with FP16-stored temperature populations: stated (printed), bounded
  by 1e-3 on density and temperature and 2e-2 on velocity.

Configurations:

* the 256 x 256 droplet evaporating in open space (Section 4.1 shape),
* the 400 x 200 droplet on a heated wall (Section 4.2 shape; FP32, FP64 and
  the FP16-stored temperature lattice it is specified for),
* the 300 x 600 boiling pool (Section 4.3 shape, 20-node heater at 1.1 T_c)
  started filled with saturated liquid as Section 4.3 states, at the
  smallest and the largest gravity of the Fritz sweep (1e-5, 8e-5), and
  started with the benchmark configuration's vapour layer in the top sixth
  at g = 1e-5.  That layer, pushed up by (rho - rho_ave) g against the open
  top, is physically unstable (in the oracle it leaves the EOS range at step
  1994 for g = 2e-5, 511 for 4e-5, 300 for 8e-5) and amplifies FP32 rounding
  like any other perturbation,
* a seeded sample of 16 of the 512 batched / served domains, advanced
  together in one FP32 batch.

The oracle runs start together in a thread pool when the module loads (the
ctypes calls release the GIL, so they use the host's cores) and are read
back by the tests; no oracle input or expected value comes from the GPU.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import parity as P
from paper_2205_00686_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64, TOL32, TOL32_U = 1e-10, 2e-4, 1e-3
CHECKPOINTS = (250, 500, 750, 1000)

CASES = {
    "open_evaporation_256": lambda: W.open_evaporation(256, 256, steps=0),
    "heated_surface_400x200": lambda: W.heated_surface(400, 200, steps=0),
    "boiling_300x600_liquid_g1e-5": lambda: W.nucleate_boiling(300, 600, gravity=1e-5, steps=0,
                                                               vapour_layer=False),
    "boiling_300x600_liquid_g8e-5": lambda: W.nucleate_boiling(300, 600, gravity=8e-5, steps=0,
                                                               vapour_layer=False),
    "boiling_300x600_vapour_layer_g1e-5": lambda: W.nucleate_boiling(300, 600, gravity=1e-5,
                                                                     steps=0),
}


def batch_sample():
    pop = W.batch_instances()
    idx = sorted(int(i) for i in np.argsort(W.uniform(99, len(pop)))[:16])
    return [pop[i] for i in idx]


def _oracle_checkpoints(case):
    s = oracle.Sim(case.nx, case.ny, case.params, case.bc)
    s.init(*case.fields())
    out, done = {}, 0
    for t in CHECKPOINTS:
        s.step(t - done)
        done = t
        out[t] = s.fields()
    return out


_POOL = {}


def oracle_runs():
    """name -> future of {step: oracle fields}; started once per session."""
    if not _POOL:
        ex = cf.ThreadPoolExecutor(max_workers=max(2, min(20, os.cpu_count() or 2)))
        jobs = {n: f() for n, f in CASES.items()}
        for i, c in enumerate(batch_sample()):
            jobs["batch_%02d" % i] = c
        # the longest runs first
        for n, c in sorted(jobs.items(), key=lambda kv: -kv[1].nx * kv[1].ny):
            _POOL[n] = ex.submit(_oracle_checkpoints, c)
    return _POOL


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()
    oracle_runs()


def gpu_checkpoints(case, prec):
    import paper_2205_00686_gb300 as lbm
    d = lbm.Domain(case.nx, case.ny, case.params, case.bc, prec=prec)
    d.init_fields(*case.fields())
    out, done = {}, 0
    for t in CHECKPOINTS:
        d.step(t - done)
        done = t
        out[t] = d.get_rho_u_T()
    d.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config_1000_steps(name, prec):
    case = CASES[name]()
    g = gpu_checkpoints(case, prec)
    o = oracle_runs()[name].result()
    errs = {t: P.field_errors(g[t], o[t]) for t in CHECKPOINTS}
    for t in CHECKPOINTS:
        print("%s %s step %d: %s" % (name, prec, t,
                                     " ".join("%s %.3e" % kv for kv in errs[t].items())))
    e = errs[1000]
    if prec == "fp64":
        assert max(e.values()) <= TOL64, e
    else:
        assert e["rho"] <= TOL32 and e["T"] <= TOL32, e
        assert e["ux"] <= TOL32_U and e["uy"] <= TOL32_U, e


def test_heated_surface_fp16_g_1000_steps():
    """The FP16-stored temperature lattice on the configuration it is
    specified for: its error is stated (printed) and loosely bounded (FP16
    keeps 11 bits of each population's deviation from w_i T_ref)."""
    name = "heated_surface_400x200"
    case = CASES[name]()
    g = gpu_checkpoints(case, "fp32_g16")
    o = oracle_runs()[name].result()
    errs = {t: P.field_errors(g[t], o[t]) for t in CHECKPOINTS}
    for t in CHECKPOINTS:
        print("%s fp32_g16 step %d: %s" % (name, t,
                                          " ".join("%s %.3e" % kv for kv in errs[t].items())))
    e = errs[1000]
    assert e["rho"] <= 1e-3 and e["T"] <= 1e-3, e
    assert e["ux"] <= 2e-2 and e["uy"] <= 2e-2, e


def test_batched_sample_fp32_1000_steps():
    """16 of the 512 batched domains (sides 64-512, edge temperatures
    0.90-0.98 T_c) advanced together in one FP32 batch: density and
    temperature within 2e-4 of each member's own oracle run after 1000
    steps, velocity within 1e-3 (normalised by the field's maximum, which
    decays five-fold as the start-up flow dies down, to 5e-3 on the 448^2
    member; the largest absolute error, 4e-6, sits at the corners of the open
    edges)."""
    import paper_2205_00686_gb300 as lbm
    sample = batch_sample()
    b = lbm.Batch()
    doms = []
    for c in sample:
        d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
        d.init_fields(*c.fields())
        b.attach(d)
        doms.append(d)
    b.step(1000)
    assert b.sync() == 0
    worst = 0.0
    for i, (c, d) in enumerate(zip(sample, doms)):
        b.detach(d)
        o = oracle_runs()["batch_%02d" % i].result()
        fe = P.field_errors(d.get_rho_u_T(), o[1000])
        print("batch member %d (%dx%d): %s" % (i, c.nx, c.ny,
                                               " ".join("%s %.3e" % kv for kv in fe.items())))
        worst = max(worst, max(fe.values()))
        assert fe["rho"] <= TOL32 and fe["T"] <= TOL32, (c.name, fe)
        assert fe["ux"] <= TOL32_U and fe["uy"] <= TOL32_U, (c.name, fe)
        d.close()
    b.close()
    print("batched sample worst FP32 error after 1000 steps: %.3e" % worst)
