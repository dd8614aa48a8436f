"""The allocation-free diagnostics entry point (lbm_diag_reduce_noalloc), for
callers that must not allocate device memory: its sums must match the regular
lbm_diagnostics of the same state, on two calls in a row that share the
library's fixed scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.  It also passes on its own in a
fresh process (the fixture builds the library)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def test_noalloc_matches_lbm_diagnostics_twice():
    import torch

    import paper_2205_00686_gb300 as lbm
    from paper_2205_00686_gb300 import workloads as W

    c = W.open_evaporation(200, 150, R=40.0, steps=0)
    d = lbm.Domain(c.nx, c.ny, c.params, c.bc, prec="fp32")
    d.init_fields(*c.fields())
    d.step(60)
    ref = d.diagnostics(c.rho_l, c.rho_g)
    fields = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in d.get_rho_u_T()]
    out = torch.full((7,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    n = c.nx * c.ny
    keys = ("mass", "energy", "liquid_mass", "liquid_area", "liquid_area_smooth", "max_u",
            "nonfinite")
    results = []
    for _ in range(2):
        out.fill_(-1.0)
        rc = lbm.lbm_diag_reduce_noalloc(*[f.data_ptr() for f in fields], n, c.params["cv"],
                                         c.rho_l, c.rho_g, out.data_ptr(), stream.cuda_stream)
        assert rc == lbm.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        results.append(got.copy())
        for k, v in zip(keys, got):
            assert abs(v - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, v, ref[k])
    assert np.array_equal(results[0], results[1])
    d.close()


def test_noalloc_rejects_sizes_beyond_its_capacity():
    import torch

    import paper_2205_00686_gb300 as lbm
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = lbm.lbm_diag_reduce_noalloc(p, p, p, p, lbm.LBM_NOALLOC_MAX_NODES + 1, 5.0, 6.5, 0.38,
                                     p, None)
    assert rc == lbm.LBM_ETOOBIG
    rc = lbm.lbm_diag_reduce_noalloc(p, p, p, p, 0, 5.0, 6.5, 0.38, p, None)
    assert rc == lbm.LBM_OK
    torch.cuda.synchronize()
    assert float(buf[:7].abs().sum()) == 0.0


def test_noalloc_at_capacity_and_allocates_nothing():
    """At the largest accepted size (LBM_NOALLOC_MAX_NODES nodes, every one of
    the 4096 blocks of the fixed array in use) the sums equal a plain PyTorch
    FP64 reduction of the same fields; and a call after the first one leaves
    the device's free memory exactly as it was: nothing is allocated."""
    import torch

    import paper_2205_00686_gb300 as lbm
    n = lbm.LBM_NOALLOC_MAX_NODES
    g = torch.Generator(device="cuda").manual_seed(5)
    rho = 0.38 + 6.2 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    ux = 0.02 * (torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5)
    uy = 0.02 * (torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5)
    T = 0.09 + 0.01 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    cv, rl, rg = 5.0, 6.5, 0.38
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    args = [rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), T.data_ptr(), n, cv, rl, rg,
            out.data_ptr(), stream.cuda_stream]
    assert lbm.lbm_diag_reduce_noalloc(*args) == lbm.LBM_OK
    torch.cuda.synchronize()
    first = out.clone()
    free0 = torch.cuda.mem_get_info()[0]
    out.fill_(-1.0)
    assert lbm.lbm_diag_reduce_noalloc(*args) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)
    mid = 0.5 * (rl + rg)
    liq = rho > mid
    ref = [rho.sum(), (rho * cv * T).sum(), rho[liq].sum(), liq.sum().double(),
           ((rho - rg) / (rl - rg)).clamp(0, 1).sum(), torch.sqrt(ux * ux + uy * uy).max(), 0.0]
    for k, (a, b) in enumerate(zip(out.tolist(), [float(r) for r in ref])):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (k, a, b)
