"""Host-side run records, field dumps and the named configurations (no GPU)."""
import json
import os

import numpy as np
import pytest

from paper_2205_00686_gb300 import runlog as RL
from paper_2205_00686_gb300 import workloads as W


class FakeDomain:
    """Mass leaks 1e-6 per step; diameter shrinks linearly."""

    def __init__(self):
        self.step_count = 0

    def step(self, n):
        self.step_count += n

    def diagnostics(self, rho_l, rho_g, sessile=False):
        s = self.step_count
        return {"mass": 1000.0 * (1 - 1e-6 * s), "energy": 50.0, "liquid_area": 300.0 - s,
                "diameter": 20.0 - 0.01 * s, "diameter_smooth": 20.5 - 0.01 * s,
                "max_u": 1e-3}

    def get_rho_u_T(self):
        return tuple(np.full((3, 4), float(k + self.step_count)) for k in range(4))


def test_runlog_records_and_mass_drift(tmp_path):
    log = RL.RunLog(str(tmp_path / "runs" / "log.jsonl"))
    log.run("evaporation_4096", "fp32", 38500.0, gbs=4620.0, roofline_frac=0.69, tile=[128, 256])
    d = FakeDomain()
    recs = RL.advance_logged(d, 250, 100, log, 6.5, 0.38, dump_dir=str(tmp_path / "dump"))
    assert [r["step"] for r in recs] == [0, 100, 200, 250]
    assert recs[-1]["mass_drift"] == pytest.approx(-250e-6)
    lines = open(log.path).read().splitlines()
    assert len(lines) == 5 and json.loads(lines[0])["kind"] == "run"
    assert [r["step"] for r in log.records("sample")] == [0, 100, 200, 250]
    assert log.records("run")[0]["tile"] == [128, 256]
    f = np.load(str(tmp_path / "dump" / "T_00000250.npy"))
    assert f.shape == (3, 4) and f[0, 0] == 253.0


def test_named_configurations_build_their_inputs():
    names = sorted(f[:-5] for f in os.listdir(W.CONFIG_DIR) if f.endswith(".json"))
    assert {"static_droplet_64", "open_evaporation_256", "heated_surface_400x200",
            "nucleate_boiling_300x600", "batched_512", "evaporation_4096",
            "droplet_cloud_256"} <= set(names)
    for n in names:
        cfg = W.load_config(n)
        assert cfg["name"] == n and cfg["precisions"] and cfg["steps"] > 0
        assert callable(getattr(W, cfg["case"]))
    c = W.config_case(W.load_config("static_droplet_64"))
    ref = W.static_droplet(64, 64, R=16.0, seed=1)
    assert np.array_equal(c.rho, ref.rho)
    c = W.config_case(W.load_config("open_evaporation_256"), nx=64, ny=64, R=10.0)
    assert (c.nx, c.ny) == (64, 64)
