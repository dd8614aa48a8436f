"""Run records and field dumps.

* `RunLog` appends one JSON object per line to a file: a run record (the
  configuration's name, precision, MLUPS, GB/s, roofline fraction) and,
  while a run advances, samples of its diagnostics (mass and its drift from
  the first sample, energy, liquid area or volume, equivalent diameter,
  max |u|) -- the D(t) and mass-drift series of the paper's droplet runs.
* `dump_fields` writes fields as .npy files (headless: figures are drawn
  offline from the files).
* `advance_logged` steps a domain in chunks and logs a sample after each.

Host-side bookkeeping only; every number comes from the library.
"""
from __future__ import annotations

import json
import os
import time
from typing import Optional, Sequence

import numpy as np


class RunLog:
    def __init__(self, path: str):
        self.path = path
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        self._mass0: Optional[float] = None

    def _write(self, rec: dict) -> dict:
        with open(self.path, "a") as fh:
            fh.write(json.dumps(rec) + "\n")
        return rec

    def run(self, config: str, prec: str, mlups: float, gbs: Optional[float] = None,
            roofline_frac: Optional[float] = None, **extra) -> dict:
        rec = {"kind": "run", "config": config, "prec": prec, "mlups": mlups, "gbs": gbs,
               "roofline_frac": roofline_frac, "time": time.time()}
        rec.update(extra)
        return self._write(rec)

    def sample(self, step: int, diag: dict) -> dict:
        """One diagnostics sample (`diag` as returned by Domain.diagnostics)."""
        m = float(diag["mass"])
        if self._mass0 is None:
            self._mass0 = m
        rec = {"kind": "sample", "step": int(step), "mass": m,
               "mass_drift": (m - self._mass0) / self._mass0 if self._mass0 else 0.0,
               "energy": float(diag["energy"]), "liquid": float(diag["liquid_area"]),
               "diameter": float(diag["diameter"]),
               "diameter_smooth": float(diag["diameter_smooth"]),
               "max_u": float(diag["max_u"])}
        return self._write(rec)

    def records(self, kind: Optional[str] = None) -> list:
        out = []
        if not os.path.exists(self.path):
            return out
        with open(self.path) as fh:
            for line in fh:
                r = json.loads(line)
                if kind is None or r.get("kind") == kind:
                    out.append(r)
        return out


def dump_fields(directory: str, step: int, fields: Sequence[np.ndarray],
                names: Sequence[str] = ("rho", "ux", "uy", "T")) -> list:
    """Writes <directory>/<name>_<step>.npy for each field; returns the paths."""
    os.makedirs(directory, exist_ok=True)
    paths = []
    for name, f in zip(names, fields):
        p = os.path.join(directory, "%s_%08d.npy" % (name, step))
        np.save(p, np.asarray(f))
        paths.append(p)
    return paths


def advance_logged(domain, steps: int, every: int, log: RunLog, rho_l: float, rho_g: float,
                   sessile: bool = False, dump_dir: Optional[str] = None) -> list:
    """Advances `domain` by `steps` in chunks of `every`, logging a sample
    (and, with `dump_dir`, the fields) after each chunk."""
    out = [log.sample(domain.step_count, domain.diagnostics(rho_l, rho_g, sessile))]
    done = 0
    while done < steps:
        n = min(every, steps - done)
        domain.step(n)
        done += n
        out.append(log.sample(domain.step_count, domain.diagnostics(rho_l, rho_g, sessile)))
        if dump_dir:
            dump_fields(dump_dir, domain.step_count, domain.get_rho_u_T())
    return out
