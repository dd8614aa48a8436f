"""Run protocols of the paper's wall experiments, on top of the C ABI.

* Section 4.2: a sessile droplet is first run without evaporation until it
  shows the prescribed contact angle, then the wall is heated.
  `relax_wetting` runs the isothermal phase (frozen thermal lattice) and
  watches the measured angle until it settles; `start_heating` switches to
  the heated configuration in place (`lbm_reconfigure`).
* Section 4.3: bubbles grow on a heater and depart; the departure diameter
  D_d follows Fritz's D_d ~ g^(-1/2).  `watch_departure` steps a domain and
  labels its vapour regions on the device (`lbm_regions`) until one no longer
  touches the heated wall; `fritz_sweep` repeats that over gravities and fits
  the log-log slope.

Everything numeric runs in the CUDA library; these functions only schedule
steps and read back the device's measurements.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional, Sequence


def equivalent_diameter(area: float) -> float:
    """Diameter of the disc with the given area (lattice units)."""
    return 2.0 * math.sqrt(max(area, 0.0) / math.pi)


def relax_wetting(domain, rho_l: float, rho_g: float, check_every: int = 1000,
                  tol_deg: float = 0.05, window: int = 3, max_steps: int = 200000,
                  skip_rows: int = 3) -> List[dict]:
    """Steps `domain` (already configured with frozen_thermal = 1) in chunks
    of `check_every` until the contact angle changed by less than `tol_deg`
    over the last `window` chunks, or `max_steps` have run.  Returns the
    history of {"step", "theta_deg", "radius", "base_width", "height"}."""
    hist: List[dict] = []
    steps = 0
    while steps < max_steps:
        domain.step(check_every)
        steps += check_every
        m = domain.contact_angle(rho_l, rho_g, skip_rows)
        m["step"] = domain.step_count
        hist.append(m)
        if len(hist) > window:
            recent = [h["theta_deg"] for h in hist[-window - 1:]]
            if max(recent) - min(recent) < tol_deg:
                break
    return hist


def start_heating(domain, params: dict, bc: dict) -> None:
    """Switches a relaxed domain to the heated configuration (thermal lattice
    running, wall temperatures of `bc`)."""
    p = dict(params)
    p["frozen_thermal"] = 0
    domain.reconfigure(p, bc)


def departed(regions: Sequence[dict], min_area: int = 1, wall: str = "s") -> List[dict]:
    """Vapour regions that have left the wall (no node on its edge row) and
    hold at least `min_area` nodes."""
    key = "touches_" + wall
    return [r for r in regions if not r[key] and r["area"] >= min_area]


def _touches_top(r: dict) -> bool:
    return bool(r["touches_n"])


def watch_departure(domain, rho_l: float, rho_g: float, check_every: int = 200,
                    max_steps: int = 100000, min_area: int = 8,
                    exclude: Optional[Callable[[dict], bool]] = _touches_top) -> Optional[dict]:
    """Steps `domain` until a vapour region of at least `min_area` nodes no
    longer touches the south wall.  Regions for which `exclude(region)` is
    true are ignored; by default those touching the north edge (the vapour
    layer above a pool).  Returns {"step", "diameter", "area", "centroid_y",
    "region"} of the first departure, or None if none happened within
    `max_steps`."""
    thr = 0.5 * (rho_l + rho_g)
    steps = 0
    while steps < max_steps:
        domain.step(check_every)
        steps += check_every
        regs = domain.regions(thr, below=True)
        for r in departed(regs, min_area):
            if exclude is not None and exclude(r):
                continue
            return {"step": domain.step_count, "diameter": equivalent_diameter(r["area"]),
                    "area": r["area"], "centroid_y": r["sum_y"] / r["area"], "region": r}
    return None


def loglog_slope(xs: Sequence[float], ys: Sequence[float]) -> float:
    """Least-squares slope of log y against log x."""
    lx = [math.log(x) for x in xs]
    ly = [math.log(y) for y in ys]
    n = len(lx)
    if n < 2:
        raise ValueError("need two points for a slope")
    mx, my = sum(lx) / n, sum(ly) / n
    sxx = sum((a - mx) ** 2 for a in lx)
    sxy = sum((a - mx) * (b - my) for a, b in zip(lx, ly))
    return sxy / sxx


def fritz_sweep(make_domain: Callable[[float], object], gravities: Sequence[float],
                rho_l: float, rho_g: float, **watch) -> Dict[str, object]:
    """For each gravity g, builds a fresh domain with `make_domain(g)`, waits
    for the first departure and records D_d.  Returns the per-g results and,
    when at least two departures were seen, the fitted slope of log D_d
    against log g (Fritz: -1/2)."""
    rows = []
    for g in gravities:
        d = make_domain(g)
        try:
            res = watch_departure(d, rho_l, rho_g, **watch)
            err = None
        except Exception as e:   # a run that left the EOS range
            res, err = None, str(e)
        finally:
            d.close()
        rows.append({"g": g, "departure": res, "error": err})
    ok = [(r["g"], r["departure"]["diameter"]) for r in rows if r["departure"]]
    slope = loglog_slope([a for a, _ in ok], [b for _, b in ok]) if len(ok) >= 2 else None
    return {"runs": rows, "slope": slope}
