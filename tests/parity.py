"""Helpers for GPU-vs-oracle parity tests (test infrastructure)."""
import numpy as np

import oracle
from paper_2205_00686_gb300 import workloads as W


def rel_err(a, b):
    """max |a - b| / max |b| (the max-normalised field error)."""
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def field_errors(gpu_fields, ref_fields):
    return {k: rel_err(a, b) for k, a, b in zip(("rho", "ux", "uy", "T"), gpu_fields, ref_fields)}


def run_oracle(case, steps):
    s = oracle.Sim(case.nx, case.ny, case.params, case.bc)
    s.init(*case.fields())
    if steps:
        s.step(steps)
    return s


def run_gpu(case, steps, prec, tile=None, chunks=None, staged=None):
    import paper_2205_00686_gb300 as lbm
    d = lbm.Domain(case.nx, case.ny, case.params, case.bc, prec=prec)
    if tile:
        d.set_tile(*tile)
    if staged is not None:
        d.staged = staged
    d.init_fields(*case.fields())
    if chunks:
        for c in chunks:
            d.step(c)
    elif steps:
        d.step(steps)
    d.sync()
    return d


def compare(case, steps, prec, tile=None, chunks=None):
    """Runs both sides; returns (field errors, population errors, gpu, oracle)."""
    o = run_oracle(case, steps)
    g = run_gpu(case, steps, prec, tile, chunks)
    fe = field_errors(g.get_rho_u_T(), o.fields())
    gf, gg, gP = g.populations()
    of, og, oP = o.populations()
    pe = {"f": rel_err(gf, of), "g": rel_err(gg, og)}
    return fe, pe, g, o


def bc_variants():
    """Every boundary kind and corner combination the library accepts."""
    Tc = W.TC
    T1, T2 = 0.86 * Tc, 0.95 * Tc
    return {
        "periodic": W.periodic_bc(),
        "open_dirichlet": W.bc_spec([W.OPEN] * 4, [W.T_DIRICHLET] * 4, T_edge=[T2, T2, T1, T2]),
        "wall_open_heater": W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.OPEN],
                                      [W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET],
                                      T_edge=[0, 0, T1, T1], theta_deg=75.0, heater=(3, 7),
                                      T_heater=1.05 * Tc),
        "two_walls_adiabatic": W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                                         [W.T_PERIODIC, W.T_PERIODIC, W.T_ADIABATIC,
                                          W.T_DIRICHLET], T_edge=[0, 0, 0, T2], theta_deg=110.0),
        "open_x_walls_y": W.bc_spec([W.OPEN, W.OPEN, W.WALL, W.WALL],
                                    [W.T_ADIABATIC, W.T_DIRICHLET, W.T_DIRICHLET, W.T_ADIABATIC],
                                    T_edge=[0, T2, T2, 0], theta_deg=60.0),
        "periodic_x_open_y": W.bc_spec([W.PERIODIC, W.PERIODIC, W.OPEN, W.OPEN],
                                       [W.T_PERIODIC, W.T_PERIODIC, W.T_ADIABATIC,
                                        W.T_DIRICHLET], T_edge=[0, 0, 0, T2]),
        "open_x_periodic_y": W.bc_spec([W.OPEN, W.OPEN, W.PERIODIC, W.PERIODIC],
                                       [W.T_DIRICHLET, W.T_ADIABATIC, W.T_PERIODIC,
                                        W.T_PERIODIC], T_edge=[T2, 0, 0, 0]),
        # Section 4.1: periodic flow, temperature held at the edges
        "periodic_flow_fixed_T": W.bc_spec([W.PERIODIC] * 4,
                                           [W.T_DIRICHLET, W.T_ADIABATIC, W.T_DIRICHLET,
                                            W.T_DIRICHLET], T_edge=[T2, 0, T1, 1.0 * Tc]),
    }


def droplet_case(nx, ny, bc, amp=1e-3, seed=7, gravity=0.0, Tr=0.86, R=None):
    """A droplet with noise and a temperature bump: exercises every term."""
    rg, rl = W.COEXISTENCE[Tr]
    R = R if R is not None else 0.3 * min(nx, ny)
    rho = W.tanh_disc(nx, ny, 0.45 * nx, 0.4 * ny, R, 4.0, rl, rg)
    rho = rho + W.noise(seed, (ny, nx), amp)
    T = W.tanh_disc(nx, ny, 0.45 * nx, 0.4 * ny, R, 4.0, Tr * W.TC, 0.93 * W.TC)
    T = T + W.noise(seed + 1, (ny, nx), 1e-4 * W.TC)
    z = np.zeros((ny, nx))
    return W.Case("droplet_%dx%d" % (nx, ny), nx, ny, W.params(gravity=gravity), bc, rho, z,
                  z.copy(), T, 0, rl, rg)
