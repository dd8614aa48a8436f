"""Pins of the CPU oracle's closed forms against what the paper and the
mathematics fix (no GPU).

Each test names the passage it follows.  None re-types an oracle formula:
they check identities, textbook properties and independent library routines.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2205_00686_gb300 import workloads as W

P = W.params()
CX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
CX5 = np.array([0, 1, 0, -1, 0])
CY5 = np.array([0, 0, 1, 0, -1])


def test_velocity_sets_follow_eq2_and_eq26():
    # Eq. 2: c_i = (cos((i-1) pi/2), sin((i-1) pi/2)) for i = 1..4 and
    # sqrt(2) (cos((2i-9) pi/4), sin((2i-9) pi/4)) for i = 5..8.
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        assert (CX9[i], CY9[i]) == (round(math.cos(a)), round(math.sin(a)))
        assert (CX5[i], CY5[i]) == (CX9[i], CY9[i])
    for i in range(5, 9):
        a = (2 * i - 9) * math.pi / 4
        assert (CX9[i], CY9[i]) == (round(math.sqrt(2) * math.cos(a)),
                                     round(math.sqrt(2) * math.sin(a)))


def test_transformation_matrices():
    M, Mi, Mh, Mhi = O.matrices()
    # Eq. 4 is the Lallemand-Luo matrix: rows mutually orthogonal
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)), atol=0)
    # the rows are the moments rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy of c
    c2 = CX9 ** 2 + CY9 ** 2
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[1], -4 + 3 * c2)
    assert np.array_equal(M[2], 4 - 21 / 2 * c2 + 9 / 2 * c2 ** 2)
    assert np.array_equal(M[3], CX9) and np.array_equal(M[5], CY9)
    assert np.array_equal(M[4], (-5 + 3 * c2) * CX9)
    assert np.array_equal(M[6], (-5 + 3 * c2) * CY9)
    assert np.array_equal(M[7], CX9 ** 2 - CY9 ** 2)
    assert np.array_equal(M[8], CX9 * CY9)
    assert np.abs(M @ Mi - np.eye(9)).max() < 1e-14
    assert np.abs(Mh @ Mhi - np.eye(5)).max() < 1e-15
    # Eq. 40: rows 1, c_x, c_y, |c|^2, c_x^2 - c_y^2 of the D2Q5 set
    assert np.array_equal(Mh[0], np.ones(5))
    assert np.array_equal(Mh[1], CX5) and np.array_equal(Mh[2], CY5)
    assert np.array_equal(Mh[3], CX5 ** 2 + CY5 ** 2)
    assert np.array_equal(Mh[4], CX5 ** 2 - CY5 ** 2)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (6.5, 0.03, -0.01),
                                       (0.38, -0.05, 0.07), (2.2, 0.1, 0.1)])
def test_feq_moments_and_meq(rho, ux, uy):
    M = O.matrices()[0]
    f = O.feq(rho, ux, uy)
    # textbook moments of the second-order Maxwellian (Eq. 3, c_s^2 = 1/3)
    assert abs(f.sum() - rho) < 1e-14 * rho
    assert abs((CX9 * f).sum() - rho * ux) < 1e-14
    assert abs((CY9 * f).sum() - rho * uy) < 1e-14
    Pxx = (CX9 * CX9 * f).sum()
    Pxy = (CX9 * CY9 * f).sum()
    assert abs(Pxx - rho * (1 / 3 + ux * ux)) < 1e-14 * rho
    assert abs(Pxy - rho * ux * uy) < 1e-14 * rho
    # M f^eq = m^eq (Eq. 7)
    assert np.abs(M @ f - O.meq(rho, ux, uy)).max() < 1e-13 * rho


@pytest.mark.parametrize("wdot", [0.2, 2 / 3, 0.9])
def test_d2q5_equilibrium_eq33_and_eq47(wdot):
    p = W.params(w_dot=wdot)
    Mh = O.matrices()[2]
    T = 0.0937
    g = O.geq(p, T)
    # Eq. 33: sum g = T, sum c g = 0, sum c c g = cs2h T I with cs2h = w_dot/2
    assert abs(g.sum() - T) < 4e-17
    assert abs((CX5 * g).sum()) == 0 and abs((CY5 * g).sum()) == 0
    assert abs((CX5 * CX5 * g).sum() - wdot / 2 * T) < 4e-17
    assert abs((CX5 * CY5 * g).sum()) == 0
    # Eq. 47: Mh g^eq = [T, 0, 0, w_dot T, 0]
    assert np.abs(Mh @ g - np.array([T, 0, 0, wdot * T, 0])).max() < 4e-17


def test_critical_point_of_peng_robinson():
    """Section 2: a = 0.45724 R^2 Tc^2/pc, b = 0.0778 R Tc/pc.  At T = Tc the
    isotherm has a horizontal inflection at p = pc; the Peng-Robinson critical
    compressibility is Z_c = pc / (rho_c R Tc) = 0.3074."""
    from scipy.optimize import minimize_scalar
    Tc = O.Tc(P)
    assert abs(Tc - 0.109383) < 1e-6

    def dpdr(r, h=1e-5):
        return (O.p_eos(P, r + h, Tc) - O.p_eos(P, r - h, Tc)) / (2 * h)

    res = minimize_scalar(dpdr, bounds=(1.0, 5.0), method="bounded",
                          options={"xatol": 1e-10})
    rc = res.x
    # horizontal at the inflection, up to the rounding of 0.45724 and 0.0778
    # (their exact Peng-Robinson values are 0.4572355 and 0.0777961)
    assert abs(res.fun) < 1e-4 * Tc
    pc = O.p_eos(P, rc, Tc)
    assert abs(pc - 0.0778 * Tc / P["b"]) < 1e-3 * pc
    assert abs(pc / (rc * Tc) - 0.3074) < 2e-3


def test_acentric_factor_reproduced():
    """omega = -1 - log10(p_sat(0.7 Tc) / pc) by definition; the
    Peng-Robinson alpha(T) of Section 2 is built to reproduce it."""
    Tc = O.Tc(P)
    pc = 0.0778 * Tc / P["b"]
    rg, rl = O.maxwell(P, 0.7 * Tc)
    psat = O.p_eos(P, rg, 0.7 * Tc)
    omega = -1 - math.log10(psat / pc)
    assert abs(omega - 0.344) < 0.03


@pytest.mark.parametrize("rho,Tr", [(0.38, 0.86), (6.5, 0.86), (3.0, 0.95), (1.0, 1.1)])
def test_dpdT_against_finite_difference(rho, Tr):
    T = Tr * O.Tc(P)
    h = 1e-6 * T
    fd = (O.p_eos(P, rho, T + h) - O.p_eos(P, rho, T - h)) / (2 * h)
    assert abs(O.dpdT(P, rho, T) - fd) < 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("Tr", [0.8, 0.86, 0.9, 0.95])
def test_maxwell_against_scipy(Tr):
    """Equal pressure and equal area, solved independently with scipy's
    root finder and adaptive quadrature on the oracle's p_EOS."""
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    T = Tr * O.Tc(P)
    rg0, rl0 = O.maxwell(P, T)

    def eqs(v):
        rg, rl = v
        pg, pl = O.p_eos(P, rg, T), O.p_eos(P, rl, T)
        area = quad(lambda r: (O.p_eos(P, r, T) - pg) / r ** 2, rg, rl,
                    epsabs=1e-14, epsrel=1e-12, limit=200)[0]
        return [pg - pl, area]

    rg, rl = fsolve(eqs, [rg0 * 1.02, rl0 * 0.99], xtol=1e-13)
    assert abs(rg - rg0) < 1e-7 * rg0
    assert abs(rl - rl0) < 1e-7 * rl0


def test_coexistence_table_matches_oracle():
    for Tr, (rg, rl) in W.COEXISTENCE.items():
        g, l = O.maxwell(P, Tr * W.TC)
        assert abs(g - rg) < 1e-10 and abs(l - rl) < 1e-10


def test_psi_radicand_sign():
    """psi^2 = 2 (p_EOS - rho c_s^2)/G with G = -1 must be positive in both
    bulk phases (Section 2) and turns negative only at very high density."""
    Tc = O.Tc(P)
    for Tr, (rg, rl) in W.COEXISTENCE.items():
        assert O.psi2(P, rg, Tr * Tc) > 0 and O.psi2(P, rl, Tr * Tc) > 0
    assert O.psi2(P, 9.5, 0.86 * Tc) < 0
