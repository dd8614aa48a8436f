"""The OpenMP build of the oracle (per-node loops over all host cores) gives
the serial build's results bit for bit: every node's arithmetic is the same
and every sum keeps its serial order (no GPU)."""
import numpy as np
import pytest

import oracle as O
import parity as P


@pytest.mark.parametrize("bc", ["wall_open_heater", "open_dirichlet", "periodic"])
def test_openmp_build_is_bit_identical(bc):
    c = P.droplet_case(61, 47, P.bc_variants()[bc], seed=5, gravity=3e-5)
    runs = []
    for omp in (False, True):
        s = O.Sim(c.nx, c.ny, c.params, c.bc, omp=omp)
        s.init(*c.fields())
        s.step(40)
        runs.append(s.populations() + s.fields())
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
