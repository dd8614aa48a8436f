"""Host logic of the slab split of one domain (no GPU): the partition of the
rows, the slabs' boundary specs, the halo moves, and the halo exchange
between ranks over torch.distributed (gloo, world size 2 and 3) with
host-memory stand-ins for the slabs' state."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2205_00686_gb300 import slabs as S
from paper_2205_00686_gb300 import workloads as W


@pytest.mark.parametrize("ny,n,per,ghost", [(40, 2, False, 3), (41, 3, False, 3), (37, 3, True, 6),
                                             (12, 4, True, 3), (9, 1, False, 3)])
def test_partition_covers_every_row_once(ny, n, per, ghost):
    sl = S.partition(ny, n, per, ghost)
    own = np.concatenate([np.arange(s.own0, s.own1) for s in sl])
    assert np.array_equal(own, np.arange(ny))
    for s in sl:
        assert (s.lo == ghost) == (s.prev is not None)
        assert (s.hi == ghost) == (s.next is not None)
        assert s.rows == s.lo + s.own1 - s.own0 + s.hi
    if n > 1:
        assert (sl[0].prev is not None) == per and (sl[-1].next is not None) == per
    heights = [s.own1 - s.own0 for s in sl]
    assert max(heights) - min(heights) <= 1


def test_partition_refuses_thin_slabs_and_bad_ghosts():
    with pytest.raises(ValueError):
        S.partition(10, 4, False, 3)          # 2-row slabs cannot feed 3 halo rows
    with pytest.raises(ValueError):
        S.partition(40, 2, False, 4)          # not a multiple of the stencil depth
    with pytest.raises(ValueError):
        S.partition(3, 4, False, 3)


def emulate(ny, n, per, ghost):
    """Global rows tagged by their index; each slab's local rows copied from
    them (wrapping on a periodic axis); halos then spoiled."""
    glob = np.arange(ny, dtype=float)[:, None] * np.ones((1, 5))
    sl = S.partition(ny, n, per, ghost)
    loc = []
    for s in sl:
        a = glob[s.local_rows() % ny].copy()
        a[:s.lo] = -1
        a[s.lo + s.own1 - s.own0:] = -1
        loc.append(a)
    return glob, sl, loc


@pytest.mark.parametrize("ny,n,per,ghost", [(40, 2, False, 3), (41, 3, False, 6), (37, 3, True, 3),
                                             (12, 4, True, 3)])
def test_halo_moves_fill_every_halo_from_its_neighbour(ny, n, per, ghost):
    glob, sl, loc = emulate(ny, n, per, ghost)
    for (si, sy, di, dy, k) in S.halo_moves(sl):
        loc[di][dy:dy + k] = loc[si][sy:sy + k]
    for s, a in zip(sl, loc):
        assert np.array_equal(a, glob[s.local_rows() % ny]), s


def test_slab_boundaries():
    T = 0.86 * W.TC
    bc = W.bc_spec([W.PERIODIC, W.PERIODIC, W.WALL, W.OPEN],
                   [W.T_PERIODIC, W.T_PERIODIC, W.T_DIRICHLET, W.T_DIRICHLET],
                   T_edge=[0, 0, T, T], theta_deg=75.0, heater=(10, 20), T_heater=1.1 * W.TC)
    sl = S.partition(60, 3, False)
    b0, b1, b2 = (S.slab_bc(bc, s) for s in sl)
    assert b0["flow"] == [W.PERIODIC, W.PERIODIC, W.WALL, W.OPEN]
    assert b0["therm"][3] == W.T_ADIABATIC and b0["heater_x1"] == 20
    assert b1["flow"][2:] == [W.OPEN, W.OPEN] and b1["therm"][2:] == [W.T_ADIABATIC] * 2
    assert b1["heater_x1"] == 0
    assert b2["flow"][2:] == [W.OPEN, W.OPEN] and b2["therm"][3] == W.T_DIRICHLET
    one = S.slab_bc(bc, S.partition(60, 1, False)[0])
    assert one["flow"] == bc["flow"] and one["therm"] == bc["therm"]


# ---------------------------------------------------------------------------
# the exchange between ranks (gloo)

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ny, per, ghost, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    glob, sl, loc = emulate(ny, world, per, ghost)
    mine = sl[rank]
    state = torch.from_numpy(loc[rank])

    def pack(y0, n):
        return state[y0:y0 + n].clone()

    def unpack(y0, n, t):
        state[y0:y0 + n] = t

    S.exchange_halos(mine, sl, pack, unpack, lambda n: torch.empty((n, 5), dtype=torch.float64),
                     dist, lambda s: s)
    ok = torch.equal(state, torch.from_numpy(glob[mine.local_rows() % ny]))
    out[rank] = int(ok)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,ny,per,ghost", [(2, 30, False, 3), (3, 37, True, 6), (2, 20, True, 3)])
def test_exchange_between_ranks(world, ny, per, ghost):
    ctx = mp.get_context("spawn")
    out = ctx.Array("i", world)
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ny, per, ghost, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert list(out) == [1] * world
