"""One domain split into slabs of rows (y), each slab a context of its own.

A slab holds its own rows and `ghost` halo rows copied from each neighbour.
One coupled step reads rows up to three away (psi at depth three feeds the
force, the velocity, its divergence and both collisions, then the pull
streaming), so after an exchange a slab can take ghost // 3 steps before its
own rows would read stale halo rows.  The slab's inner edges are open with
adiabatic temperature: they only shape halo rows, which the next exchange
overwrites.  Every slab uses the whole domain's rho_ref and T_ref, so that raw
rows move between slabs unchanged, and with buoyancy the slabs' density sums
are added after every step (rho_ave of Section 4.3 is the mean over the whole
domain; the slabs then step one at a time between exchanges).

`SlabRunner` keeps all slabs in one process on one device (exchanges are
device-to-device copies): it is how the split is tested against the oracle
on one GPU.  `exchange_halos` does the same exchange between ranks with
torch.distributed point-to-point transfers (NCCL between GPUs, gloo on CPU);
the CPU tests drive it with host-memory stand-ins for the slabs.  All numeric
work runs in the CUDA library; this module moves rows and schedules steps.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence

import numpy as np

STENCIL_DEPTH = 3    # rows a step reads on each side of an output row

PERIODIC, WALL, OPEN = 0, 1, 2
T_PERIODIC, T_DIRICHLET, T_ADIABATIC = 0, 1, 2
EDGE_S, EDGE_N = 2, 3


@dataclasses.dataclass
class Slab:
    index: int
    own0: int            # first own row (global index)
    own1: int            # one past the last own row
    lo: int              # halo rows below the own rows
    hi: int              # halo rows above
    prev: Optional[int]  # neighbour slab below (None at a non-periodic edge)
    next: Optional[int]  # neighbour slab above

    @property
    def rows(self) -> int:
        return self.lo + (self.own1 - self.own0) + self.hi

    def local_rows(self) -> np.ndarray:
        """Global row index of each local row (unwrapped: may leave [0, ny))."""
        return np.arange(self.own0 - self.lo, self.own1 + self.hi)


def partition(ny: int, n_slabs: int, periodic_y: bool, ghost: int = STENCIL_DEPTH) -> List[Slab]:
    """Splits ny rows into n_slabs slabs of near-equal height (the lower ones
    one row taller when ny does not divide), each with `ghost` halo rows on
    every side that has a neighbour.  `ghost` must be a positive multiple of
    three and no taller than the thinnest slab."""
    if n_slabs < 1 or ny < n_slabs:
        raise ValueError("need 1 <= n_slabs <= ny")
    if ghost < STENCIL_DEPTH or ghost % STENCIL_DEPTH:
        raise ValueError("ghost must be a positive multiple of %d" % STENCIL_DEPTH)
    base, extra = divmod(ny, n_slabs)
    if n_slabs > 1 and base < ghost:
        raise ValueError("slabs of %d rows cannot feed %d halo rows" % (base, ghost))
    out, y = [], 0
    for s in range(n_slabs):
        h = base + (1 if s < extra else 0)
        prev = s - 1 if s > 0 else (n_slabs - 1 if periodic_y and n_slabs > 1 else None)
        nxt = s + 1 if s < n_slabs - 1 else (0 if periodic_y and n_slabs > 1 else None)
        out.append(Slab(s, y, y + h, ghost if prev is not None else 0,
                        ghost if nxt is not None else 0, prev, nxt))
        y += h
    return out


def slab_bc(bc: dict, slab: Slab) -> dict:
    """Boundary spec of one slab: the domain's x edges; the domain's south
    (north) edge where the slab has no neighbour below (above); an open edge
    with adiabatic temperature towards a neighbour.  With a single slab of a
    periodic axis the domain's own spec stands."""
    out = dict(bc)
    flow, therm = list(bc["flow"]), list(bc["therm"])
    T_edge = list(bc.get("T_edge", (0.0,) * 4))
    if slab.prev is not None or slab.next is not None:
        for edge, nb in ((EDGE_S, slab.prev), (EDGE_N, slab.next)):
            if nb is not None:
                flow[edge], therm[edge], T_edge[edge] = OPEN, T_ADIABATIC, 0.0
    out.update(flow=flow, therm=therm, T_edge=T_edge)
    if slab.prev is not None:       # the heater lies on the domain's south wall
        out.update(heater_x0=0, heater_x1=0)
    return out


def halo_moves(slabs: Sequence[Slab]):
    """(src slab, src local row, dst slab, dst local row, rows) for every
    halo block: a slab's lower halo is its lower neighbour's top own rows,
    its upper halo its upper neighbour's bottom own rows."""
    moves = []
    for d in slabs:
        if d.prev is not None:
            s = slabs[d.prev]
            moves.append((s.index, s.lo + (s.own1 - s.own0) - d.lo, d.index, 0, d.lo))
        if d.next is not None:
            s = slabs[d.next]
            moves.append((s.index, s.lo, d.index, d.lo + (d.own1 - d.own0), d.hi))
    return moves


def exchange_halos(rank_slab: Slab, slabs: Sequence[Slab], pack: Callable[[int, int], object],
                   unpack: Callable[[int, int, object], None],
                   empty: Callable[[int], object], dist, rank_of: Callable[[int], int]):
    """One halo exchange between ranks, each owning one slab: every rank
    sends the own rows its neighbours need and receives its halo rows, with
    batched point-to-point transfers (no rank waits on a fixed order, so
    there is no deadlock on a ring).  pack(y0, n) returns a tensor of those
    local rows, unpack(y0, n, t) writes one, empty(n) allocates a receive
    tensor for n rows."""
    ops, recvs = [], []
    for (si, sy, di, dy, n) in halo_moves(slabs):
        if si == rank_slab.index and n:
            ops.append(dist.P2POp(dist.isend, pack(sy, n), rank_of(di)))
        if di == rank_slab.index and n:
            t = empty(n)
            recvs.append((dy, n, t))
            ops.append(dist.P2POp(dist.irecv, t, rank_of(si)))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()
    for dy, n, t in recvs:
        unpack(dy, n, t)


class _DeviceDouble:
    """A device double at a raw address, for torch (zero copy)."""

    def __init__(self, ptr: int):
        self.__cuda_array_interface__ = {"shape": (3,), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3}


class SlabRunner:
    """An nx x ny domain advanced as n_slabs slab contexts on one device.

    The result equals that of one context of the whole domain: own rows are
    computed from exactly the rows the whole-domain step reads, and with
    buoyancy the mean density is the whole domain's.  FP64 slabs match the
    oracle element by element; the exchange costs two halo blocks of 15
    planes per slab every ghost // 3 steps."""

    def __init__(self, nx, ny, params: dict, bc: dict, n_slabs: int, prec: str = "fp64",
                 ghost: int = STENCIL_DEPTH, stream=None):
        import torch

        import paper_2205_00686_gb300 as lbm
        self.torch, self.lbm = torch, lbm
        self.nx, self.ny, self.prec = nx, ny, prec
        self.periodic_y = bc["flow"][EDGE_S] == PERIODIC
        if self.periodic_y and bc["therm"][EDGE_S] != T_PERIODIC and n_slabs > 1:
            # a periodic flow axis whose temperature is held at the edges
            # (Section 4.1): the halo that wraps the flow would have to carry
            # the thermal edge inside a slab, which the slabs' edge-based
            # boundaries cannot express
            raise ValueError("slabs need the y axis periodic for both lattices or for neither")
        self.slabs = partition(ny, n_slabs, self.periodic_y, ghost)
        self.ghost = ghost
        self.params, self.bc = dict(params), bc
        self.gravity = float(params.get("gravity", 0.0)) != 0.0
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.doms = []
        self.step_count = 0

    def init_fields(self, rho, ux, uy, T):
        torch = self.torch
        rho, ux, uy, T = (np.asarray(a, dtype=np.float64).reshape(self.ny, self.nx)
                          for a in (rho, ux, uy, T))
        p = dict(self.params)
        # one storage reference for every slab, so rows move unchanged
        p.setdefault("rho_ref", 0.0)
        p.setdefault("T_ref", 0.0)
        if not p["rho_ref"] > 0:
            p["rho_ref"] = float(rho.mean())
        if not p["T_ref"] > 0:
            p["T_ref"] = float(T.mean())
        for d in self.doms:
            d.close()
        self.doms = []
        for sl in self.slabs:
            rows = sl.local_rows() % self.ny
            d = self.lbm.Domain(self.nx, sl.rows, p, slab_bc(self.bc, sl), prec=self.prec,
                                stream=self.stream.cuda_stream)
            d.set_partition(sl.lo, sl.lo + sl.own1 - sl.own0, self.nx * self.ny)
            d.init_fields(rho[rows], ux[rows], uy[rows], T[rows])
            self.doms.append(d)
        # step 0 reads the whole domain's initial density sum from slot 2
        self._rings = [torch.as_tensor(_DeviceDouble(d.mass_ring()), device="cuda")
                       for d in self.doms]
        with torch.cuda.stream(self.stream):
            total = torch.full((1,), float(rho.sum()), dtype=torch.float64, device="cuda")
            for r in self._rings:
                r[2:3].copy_(total)
        self.step_count = 0
        nb = max(self.doms[0].rows_bytes(self.ghost), 1)
        self._buf = torch.empty(nb, dtype=torch.uint8, device="cuda")

    def exchange(self):
        """Copies every halo block from its neighbour's own rows (device to
        device, in stream order)."""
        for (si, sy, di, dy, n) in halo_moves(self.slabs):
            if n:
                self.doms[si].pack_rows(sy, n, self._buf.data_ptr())
                self.doms[di].unpack_rows(dy, n, self._buf.data_ptr())

    def _combine_mass(self, s: int):
        torch = self.torch
        with torch.cuda.stream(self.stream):
            tot = sum(r[s % 3:s % 3 + 1] for r in self._rings)
            for r in self._rings:
                r[s % 3:s % 3 + 1].copy_(tot)

    def step(self, n: int):
        per = 1 if self.gravity else self.ghost // STENCIL_DEPTH
        done = 0
        while done < n:
            k = min(per, n - done)
            self.exchange()
            for d in self.doms:
                d.step(k)
            if self.gravity:
                self._combine_mass(self.step_count)
            self.step_count += k
            done += k

    def _own(self, a, sl):
        return a[..., sl.lo:sl.lo + sl.own1 - sl.own0, :]

    def get_rho_u_T(self):
        """rho, u, T of the whole domain [ny][nx] (the halos are refreshed
        first: an own row next to a halo needs its psi for the force)."""
        self.exchange()
        parts = [[self._own(a, sl) for a in d.get_rho_u_T()] for d, sl in zip(self.doms, self.slabs)]
        return tuple(np.concatenate([p[i] for p in parts], axis=0) for i in range(4))

    def populations(self):
        """f [9][ny][nx], g [5][ny][nx], P [ny][nx] of the whole domain."""
        parts = [[self._own(a, sl) for a in d.populations()] for d, sl in zip(self.doms, self.slabs)]
        return tuple(np.concatenate([p[i] for p in parts], axis=-2) for i in range(3))

    def set_tile(self, threads: int, rows: int, staged: Optional[bool] = None):
        for d in self.doms:
            d.set_tile(threads, rows)
            if staged is not None:
                d.staged = staged

    def close(self):
        for d in self.doms:
            d.close()
        self.doms = []
