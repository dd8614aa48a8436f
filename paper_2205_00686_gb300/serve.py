"""Continuous-batching request loop for many independent simulations.

A request is one simulation (a `workloads.Case`-like object: sizes, params,
boundary spec, initial fields) to be advanced by a number of steps.  The
server

* admits waiting requests while their device memory fits the budget (each
  domain's state lives in a PyTorch-allocated device buffer handed to
  `lbm_create`, so the budget is real memory, and is returned to PyTorch's
  caching allocator when the request retires);
* keeps every admitted domain resident and advances all of them together
  with `lbm_batch_step`: one persistent kernel launch per step walks the
  work units of every domain, so requests that arrived at different times
  overlap on the GPU;
* between chunks of steps, retires the domains that reached their target,
  copies their fields to the host, frees their memory and admits new
  requests into the freed space (continuous batching: no request waits for
  the whole batch to finish).  The loop is pipelined: the next chunk is
  queued before the host waits for the previous one, and admission and
  read-back run on each domain's own stream, so the device is not left idle
  while the host schedules;
* records, per request, the time from arrival to completion, and overall
  the aggregate node updates per second.

Requests in one batch must share precision and physical parameters (the
library's batch rule); the server keeps one batch per distinct parameter
set.  All numerics run in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np


# request outcomes besides the library's own negative codes
CANCELLED = -100      # withdrawn by the client before it finished
ADMIT_FAILED = -101   # its domain could not be created (device memory, bad input)


@dataclasses.dataclass
class Request:
    rid: int
    case: object            # nx, ny, params, bc, fields()
    steps: int
    arrival: float = 0.0
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[tuple] = None      # (rho, ux, uy, T) host arrays
    error: int = 0
    done_steps: int = 0       # steps known to have completed on the device
    planned: int = 0          # steps queued
    detail: str = ""

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class CudaBackend:
    """The real engine: PyTorch device buffers + the library's C ABI.

    Each domain is created and initialised on a stream of its own, and the
    batches step on the backend's stream; attach and detach only order the
    two streams (no host wait), so a domain can be initialised, or read back
    after it left the batch, while the next chunk of steps runs."""

    def __init__(self, prec: str = "fp32", stream=None, autotune_steps: int = 0,
                 autotune_at: int = 1):
        import torch

        import paper_2205_00686_gb300 as lbm
        self.torch = torch
        self.lbm = lbm
        self.prec = prec
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.batches: Dict[tuple, object] = {}
        self.handles: Dict[int, tuple] = {}
        self.handle_of: Dict[int, tuple] = {}   # id(domain) -> its handle
        self.attached: Dict[int, bool] = {}
        # with autotune_steps > 0, a batch's tile is chosen by
        # lbm_batch_autotune (trials of that many steps on a shadow batch of
        # its members' shapes) before the first chunk in which it holds at
        # least autotune_at domains, and kept after: tuned on the first
        # arrival alone, a batch keeps a tile made for one small domain
        self.autotune_steps = int(autotune_steps)
        self.autotune_at = max(1, int(autotune_at))
        self.tuned = set()

    def bytes_for(self, case) -> int:
        # state (both ping-pong copies) plus the field buffers read at retirement
        return self.lbm.lbm_state_bytes(case.nx, case.ny, self.prec) + 32 * case.nx * case.ny

    def _key(self, case):
        return tuple(sorted((k, float(v)) for k, v in case.params.items()))

    def open(self, case, steps: int):
        torch = self.torch
        nbytes = self.lbm.lbm_state_bytes(case.nx, case.ny, self.prec)
        own = torch.cuda.Stream()
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        d = self.lbm.Domain(case.nx, case.ny, case.params, case.bc, prec=self.prec,
                            stream=own.cuda_stream, device_mem=buf.data_ptr(),
                            device_bytes=nbytes)
        try:
            d.init_fields(*case.fields())
            # the domain stops at its own step count inside shared chunks
            d.set_target(int(steps))
        except Exception:
            d.close()
            del buf
            raise
        key = self._key(case)
        if key not in self.batches:
            self.batches[key] = self.lbm.Batch(stream=self.stream.cuda_stream)
        self.batches[key].attach(d)
        h = (d, buf, key, own)
        self.handles[id(h)] = h
        self.handle_of[id(d)] = h
        self.attached[id(h)] = True
        return h

    def step(self, n: int):
        """Queues n steps of every attached domain, then a copy of their error
        words into pinned memory; returns a token for wait()."""
        torch = self.torch
        parts = []
        for key, b in self.batches.items():
            if not len(b):
                continue
            if self.autotune_steps and key not in self.tuned and len(b) >= self.autotune_at:
                b.autotune(self.autotune_steps)
                self.tuned.add(key)
            b.step(n)
            errs = torch.zeros(len(b), dtype=torch.int32).pin_memory()
            b.errors_async(errs.data_ptr())
            parts.append((errs, [id(self.handle_of[id(d)]) for d in b.members]))
        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev, parts

    def wait(self, token) -> Dict[int, int]:
        """Waits for the chunk of `token` only; returns {id(handle): error}
        for the domains whose error word was set by then."""
        ev, parts = token
        ev.synchronize()
        out = {}
        for errs, hids in parts:
            for hid, e in zip(hids, errs.tolist()):
                if e:
                    out[hid] = self.lbm.LBM_ETIMEOUT if e & 4 else (
                        self.lbm.LBM_EPSI if e & 1 else self.lbm.LBM_ENONFINITE)
        return out

    def detach(self, handle):
        if self.attached.get(id(handle)):
            d, buf, key, own = handle
            self.batches[key].detach(d)
            self.attached[id(handle)] = False

    def close(self, handle, read: bool = True):
        self.detach(handle)
        d, buf, key, own = handle
        self.handles.pop(id(handle), None)
        self.handle_of.pop(id(d), None)
        self.attached.pop(id(handle), None)
        out = None
        try:
            if read:
                out = d.get_rho_u_T()
        finally:
            d.close()
            del buf
        return out


class Server:
    """Admission by device memory + chunked continuous batching."""

    def __init__(self, backend, mem_budget: int, chunk: int = 100,
                 clock: Callable[[], float] = time.perf_counter, pipeline: int = 1):
        self.backend = backend
        self.mem_budget = int(mem_budget)
        self.chunk = int(chunk)
        # chunks queued ahead of the one the host waits for: with 2 the device
        # keeps a chunk of work while the host's admissions and read-backs of
        # one round outlast the chunk before it
        self.pipeline = max(1, int(pipeline))
        self.clock = clock
        self.waiting: collections.deque = collections.deque()
        self.active: Dict[int, tuple] = {}       # rid -> (request, handle, bytes)
        self.finished: List[Request] = []
        self.mem_used = 0
        self.node_updates = 0
        self.t_start: Optional[float] = None
        self.max_active = 0
        self._next = 0
        self.retiring = set()                    # rids whose steps are all queued
        self._inflight = collections.deque()    # (token, [(rid, n)], at capacity) of the queued chunks
        # chunks queued while requests were still waiting for memory (the
        # device holds as much as the budget allows): their node updates and
        # the time from the previous chunk's completion to theirs
        self._cap_nodes = 0
        self._cap_time = 0.0
        self._last_done = None

    # ---- request side -------------------------------------------------------
    def submit(self, case, steps: int, arrival: Optional[float] = None) -> Request:
        if steps < 1:
            raise ValueError("steps must be >= 1")
        need = self.backend.bytes_for(case)
        if need > self.mem_budget:
            raise ValueError("request needs %d bytes, more than the whole budget" % need)
        r = Request(self._next, case, int(steps), self.clock() if arrival is None else arrival)
        self._next += 1
        self.waiting.append(r)
        return r

    # ---- scheduling ---------------------------------------------------------
    def _admit(self):
        # first come, first served; a request that does not fit blocks the
        # ones behind it (no starvation of large requests)
        while self.waiting:
            r = self.waiting[0]
            need = self.backend.bytes_for(r.case)
            if self.mem_used + need > self.mem_budget:
                break
            self.waiting.popleft()
            try:
                h = self.backend.open(r.case, r.steps)
            except Exception as e:      # allocation or creation failed: this request only
                r.admitted = r.finished = self.clock()
                r.error = ADMIT_FAILED
                r.detail = str(e)
                self.finished.append(r)
                continue
            r.admitted = self.clock()
            self.active[r.rid] = (r, h, need)
            self.mem_used += need
            self.max_active = max(self.max_active, len(self.active))

    def cancel(self, rid: int) -> bool:
        """Withdraws a request: a waiting one leaves the queue, an active one is
        retired between chunks without reading its fields.  Returns False if it
        had already finished (or never existed)."""
        for r in list(self.waiting):
            if r.rid == rid:
                self.waiting.remove(r)
                r.finished = self.clock()
                r.error = CANCELLED
                self.finished.append(r)
                return True
        if rid in self.active:
            self._retire(rid, error=CANCELLED)
            return True
        return False

    def _retire(self, rid, error=0):
        r, h, need = self.active.pop(rid)
        self.retiring.discard(rid)
        try:
            r.result = self.backend.close(h, read=error == 0)
        except Exception as e:      # a device error that surfaced at the read-back
            r.result = None
            error = error or getattr(e, "code", ADMIT_FAILED)
        r.error = error
        r.finished = self.clock()
        self.mem_used -= need
        self.finished.append(r)

    def tick(self) -> bool:
        """One scheduling round, pipelined so that the device always has a
        chunk of steps queued while the host schedules:

        1. domains whose steps are all queued leave the batch (stream-ordered);
        2. waiting requests are admitted into the freed memory;
        3. the next chunk of steps is queued for the domains still running;
        4. the oldest queued chunk is waited for once more than `pipeline`
           chunks are queued (the newer ones keep the device busy), and its
           error words are checked: a failed domain is retired at once, alone;
        5. domains whose last step has completed are read back and retired.

        Returns False when there is nothing left to do."""
        if self.t_start is None:
            self.t_start = self.clock()
        for rid, (r, h, _) in self.active.items():
            if r.planned >= r.steps and rid not in self.retiring:
                self.backend.detach(h)
                self.retiring.add(rid)
        self._admit()
        running = [(rid, r) for rid, (r, _, _) in self.active.items() if rid not in self.retiring]
        chunk = None
        if running:
            # every running domain advances together by a full chunk; each
            # stops at its own step count inside it (the library's per-domain
            # target), so no domain overshoots and no chunk is cut short
            n = self.chunk
            token = self.backend.step(n)
            moved = []
            for rid, r in running:
                k = min(n, r.steps - r.planned)
                r.planned += k
                moved.append((rid, k))
            chunk = (token, moved, bool(self.waiting))
        if chunk is not None:
            self._inflight.append(chunk)
        if self._inflight and (len(self._inflight) > self.pipeline or chunk is None):
            token, members, at_cap = self._inflight.popleft()
            errs = self.backend.wait(token)
            now = self.clock()
            nodes = 0
            for rid, n in members:
                if rid not in self.active:        # cancelled meanwhile
                    continue
                r, h, _ = self.active[rid]
                r.done_steps += n
                nodes += n * r.case.nx * r.case.ny
                self.node_updates += n * r.case.nx * r.case.ny
                e = errs.get(id(h))
                if e:
                    self._retire(rid, error=e)
            if at_cap and self._last_done is not None:
                self._cap_nodes += nodes
                self._cap_time += now - self._last_done
            self._last_done = now
        for rid in list(self.retiring):
            r = self.active[rid][0]
            if r.done_steps >= r.steps:
                self._retire(rid)
        return bool(self.active or self.waiting or self._inflight)

    def run(self, arrivals=None):
        """Runs until every request is done.  `arrivals` optionally lists
        (time_offset_s, case, steps) submitted when the clock passes them
        (requests arriving while others are on the GPU)."""
        pending = collections.deque(sorted(arrivals or [], key=lambda a: a[0]))
        t0 = self.clock()
        if self.t_start is None:
            self.t_start = t0
        while True:
            now = self.clock()
            while pending and pending[0][0] <= now - t0:
                off, case, steps = pending.popleft()
                self.submit(case, steps, arrival=t0 + off)
            busy = self.tick()
            if not busy and not pending:
                break
            if not busy and pending:
                # idle until the next arrival
                wait = pending[0][0] - (self.clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        return self.stats()

    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.finished if r.latency is not None and not r.error])
        wall = (self.clock() - self.t_start) if self.t_start is not None else 0.0
        return {
            "requests": len(self.finished),
            "failed": sum(1 for r in self.finished if r.error and r.error != CANCELLED),
            "cancelled": sum(1 for r in self.finished if r.error == CANCELLED),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "node_updates": int(self.node_updates),
            "wall_s": wall,
            "mlups": self.node_updates / wall / 1e6 if wall > 0 else None,
            # while requests waited for memory: the device as full as the budget allows
            "mlups_at_capacity": self._cap_nodes / self._cap_time / 1e6 if self._cap_time > 0 else None,
            "max_active": self.max_active,
        }
