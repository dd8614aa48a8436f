"""The plane schedule of the fused 3-D step (no GPU).  Each CTA marches k
through z0 - 2 .. z1 + 2; within an iteration, phase 1 runs stage A on plane k
and stage C on plane k - 3, then a barrier, phase 2 runs stage B on plane
k - 1, then a barrier.  Shared-memory rings carry each stage's outputs by
plane modulo the ring size.  This model replays that schedule for segments,
walls and periodic domains and checks that every read finds the value
written for the plane it wants (no ring slot was overwritten first), that no
slot is written in the phase in which another plane's value is read from it,
and that every plane of the segment is collided and blended exactly once."""
import itertools

import pytest

# ring sizes of the kernel's shared-memory arrays
RING = {"psi": 3, "rho": 4, "ic": 5, "j": 2, "tdp": 4, "u": 3}


def schedule(z0, z1, nz, walls):
    """(iteration, phase, op, array, plane) for one unit; planes unwrapped."""
    ev = []
    beyond = lambda z: walls and (z < 0 or z >= nz)
    for k in range(z0 - 2, z1 + 3):
        # phase 1: A(k) (ghost psi beyond a wall), C(k - 3)
        if k <= z1 + 1:
            if beyond(k):
                if k in (-1, nz):
                    ev.append((k, 1, "w", "psi", k))
            else:
                for a in ("psi", "rho", "ic", "j", "tdp"):
                    ev.append((k, 1, "w", a, k))
        q = k - 3
        if z0 <= q < z1:
            for dz in (-1, 0, 1):
                if not beyond(q + dz):
                    ev.append((k, 1, "r", "u", q + dz))
                    ev.append((k, 1, "r", "ic", q + dz))
            ev.append((k, 1, "r", "rho", q))
            ev.append((k, 1, "r", "tdp", q))
            ev.append((k, 1, "collide_g", None, q))
        # phase 2: B(k - 1)
        p = k - 1
        if z0 - 1 <= p <= z1 and not beyond(p):
            for dz in (-1, 0, 1):
                ev.append((k, 2, "r", "psi", p + dz))
            ev.append((k, 2, "r", "rho", p))
            ev.append((k, 2, "r", "j", p))
            ev.append((k, 2, "w", "u", p))
            if z0 <= p < z1:
                ev.append((k, 2, "collide_f", None, p))
    return ev


def check(z0, z1, nz, walls):
    slots = {a: {} for a in RING}            # array -> slot -> plane held
    done_f, done_g = [], []
    for (k, ph), group in itertools.groupby(schedule(z0, z1, nz, walls), key=lambda e: e[:2]):
        group = list(group)
        writes = {(a, z % RING[a]): z for _, _, op, a, z in group if op == "w"}
        for _, _, op, a, z in group:
            if op == "r":
                s = z % RING[a]
                assert slots[a].get(s) == z, (z0, z1, nz, walls, k, ph, a, z, slots[a].get(s))
                # a slot another plane is being written into in this phase
                assert writes.get((a, s), z) == z, (k, ph, a, z)
            elif op == "collide_f":
                done_f.append(z)
            elif op == "collide_g":
                done_g.append(z)
        for (a, s), z in writes.items():
            slots[a][s] = z
    assert done_f == list(range(z0, z1)) and done_g == list(range(z0, z1))


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("nz,zseg", [(1, 1), (2, 1), (2, 2), (7, 3), (7, 1), (16, 16), (70, 16),
                                     (256, 48), (5, 2)])
def test_every_read_finds_its_plane(nz, zseg, walls):
    if walls and nz < 2:
        pytest.skip("walls need two planes")
    for z0 in range(0, nz, zseg):
        check(z0, min(nz, z0 + zseg), nz, walls)


def test_a_smaller_ring_is_caught():
    """The model is sharp: with one slot fewer in any ring some read finds
    another plane's value."""
    for a in RING:
        RING[a] -= 1
        try:
            with pytest.raises(AssertionError):
                for walls in (False, True):
                    check(0, 16, 16, walls)
        finally:
            RING[a] += 1
