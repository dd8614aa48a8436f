"""The bulk copies of the staged step, checked on the CPU for every strip of
every domain width up to 700 (and 4096), all four tile widths, FP32 and FP16
g, open and periodic x: each copy starts on a 16-byte boundary in global and
in shared memory, moves a multiple of 16 bytes, stays inside the row pitch
and the staging row, and every thread's staged index holds the column it
reads.  The window arithmetic below restates the kernel's (a strip of
NT - 8 output columns with a 4-column halo, pitch = nx rounded up to 64,
FP16 g rows copied from the 8-column boundary with 8 columns of slack); the
eligibility rule is the library's (periodic x needs nx >= 32 a multiple of
16 bytes' worth of g elements)."""
import pytest


def segments(nx, NT, perx, es):
    """Pieces (source column, staged column, columns) of one plane row of
    the strip starting at output column x0, for element size es."""
    ga = 16 // es                          # columns per 16 bytes
    ntg = NT + (8 if es == 2 else 0)       # staged row length
    W = NT - 8
    out = []
    for x0 in range(0, nx, W):
        X0w = x0 - 4
        w0 = X0w & ~(ga - 1)
        segs = []
        if not perx:
            cs = max(w0, 0)
            ce = (min(w0 + ntg, nx) + ga - 1) & ~(ga - 1)
            segs.append((cs, cs - w0, ce - cs))
        else:
            c, end = w0, w0 + ntg
            while c < end:
                wc = c % nx
                n = min(end - c, nx - wc)
                segs.append((wc, c - w0, n))
                c += n
        out.append((x0, X0w, w0, ntg, segs))
    return out


def eligible(nx, perx, es):
    return (not perx) or (nx % (16 // es) == 0 and nx >= 32)


@pytest.mark.parametrize("NT", [128, 192, 224, 256])
@pytest.mark.parametrize("es", [4, 2])
def test_every_copy_is_aligned_in_bounds_and_covering(NT, es):
    for nx in list(range(1, 701)) + [4096]:
        pitch = (nx + 63) // 64 * 64
        for perx in (False, True):
            if not eligible(nx, perx, es):
                continue
            for x0, X0w, w0, ntg, segs in segments(nx, NT, perx, es):
                assert X0w % 4 == 0
                for src, dst, n in segs:
                    assert n > 0
                    assert (src * es) % 16 == 0 and (dst * es) % 16 == 0 and (n * es) % 16 == 0
                    assert 0 <= src and src + n <= pitch
                    assert 0 <= dst and dst + n <= ntg
                for t in range(NT):
                    X = X0w + t
                    gxl = X % nx if perx else min(max(X, 0), nx - 1)
                    sidx = t if perx else gxl - X0w
                    i = sidx + (X0w - w0)
                    assert 0 <= i < ntg
                    assert any(d <= i < d + n and s + i - d == gxl for s, d, n in segs), \
                        (NT, es, nx, perx, x0, t)
