"""CPU restatement of the tensor-core product's schedule (tccore.cuh: the
layout, the tile loop with band anchoring and split tiles, the per-group MMA
spans, clearing MMAs and drains), checked for every shape family the
library launches: each MMA stays inside its accumulator (TMEM columns) and
reads x chunks inside the stored, zero-padded x (shared memory); every
digit product of a computed column is taken exactly once; columns a span
widens into read only zero chunks; the accumulator a group writes is
cleared or overwritten first and drained over all it holds."""
import pytest


def layout(NT, G, XC, nx, ny):
    mx = (8 * nx + (1 if XC else 0) + 127) // 128
    ey = (8 * ny + 127) // 128
    ctot = mx + ey
    ptot = (mx + 32) | 1
    return dict(mx=mx, ey=ey, ctot=ctot, ptot=ptot)


def group_span(c0, W, ea, eb, mx):
    lo = (max(c0, ea) - c0) & ~15
    hi = (min(c0 + W, eb + mx) - c0 + 15) & ~15
    return lo, hi


def schedule(NT, G, XC, nx, ny, nout, lo_band=0, tile=None):
    """Yields (c0, W, groups); groups = list of (ea, eb, [(e, lo, hi)])."""
    L = layout(NT, G, XC, nx, ny)
    cfirst = lo_band // 16 if lo_band > 0 else 0
    c0 = cfirst
    while 16 * c0 < nout:
        W = min(L["ctot"] - c0, NT, (nout - 16 * c0 + 15) // 16)
        W = (W + 15) & ~15
        skip = 16 * (c0 + W) <= lo_band or (tile is not None and c0 != NT * tile)
        if not skip:
            e_lo = max(0, c0 - L["mx"] + 1)
            e_hi = min(c0 + W - 1, L["ey"])
            groups = []
            ea = e_lo
            while ea <= e_hi:
                eb = min(ea + G - 1, e_hi)
                mmas = []
                for e in range(ea, eb + 1):
                    ca = max(c0, e) - c0
                    cb = min(c0 + W, e + L["mx"]) - c0
                    mmas.append((e, ca & ~15, (cb + 15) & ~15))
                groups.append((ea, eb, mmas))
                ea += G
            yield c0, W, groups
        c0 += NT


def check(NT, G, XC, nx, ny, nout, lo_band=0, tile=None):
    L = layout(NT, G, XC, nx, ny)
    mx, ptot = L["mx"], L["ptot"]
    computed = set()
    for c0, W, groups in schedule(NT, G, XC, nx, ny, nout, lo_band, tile):
        assert W % 16 == 0 and 16 <= W <= NT
        taken = {}
        for ea, eb, mmas in groups:
            slo, shi = group_span(c0, W, ea, eb, mx)
            assert 0 <= slo < shi <= NT
            # the first MMA overwrites [slo, shi) when its span is the group's,
            # else a clearing MMA of N = shi - slo comes first
            assert shi - slo <= 256
            for e, lo, hi in mmas:
                assert lo % 16 == 0 and hi % 16 == 0 and lo < hi
                assert slo <= lo and hi <= shi          # drained, and cleared first
                assert 0 <= lo and hi <= NT             # inside the accumulator
                assert hi - lo <= 256                   # MMA N
                # x chunks read: p = c - e for tile columns c in [c0 + lo, c0 + hi),
                # stored at p + 16 in [0, ptot); outside [0, mx) they are zero
                p_first, p_last = c0 + lo - e, c0 + hi - 1 - e
                assert 0 <= p_first + 16 and p_last + 16 < ptot
                for c in range(c0 + lo, c0 + hi):
                    p = c - e
                    if 0 <= p < mx:
                        taken[(c, e)] = taken.get((c, e), 0) + 1
                    else:
                        assert -16 <= p < ptot - 16  # a zero chunk
        # every (column, block) pair of the tile with x in range: exactly once
        for c in range(c0, c0 + W):
            if c >= L["ctot"]:
                continue
            for e in range(max(0, c - mx + 1), min(c, L["ey"]) + 1):
                assert taken.get((c, e), 0) == 1, (c, e)
            computed.add(c)
    return computed


SQUARE = [1, 15, 16, 17, 100, 255, 256, 257, 511, 512, 513, 1000, 1023, 1024, 1031,
          2047, 2048, 2049, 4095, 4096, 4097, 8191, 8192, 10000]


def shape_of(nx, ny):
    """tc_shape of tcmul.cu (nx <= ny)."""
    ey = (8 * ny + 127) // 128
    cx, c0 = (8 * nx + 1 + 127) // 128 + ey, (8 * nx + 127) // 128 + ey
    if cx <= 64:
        return 64, 7, True
    if c0 <= 64:
        return 64, 7, False
    if cx <= 128:
        return 128, 8, True
    if c0 <= 128:
        return 128, 8, False
    return 256, 8, True


@pytest.mark.parametrize("n", SQUARE)
def test_full_products(n):
    NT, G, XC = shape_of(n, n)
    cols = check(NT, G, XC, n, n, 2 * n)
    # every column holding a limb of the product is computed
    assert set(range(min(layout(NT, G, XC, n, n)["ctot"], (2 * n + 15) // 16))) <= cols
    if NT == 256:
        check(256, 4, True, n, n, 2 * n)


@pytest.mark.parametrize("nx,ny", [(1, 4200), (3, 4150), (300, 4000), (700, 9000),
                                   (2100, 2100), (5000, 9999), (33, 40), (100, 37)])
def test_ragged_products(nx, ny):
    nx, ny = min(nx, ny), max(nx, ny)
    NT, G, XC = shape_of(nx, ny)
    check(NT, G, XC, nx, ny, nx + ny)


@pytest.mark.parametrize("nx,ny,m", [(512, 512, 513), (512, 512, 1), (300, 4000, 2100),
                                     (4096, 4096, 4096), (8192, 8192, 8193)])
def test_low_parts(nx, ny, m):
    NT, G, XC = shape_of(nx, ny)
    cols = check(NT, G, XC, nx, ny, m)
    assert all(16 * c < m for c in cols if c % NT == 0)


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_band_mode_of_the_quotient_product(n):
    """u (2n limbs) times w (n + 1 limbs), band below limb h - 2 = 2n - 2:
    the first computed column is the one holding that limb."""
    nx, ny = n + 1, 2 * n
    lo = 2 * n - 2
    cols = check(256, 8, True, nx, ny, nx + ny, lo_band=lo)
    assert min(cols) == lo // 16
    check(256, 4, True, nx, ny, nx + ny, lo_band=lo)


@pytest.mark.parametrize("n", [2049, 4096, 8192, 10000])
def test_split_tiles_cover_the_product_once(n):
    T = -(-(2 * n) // 4096)
    seen = []
    for t in range(T):
        seen += sorted(check(256, 8, True, n, n, 2 * n, tile=t))
    assert len(seen) == len(set(seen))
    assert set(seen) == check(256, 8, True, n, n, 2 * n)
