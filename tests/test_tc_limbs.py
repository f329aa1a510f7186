"""CPU checks, in exact Python integers, of the limb formation the
tensor-core product uses after its MMAs (tccore.cuh, tcmul.cu): biased
column sums V_j = sum_k (coef(8j+k) + 2^31) 2^(8k), the carry and bias
passes per tile, the split form (tiles with no carry in, linked by the
finishing kernel's sum of (H_t + k_t) B^((t+1) L)), and the band mode of
the division's quotient product (tiles anchored at the column of limb lo,
2^32 added at L0, quotient q or q + 1).  The kernels are checked against
the oracle on the GPU; these pin the algebra they implement."""
import numpy as np
import pytest

B = 1 << 64
M64 = B - 1
BIAS_L0, BIAS = 0x8080808080000000, 0x8080808080808080


def to_int(limbs):
    return sum(int(x) << (64 * i) for i, x in enumerate(limbs))


def digits(limbs, carry):
    """Signed base-256 digits: byte k sign-extended plus the top bit of byte
    k - 1; with `carry` the carry digit (top bit of the last byte) on top,
    without it the digits spell x - top_bit(x) B^n."""
    by = [(int(x) >> (8 * k)) & 0xFF for x in limbs for k in range(8)]
    out = []
    for i, b in enumerate(by):
        prev = by[i - 1] if i > 0 else 0
        out.append((b - 256 if b & 0x80 else b) + (prev >> 7))
    if carry:
        out.append(by[-1] >> 7)
    return out


def column_sums(x, y, xc=True):
    dx = np.array(digits(x, xc), dtype=np.int64)
    dy = np.array(digits(y, True), dtype=np.int64)
    return [int(c) for c in np.convolve(dx, dy)]


def biased_limbs(coef, j0, n):
    """V_j for limbs j0 .. j0 + n - 1 (coef beyond its end is 0, still biased)."""
    out = []
    for j in range(j0, j0 + n):
        v = 0
        for k in range(8):
            s = 8 * j + k
            c = coef[s] if s < len(coef) else 0
            v += (c + (1 << 31)) << (8 * k)
        out.append(v)
    return out


def carry_pass(V, hprev, cin):
    """One tile's pass: out_j = low(V_j) + high(V_(j-1)) + carry; returns the
    limbs, the carry out and the high word of the last limb."""
    out, c = [], cin
    for j, v in enumerate(V):
        h = hprev if j == 0 else V[j - 1] >> 64
        t = (v & M64) + h + c
        out.append(t & M64)
        c = t >> 64
    return out, c, V[-1] >> 64


def operands(seed, nx, ny, pattern=None):
    rng = np.random.default_rng(seed)
    if pattern is not None:
        x = [pattern] * nx
        y = [pattern ^ M64] * ny
    else:
        x = [int(v) | (int(rng.integers(0, 2)) << 63)
             for v in rng.integers(0, 1 << 63, nx, dtype=np.uint64)]
        y = [int(v) | (int(rng.integers(0, 2)) << 63)
             for v in rng.integers(0, 1 << 63, ny, dtype=np.uint64)]
    return x, y


SHAPES = [(1, 1), (3, 5), (16, 16), (17, 40), (33, 33), (64, 64)]
PATTERNS = [None, 0xFFFFFFFFFFFFFFFF, 0x7F807F807F807F80, 0x8080808080808080]


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("tile_limbs", [16, 32, 4096])
def test_tiles_with_fused_bias(nx, ny, pattern, tile_limbs):
    """Tiles in order, each pass adding the previous limb's high word and
    subtracting the bias (carry and borrow handed on): the product mod
    B^nout, for full and low-part products."""
    x, y = operands(nx * 100 + ny, nx, ny, pattern)
    coef = column_sums(x, y)
    for nout in sorted({nx + ny, max(1, (nx + ny) // 2), 1}):
        out, c, h, borrow = [], 0, 0, 0
        for j0 in range(0, nout, tile_limbs):
            n = min(tile_limbs, nout - j0)
            limbs, c, h = carry_pass(biased_limbs(coef, j0, n), h, c)
            for j, v in enumerate(limbs):  # the bias, as a borrow chain across tiles
                beta = BIAS_L0 if j0 + j == 0 else BIAS
                t = v - beta - borrow
                borrow = 1 if t < 0 else 0
                out.append(t & M64)
        assert to_int(out) == (to_int(x) * to_int(y)) % (1 << (64 * nout))


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("pattern", PATTERNS)
def test_x_without_carry_digit(nx, ny, pattern):
    """Without x's carry digit the digits spell x_s = x - t_x B^nx, and
    x y = x_s y + t_x y B^nx (the correction addition)."""
    x, y = operands(nx * 7 + ny, nx, ny, pattern)
    coef = column_sums(x, y, xc=False)
    value = sum(c << (8 * s) for s, c in enumerate(coef))
    tx = x[-1] >> 63
    assert value + tx * to_int(y) * (1 << (64 * nx)) == to_int(x) * to_int(y)


@pytest.mark.parametrize("nx,ny", [(16, 16), (40, 33), (64, 64), (1, 100)])
@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("tile_limbs", [16, 48])
def test_split_tiles_and_finish(nx, ny, pattern, tile_limbs):
    """Each tile computed with no carry in gives limbs L_t, carry k_t and
    high word H_t; the product is concat(L) + sum_t (H_t + k_t) B^((t+1) L)
    minus the bias sum, mod B^nout."""
    x, y = operands(nx + 3 * ny, nx, ny, pattern)
    coef = column_sums(x, y)
    nout = nx + ny
    limbs, links = [], 0
    for t, j0 in enumerate(range(0, nout, tile_limbs)):
        n = min(tile_limbs, nout - j0)
        lt, kt, ht = carry_pass(biased_limbs(coef, j0, n), 0, 0)
        limbs += lt
        assert ht + kt < B
        links += (ht + kt) << (64 * (j0 + n))
    bias = BIAS_L0 + sum(BIAS << (64 * j) for j in range(1, nout))
    got = (to_int(limbs) + links - bias) % (1 << (64 * nout))
    assert got == to_int(x) * to_int(y)


@pytest.mark.parametrize("nx,ny", [(9, 17), (20, 33), (40, 64), (64, 64)])
@pytest.mark.parametrize("pattern", PATTERNS)
def test_band_mode_quotient(nx, ny, pattern):
    """Band mode: columns below the one holding limb lo are skipped (D),
    the first computed limb is L0 = 16 floor(lo / 16), 2^32 is added there;
    floor(value / B^(h - L0)) is floor(x y / B^h) or one more, h >= lo + 2,
    and the value fits nout - L0 limbs while x y + B^h < B^nout."""
    x, y = operands(nx * 11 + ny, nx, ny, pattern)
    coef = column_sums(x, y)
    X, Y, nout = to_int(x), to_int(y), nx + ny
    for lo in range(1, nout - 2, 3):
        L0 = 16 * (lo // 16)
        D = sum(c << (8 * s) for s, c in enumerate(coef) if s < 8 * L0)
        assert abs(D) < (1 << 31) * (1 << (64 * L0)) // 255 + 1
        value = (X * Y - D) // (1 << (64 * L0)) + (1 << 32)
        assert (X * Y - D) % (1 << (64 * L0)) == 0
        for h in range(lo + 2, nout):
            if X * Y + (1 << (64 * h)) >= 1 << (64 * nout):
                continue
            assert 0 <= value < 1 << (64 * (nout - L0))
            q = X * Y // (1 << (64 * h))
            assert value // (1 << (64 * (h - L0))) in (q, q + 1)
