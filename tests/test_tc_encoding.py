"""CPU checks of the encoding identities the tensor-core product relies on
(tccore.cuh), restated in numpy: the signed base-256 digits of a limb, their
16-bit lane form with the 0x6600 bias, the byte permutations that order the
lanes into fp16 pairs, the exactness of the fp16 unbiasing, and the Hankel
rows read from the two staging copies of a reversed digit run.  GPU parity
tests check the kernels themselves; these pin the arithmetic they are built
on, so a wrong constant or selector shows up without a GPU."""
import numpy as np

M64 = (1 << 64) - 1
LANE, TOP = 0x00FF00FF00FF00FF, 0x0080008000800080
ONE, BIAS = 0x0001000100010001, 0x6600660066006600


def digit(v, below, k):
    """Digit k (k = -1 .. 7) of limb v by the definition: byte k sign
    extended plus the top bit of byte k - 1 (byte -1 = top byte of below)."""
    word = (v << 16) | (below >> 48)  # bytes -2 .. 7 at byte positions 0 .. 9
    b = (word >> (8 * (k + 2))) & 0xFF
    p = (word >> (8 * (k + 1))) & 0xFF
    return (b - 256 if b & 0x80 else b) + (p >> 7)


def recode16(v, below):
    """The lane computation of the kernel's recode16, in Python integers."""
    E, O = v & LANE, (v >> 8) & LANE
    ev = (BIAS + E - ((E & TOP) << 1) + (((O >> 7) & ONE) << 16) + (below >> 63)) & M64
    od = (BIAS + O - ((O & TOP) << 1) + ((E >> 7) & ONE)) & M64
    b7 = below >> 56
    dm1 = (0x6600 + b7 - ((b7 & 0x80) << 1) + ((below >> 55) & 1)) & 0xFFFFFFFF
    return ev, od, dm1


def byte_perm(x, y, s):
    """__byte_perm for selectors 0..7 (no sign replication)."""
    src = (y << 32) | x
    out = 0
    for n in range(4):
        sel = (s >> (4 * n)) & 7
        out |= ((src >> (8 * sel)) & 0xFF) << (8 * n)
    return out


def halves(words):
    """The 16-bit halves of 32-bit words, low half first."""
    out = []
    for w in words:
        out += [w & 0xFFFF, w >> 16]
    return out


def limbs_under_test():
    rng = np.random.default_rng(20261203)
    edge = [0, 1, M64, 1 << 63, (1 << 63) - 1, 0x8080808080808080, 0x7F7F7F7F7F7F7F7F,
            0x7F807F807F807F80, 0x807F807F807F807F, 0x00FF00FF00FF00FF, 0xFF00FF00FF00FF00]
    rand = [int(x) for x in rng.integers(0, 1 << 63, 300, dtype=np.uint64)]
    rand += [int(x) | (1 << 63) for x in rng.integers(0, 1 << 63, 300, dtype=np.uint64)]
    vals = edge + rand
    return [(v, b) for v in vals[:40] for b in vals[:40]] + list(zip(vals, reversed(vals)))


def test_lanes_are_biased_digits():
    for v, below in limbs_under_test():
        ev, od, dm1 = recode16(v, below)
        for j in range(4):
            assert (ev >> (16 * j)) & 0xFFFF == 0x6600 + digit(v, below, 2 * j)
            assert (od >> (16 * j)) & 0xFFFF == 0x6600 + digit(v, below, 2 * j + 1)
        assert dm1 == 0x6600 + digit(v, below, -1)


def test_digits_spell_the_limb():
    """sum_k e_k 256^k over the digits of a number (with the carry digit on
    top) is the number again."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = int(rng.integers(1, 6))
        limbs = [int(x) for x in rng.integers(0, 1 << 63, n, dtype=np.uint64)]
        limbs = [x | (int(rng.integers(0, 2)) << 63) for x in limbs]
        value = sum(x << (64 * i) for i, x in enumerate(limbs))
        total = 0
        for i, x in enumerate(limbs):
            below = limbs[i - 1] if i > 0 else 0
            total += sum(digit(x, below, k) << (8 * (8 * i + k)) for k in range(8))
        total += (limbs[-1] >> 63) << (64 * n)  # the carry digit at position 8n
        assert total == value


def test_lanes_never_carry_into_each_other():
    for v, below in limbs_under_test():
        for k in range(-1, 8):
            assert 0x6580 <= 0x6600 + digit(v, below, k) <= 0x6680


def test_fp16_unbias_is_exact():
    v = np.arange(-128, 129)
    pattern = (0x6600 + v).astype(np.uint16).view(np.float16)
    got = (pattern.astype(np.float32) - np.float32(1536)).astype(np.float16)
    assert np.array_equal(pattern - np.float16(1536), got)
    assert np.array_equal(got.astype(np.int64), v)


def test_x_chunk_order():
    """fill_x: element w of a limb's 16-byte chunk is digit w."""
    for v, below in limbs_under_test()[:500]:
        ev, od, _ = recode16(v, below)
        el, eh, ol, oh = ev & 0xFFFFFFFF, ev >> 32, od & 0xFFFFFFFF, od >> 32
        words = [byte_perm(el, ol, 0x5410), byte_perm(el, ol, 0x7632),
                 byte_perm(eh, oh, 0x5410), byte_perm(eh, oh, 0x7632)]
        assert halves(words) == [0x6600 + digit(v, below, w) for w in range(8)]


def staged_run(v, below):
    """The two staging words of one limb in hank_build: D0 = digits 7..0,
    D1 = digits 6..-1."""
    ev, od, dm1 = recode16(v, below)
    el, eh, ol, oh = ev & 0xFFFFFFFF, ev >> 32, od & 0xFFFFFFFF, od >> 32
    d0 = [byte_perm(oh, eh, 0x7632), byte_perm(oh, eh, 0x5410),
          byte_perm(ol, el, 0x7632), byte_perm(ol, el, 0x5410)]
    d1 = [byte_perm(eh, oh, 0x5432), byte_perm(eh, ol, 0x7610),
          byte_perm(el, ol, 0x5432), byte_perm(el, dm1, 0x5410)]
    return d0, d1


def test_staging_copies_hold_the_reversed_run():
    for v, below in limbs_under_test()[:500]:
        d0, d1 = staged_run(v, below)
        assert halves(d0) == [0x6600 + digit(v, below, 7 - w) for w in range(8)]
        assert halves(d1) == [0x6600 + digit(v, below, 6 - w) for w in range(8)]


def test_hankel_rows_from_the_staging_copies():
    """Row s of a group's Hankel matrices (last block eb) holds the digits
    at 128 eb + 127 - s - w, w = 0..7, read as four 32-bit words from the
    copy whose words start on it (D0 for even s, D1 for odd s)."""
    rng = np.random.default_rng(11)
    for ny, eb, G in ((40, 3, 8), (40, 0, 4), (17, 1, 7), (5, 2, 8)):
        y = [int(x) for x in rng.integers(0, 1 << 63, ny, dtype=np.uint64)]
        y = [x | (int(rng.integers(0, 2)) << 63) for x in y]
        HB = 16 * G + 15

        def limb(i):
            return y[i] if 0 <= i < ny else 0

        def dig(pos):  # digit at position pos of y (0 outside, carry digit at 8 ny)
            i, k = divmod(pos, 8)
            return digit(limb(i), limb(i - 1), k)

        D0, D1 = [], []
        for t in range(HB + 1):
            U = 16 * eb + 15 - t
            d0, d1 = staged_run(limb(U), limb(U - 1))
            D0 += d0
            D1 += d1
        ytop = 128 * eb + 127
        for s in range(8 * HB):
            src = D1 if s & 1 else D0
            row = halves(src[(s >> 1):(s >> 1) + 4])
            assert row == [0x6600 + dig(ytop - s - w) for w in range(8)], (s, eb, G)


def test_group_partial_sums_fit_fp32():
    """An accumulator sums G blocks of 128 digit products between drains:
    at most G 2^21 <= 2^24 in magnitude for G <= 8, the range in which fp32
    holds every integer; the all +-128 byte pattern 0x7F80... reaches 2^24
    with G = 8, so the bound is tight."""
    def group_max(x_limbs, y_limbs, G):
        dx = np.array([digit(int(v), int(x_limbs[i - 1]) if i else 0, k)
                       for i, v in enumerate(x_limbs) for k in range(8)], dtype=np.int64)
        dy = np.array([digit(int(v), int(y_limbs[i - 1]) if i else 0, k)
                       for i, v in enumerate(y_limbs) for k in range(8)], dtype=np.int64)
        nb = len(dy) // 128
        best = 0
        for c in range(nb + len(dx) // 128):      # output column c, coefficient 128 c + t
            for e0 in range(0, nb, G):            # a group of blocks e0 .. e0 + G - 1
                for t in (0, 63, 127):
                    acc = 0
                    for e in range(e0, min(e0 + G, nb)):
                        for i in range(128):
                            xi = 128 * (c - e) + i
                            yi = 128 * e + t - i
                            if 0 <= xi < len(dx) and 0 <= yi < len(dy):
                                acc += int(dx[xi]) * int(dy[yi])
                    best = max(best, abs(acc))
        return best

    pat = [0x7F807F807F807F80] * 128  # 8 blocks of digits alternating -128 / +128
    assert group_max(pat, pat, 8) == 1 << 24
    rng = np.random.default_rng(3)
    x = [int(v) for v in rng.integers(0, 1 << 63, 128, dtype=np.uint64)]
    y = [int(v) for v in rng.integers(0, 1 << 63, 128, dtype=np.uint64)]
    for G in (4, 7, 8):
        assert group_max(x, y, G) <= G << 21 <= 1 << 24
    assert float(np.float32(1 << 24)) == 1 << 24
    assert float(np.float32((1 << 24) - 1)) == (1 << 24) - 1
