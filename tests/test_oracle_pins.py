"""Pins of the CPU oracle against facts that do not come from the oracle.

The oracle (``oracle/oracle.c``) is written on 32-bit half-digits.  Here it
is checked against CPython's arbitrary-precision ``int`` (an independent
library implementation, run, not copied), against brute force on 1- and
2-limb inputs, against closed forms, and against invariants that any correct
implementation must satisfy.  Each group targets a class of plausible bugs:
dropped carries (all-ones chains), wrong digit index (random multi-limb),
transposed operands (non-square products), the add-back branch of long
division (adversarial divisors), the sign/rounding of the Newton step
(the exact error identity of Sec. V-C, Fig. 6).
"""
import random
from fractions import Fraction

import numpy as np
import pytest

B = 1 << 64
EDGE = [0, 1, (1 << 32) - 1, 1 << 32, 1 << 63, B - 1]


def to_int(x) -> int:
    v = 0
    for limb in reversed([int(t) for t in np.asarray(x, dtype=np.uint64)]):
        v = (v << 64) | limb
    return v


def from_int(v: int, n: int) -> np.ndarray:
    assert v >= 0
    out = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        out[i] = v & (B - 1)
        v >>= 64
    assert v == 0, "value does not fit"
    return out


def rand_int(rng, n, top_nonzero=False):
    v = rng.getrandbits(64 * n)
    if top_nonzero and n > 0:
        v |= (rng.getrandbits(64) | 1) << (64 * (n - 1))
        v &= (1 << (64 * n)) - 1
        if v >> (64 * (n - 1)) == 0:
            v |= 1 << (64 * (n - 1))
    return v


def edge_values(n):
    """All n-limb numbers whose limbs are edge values (n <= 2)."""
    if n == 1:
        return list(EDGE)
    return [lo | (hi << 64) for hi in EDGE for lo in EDGE]


# ---------------------------------------------------------------- add / sub
@pytest.mark.parametrize("n", [1, 2])
def test_add_sub_bruteforce_edges(orc, n):
    vals = edge_values(n)
    mod = 1 << (64 * n)
    for x in vals:
        for y in vals:
            s, c = orc.add(from_int(x, n), from_int(y, n))
            assert to_int(s) == (x + y) % mod and c == (x + y) // mod
            d, br = orc.sub(from_int(x, n), from_int(y, n))
            assert to_int(d) == (x - y) % mod and br == int(x < y)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 129, 512, 600])
def test_add_sub_random_vs_python_int(orc, n):
    rng = random.Random(1000 + n)
    mod = 1 << (64 * n)
    for _ in range(20):
        x, y = rand_int(rng, n), rand_int(rng, n)
        s, c = orc.add(from_int(x, n), from_int(y, n))
        assert to_int(s) == (x + y) % mod and c == (x + y) >> (64 * n)
        d, br = orc.sub(from_int(x, n), from_int(y, n))
        assert to_int(d) == (x - y) % mod and br == int(x < y)


@pytest.mark.parametrize("n", [2, 5, 512])
def test_add_sub_closed_forms(orc, n):
    ones = (1 << (64 * n)) - 1
    # (B^n - 1) + 1 = B^n: all limbs zero, carry 1 (the longest carry chain)
    s, c = orc.add(from_int(ones, n), from_int(1, n))
    assert not s.any() and c == 1
    # B^(n-1) - 1: a borrow through n-1 limbs
    d, br = orc.sub(from_int(1 << (64 * (n - 1)), n), from_int(1, n))
    assert br == 0 and all(d[:-1] == np.uint64(B - 1)) and d[-1] == 0
    # 0 - 1 wraps to all ones with borrow out
    d, br = orc.sub(from_int(0, n), from_int(1, n))
    assert br == 1 and all(d == np.uint64(B - 1))
    # a carry chain stopped by one zero limb in the middle
    holed = ones - (((1 << 64) - 1) << (64 * (n // 2)))
    s, c = orc.add(from_int(holed, n), from_int(1, n))
    assert c == 0 and to_int(s) == holed + 1


@pytest.mark.parametrize("n", [1, 4, 300])
def test_add_sub_inverse(orc, n):
    rng = random.Random(7 + n)
    for _ in range(10):
        x, y = rand_int(rng, n), rand_int(rng, n)
        s, c = orc.add(from_int(x, n), from_int(y, n))
        back, br = orc.sub(s, from_int(y, n))
        assert to_int(back) == x and br == c  # (a+b)-b = a; the wrap matches


# ---------------------------------------------------------------- multiply
def test_mul_bruteforce_edges(orc):
    for na in (1, 2):
        for nb in (1, 2):
            for x in edge_values(na):
                for y in edge_values(nb):
                    p = orc.mul(from_int(x, na), from_int(y, nb))
                    assert to_int(p) == x * y


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 1), (1, 3), (5, 9), (64, 64),
                                   (127, 300), (512, 512), (600, 17)])
def test_mul_random_vs_python_int(orc, na, nb):
    rng = random.Random(na * 1000 + nb)
    for _ in range(5):
        x, y = rand_int(rng, na), rand_int(rng, nb)
        p = orc.mul(from_int(x, na), from_int(y, nb))
        assert p.size == na + nb and to_int(p) == x * y
        q = orc.mul(from_int(y, nb), from_int(x, na))
        assert np.array_equal(p, q)  # a b = b a


@pytest.mark.parametrize("n", [1, 2, 3, 16, 512, 1024])
def test_mul_all_ones_closed_form(orc, n):
    """(B^n - 1)^2 = B^2n - 2 B^n + 1: limb 0 is 1, limbs 1..n-1 are 0,
    limb n is B-2, limbs n+1..2n-1 are B-1."""
    ones = np.full(n, np.uint64(B - 1), dtype=np.uint64)
    p = orc.mul(ones, ones)
    assert p[0] == 1
    assert not p[1:n].any()
    assert p[n] == np.uint64(B - 2)
    assert all(p[n + 1:] == np.uint64(B - 1))


def test_mul_residues_commute(orc):
    # the Mersenne prime 2^61 - 1 and two more primes below 2^61 found by a
    # deterministic Miller-Rabin search
    primes = [(1 << 61) - 1, _prev_prime((1 << 61) - 2), _prev_prime((1 << 60) + 12345)]
    rng = random.Random(99)
    for n in (8, 200, 777):
        x, y = rand_int(rng, n), rand_int(rng, n)
        p = to_int(orc.mul(from_int(x, n), from_int(y, n)))
        s, c = orc.add(from_int(x, n), from_int(y, n))
        s = to_int(s) + (c << (64 * n))
        for m in primes:
            assert p % m == (x % m) * (y % m) % m
            assert s % m == (x % m + y % m) % m


def _is_prime(m: int) -> bool:
    if m < 2:
        return False
    small = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    for p in small:
        if m % p == 0:
            return m == p
    d, s = m - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:  # deterministic for m < 3.3e24
        x = pow(a, d, m)
        if x in (1, m - 1):
            continue
        for _ in range(s - 1):
            x = x * x % m
            if x == m - 1:
                break
        else:
            return False
    return True


def _prev_prime(m: int) -> int:
    while not _is_prime(m):
        m -= 1
    return m


def test_residue_primes_are_prime():
    assert _is_prime((1 << 61) - 1) and _is_prime(1000003)
    assert not _is_prime((1 << 61) + 1) and not _is_prime(1000001)


@pytest.mark.parametrize("na,nb,m", [(4, 4, 4), (10, 3, 7), (3, 10, 12), (64, 64, 100),
                                     (512, 512, 512)])
def test_mul_lo_vs_python_int(orc, na, nb, m):
    rng = random.Random(na + 31 * nb + m)
    x, y = rand_int(rng, na), rand_int(rng, nb)
    lo = orc.mul_lo(from_int(x, na), from_int(y, nb), m)
    assert to_int(lo) == (x * y) % (1 << (64 * m))


# ---------------------------------------------------------------- division
def test_divmod_bruteforce_small(orc):
    for nu in (1, 2):
        for nv in (1, 2):
            for x in edge_values(nu):
                for y in edge_values(nv):
                    q, r, s = orc.divmod_(from_int(x, nu), from_int(y, nv))
                    if y == 0:
                        assert s == orc.EDIVZERO and not q.any() and not r.any()
                        continue
                    nq = max(nu - nv + 1, 1)
                    fits = x // y < (1 << (64 * nq))
                    assert s == (orc.OK if fits else orc.EINVAL)
                    assert to_int(q) == (x // y) % (1 << (64 * nq))
                    assert to_int(r) == x % y


@pytest.mark.parametrize("nu,nv", [(2, 1), (3, 2), (8, 3), (17, 16), (64, 32), (600, 300),
                                   (1024, 512), (300, 299), (5, 7)])
def test_divmod_random_vs_python_int(orc, nu, nv):
    rng = random.Random(nu * 7 + nv)
    for t in range(6):
        x = rand_int(rng, nu, top_nonzero=True)
        y = rand_int(rng, nv, top_nonzero=True)
        if t % 2:
            # small top limb of the divisor: large normalisation shift
            y = (y & ((1 << (64 * (nv - 1))) - 1)) | (rng.randrange(1, 1 << 32) << (64 * (nv - 1)))
        q, r, s = orc.divmod_(from_int(x, nu), from_int(y, nv))
        assert s == orc.OK
        assert to_int(q) == x // y and to_int(r) == x % y
        assert to_int(q) * y + to_int(r) == x and to_int(r) < y


def test_divmod_adversarial_divisors(orc):
    """Divisors that make the quotient-digit estimate of long division wrong
    and exercise the add-back branch: B^k + 1, B^(k+1) - 1, top limb 1,
    and divisors with leading zero limbs (declared longer than their value)."""
    rng = random.Random(5)
    for k in (1, 2, 5, 31):
        for y in ((1 << (64 * k)) + 1, (1 << (64 * (k + 1))) - 1, 1 << (64 * k),
                  (1 << (64 * k)) | rng.getrandbits(64 * k)):
            nv = k + 2  # one leading zero limb at least
            for x in (rand_int(rng, 2 * k + 2), (1 << (64 * (2 * k + 2))) - 1,
                      y * ((1 << 64) - 1) + y - 1):
                nu = 2 * k + 3
                q, r, s = orc.divmod_(from_int(x, nu), from_int(y, nv))
                assert s == orc.OK
                assert to_int(q) == x // y and to_int(r) == x % y
    # the classic hard case for the two-digit quotient estimate
    x = (1 << 128) - 1
    y = (1 << 64) + (1 << 63) - 1
    q, r, s = orc.divmod_(from_int(x, 3), from_int(y, 2))
    assert to_int(q) == x // y and to_int(r) == x % y


def test_divmod_quotient_overflow_flag(orc):
    """q has nu - nv + 1 limbs; a divisor with leading zero limbs can make the
    true quotient longer, which is reported (EINVAL) with r still exact."""
    x = (1 << 256) - 1
    y = 3  # declared with 4 limbs
    q, r, s = orc.divmod_(from_int(x, 4), from_int(y, 4))
    assert s == orc.EINVAL and to_int(r) == x % y
    assert to_int(q) == (x // y) % B


def test_divmod_u_less_than_v(orc):
    q, r, s = orc.divmod_(from_int(12345, 2), from_int(1 << 100, 3))
    assert s == orc.OK and to_int(q) == 0 and to_int(r) == 12345


# ---------------------------------------------------------------- shinv / step
@pytest.mark.parametrize("k,h", [(0, 3), (2, 5), (7, 30), (100, 201)])
def test_shinv_power_of_base(orc, k, h):
    """shinv_h(B^k) = B^(h-k)."""
    v = from_int(1 << (64 * k), k + 1)
    w, s = orc.shinv(v, h, h - k + 1)
    assert s == orc.OK and to_int(w) == 1 << (64 * (h - k))


@pytest.mark.parametrize("nv,h", [(1, 2), (3, 6), (40, 81), (256, 512)])
def test_shinv_random_vs_python_int(orc, nv, h):
    rng = random.Random(nv + h)
    y = rand_int(rng, nv, top_nonzero=True)
    w, s = orc.shinv(from_int(y, nv), h, h - nv + 2)
    assert s == orc.OK and to_int(w) == (1 << (64 * h)) // y


def _step_error_identity(v, w, h, m, wp):
    """Sec. V-C, Fig. 6 step: with w = B^(h-m)/v - e (e real), the exact real
    Newton update equals B^h/v - v e^2 B^(2m-h); the floor/ceiling of the step
    lowers it by delta in [0, 1).  Return delta."""
    e = Fraction(B ** (h - m), v) - w
    predicted = Fraction(B ** h, v) - v * e * e * Fraction(B ** (2 * m)) / B ** h
    return predicted - wp


@pytest.mark.parametrize("k,l,m", [(0, 3, 1), (3, 3, 1), (5, 4, 2), (9, 10, 8), (40, 18, 16),
                                   (3, 6, 4)])
def test_step_newton_error_identity(orc, k, l, m):
    rng = random.Random(k * 100 + l * 10 + m)
    for t in range(8):
        v = rand_int(rng, k + 1, top_nonzero=True)
        h = k + l + m
        exact = B ** (h - m) // v
        # perturb the iterate on both sides of B^(h-m)/v
        w = max(exact + rng.randrange(-3, 4) * (t % 3), 1)
        wp, s = orc.step(h, m, from_int(v, k + 1), from_int(w, l + 2), l + m + 3)
        assert s == orc.OK
        delta = _step_error_identity(v, w, h, m, to_int(wp))
        assert 0 <= delta < 1, (t, delta)
        # Newton from below: the result never exceeds B^h / v
        assert to_int(wp) <= B ** h // v


def test_step_exact_power_of_base(orc):
    """v = B^k and w = B^(h-m-k) exactly: d = 0 and w' = w B^m = B^(h-k)."""
    k, l, m = 4, 6, 4
    h = k + l + m
    v = from_int(1 << (64 * k), k + 1)
    w = from_int(1 << (64 * (h - m - k)), l + 1)
    wp, s = orc.step(h, m, v, w, l + m + 2)
    assert s == orc.OK and to_int(wp) == 1 << (64 * (h - k))


def test_prec(orc):
    assert orc.prec(np.zeros(5, dtype=np.uint64)) == 0
    x = np.zeros(9, dtype=np.uint64)
    x[3] = 1
    assert orc.prec(x) == 4
    x[8] = 7
    assert orc.prec(x) == 9


# ---------------------------------------------------------------- batches
def test_batches_match_single(orc):
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_small(seed=11, n=16, count=5)
    out, carry = orc.batch_add(a, b)
    for i in range(a.shape[0]):
        s, c = orc.add(a[i], b[i])
        assert np.array_equal(out[i], s) and carry[i] == c
    sa, sb = inputs.order_pairs(a, b)
    out, borrow = orc.batch_sub(sa, sb)
    assert not borrow.any()
    p = orc.batch_mul(a, b)
    for i in range(a.shape[0]):
        assert to_int(p[i]) == to_int(a[i]) * to_int(b[i])
    u, v = inputs.config_div(8, 6, seed=4)
    q, r, st = orc.batch_divmod(u, v)
    for i in range(u.shape[0]):
        assert st[i] == 0
        assert to_int(q[i]) == to_int(u[i]) // to_int(v[i])
        assert to_int(r[i]) == to_int(u[i]) % to_int(v[i])


# ---- fused programs (Sec. VI, Tables I and II) ------------------------------
@pytest.mark.parametrize("n,k", [(1, 1), (1, 6), (3, 6), (17, 6), (64, 13), (5, 255)])
def test_add_chain_vs_python_int(orc, n, k):
    """a + k b mod B^n and floor((a + k b) / B^n): random and all-ones
    operands (the carry count reaches k)."""
    rng = random.Random(100 * n + k)
    for av, bv in ((rng.getrandbits(64 * n), rng.getrandbits(64 * n)),
                   (B ** n - 1, B ** n - 1), (B ** n - 1, 1), (0, 0)):
        out, c = orc.add_chain(from_int(av, n), from_int(bv, n), k)
        s = av + k * bv
        assert to_int(out) == s % (B ** n)
        assert c == s // (B ** n)


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_poly_vs_python_int(orc, n):
    """(a a + b)(b b + b) + a b mod B^n: every product and sum reduced mod
    B^n gives the residue of the exact polynomial."""
    rng = random.Random(7 * n)
    for av, bv in ((rng.getrandbits(64 * n), rng.getrandbits(64 * n)),
                   (B ** n - 1, B ** n - 1), (1, 0), (0, B ** n - 1)):
        out = orc.poly(from_int(av, n), from_int(bv, n))
        assert to_int(out) == ((av * av + bv) * (bv * bv + bv) + av * bv) % (B ** n)
