"""Pass 2's per-pixel accept bounds (Section 2.2 band test): the band test on u64 integers,
eps_den * (q - qmin) <= eps_num * (qmin + Nq) with both products taken mod 2^64, decides exactly as
bounds.x <= q <= bounds.y with bounds = {qmin, qmin + floor(eps_num (qmin + Nq) / eps_den)} whenever
eps_num (2^40 + Nq) + eps_den 2^40 <= 2^64 (the host condition under which the kernels use the bounds), and
not always beyond it. Python integers, wrap written out, no GPU."""
from __future__ import annotations

import random

M64 = (1 << 64) - 1
QMAX = (1 << 40) - 2      # largest depth code
EMPTY_Q = (1 << 40) - 1   # code of an empty pixel (key all ones >> 24)


def in_band_u64(q, qmin, nq, num, den):
    return (den * ((q - qmin) & M64)) & M64 <= (num * (qmin + nq)) & M64


def bounds(qmin, nq, num, den):
    lo, hi = qmin, qmin + (num * (qmin + nq)) // den
    assert hi <= M64  # the kernel's u64 sum does not wrap either
    return lo, hi


def condition(nq, num, den):
    return num * ((1 << 40) + nq) + (den << 40) <= 1 << 64


def api_valid(nq, num, den):
    return 1 <= den <= 1 << 20 and num * ((1 << 40) + nq) < 1 << 64


def _cases(rng, nq, num, den, k):
    for _ in range(k):
        qmin = rng.choice([0, 1, EMPTY_Q, QMAX, rng.randrange(1 << 40), rng.randrange(1 << 20)])
        _, hi = bounds(qmin, nq, num, den)
        near = [qmin, qmin - 1, qmin + 1, hi, hi + 1, hi - 1, 0, QMAX, rng.randrange(1 << 40)]
        for q in near:
            if 0 <= q <= QMAX:
                yield q, qmin


def test_bounds_decide_like_the_band_test():
    rng = random.Random(7)
    nqs = [0, 1, 1 << 20, 123456789, (1 << 40) - 1]
    eps = [(1, 100), (1, 1), (0, 1), (3, 7), (1, 1 << 20), ((1 << 20) - 1, 1 << 20), (1000, 3)]
    n = 0
    for nq in nqs:
        for num, den in eps:
            if not (api_valid(nq, num, den) and condition(nq, num, den)):
                continue
            for q, qmin in _cases(rng, nq, num, den, 200):
                lo, hi = bounds(qmin, nq, num, den)
                assert in_band_u64(q, qmin, nq, num, den) == (lo <= q <= hi), (q, qmin, nq, num, den)
                n += 1
    assert n > 10000


def test_largest_eps_inside_the_condition():
    """The largest eps_num the condition admits for a few (Nq, eps_den): still the same decisions."""
    rng = random.Random(8)
    for nq in (0, 1 << 30, (1 << 40) - 1):
        for den in (1, 2, 100, 1 << 20):
            num = ((1 << 64) - (den << 40)) // ((1 << 40) + nq)
            assert condition(nq, num, den) and not condition(nq, num + 1, den)
            if not api_valid(nq, num, den):
                continue
            for q, qmin in _cases(rng, nq, num, den, 300):
                lo, hi = bounds(qmin, nq, num, den)
                assert in_band_u64(q, qmin, nq, num, den) == (lo <= q <= hi), (q, qmin, nq, num, den)


def test_beyond_the_condition_the_wrap_accepts_nearer_codes():
    """Outside the condition (a valid eps for the API), the u64 test accepts some q < qmin: the bounds would
    not, which is why the kernels fall back to the stored-key test there."""
    nq, den = 0, 2
    num = (1 << 24) - 1
    assert api_valid(nq, num, den) and not condition(nq, num, den)
    qmin = QMAX
    # den * (qmin - q) = 2^40 + 2^25: the wrapped left side 2^64 - 2^40 - 2^25 is below
    # eps_num * qmin = 2^64 - 2^40 - 2^25 + 2
    q = qmin - (1 << 39) - (1 << 24)
    assert in_band_u64(q, qmin, nq, num, den)
    lo, hi = bounds(qmin, nq, num, den)
    assert not (lo <= q <= hi)


def div_magic(d):
    """k_band_bounds' invariant-divisor constants (Granlund and Montgomery 1994, unsigned, N = 64)."""
    l = 0
    while (1 << l) < d:
        l += 1
    m = (((1 << l) - d) << 64) // d + 1
    assert m < 1 << 64
    return m, min(l, 1), max(l - 1, 0)


def div_by(n, magic):
    m, sh1, sh2 = magic
    t = (m * n) >> 64
    return ((t + (((n - t) & M64) >> sh1)) & M64) >> sh2


def test_invariant_divisor_division_is_exact():
    """floor(n / d) for every divisor the API admits (1..2^20), sampled, and n at the ends of the u64 range,
    near multiples of d and at random."""
    rng = random.Random(9)
    ds = list(range(1, 300)) + [1 << k for k in range(21)] + [(1 << k) + 1 for k in range(1, 20)] + \
        [(1 << k) - 1 for k in range(2, 21)] + [rng.randrange(1, (1 << 20) + 1) for _ in range(300)]
    for d in ds:
        mg = div_magic(d)
        ns = [0, 1, d - 1, d, d + 1, M64, M64 - 1, M64 - d, (M64 // d) * d, (M64 // d) * d - 1]
        ns += [rng.randrange(1 << 64) for _ in range(20)]
        ns += [k * d + r for k in (rng.randrange(1 << 40), rng.randrange(1 << 60)) for r in (0, d - 1)]
        for n in ns:
            n &= M64
            assert div_by(n, mg) == n // d, (n, d)


def band_record_constants(num, den, nq):
    """band_mask restated: 1 + E, mf = ceil(f 2^32) (with the carry into E), C + 1."""
    e1p = 1 + num // den
    mf = -(-((num % den) << 32) // den)
    if mf >> 32:
        e1p, mf = e1p + 1, 0
    c = -(-(255 * (den + num) + num * nq + den) // (256 * den))
    if e1p > 1 << 24 or c > 1 << 56:
        return 0, 0, 1 << 62
    return e1p, mf, c + 1


def band_record_out(key, sk, consts):
    """Pass 1's band-record test on the keys' high words: the point is dropped when this is true."""
    e1p, mf, c1 = consts
    kh, sh = key >> 32, sk >> 32
    return kh >= sh * e1p + c1 + ((sh * mf) >> 32)


def test_band_record_test_is_conservative():
    """Pass 1's band record drops a point only when kh >= sh (1 + E) + floor(sh mf / 2^32) + C + 1 on the keys'
    high words: this must imply the exact u64 condition q > qs and eps_den (q - qs) > eps_num (qs + Nq) for
    q = key >> 24, qs = sk >> 24, at keys placed just below, on and above the band's edge, for empty pixels and
    several eps and Nq; and it must still drop points well beyond the band."""
    rng = random.Random(10)
    n_out = 0
    for nq in (0, 1 << 20, 109951162777, (1 << 40) - 1):
        for num, den in ((1, 100), (3, 7), (1, 1 << 20), (5, 3), (100, 1), ((1 << 20) - 1, 1 << 20)):
            consts = band_record_constants(num, den, nq)
            for _ in range(300):
                qs = rng.choice([rng.randrange(1 << 40), rng.randrange(1 << 30), (1 << 40) - 1, 1])
                sk = (qs << 24) | rng.randrange(1 << 24)
                if rng.random() < 0.05:
                    sk = M64  # empty pixel
                edge = qs + (num * (qs + nq)) // den  # the last code in the band
                for dq in (-2, -1, 0, 1, 2, 3, 1 << 8, 1 << 10, 1 << 20, rng.randrange(1 << 30)):
                    q = min(max(edge + dq, 0), (1 << 40) - 2)
                    key = (q << 24) | rng.randrange(1 << 24)
                    if not band_record_out(key, sk, consts):
                        continue
                    n_out += 1
                    qq, qqs = key >> 24, sk >> 24
                    assert qq > qqs and den * (qq - qqs) > num * (qqs + nq), (key, sk, num, den, nq)
    assert n_out > 1000  # the test does drop points


def test_band_record_constants_never_wrap():
    """At the largest eps and Nq the API admits, the record's 64-bit bound sh (1 + E) + C + 1 + floor(sh mf /
    2^32) stays below 2^64, and where it would not, the record keeps every point."""
    for nq in (0, (1 << 40) - 1):
        for num, den in (((1 << 32) - 1, 1), ((1 << 24) - 1, 1), (1, 1), ((1 << 20) - 1, 1 << 20), (1 << 31, 3)):
            e1p, mf, c1 = band_record_constants(num, den, nq)
            sh = (1 << 32) - 1
            assert sh * e1p + c1 + ((sh * mf) >> 32) < 1 << 63
            if (e1p, mf, c1) == (0, 0, 1 << 62):
                assert not band_record_out(M64 - 1, 0, (e1p, mf, c1))  # nothing is dropped
