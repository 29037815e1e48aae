"""CPU check of the first-tier arithmetic of the CUDA rasterizer (csrc/pcr_certified.cuh, classify_fast),
restated step by step in IEEE float32 (numpy rounds every float32 operation to nearest, as the kernel's
__fadd_rn / __fsub_rn / __fmaf_rn do; a directed rounding is restated with nextafter).

Pixel axis. The kernel holds fm, a float estimate of fx - 1/2 for the definition's pixel coordinate fx, and
hE < 1/2 - E, E a bound on |fx - (fm + 1/2)| for a point inside the image. It floors without a conversion
instruction: g = fm + 1.5 * 2^23 rounds fm to the nearest integer k because the sum lies in [2^23, 2^24), where
floats are the integers; k is the difference of the bit patterns of g and 1.5 * 2^23. The axis is decided when
k < size and |fm - k| < hE: every fx within E of fm + 1/2 must then floor to k. A point the kernel does not
decide is certainly outside when fm < -RU(1/2 + Eg) or fm >= RU(size - 1/2 + Eg), Eg the kernel's bound of E
that holds at any |fm|.

Depth code. frac is the fixed-point fraction of t truncated to 23 bits; the code is certain when every t
within D of the fixed-point value has the same floor. The kernel tests |frac - 1/2| < hD with
hD <= 1/2 - D - 2^-22 + 2^-25.
"""
import numpy as np

F32 = np.float32
MAGIC = F32(12582912.0)  # 1.5 * 2^23


def _ru(a):
    """The next float32 above a float64 value that float32 rounding may have lowered (directed rounding up)."""
    f = F32(a)
    return f if np.float64(f) >= a else np.nextafter(f, F32(np.inf))


def pixel_axis(fm, hE, size, eg=None):
    """float32 restatement: returns (state, k); state 0 decided, 1 outside, 2 undecided. eg: the bound used for
    the outside test (default: the largest bound a decided point may have, 1/2 - hE)."""
    fm, hE, size = F32(fm), F32(hE), np.uint32(size)
    with np.errstate(all="ignore"):
        if eg is None:
            eg = _ru(0.5 - np.float64(hE)) if np.isfinite(hE) else F32(np.nan)
        eg = F32(eg)
        g = F32(fm + MAGIC)
        k = np.uint32((int(np.array(g, np.float32).view(np.int32)) - 0x4B400000) & 0xFFFFFFFF)
        d = F32(fm - F32(g - MAGIC))
        if k < size and abs(d) < hE:
            return 0, int(k)
        left = _ru(0.5 + np.float64(eg))
        right = _ru(np.float64(F32(np.float64(size) - 0.5)) + np.float64(eg))
        if (fm < -left or fm >= right) and F32(eg + eg) < F32(3.0e38):  # a finite bound only
            return 1, None
    return 2, None


def _check(values, hE, size, eg=None):
    for fm in values:
        st, k = pixel_axis(fm, hE, size, eg)
        f = np.float64(F32(fm)) + 0.5
        E = 0.5 - np.float64(F32(hE))  # the largest bound the kernel may have been given
        if st == 0:
            assert 0 <= k < size
            assert np.floor(f - E) == k and f + E < k + 1, (fm, k)
        elif st == 1:
            Eo = E if eg is None else np.float64(F32(eg))
            assert f + Eo < 0 or f - Eo >= size, fm


def test_low_range_that_once_faulted():
    # fx in [0, 0.5): fm is negative; an older 2^23 shift left the binade of integers here
    vals = np.concatenate([np.linspace(-0.5, 0.0, 20001), -(np.float32(2.0) ** -np.arange(1, 150, dtype=np.float64))])
    _check(vals, 0.5 - 1e-3, 640)
    _check(vals, 0.5 - 2.0 ** -19, 1)


def test_every_integer_neighbourhood():
    for size in (1, 2, 33, 640, 1920, 16384):
        ks = np.arange(-1, size + 2, dtype=np.float64)
        eps = np.array([-0.5, -3e-3, -1e-3, -2.0 ** -20, 0.0, 2.0 ** -20, 1e-3, 3e-3, 0.25, 0.5])
        vals = (ks[:, None] + eps[None, :]).ravel()
        for hE in (0.5 - 1e-3, 0.5 - 2.0 ** -19, 0.25):
            _check(vals, hE, size)
            _check(np.nextafter(vals.astype(np.float32), np.float32(np.inf)), hE, size)
            _check(np.nextafter(vals.astype(np.float32), np.float32(-np.inf)), hE, size)


def test_random_and_special_values():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.uniform(-10, 17000, 100000), rng.uniform(-1e9, 1e9, 20000),
                           [np.nan, np.inf, -np.inf, -0.0, 16383.5, 16384.5, 2.0 ** 22, -2.0 ** 22, 3e38]])
    for hE in (0.5 - 2.0 ** -19, 0.49, 0.4, 0.1, 0.0, -5.0, -1e6, np.nan, -np.inf):
        _check(vals, hE, 16384)
    assert pixel_axis(np.nan, 0.49, 100)[0] == 2 and pixel_axis(1.5, np.nan, 100)[0] == 2
    assert pixel_axis(np.inf, 0.49, 100)[0] == 1 and pixel_axis(np.inf, 0.49, 100, np.inf)[0] == 2
    # a large bound still culls what is far enough outside, and decides nothing
    assert pixel_axis(-1e6, -100.0, 100)[0] == 1 and pixel_axis(50.0, -100.0, 100)[0] == 2
    # the outside test with its own bound, as the kernel's cull branch takes it
    for eg in (0.0, 2.0 ** -20, 1e-3, 0.3, 7.5, 1e6, np.inf, np.nan):
        _check(vals, 0.49, 16384, eg)
        _check(vals, -1.0, 1920, eg)
    assert pixel_axis(-3e38, 0.49, 100, 1e30)[0] == 1


def test_depth_fraction_test():
    """|frac - 1/2| < hD, with hD as small as 1/2 - D - 2^-22 + 2^-25 allows, certifies D < frac_exact < 1 - D
    for the exact 40-bit fraction; hD > 1/4 certifies D < 1/4."""
    rng = np.random.default_rng(1)
    n = 200000
    frac40 = rng.integers(0, 2 ** 40, n, dtype=np.uint64)
    edges = np.array([0, 1, 2 ** 17 - 1, 2 ** 17, 2 ** 39 - 1, 2 ** 39, 2 ** 40 - 2 ** 17, 2 ** 40 - 1], np.uint64)
    frac40 = np.concatenate([frac40, edges])
    frac_exact = frac40.astype(np.float64) / 2.0 ** 40  # exact in float64 (40 bits)
    frac23 = (frac40 >> np.uint64(17)).astype(np.float64) / 2.0 ** 23  # the kernel's truncated fraction
    for D in (0.0, 1e-9, 3e-4, 0.01, 0.2, 0.2499, 0.3, 0.49):
        hD = F32(0.5 - D - 2.0 ** -22 + 2.0 ** -25)  # the largest value the kernel's fma may produce
        ok = np.abs(frac23.astype(np.float32) - F32(0.5)) < hD  # frac - 1/2 is exact in float32
        assert np.all(frac_exact[ok] > D) and np.all(frac_exact[ok] < 1.0 - D)
        if hD > F32(0.25):
            assert D < 0.25
