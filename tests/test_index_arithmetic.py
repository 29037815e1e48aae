"""CPU check of the first-tier pixel index arithmetic of the CUDA rasterizer (csrc/pcr_certified.cuh,
pixel_axis), restated step by step in IEEE float32 (numpy rounds every float32 operation to nearest, as
the kernel's __fadd_rn / __fsub_rn do).

The kernel floors the pixel coordinate f without a conversion instruction: g = (f - 0.5) + 1.5 * 2^23
rounds f - 0.5 to the nearest integer because the sum lies in [2^23, 2^24), where floats are the
integers; the pixel is then the difference of the bit patterns of g and 1.5 * 2^23. Every index the
kernel produces must be floor(f), inside [0, size), whenever it reports the axis as decided.
"""
import numpy as np

F32 = np.float32


def pixel_axis(f, E, size):
    """float32 restatement: returns (state, px); state 0 decided, 1 outside, 2 undecided."""
    f, E, size = F32(f), F32(E), F32(size)
    if not (E < F32(0.25)):
        return 2, None
    if not (f >= F32(0)):
        return (1 if f < -E else 2), None
    if not (f < size + F32(1)):
        return (1 if f >= size + F32(1) else 2), None
    g = (f - F32(0.5)) + F32(12582912.0)
    fl = g - F32(12582912.0)
    fr = f - fl
    if not (fr >= E and fr < F32(1) - E):
        return 2, None
    k = int(np.array(g, np.float32).view(np.int32)) - 0x4B400000
    if fl >= size:
        return 1, None
    return 0, k


def _check(values, E, size):
    for f in values:
        st, k = pixel_axis(f, E, size)
        if st == 0:
            exact = np.floor(np.float64(F32(f)))
            assert k == int(exact), (f, k)
            assert 0 <= k < size
            assert np.floor(np.float64(F32(f)) - E) == k and np.floor(np.float64(F32(f)) + E) == k
        elif st == 1:
            ff = np.float64(F32(f))
            assert ff + E < 0 or ff - E >= size, f


def test_low_range_that_once_faulted():
    # f in [0, 0.5): f - 0.5 is negative; the old 2^23 shift left the binade of integers here
    vals = np.concatenate([np.linspace(0, 0.5, 20001), np.float32(2.0) ** -np.arange(1, 150, dtype=np.float64)])
    _check(vals, 1e-3, 640)
    _check(vals, 2.0 ** -20, 1)


def test_every_integer_neighbourhood():
    for size in (1, 2, 33, 640, 1920, 16384):
        ks = np.arange(0, size + 2, dtype=np.float64)
        eps = np.array([-3e-3, -1e-3, -2.0 ** -20, 0.0, 2.0 ** -20, 1e-3, 3e-3, 0.25, 0.5, 0.75])
        vals = (ks[:, None] + eps[None, :]).ravel()
        _check(vals, 1e-3, size)
        _check(np.nextafter(vals.astype(np.float32), np.float32(np.inf)), 1e-3, size)
        _check(np.nextafter(vals.astype(np.float32), np.float32(-np.inf)), 1e-3, size)


def test_random_and_special_values():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.uniform(-10, 17000, 200000), [np.nan, np.inf, -np.inf, -0.0, 16384.0, 16385.0]])
    for E in (2.0 ** -20, 1e-4, 1e-3, 0.1, 0.3, np.nan):
        _check(vals, E, 16384)
    assert pixel_axis(np.nan, 1e-3, 100)[0] == 2 and pixel_axis(1.5, np.nan, 100)[0] == 2
    assert pixel_axis(np.inf, 1e-3, 100)[0] == 1
