"""The erf inside the tcgen05 surrogate forward's GELU: Abramowitz & Stegun
7.1.28, erf(x) = 1 - (1 + a1 x + ... + a6 x^6)^-16 (x >= 0, odd), with a
published absolute error bound of 3e-7.  Pinned here against the exact erf
(scipy): the coefficients in FP64 must meet the published bound, and the
kernel's FP32 operation sequence (fused multiply-adds, four squarings, a
reciprocal) must stay within that bound plus its FP32 evaluation error,
far below the 2^-9 relative rounding of the BF16 activation it feeds.
The kernel evaluates twice GELU on pairs in the rearranged form
2 z Phi(z) = (z + |z|) - |z| (1 + p(|z|))^-16, with the coefficients scaled
by 2^(-i/2) so the polynomial takes |z| instead of |z| / sqrt 2 (the factor
1/2 sits, exactly, in the next layer's weights); that FP32 sequence is
pinned against the exact GELU as well."""
import numpy as np
from scipy.special import erf

A = [7.05230784e-2, 4.22820123e-2, 9.2705272e-3, 1.520143e-4, 2.765672e-4, 4.30638e-5]


def erf_as_f64(x):
    ax = np.abs(x)
    p = np.zeros_like(ax)
    for a in reversed(A):
        p = (p + a) * ax
    p = p + 1.0
    return np.sign(x) * (1.0 - p ** -16)


def f32(v):
    return np.asarray(v, np.float64).astype(np.float32).astype(np.float64)


def fma32(a, b, c):
    return f32(a * b + c)  # one rounding of the exact product-sum


def erf_as_f32(x):
    ax = np.abs(f32(x))
    p = fma32(ax, f32(A[5]), f32(A[4]))
    for a in (A[3], A[2], A[1], A[0], 1.0):
        p = fma32(ax, p, f32(a))
    q = f32(p * p)
    for _ in range(3):
        q = f32(q * q)
    with np.errstate(over="ignore", divide="ignore"):
        r = f32(np.where(np.isinf(q), 0.0, 1.0 / q))
    return np.sign(x) * f32(1.0 - r)


def test_published_bound_in_fp64():
    x = np.linspace(-8.0, 8.0, 400001)
    assert np.max(np.abs(erf_as_f64(x) - erf(x))) <= 3.0e-7


def test_fp32_sequence_and_gelu():
    x = np.linspace(-12.0, 12.0, 200001)
    e = erf_as_f32(x)
    # published bound + FP32 evaluation (16-fold growth of p's relative error)
    assert np.max(np.abs(e - erf(x))) <= 3.0e-6
    z = x * np.sqrt(2.0)
    gelu = z * (0.5 + 0.5 * e)
    exact = z * 0.5 * (1.0 + erf(x))
    assert np.max(np.abs(gelu - exact) / np.maximum(np.abs(z), 1.0)) <= 2.0e-6
    assert np.all(np.abs(e) <= 1.0) and e[-1] == 1.0 and e[0] == -1.0


def gelu_packed_f32(z):
    """The kernel's pair sequence, one lane: scaled coefficients rounded to
    FP32 once, Horner by fused multiply-adds, four squarings, reciprocal,
    one add and one fused multiply-add giving 2 GELU(z); halved here (exact)."""
    z = f32(z)
    a = np.abs(z)
    K = [f32(c * 2.0 ** (-(i + 1) / 2)) for i, c in enumerate(A)]
    p = fma32(a, K[5], K[4])
    for c in (K[3], K[2], K[1], K[0], 1.0):
        p = fma32(a, p, c)
    q = f32(p * p)
    for _ in range(3):
        q = f32(q * q)
    with np.errstate(over="ignore", divide="ignore"):
        r = f32(np.where(np.isinf(q), 0.0, 1.0 / q))
    return 0.5 * fma32(a, -r, f32(z + a))


def test_packed_gelu_sequence():
    # the rearrangement is exact algebra: (z + |z| E) / 2 = z (1 + erf(z / sqrt 2)) / 2
    z = np.linspace(-16.0, 16.0, 320001)
    exact = z * 0.5 * (1.0 + erf(z / np.sqrt(2.0)))
    with np.errstate(over="ignore"):
        g = gelu_packed_f32(z)
    assert np.max(np.abs(g - exact) / np.maximum(np.abs(z), 1.0)) <= 2.0e-6
    # limits: relu for large |z| (the 16th power overflows to inf), 0 at 0
    assert gelu_packed_f32(np.array([0.0]))[0] == 0.0
    with np.errstate(over="ignore"):
        big = gelu_packed_f32(np.array([-30.0, 30.0]))
    assert big[0] == 0.0 and big[1] == 30.0
    # a dropped scale on the coefficients (unscaled a_i acting on |z|) is caught
    wrong = np.sign(z) * (1.0 - (1.0 + sum(c * np.abs(z) ** (i + 1) for i, c in enumerate(A))) ** -16.0)
    assert np.max(np.abs(z * 0.5 * (1.0 + wrong) - exact)) > 1e-2
