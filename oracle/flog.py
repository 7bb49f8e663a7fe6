"""Natural logarithms in float32 and float64 arithmetic with a fixed
operation order (oracle; test infrastructure only).

The energy of the prior cells (Section 2.1) contains ln D for the
logarithmic potential.  Library logarithms round differently on different
machines, so a particle near a cell edge could change cell between two
implementations; this one is defined by its float32 operations alone, and
the GPU path evaluates the same definition.  It follows from the series

    ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...),  s = (m - 1)/(m + 1),

after the reduction x = 2^k m with m in [sqrt(1/2), sqrt(2)] (|s| <= 0.1716,
so the terms to s^9 leave a truncation error below 1e-9 relative):

    b = the bits of x;  k = (b >> 23) - 127;  m = the float with b's mantissa
    and exponent 0 (m in [1, 2)); if m > sqrt 2 (above 0x3fb504f3): m = m/2,
    k = k + 1;  s = (m - 1)/(m + 1);  z = s*s;
    p = ((((2/9) z + 2/7) z + 2/5) z + 2/3) z + 2;  ln m = s*p;
    ln x = k*LN2_HI + (k*LN2_LO + ln m)

with every product and sum a separate float32 operation (no fused
multiply-add), the coefficients 2/(2j+1) rounded to float32, and ln 2 split
into LN2_HI = 0x3f317200 (k*LN2_HI exact for |k| < 256) and LN2_LO, ln 2 -
LN2_HI rounded to float32.  Subnormal x are scaled by 2^24 first; x = 0
gives -inf, negative x or NaN give NaN, +inf gives +inf.
"""
import numpy as np

F = np.float32
C = [F(2.0 / 9.0), F(2.0 / 7.0), F(2.0 / 5.0), F(2.0 / 3.0), F(2.0)]
LN2_HI = np.array([0x3F317200], dtype=np.uint32).view(np.float32)[0]
LN2_LO = F(np.float64(np.log(2.0)) - np.float64(LN2_HI))
SQRT2_BITS = 0x3FB504F3


def log_f32(x):
    """ln x elementwise for a float32 array (see the module docstring)."""
    x = np.asarray(x, dtype=np.float32)
    shape = x.shape
    x = np.atleast_1d(x).copy()
    out = np.empty_like(x)
    finite_pos = np.isfinite(x) & (x > 0)
    xs = x[finite_pos]
    sub = xs < np.finfo(np.float32).tiny
    ks = np.where(sub, -24, 0).astype(np.int32)
    xs[sub] = xs[sub] * F(16777216.0)
    b = xs.view(np.uint32)
    k = ((b >> np.uint32(23)).astype(np.int32) - 127) + ks
    mb = (b & np.uint32(0x007FFFFF)) | np.uint32(0x3F800000)
    up = mb > np.uint32(SQRT2_BITS)
    mb = np.where(up, mb - np.uint32(0x00800000), mb).astype(np.uint32)
    k = k + up.astype(np.int32)
    m = mb.view(np.float32)
    s = (m - F(1)) / (m + F(1))
    z = s * s
    p = C[0]
    for c in C[1:]:
        p = (p * z) + c
    lm = s * p
    kf = k.astype(np.float32)
    res = (kf * LN2_HI) + ((kf * LN2_LO) + lm)
    out[finite_pos] = res
    out[x == 0] = -np.inf
    out[np.isposinf(x)] = np.inf
    out[np.isnan(x) | (x < 0)] = np.nan
    return out.reshape(shape)


def log_f64(x):
    """ln x elementwise for a float64 array by the same reduction and series
    in float64 operations (terms to s^21: truncation below 1e-17 relative):

        b = the bits of x;  k = (b >> 52) - 1023;  m = the double with b's
        mantissa and exponent 0; if m > sqrt 2 (above 0x3ff6a09e667f3bcc):
        m = m/2, k = k + 1;  s = (m - 1)/(m + 1);  z = s*s;
        p = (...((2/21) z + 2/19) z + ... + 2/3) z + 2;  ln m = s*p;
        ln x = k*LN2_HI + (k*LN2_LO + ln m)

    with LN2_HI = ln 2 with its low 32 mantissa bits cleared (k*LN2_HI exact
    for |k| < 2^11) and LN2_LO = ln 2 - LN2_HI rounded to double.  Subnormal x
    are scaled by 2^54 first; 0 -> -inf, negative or NaN -> NaN, +inf -> +inf.
    """
    x = np.asarray(x, dtype=np.float64)
    shape = x.shape
    x = np.atleast_1d(x).copy()
    out = np.empty_like(x)
    ok = np.isfinite(x) & (x > 0)
    xs = x[ok]
    sub = xs < np.finfo(np.float64).tiny
    ks = np.where(sub, -54, 0).astype(np.int64)
    xs[sub] = xs[sub] * 18014398509481984.0
    b = xs.view(np.uint64)
    k = ((b >> np.uint64(52)).astype(np.int64) - 1023) + ks
    mb = (b & np.uint64(0x000FFFFFFFFFFFFF)) | np.uint64(0x3FF0000000000000)
    up = mb > np.uint64(SQRT2_BITS64)
    mb = np.where(up, mb - np.uint64(0x0010000000000000), mb).astype(np.uint64)
    k = k + up.astype(np.int64)
    m = mb.view(np.float64)
    s = (m - 1.0) / (m + 1.0)
    z = s * s
    p = C64[0]
    for c in C64[1:]:
        p = (p * z) + c
    lm = s * p
    kf = k.astype(np.float64)
    out[ok] = (kf * LN2_HI64) + ((kf * LN2_LO64) + lm)
    out[x == 0] = -np.inf
    out[np.isposinf(x)] = np.inf
    out[np.isnan(x) | (x < 0)] = np.nan
    return out.reshape(shape)


SQRT2_BITS64 = 0x3FF6A09E667F3BCC
C64 = [2.0 / (2 * j + 1) for j in range(10, -1, -1)]
LN2_HI64 = np.array([np.array([np.log(2.0)]).view(np.uint64)[0] & np.uint64(0xFFFFFFFF00000000)],
                    dtype=np.uint64).view(np.float64)[0]
LN2_LO64 = float(np.log(2.0) - LN2_HI64)
