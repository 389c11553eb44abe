"""Accuracy of the radix-9 twiddles that the specialised FFT stages form as products instead of
reading them (the HOM_TW_POW choice): from the FP32 table entries w = w_j and w^4, the powers
w^2 = w w, w^3 = w^2 w, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3, w^8 = w^4 w^4, each complex
product taken as (fma(a.x, b.x, -rn(a.y b.y)), fma(a.x, b.y, rn(a.y b.x))) in FP32.  For every
radix-9 stage with a span L > 1 of every specialised size, the products stay within a few FP32
ulps of the exact twiddles (the table entries themselves are within half an ulp)."""
import numpy as np
import pytest

# DIT radix orders of the specialised sizes with a radix-9 stage (75 = 5 x 15 and 225 = 15 x 15 have none)
PLANS = {45: (5, 9), 135: (15, 9), 405: (5, 9, 9), 1215: (15, 9, 9), 27: (3, 9), 81: (9, 9), 243: (3, 9, 9)}


def _f32(x):
    return np.float32(x)


def _fma(a, b, c):
    # a b + c with one rounding to FP32 (the FP64 product of two FP32 values is exact)
    return _f32(np.float64(a) * np.float64(b) + np.float64(c))


def _cmul(a, b):
    return (_fma(a[0], b[0], -_f32(np.float64(a[1]) * np.float64(b[1]))),
            _fma(a[0], b[1], _f32(np.float64(a[1]) * np.float64(b[0]))))


def _entry(n, t):
    ang = 2.0 * np.pi * (t % n) / n
    return (_f32(np.cos(ang)), _f32(-np.sin(ang)))


@pytest.mark.parametrize("n", sorted(PLANS))
def test_radix9_twiddle_products_stay_within_a_few_ulps(n):
    radices = PLANS[n]
    worst = 0.0
    span = 1
    for R in radices:
        L = span
        span *= R
        if R != 9 or L == 1:
            continue
        ts = n // (L * R)
        for j in range(L):
            w = {1: _entry(n, j * ts), 4: _entry(n, 4 * j * ts)}
            w[2] = _cmul(w[1], w[1])
            w[3] = _cmul(w[2], w[1])
            w[5] = _cmul(w[4], w[1])
            w[6] = _cmul(w[4], w[2])
            w[7] = _cmul(w[4], w[3])
            w[8] = _cmul(w[4], w[4])
            for q in range(1, 9):
                ang = 2.0 * np.pi * ((j * q * ts) % n) / n
                err = max(abs(float(w[q][0]) - np.cos(ang)), abs(float(w[q][1]) + np.sin(ang)))
                worst = max(worst, err)
    assert worst > 0.0
    # FP32 ulp at 1 is 1.19e-7: the table entries are within 6e-8, the products within 2 ulps
    # (measured worst 1.43e-7 at 405 and 1215)
    assert worst < 2.4e-7, worst
