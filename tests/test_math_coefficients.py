"""The polynomial coefficients in the kernels' math header are the ones the
committed fit script (csrc/fit_poly.py: least-squares fits at 64 Chebyshev
points, rounded to float32) produces, literal for literal."""
import os
import re
import sys

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_26089_b300", "csrc")


def _function_literals(src, name):
    body = src[src.index(f"float {name}("):]
    body = body[:body.index("\n}\n")]
    return [np.float32(float(x)) for x in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]


def test_header_coefficients_come_from_the_fit_script():
    sys.path.insert(0, CSRC)
    try:
        import fit_poly as F
    finally:
        sys.path.pop(0)
    src = open(os.path.join(CSRC, "pdr_math.cuh")).read()
    for fn, key in (("asin_half", "asin_half (P)"), ("sin_quarter", "sin_quarter (Q)"),
                    ("ln_unit", "ln_unit (L)"), ("log1p_pos", "log1p_pos (M)")):
        g, a, b, deg = F.FITS[key][:4]
        want = set(F.fit(g, a, b, deg).tolist())
        got = [v for v in _function_literals(src, fn) if v not in (np.float32(0.75), np.float32(0.25))]
        # every coefficient the script gives appears in the function (the
        # constant 1 of L and M is written as the fma's last addend)
        assert want <= set(float(v) for v in got) | {1.0}, (fn, sorted(want), got)


def test_fits_are_accurate():
    sys.path.insert(0, CSRC)
    try:
        import fit_poly as F
    finally:
        sys.path.pop(0)
    for key, (g, a, b, deg, poly, f, lo, hi) in F.FITS.items():
        c = F.fit(g, a, b, deg).astype(np.float64)
        x = np.linspace(lo, hi, 200_001)[1:]
        err = np.max(np.abs(poly(x, c) - f(x)) / np.abs(f(x)))
        assert err < 3e-8, (key, err)
