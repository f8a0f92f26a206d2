"""Constants of the float-float exponential in pdr_ff.cuh.

The exponential there follows Tang's table-driven method (P. T. P. Tang,
ACM TOMS 15(2), 1989) with 32 table entries: a = n ln2/32 + r with
n = rint(32 a / ln2) and |r| <= ln2/64, so e^a = 2^(n div 32) 2^((n mod 32)/32) e^r.
Each 2^(j/32) is stored as a pair of float32 (hi = the value rounded to
float32, lo = the remainder rounded to float32); ln2/32 is split into three
float32 parts, the first with 12 significant bits so that n * C1 is exact
for n < 4096 (arguments up to 88).

Run it to print the constants; the values are computed in 60-digit decimal
arithmetic and rounded to float32 once.
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60


def f32(d: Decimal) -> np.float32:
    """d rounded to the nearest float32 (ties to even), without double rounding."""
    x = np.float32(float(d))
    for cand in (np.nextafter(x, np.float32(-np.inf)), np.nextafter(x, np.float32(np.inf))):
        if abs(Decimal(float(cand)) - d) < abs(Decimal(float(x)) - d):
            x = cand
    return x


def fmt(v) -> str:
    """Shortest decimal that reads back as the same float32."""
    v = np.float32(v)
    if v == 0 or 1e-3 <= abs(v) < 1e3:
        return np.format_float_positional(v, unique=True, trim="0")
    return np.format_float_scientific(v, unique=True, trim="0")


def split(d: Decimal):
    hi = f32(d)
    lo = f32(d - Decimal(float(hi)))
    return hi, lo


def table():
    ln2 = Decimal(2).ln()
    return [split((ln2 * j / 32).exp()) for j in range(32)]


def ln2_over_32():
    x = Decimal(2).ln() / 32
    # 12 significant bits: x lies in [2^-6, 2^-5), so keep multiples of 2^-17
    c1 = Decimal(int((x * 2 ** 17).to_integral_value())) / 2 ** 17
    c2 = f32(x - c1)
    c3 = f32(x - c1 - Decimal(float(c2)))
    return np.float32(float(c1)), c2, c3


if __name__ == "__main__":
    c1, c2, c3 = ln2_over_32()
    print(f"ln2/32 = {fmt(c1)}f + {fmt(c2)}f + {fmt(c3)}f")
    print(f"32/ln2 = {fmt(f32(32 / Decimal(2).ln()))}f")
    for j, (hi, lo) in enumerate(table()):
        print(f"  {{{fmt(hi)}f, {fmt(lo)}f}},  // 2^({j}/32)")
