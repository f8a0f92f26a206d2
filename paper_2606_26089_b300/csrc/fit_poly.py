"""Coefficients of the polynomial approximations in pdr_math.cuh.

Each is a least-squares polynomial fit, in double precision, of the reduced
function in its reduced variable, sampled at the 64 Chebyshev points of the
first kind of the interval, with the coefficients then rounded to float32:

* asin(x) = x + x^3 P(x^2),  P fitted on t = x^2 in [0, 1/4]   (degree 5)
* sin(x)  = x + x^3 Q(x^2),  Q fitted on t = x^2 in [0, pi^2/4] (degree 4)
* ln(1 - v) = -v L(v),       L fitted on v in [0, 1/4]          (degree 6)
* ln(1 + x) = x M(x),        M fitted on x in [0, 1/4]          (degree 6)

Run it to print the coefficients (lowest order first) and the largest
difference between each fitted polynomial and the function on a fine grid
(the error of the fit itself, before float32 evaluation).  The float32
accuracy over each function's whole argument range is what the GPU test of
pdr_math_eval holds each function to.
"""
import numpy as np

NODES = 64


def chebyshev_points(a: float, b: float, n: int = NODES) -> np.ndarray:
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos((2 * k + 1) * np.pi / (2 * n))


def fit(f_reduced, a, b, degree):
    t = chebyshev_points(a, b)
    return np.polynomial.polynomial.polyfit(t, f_reduced(t), degree).astype(np.float32)


FITS = {
    "asin_half (P)": (lambda t: (np.arcsin(np.sqrt(t)) - np.sqrt(t)) / (t * np.sqrt(t)), 0.0, 0.25, 5,
                      lambda x, c: x + x ** 3 * np.polynomial.polynomial.polyval(x * x, c), np.arcsin, 0.0, 0.5),
    "sin_quarter (Q)": (lambda t: (np.sin(np.sqrt(t)) - np.sqrt(t)) / (t * np.sqrt(t)), 0.0, np.pi ** 2 / 4, 4,
                        lambda x, c: x + x ** 3 * np.polynomial.polynomial.polyval(x * x, c), np.sin, 0.0, np.pi / 2),
    "ln_unit (L)": (lambda v: -np.log1p(-v) / v, 0.0, 0.25, 6,
                    lambda v, c: -v * np.polynomial.polynomial.polyval(v, c), lambda v: np.log1p(-v), 0.0, 0.25),
    "log1p_pos (M)": (lambda x: np.log1p(x) / x, 0.0, 0.25, 6,
                      lambda x, c: x * np.polynomial.polynomial.polyval(x, c), np.log1p, 0.0, 0.25),
}

if __name__ == "__main__":
    for name, (g, a, b, deg, poly, f, lo, hi) in FITS.items():
        c = fit(g, a, b, deg)
        x = np.linspace(lo, hi, 1_000_001)[1:]
        err = np.max(np.abs(poly(x, c.astype(np.float64)) - f(x)) / np.maximum(np.abs(f(x)), 1e-300))
        print(f"{name}: " + ", ".join(f"{v!r}f" for v in c.tolist()) + f"   (max relative fit error {err:.1e})")
