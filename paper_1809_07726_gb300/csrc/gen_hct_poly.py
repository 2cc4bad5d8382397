"""Coefficients of the far-pair polynomials in cph_device.cuh.

For disjoint spheres (L = r - s) the HCT integral and its derivatives depend on
r and x = s / r only:
    H      = (1/r)   x^3 P(x^2),   P(y) = sum_{k>=1} 2k/(2k+1) y^(k-1)
    dH/dr  = -(1/r^2) x^3 Q(x^2),  Q(y) = sum_{k>=1} 2k(2k+2)/(2k+1) y^(k-1)
    dH/ds  = (1/r^2) x^2 S(x^2),   S(y) = sum_{k>=1} 2k y^(k-1) = 2 / (1 - y)^2
The kernels use them for x <= 0.35, i.e. y in [0, 0.1225].  Each function is
interpolated there by a degree-5 Chebyshev series fitted at 200 Chebyshev
nodes with relative weights (near-minimax in relative error), then written in
monomial form for Horner evaluation.  The exact functions come from their
series summed to 60 terms in FP64.

Run:  python gen_hct_poly.py   (prints the coefficients and their max relative
error on the interval).
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as Pm

XMAX = 0.35
Y = XMAX * XMAX
DEG = 5


def series(coef, y, terms=60):
    return sum(coef(k) * y ** (k - 1) for k in range(1, terms))


FUNCS = {
    "P": lambda y: series(lambda k: 2 * k / (2 * k + 1), y),
    "Q": lambda y: series(lambda k: 2 * k * (2 * k + 2) / (2 * k + 1), y),
    "S": lambda y: 2.0 / (1.0 - y) ** 2,
}


def fit(f, deg=DEG, nodes=200):
    t = np.cos(np.pi * (np.arange(nodes) + 0.5) / nodes)
    y = (t + 1.0) / 2.0 * Y
    fy = f(y)
    c = C.chebfit(t, fy, deg, w=1.0 / fy)
    in_t = Pm.Polynomial(C.cheb2poly(c))
    return in_t(Pm.Polynomial([-1.0, 2.0 / Y])).coef  # t = 2y/Y - 1


def max_rel_err(coef, f, n=20001):
    y = np.linspace(0.0, Y, n)
    return float(np.max(np.abs(Pm.polyval(y, coef) / f(y) - 1.0)))


if __name__ == "__main__":
    for name, f in FUNCS.items():
        c = fit(f)
        print(name, "max rel err %.2e" % max_rel_err(c, f), ", ".join("%.10g" % v for v in c))
