"""Coefficients of the polynomial used for the memristor current sinh(x) in k_stencil.cu.

sinh(x) / x = sum_k t^k / (2k+1)!  with t = x^2.  On |x| <= X (t in [0, X^2]) the Taylor
series is economised (Lanczos' Chebyshev economisation): the series, taken to degree 16 in t,
is written in the shifted Chebyshev basis of [0, X^2] with exact rational arithmetic, the
basis terms above degree DEG are dropped, and the result is converted back to monomials.
The bound printed for the dropped terms (the sum of their absolute Chebyshev coefficients)
is an upper bound of the truncation error relative to sinh(x)/x >= 1.

    python gen_sinh_poly.py        # prints the C initialisers used by the kernel
"""
import sympy as sp

X2 = sp.Rational(9, 16)   # |x| <= 3/4
DEG = 6
TAYLOR = 16


def coefficients(x2=X2, deg=DEG, taylor=TAYLOR):
    t, u = sp.symbols("t u")
    series = sum(t**k / sp.factorial(2 * k + 1) for k in range(taylor + 1))
    # t = x2 (u + 1) / 2 maps u in [-1, 1] onto t in [0, x2]
    pu = sp.Poly(sp.expand(series.subs(t, x2 * (u + 1) / 2)), u)
    cheb = []
    rem = pu
    for n in range(pu.degree(), -1, -1):        # peel Chebyshev terms from the top
        tn = sp.Poly(sp.chebyshevt(n, u), u)
        c = rem.coeff_monomial(u**n) / tn.coeff_monomial(u**n)
        cheb.append((n, c))
        rem = rem - tn * c
    kept = sum((sp.Poly(sp.chebyshevt(n, u), u) * c for n, c in cheb if n <= deg),
               sp.Poly(0, u))
    dropped = sum(abs(c) for n, c in cheb if n > deg)
    # back to t: u = 2 t / x2 - 1
    pt = sp.Poly(sp.expand(kept.as_expr().subs(u, 2 * t / x2 - 1)), t)
    coef = [pt.coeff_monomial(t**k) for k in range(deg + 1)]
    tail = sum(x2**k / sp.factorial(2 * k + 1) for k in range(taylor + 1, taylor + 4))
    return coef, float(dropped + tail)


if __name__ == "__main__":
    coef, bound = coefficients()
    print(f"// degree {DEG} in t on |x| <= {float(sp.sqrt(X2))}, truncation bound {bound:.2e}")
    for k in range(DEG, -1, -1):
        print(f"  {float(coef[k]):.17e},  // t^{k}")
