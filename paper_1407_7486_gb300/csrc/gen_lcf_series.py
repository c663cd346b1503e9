"""Coefficients of the small-argument series of the constant-field brackets
used by the LCF comparison in wln_stats.cu:

    x coth x  - 1 - x^2/3 = sum_{k>=2} a_k x^{2k},  a_k = 2^{2k} B_{2k} / (2k)!
    x / sinh x - 1 + x^2/6 = sum_{k>=2} b_k x^{2k},  b_k = (2 - 2^{2k}) B_{2k} / (2k)!

B_{2k} are the Bernoulli numbers, computed here exactly from their generating
recurrence sum_{j=0}^{m} C(m+1, j) B_j = 0 (m >= 1, B_0 = 1).  Run it to
print the C tables; they are pasted into wln_stats.cu (kLcfSpin, kLcfScal).
Twelve terms reach double precision for |x| < 1/2: the terms shrink like
(x/pi)^2 per order.
"""
from fractions import Fraction
from math import comb, factorial


def bernoulli(n_max):
    B = [Fraction(1)]
    for m in range(1, n_max + 1):
        B.append(-sum(comb(m + 1, j) * B[j] for j in range(m)) / (m + 1))
    return B


def tables(n_terms=12):
    B = bernoulli(2 * (n_terms + 1) + 2)
    a = [Fraction(2 ** (2 * k)) * B[2 * k] / factorial(2 * k) for k in range(2, n_terms + 2)]
    b = [Fraction(2 - 2 ** (2 * k)) * B[2 * k] / factorial(2 * k) for k in range(2, n_terms + 2)]
    return a, b


if __name__ == "__main__":
    a, b = tables()
    for name, t in (("kLcfSpin", a), ("kLcfScal", b)):
        print(f"__constant__ double {name}[{len(t)}] = {{")
        print(",\n".join(f"    {float(c)!r}" for c in t))
        print("};")
