"""Writes tests/golden/wigner_exact.json from the oracle's exact Rodrigues form.

Source formula: the Rodrigues-type expression for P^l_{mn}(x) with its
normalisation constant c^l_{mn} (Sec. 3, Euler-angle form of the matrix
coefficients), evaluated by oracle.basis.P_rodrigues_exact in exact sympy
arithmetic at x = cos(beta) = -7/25 (cos(beta/2) = 3/5, sin(beta/2) = 4/5),
for every l <= 5/2.  The stored real number is d^l_{mn}(beta) = i^{m-n} P^l_{mn}.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import sympy as sp  # noqa: E402

from oracle import basis  # noqa: E402


def main():
    x = sp.Rational(-7, 25)
    beta = 2 * sp.acos(sp.Rational(3, 5))
    vals = []
    for j in range(0, 6):
        for m2 in range(-j, j + 1, 2):
            for n2 in range(-j, j + 1, 2):
                l, m, n = sp.Rational(j, 2), sp.Rational(m2, 2), sp.Rational(n2, 2)
                P = basis.P_rodrigues_exact(l, m, n, x)
                d = sp.simplify(sp.I ** (m - n) * P)
                dv = sp.N(d, 30)
                assert abs(sp.im(dv)) < 1e-25
                vals.append({"two_l": j, "two_first": m2, "two_second": n2,
                             "d": str(sp.re(dv))})
    out = {
        "source": "Sec. 3 Rodrigues-type formula for P^l_{mn}; d = i^{m-n} P",
        "x": "-7/25",
        "beta": float(sp.N(beta, 20)),
        "values": vals,
    }
    with open(os.path.join(os.path.dirname(__file__), "wigner_exact.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
