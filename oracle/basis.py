"""Matrix coefficients of SU(2) representations (oracle side, float64).

Three independent ways to obtain the basis, used against each other in tests:

1. ``t_from_u``: t^l_{mn}(u) from the derivative definition in the Sec. 3
   Theorem (matrix coefficients of T_l acting on homogeneous polynomials),
   with u(phi, theta, psi) the matrix printed in that Theorem.  Applying
   d^{l-m}/dz1^{l-m} d^{l+m}/dz2^{l+m} to a homogeneous polynomial of degree 2l
   extracts (l-m)!(l+m)! times its z1^{l-m} z2^{l+m} coefficient; expanding both
   binomials gives

     t^l_{mn}(u) = sqrt((l-m)!(l+m)! / ((l-n)!(l+n)!))
                   * sum_i C(l-n, i) C(l+n, l-m-i) a^i b^{l-m-i} c^{l-n-i} d^{m+n+i}.

   Small l only (the alternating sum cancels badly for large l).

2. ``P_rodrigues_exact``: P^l_{mn}(x) from the Rodrigues-type formula of Sec. 3
   (the Euler-angle form t^l_{mn} = P^l_{mn}(cos theta) e^{-i(m phi + n psi)}),
   evaluated symbolically with sympy.  Small l only.

3. ``wigner_d_column``: the real small-d values by the three-term recurrence in
   l.  The paper derives the recurrence only for m = n = 0 (Sec. 4 Lemma,
   (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}) and states that the general case
   follows from the Jacobi recurrence in the same way (end of Sec. 4); the
   general form used here is that Jacobi three-term recurrence written for
   d^l_{nm}, and it reduces to the Lemma at n = m = 0.

Relation between the forms (checked in tests):
   P^l_{mn}(cos beta) = i^{n-m} d^l_{mn}(beta),
with d the standard real Wigner small-d (d^{1/2}_{1/2,-1/2} = -sin(beta/2)).

Index convention of the recurrence: ``wigner_d_column(n2, m2, ...)`` returns
d^l_{nm} with FIRST index n (= n2/2) and second index m (= m2/2), the order in
which it enters the analysis integral (conj of t^l_{nm}, Sec. 3 definition of
the Fourier transform).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# 1. Group element and the derivative definition
# ---------------------------------------------------------------------------

def u_entries(phi, theta, psi):
    """Entries (a, b, c, d) of u(phi, theta, psi) as printed in the Sec. 3 Theorem.

    a = e^{i(phi+psi)/2} cos(theta/2),  b = e^{i(phi-psi)/2} i sin(theta/2),
    c = e^{-i(phi-psi)/2} i sin(theta/2), d = e^{-i(phi+psi)/2} cos(theta/2).
    Inputs broadcast against each other.
    """
    ch = np.cos(np.asarray(theta) / 2.0)
    sh = np.sin(np.asarray(theta) / 2.0)
    sp = (np.asarray(phi) + np.asarray(psi)) / 2.0
    sm = (np.asarray(phi) - np.asarray(psi)) / 2.0
    a = np.exp(1j * sp) * ch
    b = np.exp(1j * sm) * 1j * sh
    c = np.exp(-1j * sm) * 1j * sh
    d = np.exp(-1j * sp) * ch
    return a, b, c, d


def t_from_u(j: int, m2: int, n2: int, a, b, c, d):
    """t^l_{mn}(u) with l = j/2, m = m2/2, n = n2/2 (Sec. 3 Theorem, expanded).

    Note the argument order follows the paper's t^l_{mn}: row m, column n.
    """
    lm = (j - m2) // 2   # l - m
    lp = (j + m2) // 2   # l + m
    ln = (j - n2) // 2   # l - n
    lq = (j + n2) // 2   # l + n
    mn = (m2 + n2) // 2  # m + n
    norm = math.sqrt(math.factorial(lm) * math.factorial(lp)
                     / (math.factorial(ln) * math.factorial(lq)))
    out = np.zeros(np.broadcast(a, b, c, d).shape, dtype=np.complex128)
    for i in range(max(0, -mn), min(ln, lm) + 1):
        coef = math.comb(ln, i) * math.comb(lq, lm - i)
        out = out + coef * (a ** i) * (b ** (lm - i)) * (c ** (ln - i)) * (d ** (mn + i))
    return norm * out


# ---------------------------------------------------------------------------
# 2. Rodrigues-type formula in exact arithmetic
# ---------------------------------------------------------------------------

def P_rodrigues_exact(l, m, n, x):
    """P^l_{mn}(x) from the Sec. 3 Rodrigues-type formula, as a sympy expression.

    P^l_{mn}(x) = c^l_{mn} (1-x)^{(n-m)/2} / (1+x)^{(m+n)/2}
                  * (d/dx)^{l-m} [ (1-x)^{l-n} (1+x)^{l+n} ],
    c^l_{mn} = 2^{-l} (-1)^{l-n} i^{n-m} / sqrt((l-n)!(l+n)!) * sqrt((l+m)!/(l-m)!).

    l, m, n: sympy Rationals (half-integers allowed); x: sympy number in (-1, 1).
    """
    import sympy as sp

    X = sp.Symbol("X")
    c = (sp.Integer(2) ** (-l) * sp.Integer(-1) ** (l - n) * sp.I ** (n - m)
         / sp.sqrt(sp.factorial(l - n) * sp.factorial(l + n))
         * sp.sqrt(sp.factorial(l + m) / sp.factorial(l - m)))
    inner = (1 - X) ** (l - n) * (1 + X) ** (l + n)
    k = int(l - m)
    der = sp.diff(inner, X, k) if k > 0 else inner
    expr = c * (1 - X) ** ((n - m) / 2) / (1 + X) ** ((m + n) / 2) * der
    return expr.subs(X, x)


# ---------------------------------------------------------------------------
# 3. Real small-d by the three-term recurrence in l
# ---------------------------------------------------------------------------

def seed_log(n2: int, m2: int, beta: np.ndarray):
    """Seed d^mu_{nm}(beta) at mu = max(|n|, |m|) as (sign, log|value|).

    Obtained from the Rodrigues-type formula at l = mu, where the derivative
    order l - n (or, through the symmetry of d, l - m) vanishes, with
    1 - x = 2 sin^2(beta/2), 1 + x = 2 cos^2(beta/2):

      n =  mu:  (-1)^{mu-m} sqrt((2mu)!/((mu+m)!(mu-m)!)) cos^{mu+m} sin^{mu-m}
      n = -mu:              sqrt((2mu)!/((mu+m)!(mu-m)!)) cos^{mu-m} sin^{mu+m}
      m =  mu:              sqrt((2mu)!/((mu+n)!(mu-n)!)) cos^{mu+n} sin^{mu-n}
      m = -mu:  (-1)^{mu+n} sqrt((2mu)!/((mu+n)!(mu-n)!)) cos^{mu-n} sin^{mu+n}

    (cos, sin of beta/2).  Factorial ratios are taken in log space.  Returns
    (sign, logabs) arrays; logabs = -inf where a zero power base occurs.
    """
    j = max(abs(n2), abs(m2))          # 2 mu
    if abs(n2) == j:
        other2 = m2
        if n2 > 0 or j == 0:
            pc, ps = (j + m2) // 2, (j - m2) // 2
            sgn = -1.0 if ((j - m2) // 2) % 2 else 1.0
        else:
            pc, ps = (j - m2) // 2, (j + m2) // 2
            sgn = 1.0
    else:
        other2 = n2
        if m2 > 0:
            pc, ps = (j + n2) // 2, (j - n2) // 2
            sgn = 1.0
        else:
            pc, ps = (j - n2) // 2, (j + n2) // 2
            sgn = -1.0 if ((j + n2) // 2) % 2 else 1.0
    lf = 0.5 * (math.lgamma(j + 1) - math.lgamma((j + other2) // 2 + 1)
                - math.lgamma((j - other2) // 2 + 1))
    ch = np.cos(beta / 2.0)
    sh = np.sin(beta / 2.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        lc = np.where(pc > 0, pc * np.log(np.abs(ch)), 0.0)
        ls = np.where(ps > 0, ps * np.log(np.abs(sh)), 0.0)
    logabs = lf + lc + ls
    # cos(beta/2) >= 0 and sin(beta/2) >= 0 on [0, pi]: the sign is the prefactor's.
    return np.full(beta.shape, sgn), logabs


def wigner_d_column(n2: int, m2: int, beta: np.ndarray, jmax: int):
    """d^l_{nm}(beta_k) for l = mu, mu+1, ..., up to l <= jmax/2.

    n = n2/2 (first index), m = m2/2 (second), mu = max(|n|, |m|); n2, m2 and
    jmax must have equal parity.  Returns (j0, D) with j0 = 2 mu and
    D[i, k] = d^{mu+i}_{nm}(beta_k); D has zero rows if mu > jmax/2.

    Recurrence (ascending l, fixed n, m, x = cos beta), with d^{mu-1} = 0:
      d^{l+1} = (l+1)(2l+1) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)) * (x - nm/(l(l+1))) d^l
              - (l+1)/l * sqrt((l^2-n^2)(l^2-m^2)) / sqrt(((l+1)^2-n^2)((l+1)^2-m^2)) d^{l-1}.
    At l = 0 (only when n = m = 0) the first step is d^1 = x d^0, as in the
    Sec. 4 Lemma with P_{-1} = 0.
    """
    j0 = max(abs(n2), abs(m2))
    assert (n2 - jmax) % 2 == 0 and (m2 - jmax) % 2 == 0
    if j0 > jmax:
        return j0, np.zeros((0, beta.size))
    L = (jmax - j0) // 2 + 1
    x = np.cos(beta)
    sgn, la = seed_log(n2, m2, beta)
    D = np.zeros((L, beta.size))
    D[0] = sgn * np.exp(la)
    n = n2 / 2.0
    m = m2 / 2.0
    prev = np.zeros(beta.size)
    cur = D[0].copy()
    for i in range(L - 1):
        l = j0 / 2.0 + i
        if l == 0.0:
            nxt = x * cur
        else:
            q1 = ((l + 1) ** 2 - n * n) * ((l + 1) ** 2 - m * m)
            q0 = (l * l - n * n) * (l * l - m * m)
            A = (l + 1) * (2 * l + 1) / math.sqrt(q1)
            Bv = n * m / (l * (l + 1))
            Cv = (l + 1) / l * math.sqrt(max(q0, 0.0)) / math.sqrt(q1)
            nxt = A * (x - Bv) * cur - Cv * prev
        D[i + 1] = nxt
        prev, cur = cur, nxt
    return j0, D


def wigner_d_matrix(j: int, beta: float) -> np.ndarray:
    """Full (j+1) x (j+1) matrix d^l(beta), l = j/2, rows n = -l..l, columns m.

    Assembled from ``wigner_d_column``; for tests (unitarity, group law).
    """
    out = np.zeros((j + 1, j + 1))
    b = np.array([beta], dtype=np.float64)
    for r, n2 in enumerate(range(-j, j + 1, 2)):
        for c, m2 in enumerate(range(-j, j + 1, 2)):
            j0, D = wigner_d_column(n2, m2, b, j)
            out[r, c] = D[(j - j0) // 2, 0]
    return out


def i_pow(k: int) -> complex:
    """i^k for integer k (exact)."""
    return (1.0 + 0j, 1j, -1.0 + 0j, -1j)[k % 4]
