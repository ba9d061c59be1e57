"""Shifted Legendre polynomials and the divide-and-conquer projection (Sec. 4).

These are the paper's identities for the m = n = 0 case, used as oracle pins
(tests compare every form with <s, P_{L+r}> from scipy's Legendre routine):

* ``legendre_lemma``: P_0..P_lmax by the Sec. 4 Lemma,
  P_{l+1} = (2l+1)/(l+1) x P_l - l/(l+1) P_{l-1}, P_0 = 1, P_{-1} = 0.
* ``shifted_AB``: A_r^L, B_r^L with P_{L+r} = A_r^L P_L + B_r^L P_{L-1}
  (Sec. 4 Proposition), generated by the matrix/scalar recurrence of the next
  Proposition from A_0 = 1, B_0 = 0, A_{-1} = 0, B_{-1} = 1.
* ``projection_k1``: <s, P_{L+r}> = <s^L, A_r^L> + <s^{L-1}, B_r^L>
  (Divide-and-conquer Theorem, first identity), s^j = s * P_j pointwise.
* ``projection_split``: the expansion for r = n_1 + ... + n_k obtained by
  applying the composition rule (Proposition on A_{r+s}, B_{r+s}) k-1 times.
  Each term is a Hadamard product of k shifted polynomials.  Reading: the
  general formula printed in the Theorem lowers only the first subscript by
  epsilon_1; the composition rule lowers the subscript of every factor but the
  last (n_i - epsilon_i for i < k).  The two agree for k = 2 (the worked
  Example); for k >= 3 this module follows the composition rule.

The end of Sec. 4 states that the same construction applies to the polynomials
of the other matrix entries (m, n not both 0) through their own three-term
recurrence.  ``wigner_shifted_AB`` and ``wigner_projection`` take that
statement literally for d^l_{nm}: A_r^L, B_r^L are generated by the Wigner
recurrence in r (step coefficients at degree L + r) from the same initial
values, so d^{L+r} = A_r^L d^L + B_r^L d^{L-1}, and the depth-k expansion is
the composition-rule form above.  ``forward_depth`` is the whole forward
transform with stage 2 computed that way, the split of each shift r into k
parts taken from the digits of r in base b (``digit_parts``), as in the GPU
depth-k contraction.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def legendre_lemma(lmax: int, x: np.ndarray) -> np.ndarray:
    """Rows P_0..P_lmax at x via the Sec. 4 Lemma recurrence."""
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((lmax + 1,) + x.shape)
    P[0] = 1.0
    prev = np.zeros_like(x)
    for l in range(lmax):
        P[l + 1] = (2 * l + 1) / (l + 1) * x * P[l] - l / (l + 1) * prev
        prev = P[l]
    return P


def shifted_AB(L: int, rmax: int, x: np.ndarray):
    """A_r^L(x), B_r^L(x) for r = -1..rmax; returned arrays indexed r+1."""
    x = np.asarray(x, dtype=np.float64)
    A = np.zeros((rmax + 2,) + x.shape)
    B = np.zeros((rmax + 2,) + x.shape)
    A[0], B[0] = 0.0, 1.0          # r = -1
    A[1], B[1] = 1.0, 0.0          # r = 0
    for r in range(0, rmax):
        k = L + r                  # advancing from degree L+r to L+r+1
        a = (2 * k + 1) / (k + 1)
        c = k / (k + 1)
        A[r + 2] = a * x * A[r + 1] - c * A[r]
        B[r + 2] = a * x * B[r + 1] - c * B[r]
    return A, B


def _AB(L, r, x):
    A, B = shifted_AB(L, max(r, 0), x)
    return A[r + 1], B[r + 1]


def projection_k1(s: np.ndarray, L: int, r: int, x: np.ndarray) -> float:
    """<s^L, A_r^L> + <s^{L-1}, B_r^L> (Divide-and-conquer Theorem)."""
    P = legendre_lemma(L, x)
    sL = s * P[L]
    sLm1 = s * P[L - 1]
    A, B = _AB(L, r, x)
    return float(np.dot(sL, A) + np.dot(sLm1, B))


def projection_split(s: np.ndarray, L: int, parts, x: np.ndarray) -> float:
    """<s, P_{L+r}> for r = sum(parts) as 2^k Hadamard-product terms.

    Term for tau_1 in {A, B} and eps in {0,1}^{k-1}:
      <s^{L or L-1},  tau_1[n_1 - eps_1]^{L_0} * prod_{i=2}^{k} tau_i[n_i - eps_i]^{L_{i-1}}>
    with eps_k = 0, L_0 = L, L_i = L + n_1 + ... + n_i, and tau_i = A if
    eps_{i-1} = 0 else B (the selector of the Theorem).
    """
    k = len(parts)
    P = legendre_lemma(L, x)
    svec = {"A": s * P[L], "B": s * P[L - 1]}
    Ls = [L]
    for n in parts[:-1]:
        Ls.append(Ls[-1] + n)
    total = 0.0
    for tau1 in ("A", "B"):
        for eps in itertools.product((0, 1), repeat=k - 1):
            e = list(eps) + [0]
            v = np.ones_like(x, dtype=np.float64)
            tau = tau1
            for i in range(k):
                Ai, Bi = _AB(Ls[i], parts[i] - e[i], x)
                v = v * (Ai if tau == "A" else Bi)
                tau = "A" if e[i] == 0 else "B"
            total += float(np.dot(svec[tau1], v))
    return total


def projection_printed(s: np.ndarray, L: int, parts, x: np.ndarray) -> float:
    """The Theorem's general formula as printed (only n_1 lowered by eps_1)."""
    k = len(parts)
    P = legendre_lemma(L, x)
    svec = {"A": s * P[L], "B": s * P[L - 1]}
    Ls = [L]
    for n in parts[:-1]:
        Ls.append(Ls[-1] + n)
    total = 0.0
    for tau1 in ("A", "B"):
        for eps in itertools.product((0, 1), repeat=k - 1):
            A1, B1 = _AB(L, parts[0] - (eps[0] if k > 1 else 0), x)
            v = A1 if tau1 == "A" else B1
            for i in range(1, k):
                Ai, Bi = _AB(Ls[i], parts[i], x)
                v = v * (Ai if eps[i - 1] == 0 else Bi)
            total += float(np.dot(svec[tau1], v))
    return total


# ---------------------------------------------------------------------------
# The (m, n) analogue: shifted polynomials of the Wigner-d recurrence
# ---------------------------------------------------------------------------

def _wigner_step(n2: int, m2: int, l: float):
    """Coefficients (a, b, c) of d^{l+1} = a (x - b) d^l - c d^{l-1} for the pair
    (n, m) = (n2/2, m2/2) (the Jacobi three-term recurrence in l)."""
    n, m = n2 / 2.0, m2 / 2.0
    if l == 0.0:
        return 1.0, 0.0, 0.0
    q1 = ((l + 1) ** 2 - n * n) * ((l + 1) ** 2 - m * m)
    q0 = (l * l - n * n) * (l * l - m * m)
    return ((l + 1) * (2 * l + 1) / math.sqrt(q1), n * m / (l * (l + 1)),
            (l + 1) / l * math.sqrt(max(q0, 0.0)) / math.sqrt(q1))


def wigner_shifted_AB(n2: int, m2: int, L2: int, rmax: int, x: np.ndarray):
    """A_r^L(x), B_r^L(x), r = -1..rmax, of the pair (n, m) from degree L = L2/2:
    d^{L+r}_{nm} = A_r^L d^L_{nm} + B_r^L d^{L-1}_{nm}.  Indexed r + 1."""
    x = np.asarray(x, dtype=np.float64)
    A = np.zeros((rmax + 2,) + x.shape)
    B = np.zeros((rmax + 2,) + x.shape)
    A[0], B[0] = 0.0, 1.0          # r = -1
    A[1], B[1] = 1.0, 0.0          # r = 0
    for r in range(0, rmax):
        a, b, c = _wigner_step(n2, m2, L2 / 2.0 + r)
        A[r + 2] = a * (x - b) * A[r + 1] - c * A[r]
        B[r + 2] = a * (x - b) * B[r + 1] - c * B[r]
    return A, B


def _wAB(n2, m2, L2, r, x):
    A, B = wigner_shifted_AB(n2, m2, L2, max(r, 0), x)
    return A[r + 1], B[r + 1]


def wigner_projection(s: np.ndarray, dL: np.ndarray, dLm1: np.ndarray, n2: int, m2: int, L2: int,
                      parts, x: np.ndarray) -> float:
    """<s, d^{L+r}_{nm}>, r = sum(parts), as the 2^k inner products of the
    divide-and-conquer Theorem (composition-rule reading): s^L = s d^L,
    s^{L-1} = s d^{L-1} given; each term is <s^{L or L-1}, V> with V the
    Hadamard product of k shifted polynomials at levels L_0 = L,
    L_i = L_{i-1} + n_i, orders n_i - eps_i (eps_k = 0)."""
    k = len(parts)
    svec = {"A": s * dL, "B": s * dLm1}
    Ls = [L2]
    for n in parts[:-1]:
        Ls.append(Ls[-1] + 2 * n)
    total = 0.0
    for tau1 in ("A", "B"):
        for eps in itertools.product((0, 1), repeat=k - 1):
            e = list(eps) + [0]
            v = np.ones_like(x, dtype=np.float64)
            tau = tau1
            for i in range(k):
                Ai, Bi = _wAB(n2, m2, Ls[i], parts[i] - e[i], x)
                v = v * (Ai if tau == "A" else Bi)
                tau = "A" if e[i] == 0 else "B"
            total = total + np.dot(svec[tau1], v)
    return total


def depth_base(R: int, k: int) -> int:
    """Smallest base b >= 1 with b^k >= R + 1: every shift r <= R has k digits."""
    b = 1
    while b ** k < R + 1:
        b += 1
    return b


def digit_parts(r: int, b: int, k: int):
    """Parts n_i = d_i b^{k-i} of r = sum_i d_i b^{k-i} (digits of r in base b)."""
    out = []
    for i in range(k):
        p = b ** (k - 1 - i)
        out.append((r // p) * p)
        r -= (r // p) * p
    return out


def forward_depth(f: np.ndarray, k: int, weights: str = "cc") -> np.ndarray:
    """Forward transform with stage 2 by the depth-k divide-and-conquer projection.

    Stage 1 as in ``transform.forward_separable``.  Per pair (n, m) with
    mu = max(|n|, |m|): l = mu and mu + 1 directly; from the base L = mu + 1,
    each l = L + r (r = 1..R) by ``wigner_projection`` with the parts of
    ``digit_parts(r, depth_base(R, k), k)``.  Equal to the plain definition
    up to rounding (pinned against it)."""
    from . import basis, grid, quadrature, transform
    N = f.shape[0]
    al, be, ga = grid.alpha_nodes(N), grid.beta_nodes(N), grid.gamma_nodes(N)
    w = quadrature.weights(N, weights)
    pref = transform._prefactor(N, False)
    x = np.cos(be)
    out = np.zeros(grid.num_coeffs(N), dtype=np.complex128)
    for sector in ("int", "half"):
        idx = transform.sector_indices(N, sector)
        jtop = transform._top_j(N, sector)
        F2 = transform.torus_dft(f, idx, idx, al, ga)
        for ni, n2 in enumerate(idx):
            for mi, m2 in enumerate(idx):
                j0, D = basis.wigner_d_column(n2, m2, be, jtop)
                if D.shape[0] == 0:
                    continue
                s = w * F2[:, ni, mi]
                vals = [np.dot(D[0], s)]
                if D.shape[0] > 1:
                    vals.append(np.dot(D[1], s))
                R = D.shape[0] - 2
                b = depth_base(R, k)
                for r in range(1, R + 1):
                    vals.append(wigner_projection(s, D[1], D[0], n2, m2, j0 + 2, digit_parts(r, b, k), x))
                ph = pref * basis.i_pow((n2 - m2) // 2)
                for i, v in enumerate(vals):
                    out[grid.coeff_index(j0 + 2 * i, m2, n2)] = ph * v
    return out
