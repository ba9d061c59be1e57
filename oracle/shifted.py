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
"""
from __future__ import annotations

import itertools

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
