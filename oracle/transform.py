"""Forward transform, synthesis and adjoint on the Euler-angle grid (oracle side).

Definitions followed (all float64 / complex128):

* Analysis (Sec. 3, Definition of the Fourier transform on SU(2); Sec. 4,
  Euler-angle integral with the factor 1/(8 pi^2)):
      f^(l)_{mn} = <f, t^l_{nm}> = (1/(8 pi^2)) int f conj(t^l_{nm}) sin(theta) dphi dtheta dpsi,
      t^l_{nm}(phi, theta, psi) = e^{-i(n phi + m psi)} P^l_{nm}(cos theta).
  On the grid the integral becomes the quadrature sum (Sec. 4, factorised
  Riemann-sum Proposition)
      f^(l)_{mn} = pref * sum_{j1,k,j2} w_k f(phi_j1, theta_k, psi_j2) conj(t^l_{nm}(...)),
  pref = (1/(8 pi^2)) * dphi * dpsi (= 1/(2N^2) on the periodic grid), and w_k
  the beta weights (Clenshaw-Curtis by default, or the paper-literal Riemann
  weights).  This sum is the oracle's definition of the forward transform; it
  is evaluated two independent ways:

  - ``forward_direct``   O(N^6): every coefficient summed over every grid
    point with t^l_{nm} built from the group element u (Sec. 5, direct method);
  - ``forward_separable`` O(N^4): the bracketed double sum over (j1, j2) for
    every theta_k first (Sec. 4 Proposition; Sec. 6 first-stage Proposition,
    f_2(theta_k; m, n)), then the theta contraction <s, P^l_{nm}> (Sec. 4,
    discrete Legendre transform; Sec. 6 second-stage Proposition with k = 1).
    The double sum is written as products with explicit exponential matrices
    (a plain DFT, no FFT), and P^l_{nm} = i^{m-n} d^l_{nm} with d from the
    three-term recurrence.

* Synthesis (Sec. 3, Peter-Weyl expansion):
      f(x) = sum_l (2l+1) sum_{m,n} f^(l)_{mn} t^l_{nm}(x).
* Adjoint of the forward map (conjugate transpose of the quadrature sum):
      (A^H g)(x_{j1 k j2}) = pref * w_k * sum_{l,m,n} g(l)_{mn} t^l_{nm}(x).

Sector note: on the paper's domain (phi, psi in [-pi, pi]) the integer-l and
half-integer-l basis functions are not orthogonal to each other, so the forward
map returns cross-sector leakage for functions that mix both; the oracle
computes the quadrature sum as defined, leakage included.

Full-group grid (``full=True``): psi in [-2 pi, 2 pi) with 2N nodes, so the
sampled domain is all of SU(2); the normalised Haar measure is then
(1/(16 pi^2)) sin(theta) dphi dtheta dpsi and pref = (2 pi/N)^2/(16 pi^2) =
1/(4N^2).  Grids have shape (N, N, 2N).  On this grid the two sectors are
orthogonal and band-limited functions mixing both are recovered exactly.
"""
from __future__ import annotations

import numpy as np

from . import basis, grid, quadrature


def _prefactor(N: int, literal: bool, full: bool = False) -> float:
    h = 2.0 * np.pi / ((N - 1) if literal else N)
    return h * h / ((16.0 if full else 8.0) * np.pi ** 2)


def _setup(N, weights, literal, full=False):
    al = grid.alpha_nodes(N, literal)
    ga = grid.gamma_nodes(N, literal, full)
    be = grid.beta_nodes(N)
    w = quadrature.weights(N, weights)
    return al, be, ga, w, _prefactor(N, literal, full)


def sector_indices(N: int, sector: str) -> np.ndarray:
    """Doubled indices 2n allowed for bandwidth N in one sector.

    l <= (N-1)/2.  Integer sector: n = -(N/2-1)..(N/2-1); half-integer sector:
    n = -(N-1)/2..(N-1)/2 in unit steps.  (N even.)
    """
    jmax = N - 1
    if sector == "int":
        top = jmax - 1 if jmax % 2 else jmax     # largest even 2l <= N-1
    elif sector == "half":
        top = jmax if jmax % 2 else jmax - 1     # largest odd 2l <= N-1
    else:
        raise ValueError(sector)
    return np.arange(-top, top + 1, 2)


def _top_j(N: int, sector: str) -> int:
    return int(sector_indices(N, sector)[-1])


# ---------------------------------------------------------------------------
# Direct O(N^6) forward and synthesis (t from the group element)
# ---------------------------------------------------------------------------

def forward_direct(f: np.ndarray, weights: str = "cc", literal: bool = False, full: bool = False) -> np.ndarray:
    """Quadrature sum evaluated coefficient by coefficient (Sec. 5).

    f: complex array [j1, k, j2] of shape (N, N, N) ((N, N, 2N) on the full-group
    grid).  Returns packed coefficients.
    """
    N = f.shape[0]
    al, be, ga, w, pref = _setup(N, weights, literal, full)
    a, b, c, d = basis.u_entries(al[:, None, None], be[None, :, None], ga[None, None, :])
    fw = f * w[None, :, None]
    out = np.zeros(grid.num_coeffs(N), dtype=np.complex128)
    for j in range(N):
        for m2 in grid.half_range(j):
            for n2 in grid.half_range(j):
                t = basis.t_from_u(j, n2, m2, a, b, c, d)          # t^l_{nm}
                out[grid.coeff_index(j, m2, n2)] = pref * np.sum(fw * np.conj(t))
    return out


def inverse_direct(coeffs: np.ndarray, N: int, literal: bool = False, full: bool = False) -> np.ndarray:
    """Synthesis sum_l (2l+1) sum_{m,n} f^(l)_{mn} t^l_{nm} on the grid (Sec. 3)."""
    al = grid.alpha_nodes(N, literal)
    ga = grid.gamma_nodes(N, literal, full)
    be = grid.beta_nodes(N)
    a, b, c, d = basis.u_entries(al[:, None, None], be[None, :, None], ga[None, None, :])
    f = np.zeros((N, N, len(ga)), dtype=np.complex128)
    for j in range(N):
        for m2 in grid.half_range(j):
            for n2 in grid.half_range(j):
                cval = coeffs[grid.coeff_index(j, m2, n2)]
                if cval != 0:
                    f += (j + 1) * cval * basis.t_from_u(j, n2, m2, a, b, c, d)
    return f


# ---------------------------------------------------------------------------
# Separable O(N^4) forward, synthesis and adjoint
# ---------------------------------------------------------------------------

def torus_dft(f: np.ndarray, nvals2: np.ndarray, mvals2: np.ndarray,
              alpha: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """f_2(theta_k; m, n) = sum_{j1,j2} e^{i n phi_j1} e^{i m psi_j2} f[j1, k, j2].

    Sec. 6, first-stage Proposition (the bracket of the Sec. 4 factorisation).
    nvals2 / mvals2: doubled n and m.  Returns F[k, n_index, m_index].
    """
    En = np.exp(1j * np.outer(nvals2 / 2.0, alpha))     # [n, j1]
    Em = np.exp(1j * np.outer(mvals2 / 2.0, gamma))     # [m, j2]
    N = f.shape[0]
    t = (En @ f.reshape(N, -1)).reshape(len(nvals2), f.shape[1], f.shape[2])   # [n, k, j2]
    t = t @ Em.T                                                               # [n, k, m]
    return np.transpose(t, (1, 0, 2))


def forward_separable(f: np.ndarray, weights: str = "cc", literal: bool = False,
                      row_stride: int = 1, full: bool = False) -> np.ndarray:
    """Forward transform by the two-stage separation (Sec. 4 and Sec. 6, k = 1).

    Stage 1: f_2(theta_k; m, n) by the torus double sum for every theta_k.
    Stage 2: f^(l)_{mn} = pref * sum_k w_k conj(P^l_{nm}(cos theta_k)) f_2(theta_k; m, n),
             conj(P^l_{nm}) = i^{n-m} d^l_{nm}.
    row_stride > 1 runs stage 2 only for every row_stride-th n (a bounded
    timing sample; the other coefficients stay zero).
    """
    N = f.shape[0]
    al, be, ga, w, pref = _setup(N, weights, literal, full)
    out = np.zeros(grid.num_coeffs(N), dtype=np.complex128)
    for sector in ("int", "half"):
        idx = sector_indices(N, sector)
        jtop = _top_j(N, sector)
        F2 = torus_dft(f, idx, idx, al, ga)            # [k, n, m]
        for ni, n2 in enumerate(idx):
            if ni % row_stride:
                continue
            for mi, m2 in enumerate(idx):
                j0, D = basis.wigner_d_column(n2, m2, be, jtop)
                if D.shape[0] == 0:
                    continue
                s = w * F2[:, ni, mi]                    # [s]_k with weight w_k
                vals = pref * basis.i_pow((n2 - m2) // 2) * (D @ s)
                for i in range(D.shape[0]):
                    j = j0 + 2 * i
                    out[grid.coeff_index(j, m2, n2)] = vals[i]
    return out


def _synthesis_planes(coeffs: np.ndarray, N: int, sector: str, row_weight) -> np.ndarray:
    """G[k, n, m] = sum_l row_weight(l, k) * i^{m-n} d^l_{nm}(beta_k) c(l)_{mn}."""
    be = grid.beta_nodes(N)
    idx = sector_indices(N, sector)
    jtop = _top_j(N, sector)
    G = np.zeros((N, len(idx), len(idx)), dtype=np.complex128)
    for ni, n2 in enumerate(idx):
        for mi, m2 in enumerate(idx):
            j0, D = basis.wigner_d_column(n2, m2, be, jtop)
            if D.shape[0] == 0:
                continue
            js = j0 + 2 * np.arange(D.shape[0])
            c = np.array([coeffs[grid.coeff_index(j, m2, n2)] for j in js])
            rw = row_weight(js)                          # [L] or [L, K]
            G[:, ni, mi] = basis.i_pow((m2 - n2) // 2) * np.sum(
                (rw if np.ndim(rw) == 2 else rw[:, None]) * D * c[:, None], axis=0)
    return G


def _torus_synthesis(G: np.ndarray, idx: np.ndarray, alpha, gamma) -> np.ndarray:
    """sum_{n,m} G[k, n, m] e^{-i(n phi_j1 + m psi_j2)} -> f[j1, k, j2]."""
    En = np.exp(-1j * np.outer(alpha, idx / 2.0))        # [j1, n]
    Em = np.exp(-1j * np.outer(idx / 2.0, gamma))        # [m, j2]
    t = np.einsum("an,knm->akm", En, G)
    return t @ Em


def inverse_separable(coeffs: np.ndarray, N: int, literal: bool = False, full: bool = False) -> np.ndarray:
    """Synthesis (Sec. 3) by separation: theta sum per (n, m), then torus sum."""
    al = grid.alpha_nodes(N, literal)
    ga = grid.gamma_nodes(N, literal, full)
    f = np.zeros((N, N, len(ga)), dtype=np.complex128)
    for sector in ("int", "half"):
        G = _synthesis_planes(coeffs, N, sector, lambda js: (js + 1).astype(np.float64))
        f += _torus_synthesis(G, sector_indices(N, sector), al, ga)
    return f


def adjoint_separable(g: np.ndarray, N: int, weights: str = "cc",
                      literal: bool = False, full: bool = False) -> np.ndarray:
    """Conjugate transpose of the forward quadrature map applied to g (packed)."""
    al, be, ga, w, pref = _setup(N, weights, literal, full)
    f = np.zeros((N, N, len(ga)), dtype=np.complex128)
    for sector in ("int", "half"):
        G = _synthesis_planes(g, N, sector, lambda js: np.ones(js.shape))
        f += _torus_synthesis(G, sector_indices(N, sector), al, ga)
    return f * (pref * w)[None, :, None]


# ---------------------------------------------------------------------------
# Sampled coefficients for large grids
# ---------------------------------------------------------------------------

def forward_pair(f: np.ndarray, n2: int, m2: int, weights: str = "cc",
                 literal: bool = False, full: bool = False):
    """All coefficients f^(l)_{mn}, l = mu..lmax, of one (n, m) pair.

    Same definition as ``forward_separable`` restricted to one pair: the torus
    double sum for that (n, m) on every theta_k (O(N^3)), then the theta
    contraction with the recurrence values.  Returns (j0, values[L]).
    """
    N = f.shape[0]
    al, be, ga, w, pref = _setup(N, weights, literal, full)
    sector = "int" if n2 % 2 == 0 else "half"
    jtop = _top_j(N, sector)
    en = np.exp(1j * (n2 / 2.0) * al)                    # [j1]
    em = np.exp(1j * (m2 / 2.0) * ga)                    # [j2]
    f2 = np.einsum("a,akb,b->k", en, f, em)
    j0, D = basis.wigner_d_column(n2, m2, be, jtop)
    return j0, pref * basis.i_pow((n2 - m2) // 2) * (D @ (w * f2))


def loss_and_grad(f: np.ndarray, target: np.ndarray, weights: str = "cc"):
    """L = sum_l (2l+1) ||f^(l) - target(l)||_F^2 and dL/dRe f + i dL/dIm f.

    The gradient is 2 A^H [(2l+1)(A f - target)] (A linear), the form PyTorch
    reports for a real loss of a complex tensor.
    """
    N = f.shape[0]
    c = forward_separable(f, weights)
    r = c - target
    two_l = np.concatenate([np.full((j + 1) ** 2, j) for j in range(N)])
    wl = (two_l + 1).astype(np.float64)
    L = float(np.sum(wl * np.abs(r) ** 2))
    g = 2.0 * adjoint_separable(wl * r, N, weights)
    return L, g
