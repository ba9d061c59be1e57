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
    """sum_{n,m} G[k, n, m] e^{-i(n phi_j1 + m psi_j2)} -> f[j1, k, j2].

    Two matrix products: the sum over n (t[j1, k, m]) and then the sum over m.
    """
    En = np.exp(-1j * np.outer(alpha, idx / 2.0))        # [j1, n]
    Em = np.exp(-1j * np.outer(idx / 2.0, gamma))        # [m, j2]
    K, Nn, Nm = G.shape
    t = (En @ np.transpose(G, (1, 0, 2)).reshape(Nn, K * Nm)).reshape(len(alpha), K, Nm)
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


# ---------------------------------------------------------------------------
# Row-restricted pieces: the same definitions evaluated for a subset of n, so
# that large bandwidths can be split across host processes (tests only)
# ---------------------------------------------------------------------------

def forward_rows(fs: np.ndarray, n2_list, weights: str = "cc"):
    """Coefficients f^(l)_{mn} of every pair whose n (doubled) is in n2_list,
    for a batch of grids of one bandwidth on the periodic grid.

    The definition of ``forward_separable`` restricted to those n: stage 1 is
    the torus double sum for the listed n and every m of their sector (Sec. 6,
    first-stage Proposition), as two matrix products; stage 2 the theta
    contraction with conj(P^l_{nm}) = i^{n-m} d^l_{nm} from the recurrence
    (Sec. 4, discrete Legendre transform), one d column per pair shared by
    the batch.  fs: [B, N, N, N].  Returns (idx, vals): the packed indices of
    the computed coefficients and vals[B, len(idx)].
    """
    fs = np.asarray(fs)
    B, N = fs.shape[0], fs.shape[1]
    al, be, ga, w, pref = _setup(N, weights, False)
    idx_out, vals_out = [], []
    for parity, sector in ((0, "int"), (1, "half")):
        ns = np.array(sorted(n2 for n2 in n2_list if n2 % 2 == parity), dtype=np.int64)
        if ns.size == 0:
            continue
        ms = sector_indices(N, sector)
        jtop = _top_j(N, sector)
        En = np.exp(1j * np.outer(ns / 2.0, al))             # [n, j1]
        Em = np.exp(1j * np.outer(ms / 2.0, ga))             # [m, j2]
        F2 = np.stack([((En @ fs[b].reshape(N, -1)).reshape(ns.size, N, N)) @ Em.T
                       for b in range(B)])                   # [b, n, k, m]
        for ni, n2 in enumerate(ns):
            for mi, m2 in enumerate(ms):
                j0, D = basis.wigner_d_column(int(n2), int(m2), be, jtop)
                if D.shape[0] == 0:
                    continue
                s = w[None, :] * F2[:, ni, :, mi]                           # [b, k]
                vals = pref * basis.i_pow((int(n2) - int(m2)) // 2) * (s @ D.T)   # [b, L]
                idx_out.append(np.array([grid.coeff_index(j0 + 2 * i, int(m2), int(n2))
                                         for i in range(D.shape[0])], dtype=np.int64))
                vals_out.append(vals)
    if not idx_out:
        return np.zeros(0, dtype=np.int64), np.zeros((B, 0), dtype=np.complex128)
    return np.concatenate(idx_out), np.concatenate(vals_out, axis=1)


def synthesis_rows(cs: np.ndarray, N: int, n2_list, ks, modes=("synthesis",), weights: str = "cc"):
    """Theta sums G[k, n, m] of the synthesis and/or the adjoint for the listed
    n (doubled) at the beta nodes ks, for a batch of packed coefficient vectors.

    Synthesis (Sec. 3, Peter-Weyl expansion):
        G[k, n, m] = sum_l (2l+1) i^{m-n} d^l_{nm}(beta_k) c(l)_{mn};
    adjoint of the forward quadrature map: (2l+1) replaced by pref * w_k.
    The grid values follow as sum_{n,m} G[k, n, m] e^{-i(n alpha + m gamma)}
    (``planes_from_rows``).  cs: [B, C]; modes: "synthesis" and/or "adjoint"
    (the d columns are shared).  Returns {mode: {sector: (ns, G[B, K, n, m])}}.
    """
    cs = np.asarray(cs)
    B = cs.shape[0]
    ks = np.asarray(ks, dtype=np.int64)
    be = grid.beta_nodes(N)[ks]
    w = quadrature.weights(N, weights)[ks]
    pref = _prefactor(N, False)
    out = {mode: {} for mode in modes}
    for parity, sector in ((0, "int"), (1, "half")):
        ns = np.array(sorted(n2 for n2 in n2_list if n2 % 2 == parity), dtype=np.int64)
        if ns.size == 0:
            continue
        ms = sector_indices(N, sector)
        jtop = _top_j(N, sector)
        G = {mode: np.zeros((B, ks.size, ns.size, ms.size), dtype=np.complex128) for mode in modes}
        for ni, n2 in enumerate(ns):
            for mi, m2 in enumerate(ms):
                j0, D = basis.wigner_d_column(int(n2), int(m2), be, jtop)   # [L, K]
                if D.shape[0] == 0:
                    continue
                js = j0 + 2 * np.arange(D.shape[0])
                c = cs[:, [grid.coeff_index(int(j), int(m2), int(n2)) for j in js]]   # [B, L]
                ph = basis.i_pow((int(m2) - int(n2)) // 2)
                for mode in modes:
                    if mode == "adjoint":
                        t = (c @ D) * (pref * w)[None, :]
                    elif mode == "synthesis":
                        t = (c * (js + 1)[None, :].astype(np.float64)) @ D
                    else:
                        raise ValueError(mode)
                    G[mode][:, :, ni, mi] = ph * t
        for mode in modes:
            out[mode][sector] = (ns, G[mode])
    return out


def planes_from_rows(parts, N: int) -> np.ndarray:
    """Grid values f[b, j1, k, j2] at the beta nodes of ``synthesis_rows`` from
    its outputs for disjoint n lists covering every n (summed over both
    sectors): f = sum_{n,m} G[k, n, m] e^{-i(n alpha_j1 + m gamma_j2)}."""
    al, ga = grid.alpha_nodes(N), grid.gamma_nodes(N)
    f = None
    for sector in ("int", "half"):
        idx = sector_indices(N, sector)
        pos = {int(n2): i for i, n2 in enumerate(idx)}
        G = None
        for part in parts:
            if sector not in part:
                continue
            ns, g = part[sector]
            if G is None:
                G = np.zeros(g.shape[:2] + (idx.size, idx.size), dtype=np.complex128)
            for i, n2 in enumerate(ns):
                G[:, :, pos[int(n2)], :] += g[:, :, i, :]
        if G is None:
            continue
        fs = np.stack([_torus_synthesis(G[b], idx, al, ga) for b in range(G.shape[0])])
        f = fs if f is None else f + fs
    return f
