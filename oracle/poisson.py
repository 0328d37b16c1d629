"""Pressure Poisson equation of the projection (Eqs 3.9, 3.17, 3.24; Sec. 3.3).

Discrete operator: with the auxiliary fluxes F_j = bar(rho v)^{1x_j} - delta_1 P /
delta_1 x_j (Eq 3.23) inserted into the discrete continuity equation (Eq 3.24,
plus S_m of Eq 3.33), the unknown P = p dt solves

    L P := sum_j delta_1(delta_1 P / delta_1 x_j) / delta_1 x_j = b,

the compact (2 dim + 1)-point Laplacian.  On a non-periodic side the boundary
mass flux is known, so the boundary interface carries no pressure term:
homogeneous Neumann for P (Sec. 3.3).  L annihilates constants; the zero-mean
solution is selected (augmented-matrix method, Sec. 3.3).

``solve`` diagonalises L exactly: discrete Fourier modes along periodic
directions and DCT-II modes (cell-centred Neumann) along the others; the
eigenvalue of mode k along d is -(2 - 2 cos theta_k)/h_d^2 with
theta_k = 2 pi k / n_d (periodic) or pi k / n_d (Neumann).  ``dense_solve`` is the
brute-force check: it assembles L column by column from ``apply`` and solves
the augmented system [L 1; 1^T 0].

On a stretched grid (Eq 4.18) L is no longer diagonalised by those bases.
There ``solve`` assembles L as a sum of Kronecker products of the 1D
operators delta_1(delta_1 . / delta_1 x_d) / delta_1 x_d and factors, once
per grid, the augmented system [W L, w; w^T, 0] (W the cell volumes, w their
vector): W L is symmetric (the volume-weighted sum of L P is the net
boundary flux, zero here), and the border row selects the solution with zero
volume-weighted mean.
"""

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from .operators import V, diff_to_faces, faces_diff_to_cells


def apply(P_int, g, periodic):
    """L P for an interior-shaped array (Neumann faces carry no flux)."""
    P = g.zeros()
    V(P, g)[...] = P_int
    for d in range(g.dim):
        n = g.n[d]
        a = g.ax(d)
        sl0 = [slice(None)] * g.dim
        sl1 = [slice(None)] * g.dim
        if periodic[d]:
            sl0[a], sl1[a] = 0, n
            P[tuple(sl0)] = P[tuple(sl1)]
            sl0[a], sl1[a] = n + 1, 1
            P[tuple(sl0)] = P[tuple(sl1)]
    out = np.zeros(P_int.shape)
    for j in range(g.dim):
        fv = diff_to_faces(P, g, j)
        if not periodic[j]:
            a = g.ax(j)
            sl = [slice(None)] * g.dim
            sl[a] = 0
            fv[tuple(sl)] = 0.0
            sl[a] = g.n[j]
            fv[tuple(sl)] = 0.0
        out += faces_diff_to_cells(fv, g, j)
    return out


def eigenvalues(g, periodic):
    """Eigenvalues of L on the separable basis, broadcast to the interior shape."""
    lam = np.zeros(tuple(g.n[d] for d in reversed(range(g.dim))))
    for d in range(g.dim):
        n = g.n[d]
        k = np.arange(n)
        theta = (2.0 * np.pi * k / n) if periodic[d] else (np.pi * k / n)
        ld = -(2.0 - 2.0 * np.cos(theta)) / g.h[d] ** 2
        shp = [1] * g.dim
        shp[g.ax(d)] = n
        lam = lam + ld.reshape(shp)
    return lam


def _operator_1d(g, d, periodic):
    """delta_1(delta_1 P / delta_1 x_d) / delta_1 x_d along direction d of a
    stretched grid (n_d x n_d, zero flux through non-periodic ends)."""
    n = g.n[d]
    xc, dx = g.xc[d], g.dx[d][1:-1]
    G = sp.lil_matrix((n + 1, n))              # interface gradients, faces 0..n
    for f in range(1, n):
        G[f, f] = 1.0 / (xc[f + 1] - xc[f])
        G[f, f - 1] = -1.0 / (xc[f + 1] - xc[f])
    if periodic[d]:
        for f in (0, n):                       # the same interface seen from both ends
            G[f, 0] = 1.0 / (xc[1] - xc[0])
            G[f, n - 1] = -1.0 / (xc[1] - xc[0])
    D = sp.lil_matrix((n, n + 1))
    for c in range(n):
        D[c, c + 1] = 1.0 / dx[c]
        D[c, c] = -1.0 / dx[c]
    return (D.tocsr() @ G.tocsr()).tocsr()


def _stretched_factor(g, periodic):
    key = tuple(bool(p) for p in periodic)
    cache = g.__dict__.setdefault("_poisson_lu", {})
    if key not in cache:
        L = None
        for d in range(g.dim):
            term = sp.identity(1, format="csr")
            for dd in reversed(range(g.dim)):           # x is the fastest index
                term = sp.kron(term, _operator_1d(g, dd, periodic) if dd == d
                               else sp.identity(g.n[dd], format="csr"), format="csr")
            L = term if L is None else L + term
        w = np.asarray(g.dV * np.ones(tuple(g.n[d] for d in reversed(range(g.dim))))).ravel()
        WL = sp.diags(w) @ L
        M = sp.bmat([[WL, sp.csr_matrix(w[:, None])], [sp.csr_matrix(w[None, :]), None]], format="csc")
        cache[key] = (splu(M), w, L)
    return cache[key]


def solve(b, g, periodic):
    """Zero-mean P with L P = b - mean(b) (exact: transform-diagonalised on a
    uniform grid, a sparse LU factorisation on a stretched one, where both
    means are volume-weighted).  A complex b (a complex-step perturbation)
    is solved part by part: L is real."""
    if np.iscomplexobj(b):
        return solve(b.real, g, periodic) + 1j * solve(b.imag, g, periodic)
    if not g.uniform:
        lu, w, _ = _stretched_factor(g, periodic)
        r = np.asarray(b, dtype=np.float64).ravel()
        r = r - np.dot(w, r) / np.sum(w)
        sol = lu.solve(np.concatenate([w * r, [0.0]]))
        return sol[:-1].reshape(np.asarray(b).shape)
    X = np.asarray(b, dtype=np.float64).astype(np.complex128)
    for d in range(g.dim):
        a = g.ax(d)
        if periodic[d]:
            X = sfft.fft(X, axis=a)
        else:
            X = sfft.dct(X.real, type=2, axis=a, norm="ortho") + 1j * sfft.dct(
                X.imag, type=2, axis=a, norm="ortho")
    lam = eigenvalues(g, periodic)
    zero = (lam == 0.0)
    lam_safe = np.where(zero, 1.0, lam)
    X = np.where(zero, 0.0, X / lam_safe)
    for d in reversed(range(g.dim)):
        a = g.ax(d)
        if periodic[d]:
            X = sfft.ifft(X, axis=a)
        else:
            X = sfft.idct(X.real, type=2, axis=a, norm="ortho") + 1j * sfft.idct(
                X.imag, type=2, axis=a, norm="ortho")
    P = X.real
    return P - P.mean()


def assemble(g, periodic):
    """Dense matrix of L (interior cells, x fastest)."""
    N = int(np.prod(g.n))
    shape = tuple(g.n[d] for d in reversed(range(g.dim)))
    A = np.zeros((N, N))
    e = np.zeros(N)
    for col in range(N):
        e[:] = 0.0
        e[col] = 1.0
        A[:, col] = apply(e.reshape(shape), g, periodic).ravel()
    return A


def dense_solve(b, g, periodic):
    """Brute force: augmented system [L 1; 1^T 0] [P; lambda] = [b; 0]."""
    A = assemble(g, periodic)
    N = A.shape[0]
    M = np.zeros((N + 1, N + 1))
    M[:N, :N] = A
    M[:N, N] = 1.0
    M[N, :N] = 1.0
    rhs = np.zeros(N + 1)
    rhs[:N] = np.asarray(b).ravel()
    sol = np.linalg.solve(M, rhs)
    return sol[:N].reshape(np.asarray(b).shape), sol[N]
