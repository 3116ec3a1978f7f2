"""Direct solvers of the discrete lower-boundary and interior problems.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Two solvers that share
nothing with the multigrid oracle in ``mhs_oracle.c``; they reach the exact
solution of the same discrete equations up to rounding, so they pin it:

* :func:`separable_solve2d` / :func:`separable_solve3d`: xi depends on z only
  (Sect. 2.1, eq. scalar_pot) and the side faces are Dirichlet (Sect. 2.2), so
  the discrete sine vectors sin(m pi i/(nx-1)) sin(n pi j/(ny-1)) diagonalise
  the horizontal second differences with eigenvalues
  lambda_mn = -(4/hx^2) sin^2(m pi / (2(nx-1))) - (4/hy^2) sin^2(n pi / (2(ny-1))).
  Eq. (lower_bound) is then a division per mode, and eq. (scalar_pot) one
  tridiagonal system in k per mode (Thomas algorithm).  The transform is a
  plain matrix product (no FFT library).
* :func:`kron_solve3d`: the interior matrix built from Kronecker products of
  1D second-difference matrices and solved by a sparse direct factorisation
  (scipy's SuperLU).
"""
from __future__ import annotations

import math

import numpy as np


def _sine_matrix(n: int) -> np.ndarray:
    """S[m-1, i-1] = sin(pi m i / (n-1)) for interior index i and mode m."""
    idx = np.arange(1, n - 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(idx, idx) / (n - 1))


def _eig_1d(n: int, h: float) -> np.ndarray:
    m = np.arange(1, n - 1, dtype=np.float64)
    return -(4.0 / (h * h)) * np.sin(np.pi * m / (2.0 * (n - 1))) ** 2


def _fwd(a2: np.ndarray, Sy: np.ndarray, Sx: np.ndarray) -> np.ndarray:
    """Sine transform of an interior [ny-2][nx-2] block (unnormalised)."""
    return Sy @ a2 @ Sx.T


def _inv(a2: np.ndarray, Sy: np.ndarray, Sx: np.ndarray, nx: int, ny: int) -> np.ndarray:
    # S S^T = (n-1)/2 I for the unnormalised sine matrix.
    return (2.0 / (ny - 1)) * (2.0 / (nx - 1)) * (Sy.T @ a2 @ Sx)


def _xi(pr, z):
    k = pr["xi_kind"]
    if k == 1:
        return pr["xi_a"] * np.exp(-pr["xi_kappa"] * z)
    if k == 2:
        return (pr["xi_a"] + pr["xi_b"] * np.sin(pr["xi_omega"] * z)) * np.exp(-pr["xi_kappa"] * z)
    return np.zeros_like(z)


def separable_solve2d(pr, bz: np.ndarray) -> np.ndarray:
    """Exact discrete solution of P_xx + P_yy = -B_z, P = 0 on the edges."""
    nx, ny = pr["nx"], pr["ny"]
    hx, hy = pr["Lx"] / (nx - 1), pr["Ly"] / (ny - 1)
    Sx, Sy = _sine_matrix(nx), _sine_matrix(ny)
    lam = _eig_1d(ny, hy)[:, None] + _eig_1d(nx, hx)[None, :]
    bh = _fwd(np.asarray(bz, dtype=np.float64)[1:-1, 1:-1], Sy, Sx)
    P = np.zeros((ny, nx))
    P[1:-1, 1:-1] = _inv(-bh / lam, Sy, Sx, nx, ny)
    return P


def separable_solve3d(pr, P0: np.ndarray, f: np.ndarray | None = None, top: np.ndarray | None = None) -> np.ndarray:
    """Exact discrete solution of eq. (scalar_pot) (+ optional interior RHS f)
    with P = P0 on k = 0, P = top (default 0) on k = nz-1 and P = 0 on the
    sides.  P0 and top must vanish on their edges."""
    nx, ny, nz = pr["nx"], pr["ny"], pr["nz"]
    hx, hy, hz = pr["Lx"] / (nx - 1), pr["Ly"] / (ny - 1), pr["Lz"] / (nz - 1)
    alpha2 = pr["alpha"] ** 2
    Sx, Sy = _sine_matrix(nx), _sine_matrix(ny)
    lam = _eig_1d(ny, hy)[:, None] + _eig_1d(nx, hx)[None, :]
    z = np.arange(nz, dtype=np.float64) * hz
    xi = _xi(pr, z)
    cz = 1.0 / (hz * hz)
    # transformed Dirichlet data and right-hand side per plane
    bot = _fwd(np.asarray(P0, dtype=np.float64)[1:-1, 1:-1], Sy, Sx)
    tp = np.zeros_like(bot) if top is None else _fwd(np.asarray(top, dtype=np.float64)[1:-1, 1:-1], Sy, Sx)
    m = nz - 2
    rhs = np.zeros((m,) + bot.shape)
    if f is not None:
        for k in range(1, nz - 1):
            rhs[k - 1] = _fwd(np.asarray(f[k], dtype=np.float64)[1:-1, 1:-1], Sy, Sx)
    rhs[0] -= cz * bot
    rhs[-1] -= cz * tp
    # Thomas algorithm, all modes at once: sub = sup = cz, diagonal per plane.
    diag = np.stack([(1.0 - xi[k]) * lam - 2.0 * cz + alpha2 for k in range(1, nz - 1)])
    cp = np.zeros_like(rhs)
    dp = np.zeros_like(rhs)
    cp[0] = cz / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, m):
        den = diag[k] - cz * cp[k - 1]
        cp[k] = cz / den
        dp[k] = (rhs[k] - cz * dp[k - 1]) / den
    xh = np.zeros_like(rhs)
    xh[-1] = dp[-1]
    for k in range(m - 2, -1, -1):
        xh[k] = dp[k] - cp[k] * xh[k + 1]
    P = np.zeros((nz, ny, nx))
    P[0] = P0
    if top is not None:
        P[-1] = top
    for k in range(1, nz - 1):
        P[k, 1:-1, 1:-1] = _inv(xh[k - 1], Sy, Sx, nx, ny)
    return P


def _second_diff(n: int, h: float):
    import scipy.sparse as sp
    m = n - 2
    return sp.diags([np.ones(m - 1), -2.0 * np.ones(m), np.ones(m - 1)], [-1, 0, 1], format="csr") / (h * h)


def kron_matrix3d(pr):
    """Sparse matrix of eq. (scalar_pot) on the interior unknowns (x fastest)."""
    import scipy.sparse as sp
    nx, ny, nz = pr["nx"], pr["ny"], pr["nz"]
    hx, hy, hz = pr["Lx"] / (nx - 1), pr["Ly"] / (ny - 1), pr["Lz"] / (nz - 1)
    Ix, Iy, Iz = (sp.identity(n - 2, format="csr") for n in (nx, ny, nz))
    Lxy = sp.kron(Iy, _second_diff(nx, hx)) + sp.kron(_second_diff(ny, hy), Ix)
    z = np.arange(1, nz - 1, dtype=np.float64) * hz
    W = sp.diags(1.0 - _xi(pr, z))
    A = sp.kron(W, Lxy) + sp.kron(_second_diff(nz, hz), sp.kron(Iy, Ix)) + pr["alpha"] ** 2 * sp.identity(
        (nx - 2) * (ny - 2) * (nz - 2))
    return A.tocsc()


def kron_solve3d(pr, P0: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    """Direct sparse solve with P = P0 on k = 0 and P = 0 on the other faces."""
    import scipy.sparse.linalg as spla
    nx, ny, nz = pr["nx"], pr["ny"], pr["nz"]
    hz = pr["Lz"] / (nz - 1)
    b = np.zeros((nz - 2, ny - 2, nx - 2))
    if f is not None:
        b += np.asarray(f)[1:-1, 1:-1, 1:-1]
    b[0] -= np.asarray(P0)[1:-1, 1:-1] / (hz * hz)
    x = spla.spsolve(kron_matrix3d(pr), b.ravel())
    P = np.zeros((nz, ny, nx))
    P[0] = P0
    P[1:-1, 1:-1, 1:-1] = x.reshape(nz - 2, ny - 2, nx - 2)
    return P


def kron_solve2d(pr, bz: np.ndarray) -> np.ndarray:
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    nx, ny = pr["nx"], pr["ny"]
    hx, hy = pr["Lx"] / (nx - 1), pr["Ly"] / (ny - 1)
    A = (sp.kron(sp.identity(ny - 2), _second_diff(nx, hx)) + sp.kron(_second_diff(ny, hy), sp.identity(nx - 2))).tocsc()
    x = spla.spsolve(A, -np.asarray(bz)[1:-1, 1:-1].ravel())
    P = np.zeros((ny, nx))
    P[1:-1, 1:-1] = x.reshape(ny - 2, nx - 2)
    return P


def exact_solution(pr, bz: np.ndarray) -> np.ndarray:
    """The three-step procedure of Sect. 2.2 with the separable direct solvers."""
    P0 = separable_solve2d(pr, bz)
    return separable_solve3d(pr, P0)


def continuum_mode_solution(pr, m: int = 1, n: int = 1):
    """Continuum solution for constant xi = c (xi_kind 1 with kappa = 0) and
    B_z = sin(m pi x/Lx) sin(n pi y/Ly): P = P0(x,y) sinh(k (Lz - z)) / sinh(k Lz)
    with P0 = B_z / K^2, K^2 = (m pi/Lx)^2 + (n pi/Ly)^2 and
    k^2 = (1 - c) K^2 - alpha^2 (> 0).  Returns a function of (x, y, z)."""
    c = pr["xi_a"] if pr["xi_kind"] == 1 else 0.0
    assert pr["xi_kind"] in (0, 1) and (pr["xi_kind"] == 0 or pr["xi_kappa"] == 0.0)
    K2 = (m * math.pi / pr["Lx"]) ** 2 + (n * math.pi / pr["Ly"]) ** 2
    k = math.sqrt((1.0 - c) * K2 - pr["alpha"] ** 2)
    Lz = pr["Lz"]

    def P(x, y, z):
        base = np.sin(m * math.pi * x / pr["Lx"]) * np.sin(n * math.pi * y / pr["Ly"]) / K2
        return base * np.sinh(k * (Lz - z)) / math.sinh(k * Lz)

    return P
