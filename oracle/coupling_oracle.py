"""FP64 oracle: von Karman coupling tensors of a simply supported rectangle.

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline leg.  Shares no code with the library.

Sec. 3.1, Eqs. 10-11:
    H^k_ij = int Psi_k L(Phi_i, Phi_j) dS / (|Psi_k| |Phi_i| |Phi_j|)
    C^s_ij = int Phi_s L(Phi_i, Psi_j) dS / (|Phi_s| |Phi_i| |Psi_j|)
with the von Karman operator of Eq. 7,
    L(f, g) = f_xx g_yy + f_yy g_xx - 2 f_xy g_xy,
transverse modes Phi the simply supported sin*sin modes and in-plane modes Psi
the eigenfunctions of the Airy problem Delta Delta Psi = zeta^4 Psi.  The paper
does not state the Airy boundary conditions; this file uses Psi = dPsi/dn = 0
on all four edges (the in-plane-movable simply supported plate).

Method (plain, no separability tricks):
  * Rayleigh-Ritz for Psi on the tensor basis B_a(xi) B_b(upsilon),
    B_a = (1 - xi^2)^2 P_a(xi) (Legendre P_a), which satisfies both boundary
    conditions; stiffness int (Delta Psi)^2, mass int Psi^2, both by 2D tensor
    Gauss-Legendre quadrature; generalized symmetric eigenproblem;
  * H and C by 2D tensor Gauss-Legendre quadrature of the integrands above.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import physics_oracle as phys


def _legendre_with_derivs(n_basis, xi):
    """P_a(xi), P_a'(xi), P_a''(xi), P_a'''(xi), P_a''''(xi) for a < n_basis."""
    out = []
    for a in range(n_basis):
        c = np.zeros(n_basis)
        c[a] = 1.0
        vals = [np.polynomial.legendre.legval(xi, c)]
        d = c
        for _ in range(4):
            d = np.polynomial.legendre.legder(d)
            vals.append(np.polynomial.legendre.legval(xi, d) if d.size else np.zeros_like(xi))
        out.append(vals)
    return np.array(out)  # [a][deriv][points]


def _ritz_basis_1d(n_basis, xi):
    """B_a = (1 - xi^2)^2 P_a and its first two derivatives with respect to xi."""
    P = _legendre_with_derivs(n_basis, xi)
    w = (1.0 - xi ** 2) ** 2
    w1 = -4.0 * xi * (1.0 - xi ** 2)
    w2 = -4.0 + 12.0 * xi ** 2
    B0 = w * P[:, 0]
    B1 = w1 * P[:, 0] + w * P[:, 1]
    B2 = w2 * P[:, 0] + 2.0 * w1 * P[:, 1] + w * P[:, 2]
    return B0, B1, B2


def airy_modes(Lx, Ly, n_psi, n_basis=20, n_quad=64):
    """Lowest n_psi Airy modes: returns (zeta4 [n_psi], evaluator) where
    evaluator(x, y) gives Psi, Psi_xx, Psi_yy, Psi_xy at physical points
    (flattened grids), each [points][n_psi], unit L2 norm on the rectangle."""
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    B0, B1, B2 = _ritz_basis_1d(n_basis, xg)
    sx, sy = 2.0 / Lx, 2.0 / Ly            # d xi / dx, d upsilon / dy
    # 2D values on the tensor grid: index (i, j) over quadrature points, (a, b) over basis
    Psi = np.einsum("ai,bj->ijab", B0, B0).reshape(n_quad * n_quad, -1)
    lap = (sx ** 2 * np.einsum("ai,bj->ijab", B2, B0) +
           sy ** 2 * np.einsum("ai,bj->ijab", B0, B2)).reshape(n_quad * n_quad, -1)
    W = (np.outer(wg, wg) * (Lx / 2.0) * (Ly / 2.0)).reshape(-1)
    K = lap.T @ (W[:, None] * lap)
    Mm = Psi.T @ (W[:, None] * Psi)
    vals, vecs = scipy.linalg.eigh(K, Mm)
    order = np.argsort(vals, kind="stable")[:n_psi]
    zeta4 = vals[order]
    C = vecs[:, order]                      # Mm-orthonormal: unit L2 norm in physical units
    # deterministic sign: the largest-magnitude coefficient is positive
    idx = np.argmax(np.abs(C), axis=0)
    C = C * np.sign(C[idx, np.arange(C.shape[1])])

    def evaluate(x, y):
        xi = 2.0 * np.asarray(x) / Lx - 1.0
        up = 2.0 * np.asarray(y) / Ly - 1.0
        X0, X1, X2 = _ritz_basis_1d(n_basis, xi)
        Y0, Y1, Y2 = _ritz_basis_1d(n_basis, up)
        def comb(X, Y, scale):
            # point-wise product of x- and y-factors: points are paired (x[i], y[i])
            return scale * np.einsum("ai,bi->iab", X, Y).reshape(len(xi), -1) @ C
        return (comb(X0, Y0, 1.0), comb(X2, Y0, sx ** 2), comb(X0, Y2, sy ** 2),
                comb(X1, Y1, sx * sy))

    return zeta4, evaluate


def _phi_derivs(labels, Lx, Ly, x, y):
    """Unit-norm simply supported modes and second derivatives at points (x, y)."""
    m = labels[:, 0][None, :]
    k = labels[:, 1][None, :]
    a = m * math.pi / Lx
    b = k * math.pi / Ly
    x = np.asarray(x)[:, None]
    y = np.asarray(y)[:, None]
    A = 2.0 / math.sqrt(Lx * Ly)
    sxv, cxv = np.sin(a * x), np.cos(a * x)
    syv, cyv = np.sin(b * y), np.cos(b * y)
    phi = A * sxv * syv
    return phi, -a ** 2 * phi, -b ** 2 * phi, A * a * b * cxv * cyv


def _grid(Lx, Ly, n_quad):
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    x = (xg + 1.0) * Lx / 2.0
    y = (xg + 1.0) * Ly / 2.0
    X, Y = np.meshgrid(x, y, indexing="ij")
    W = np.outer(wg, wg) * (Lx / 2.0) * (Ly / 2.0)
    return X.reshape(-1), Y.reshape(-1), W.reshape(-1)


def default_quadrature(labels, n_basis):
    kmax = int(max(labels[:, 0].max(), labels[:, 1].max()))
    return int(max(48, 2 * kmax + n_basis + 24))


def default_basis(n_psi):
    return int(max(16, math.ceil(2.0 * math.sqrt(n_psi)) + 12))


def coupling_H(inst, labels, n_psi, n_basis=None, n_quad=None):
    """H[k][i][j] (Eq. 10) for the given transverse labels, and zeta^4 [k]."""
    Lx, Ly = phys.rect_sides(inst)
    n_basis = n_basis or default_basis(n_psi)
    n_quad = n_quad or default_quadrature(labels, n_basis)
    zeta4, psi_eval = airy_modes(Lx, Ly, n_psi, n_basis=n_basis, n_quad=max(64, n_basis + 8))
    X, Y, W = _grid(Lx, Ly, n_quad)
    Psi, _, _, _ = psi_eval(X, Y)
    _, Pxx, Pyy, Pxy = _phi_derivs(labels, Lx, Ly, X, Y)
    N = labels.shape[0]
    H = np.empty((n_psi, N, N))
    for k in range(n_psi):
        wk = (W * Psi[:, k])[:, None]
        H[k] = Pxx.T @ (wk * Pyy) + Pyy.T @ (wk * Pxx) - 2.0 * Pxy.T @ (wk * Pxy)
    return H, zeta4


def coupling_C(inst, labels, n_psi, n_basis=None, n_quad=None):
    """C[s][i][j] = int Phi_s L(Phi_i, Psi_j) dS (Eq. 11), by its own quadrature."""
    Lx, Ly = phys.rect_sides(inst)
    n_basis = n_basis or default_basis(n_psi)
    n_quad = n_quad or default_quadrature(labels, n_basis)
    _, psi_eval = airy_modes(Lx, Ly, n_psi, n_basis=n_basis, n_quad=max(64, n_basis + 8))
    X, Y, W = _grid(Lx, Ly, n_quad)
    _, Sxx, Syy, Sxy = psi_eval(X, Y)
    Phi, Pxx, Pyy, Pxy = _phi_derivs(labels, Lx, Ly, X, Y)
    N = labels.shape[0]
    C = np.empty((N, N, n_psi))
    for s in range(N):
        ws = (W * Phi[:, s])[:, None]
        C[s] = Pxx.T @ (ws * Syy) + Pyy.T @ (ws * Sxx) - 2.0 * Pxy.T @ (ws * Sxy)
    return C


def oracle_coupling(inst, labels, n_psi):
    """Callable for physics_oracle.build_instance."""
    return coupling_H(inst, labels, n_psi)
