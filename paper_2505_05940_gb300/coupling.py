"""Von Karman coupling tensors of a simply supported rectangle (host, FP64).

Sec. 3.1, Eq. 10: H^k_ij = int Psi_k L(Phi_i, Phi_j) dS with unit-norm modes,
L(f, g) = f_xx g_yy + f_yy g_xx - 2 f_xy g_xy (Eq. 7), Phi the simply
supported sin*sin modes and Psi the Airy stress modes, Delta Delta Psi =
zeta^4 Psi with Psi = dPsi/dn = 0 on the edges (in-plane-movable simply
supported plate; the paper leaves these conditions to its references).

This generator is offline preprocessing for the plan (the coupling tensor is
an input of mdx_plan_create).  It exploits separability: Psi is expanded in
products B_a(x) B_b(y), B_a = (1 - xi^2)^2 P_a(xi); for sin*sin modes L(Phi_i,
Phi_j) is a sum of two products of one-dimensional functions, so H reduces to
one-dimensional Gauss-Legendre integrals contracted with the Ritz
coefficients.  The Ritz problem splits into four parity blocks (even / odd
about each mid-line).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def _basis_1d(n_basis, xi):
    """B_a(xi) = (1 - xi^2)^2 P_a(xi) and d/dxi, d^2/dxi^2 for a < n_basis."""
    V = np.polynomial.legendre.legvander(xi, n_basis - 1).T           # [a][pts]
    eye = np.eye(n_basis)
    V1 = np.array([np.polynomial.legendre.legval(xi, np.polynomial.legendre.legder(eye[a], 1))
                   if a > 0 else np.zeros_like(xi) for a in range(n_basis)])
    V2 = np.array([np.polynomial.legendre.legval(xi, np.polynomial.legendre.legder(eye[a], 2))
                   if a > 1 else np.zeros_like(xi) for a in range(n_basis)])
    w = (1 - xi ** 2) ** 2
    w1 = -4 * xi * (1 - xi ** 2)
    w2 = 12 * xi ** 2 - 4
    return w * V, w1 * V + w * V1, w2 * V + 2 * w1 * V1 + w * V2


def default_basis(n_psi):
    return int(max(16, math.ceil(2.0 * math.sqrt(n_psi)) + 12))


def airy_modes(Lx, Ly, n_psi, n_basis=None):
    """Lowest n_psi Airy eigenpairs.  Returns zeta4 [n_psi] and coefficient
    tensors C [n_psi][n_basis][n_basis] (Psi_k = sum C_kab B_a(x) B_b(y)),
    normalised to unit L2 norm on the plate."""
    nb = n_basis or default_basis(n_psi)
    xg, wg = np.polynomial.legendre.leggauss(nb + 8)
    B0, B1, B2 = _basis_1d(nb, xg)
    sx, sy = 2.0 / Lx, 2.0 / Ly
    jx, jy = Lx / 2.0, Ly / 2.0
    I00 = (B0 * wg) @ B0.T
    I22 = (B2 * wg) @ B2.T
    I20 = (B2 * wg) @ B0.T
    Mx, My = I00 * jx, I00 * jy
    Kx = [I00 * jx, I20 * sx ** 2 * jx, I22 * sx ** 4 * jx]   # [d0d0, d2d0, d2d2]
    Ky = [I00 * jy, I20 * sy ** 2 * jy, I22 * sy ** 4 * jy]
    vals, vecs = [], []
    par = np.arange(nb) % 2
    for px in (0, 1):
        for py in (0, 1):
            ia = np.where(par == px)[0]
            ib = np.where(par == py)[0]
            sub = lambda A, I: A[np.ix_(I, I)]
            K = (np.kron(sub(Kx[2], ia), sub(Ky[0], ib)) + np.kron(sub(Kx[1], ia), sub(Ky[1], ib).T)
                 + np.kron(sub(Kx[1], ia).T, sub(Ky[1], ib)) + np.kron(sub(Kx[0], ia), sub(Ky[2], ib)))
            M = np.kron(sub(Mx, ia), sub(My, ib))
            w, v = scipy.linalg.eigh(K, M)
            for j in range(min(len(w), n_psi)):
                C = np.zeros((nb, nb))
                C[np.ix_(ia, ib)] = v[:, j].reshape(len(ia), len(ib))
                vals.append(w[j])
                vecs.append(C)
    order = np.argsort(np.array(vals), kind="stable")[:n_psi]
    zeta4 = np.array(vals)[order]
    C = np.stack([vecs[o] for o in order])
    flat = C.reshape(n_psi, -1)
    idx = np.argmax(np.abs(flat), axis=1)
    C = C * np.sign(flat[np.arange(n_psi), idx])[:, None, None]
    return zeta4, C


def _one_d_integrals(L, kmax, n_basis, n_quad):
    """J_s[a, m, m'] = int_0^L B_a sin(m pi x/L) sin(m' pi x/L) dx and the cos*cos
    counterpart J_c, for m, m' = 1..kmax."""
    xg, wg = np.polynomial.legendre.leggauss(n_quad)
    B0, _, _ = _basis_1d(n_basis, xg)
    x = (xg + 1) * L / 2
    w = wg * L / 2
    m = np.arange(1, kmax + 1)
    S = np.sin(np.outer(m, x) * math.pi / L)
    Cc = np.cos(np.outer(m, x) * math.pi / L)
    Js = np.einsum("ap,mp,np->amn", B0 * w, S, S)
    Jc = np.einsum("ap,mp,np->amn", B0 * w, Cc, Cc)
    return Js, Jc


def coupling_tensor(Lx, Ly, labels, n_psi, n_basis=None, n_quad=None, airy=None):
    """H [n_psi][N][N] for transverse mode labels (m, n) and zeta4 [n_psi].

    With G^k[(m, m'), (n, n')] = sum_ab C^k_ab Jx[a, m, m'] Jy[b, n, n'] (two
    matrix products over all label pairs), H^k_ij is a gather of G^k at
    ((m_i, m_j), (n_i, n_j)) weighted by the derivative factors of L."""
    labels = np.asarray(labels, dtype=np.int64)
    nb = n_basis or default_basis(n_psi)
    zeta4, C = airy if airy is not None else airy_modes(Lx, Ly, n_psi, nb)
    mx, my = int(labels[:, 0].max()), int(labels[:, 1].max())
    kmax = max(mx, my)
    nq = n_quad or int(max(48, 2 * kmax + nb + 24))
    Jsx, Jcx = _one_d_integrals(Lx, mx, nb, nq)
    Jsy, Jcy = _one_d_integrals(Ly, my, nb, nq)
    A2 = 4.0 / (Lx * Ly)
    m = labels[:, 0]
    n = labels[:, 1]
    al = m * math.pi / Lx
    be = n * math.pi / Ly
    w1 = np.outer(al ** 2, be ** 2) + np.outer(be ** 2, al ** 2)
    w2 = 2.0 * np.outer(al * be, al * be)
    pm = ((m - 1)[:, None] * mx + (m - 1)[None, :])          # index of (m_i, m_j)
    pn = ((n - 1)[:, None] * my + (n - 1)[None, :])          # index of (n_i, n_j)

    def contract(Jx, Jy):
        Tk = np.matmul(C, Jy.reshape(nb, -1))                    # [k][a][(n, n')]
        return np.matmul(Jx.reshape(nb, -1).T[None], Tk)          # [k][(m, m')][(n, n')]

    Gs = contract(Jsx, Jsy)
    Gc = contract(Jcx, Jcy)
    H = A2 * (w1[None] * Gs[:, pm, pn] - w2[None] * Gc[:, pm, pn])
    return H, zeta4


def transverse_classes(labels):
    """Symmetry class of each simply supported mode sin(m pi x/Lx) sin(n pi y/Ly):
    bit 1 set when the mode is odd about x = Lx/2 (m even), bit 0 when odd
    about y = Ly/2 (n even)."""
    labels = np.asarray(labels, dtype=np.int64)
    return (2 * ((labels[:, 0] + 1) % 2) + ((labels[:, 1] + 1) % 2)).astype(np.int32)


def airy_classes(C):
    """Symmetry class of each Airy mode from its Ritz coefficients: the basis
    B_a(x) B_b(y) is odd about the x mid-line for odd a and about the y
    mid-line for odd b, and every eigenvector lives in one parity block."""
    nb = C.shape[1]
    par = np.arange(nb) % 2
    out = []
    for Ck in C:
        w = np.abs(Ck)
        ax = int(np.argmax([w[par == 0].sum(), w[par == 1].sum()]))
        ay = int(np.argmax([w[:, par == 0].sum(), w[:, par == 1].sum()]))
        out.append(2 * ax + ay)
    return np.array(out, dtype=np.int32)


def sides(area, aspect):
    return math.sqrt(area / aspect), math.sqrt(area * aspect)


def coupling_with_aspect_derivative(area, aspect, labels, n_psi, rel_step=1e-4, n_basis=None):
    """H, zeta4 at aspect a = Ly/Lx (area fixed) and their derivatives with
    respect to a by central differences at fixed mode labels; the Airy mode
    signs at a +- h are aligned with those at a."""
    nb = n_basis or default_basis(n_psi)
    Lx, Ly = sides(area, aspect)
    z0, C0 = airy_modes(Lx, Ly, n_psi, nb)
    H0, _ = coupling_tensor(Lx, Ly, labels, n_psi, nb, airy=(z0, C0))
    h = rel_step * aspect
    cls0 = airy_classes(C0)
    out = []
    for a in (aspect + h, aspect - h):
        lx, ly = sides(area, a)
        # a few extra modes so that a crossing at the cut cannot lose a partner
        z, C = airy_modes(lx, ly, n_psi + 4, nb)
        cls = airy_classes(C)
        # pair every mode at `aspect` with the mode of the same symmetry class
        # whose eigenvalue is closest (robust to ordering changes), then align signs
        order = []
        for k in range(n_psi):
            cand = [j for j in range(len(z)) if cls[j] == cls0[k] and j not in order]
            order.append(min(cand, key=lambda j: abs(z[j] - z0[k])))
        z, C = z[order], C[order]
        sgn = np.sign(np.einsum("kab,kab->k", C, C0))
        C = C * sgn[:, None, None]
        Ha, _ = coupling_tensor(lx, ly, labels, n_psi, nb, airy=(z, C))
        out.append((Ha, z))
    dH = (out[0][0] - out[1][0]) / (2 * h)
    dz = (out[0][1] - out[1][1]) / (2 * h)
    return H0, z0, dH, dz, airy_classes(C0)
