"""Dense brute-force assembly of the FOEED / EED operators for tiny grids.

An independent second route to the oracle's operators, used only to pin the
oracle. Instead of ghost cells with parity rules, the operators are built as
explicit matrices acting on the whole image vector (row-major, p = y*w + x):

  inner derivatives A_xx, A_xy = A_yx, A_yy with mirrored (even) ghosts,
  P = sum_{ij,kl} A_ij^T diag(d_ijkl) A_kl          (FOEED, energy form)
  P_EED = F_x^T diag(a_face) F_x + F_y^T diag(c_face) F_y
          + D_x^T diag(b) D_y + D_y^T diag(b) D_x  (EED)

so the outer operator is the transpose of the inner one by construction
(Sec. 3.3 requires P symmetric for FSI).
"""
from __future__ import annotations

import numpy as np


def mirror(i: int, n: int) -> int:
    p = 2 * n
    i %= p
    return i if i < n else p - 1 - i


def second_diff(n: int) -> np.ndarray:
    """u[i-1] - 2u[i] + u[i+1], mirrored ghosts."""
    M = np.zeros((n, n))
    for i in range(n):
        M[i, mirror(i - 1, n)] += 1.0
        M[i, i] -= 2.0
        M[i, mirror(i + 1, n)] += 1.0
    return M


def central_diff(n: int) -> np.ndarray:
    """(u[i+1] - u[i-1]) / 2, mirrored ghosts."""
    M = np.zeros((n, n))
    for i in range(n):
        M[i, mirror(i + 1, n)] += 0.5
        M[i, mirror(i - 1, n)] -= 0.5
    return M


def forward_diff(n: int) -> np.ndarray:
    """Face differences u[i+1] - u[i], i = 0..n-2 (no flux through the border faces)."""
    M = np.zeros((max(n - 1, 0), n))
    for i in range(n - 1):
        M[i, i] = -1.0
        M[i, i + 1] = 1.0
    return M


def gauss_1d(n: int, wts: np.ndarray) -> np.ndarray:
    R = (len(wts) - 1) // 2
    M = np.zeros((n, n))
    for i in range(n):
        for t in range(-R, R + 1):
            M[i, mirror(i + t, n)] += wts[t + R]
    return M


def ops2d(h: int, w: int):
    """Inner derivative matrices on the h*w image vector."""
    Ih, Iw = np.eye(h), np.eye(w)
    Axx = np.kron(Ih, second_diff(w))
    Ayy = np.kron(second_diff(h), Iw)
    Axy = np.kron(central_diff(h), central_diff(w))
    Dx = np.kron(Ih, central_diff(w))
    Dy = np.kron(central_diff(h), Iw)
    return Axx, Axy, Ayy, Dx, Dy


def foeed_P(d: np.ndarray) -> np.ndarray:
    """P = sum A_ij^T diag(d_ijkl) A_kl for a tensor field d [h, w, 2, 2, 2, 2]."""
    h, w = d.shape[:2]
    Axx, Axy, Ayy, _, _ = ops2d(h, w)
    A = {(0, 0): Axx, (0, 1): Axy, (1, 0): Axy, (1, 1): Ayy}
    n = h * w
    P = np.zeros((n, n))
    for (i, j), Aij in A.items():
        for (k, l), Akl in A.items():
            P += Aij.T @ (d[:, :, i, j, k, l].reshape(-1)[:, None] * Akl)
    return P


def eed_P(abc: np.ndarray) -> np.ndarray:
    """Symmetric EED matrix for a field (a, b, c) [h, w, 3]."""
    h, w = abc.shape[:2]
    a, b, c = abc[..., 0], abc[..., 1], abc[..., 2]
    Fx = np.kron(np.eye(h), forward_diff(w))
    Fy = np.kron(forward_diff(h), np.eye(w))
    a_face = ((a[:, :-1] + a[:, 1:]) / 2.0).reshape(-1)
    c_face = ((c[:-1, :] + c[1:, :]) / 2.0).reshape(-1)
    _, _, _, Dx, Dy = ops2d(h, w)
    bb = b.reshape(-1)[:, None]
    P = Fx.T @ (a_face[:, None] * Fx) + Fy.T @ (c_face[:, None] * Fy)
    P += Dx.T @ (bb * Dy) + Dy.T @ (bb * Dx)
    return P


def gauss_2d(h: int, w: int, wts: np.ndarray) -> np.ndarray:
    return np.kron(gauss_1d(h, wts), gauss_1d(w, wts))


def spectral_tensor(gx: float, gy: float, mu1: float, mu3: float) -> np.ndarray:
    """d = sum_r mu_r E_r (x) E_r from the eigenpairs of Sec. 3.1, built with einsum."""
    nrm = np.hypot(gx, gy)
    v1 = np.array([1.0, 0.0]) if nrm == 0 else np.array([gx, gy]) / nrm
    v2 = np.array([-v1[1], v1[0]])
    E1 = np.outer(v1, v1)
    E2 = np.outer(v2, v2)
    E3 = (np.outer(v1, v2) + np.outer(v2, v1)) / np.sqrt(2.0)
    return (mu1 * np.einsum("ij,kl->ijkl", E1, E1) + np.einsum("ij,kl->ijkl", E2, E2)
            + mu3 * np.einsum("ij,kl->ijkl", E3, E3))


def dense_foeed_fsi(f, mask, sigma, lam, tau, cycle_len, cycles, wts):
    """Whole FSI solve with dense matrices rebuilt every step (Charbonnier, mu3 = sqrt(mu1))."""
    h, w = f.shape
    G = gauss_2d(h, w, wts)
    _, _, _, Dx, Dy = ops2d(h, w)
    known = mask.reshape(-1) != 0
    fv = f.reshape(-1)
    u = np.where(known, fv, fv[known].mean() if known.any() else 0.0)
    for _ in range(cycles):
        um = u.copy()
        for k in range(cycle_len):
            alpha = (4.0 * k + 2.0) / (2.0 * k + 3.0)
            us = G @ u
            gx, gy = Dx @ us, Dy @ us
            d = np.zeros((h * w, 2, 2, 2, 2))
            for p in range(h * w):
                s2 = gx[p] ** 2 + gy[p] ** 2
                mu1 = 1.0 / np.sqrt(1.0 + s2 / lam ** 2)
                d[p] = spectral_tensor(gx[p], gy[p], mu1, np.sqrt(mu1))
            P = foeed_P(d.reshape(h, w, 2, 2, 2, 2))
            un = alpha * (u - tau * (P @ u)) + (1.0 - alpha) * um
            un[known] = u[known]
            um, u = u, un
    return u.reshape(h, w)
