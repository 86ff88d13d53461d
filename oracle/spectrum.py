"""Oracle of the dynamical correlation function (test infrastructure only).

The paper's spectrum calculation (Sec. 3.2) evaluates
    D(z) = <Phi_ex| (z I - H)^{-1} |Phi_ex>,   Phi_ex = O |Phi_0>,
with the structure factor S^zz(q, w) = -Im D(w + i eta) for
O = sum_l e^{i q l} S^z_l.  It names two algorithms: the continued fraction
built from Lanczos coefficients, and the shifted Krylov-subspace (shifted
COCG) method of its references (Frommer; Yamamoto et al.; Hoshi et al.).
Each is written here in its plain form, plus the definition itself:

  resolvent_dense      D(z) = sum_n |<n|Phi>|^2 / (z - E_n) from a full
                       eigendecomposition (small D only).
  lanczos_galerkin     the Galerkin solution on the Krylov space K_m(H, b):
                       D_m(z) = |b|^2 [(z - T_m)^{-1}]_{00} and its residual
                       |b - (z - H) x_m| / |b| = beta_m |[(z - T_m)^{-1}]_{m-1,0}|,
                       each by a dense complex solve with T_m.
  continued_fraction   |b|^2 / (z - a_0 - b_1^2 / (z - a_1 - ...)), bottom-up.
  shifted_cocg         the textbook shifted COCG: one seed system
                       (z_s - H) x = b in complex arithmetic with the bilinear
                       form u^T v, and every other shift through the collinear
                       residuals r^j = r / pi^j; keeps every solution vector
                       and reports D(z_j) = conj(b)^T x^j and the explicit
                       residual norms.

Only tests/ call these.  Nothing here is shared with the GPU library.
"""
from __future__ import annotations

import numpy as np


def resolvent_dense(H: np.ndarray, phi: np.ndarray, z) -> np.ndarray:
    """<phi|(z - H)^{-1}|phi> for every z, from numpy's Hermitian eigensolver."""
    E, U = np.linalg.eigh(H)
    w = np.abs(U.T @ np.asarray(phi, dtype=np.complex128)) ** 2  # |<n|phi>|^2
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    return np.array([np.sum(w / (zz - E)) for zz in z])


def lanczos_galerkin(alpha, beta, norm2: float, z):
    """Galerkin projection on the m-step Krylov space from its Lanczos
    coefficients: alpha[0..m-1], beta[0..m] with beta[0] unused and beta[m] the
    norm of the remainder.  Returns (D_m(z), relative residual norm) per z."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = alpha.size
    T = np.diag(alpha) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
    e0 = np.zeros(m)
    e0[0] = 1.0
    G, R = [], []
    for zz in np.atleast_1d(np.asarray(z, dtype=np.complex128)):
        y = np.linalg.solve(zz * np.eye(m) - T, e0.astype(np.complex128))
        G.append(norm2 * y[0])
        R.append(beta[m] * abs(y[m - 1]))
    return np.array(G), np.array(R)


def continued_fraction(alpha, beta, norm2: float, z) -> np.ndarray:
    """norm2 / (z - alpha_0 - beta_1^2 / (z - alpha_1 - ... - beta_{m-1}^2 / (z - alpha_{m-1})))."""
    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    m = alpha.size
    out = []
    for zz in np.atleast_1d(np.asarray(z, dtype=np.complex128)):
        f = zz - alpha[m - 1]
        for k in range(m - 2, -1, -1):
            f = zz - alpha[k] - beta[k + 1] ** 2 / f
        out.append(norm2 / f)
    return np.array(out)


def _apply_complex(model, v: np.ndarray) -> np.ndarray:
    """H v for a complex vector (H is real: it acts on both parts alike)."""
    return model.apply(np.ascontiguousarray(v.real)) + 1j * model.apply(np.ascontiguousarray(v.imag))


def shifted_cocg(model, b, z, maxiter: int, tol: float, seed: int = 0):
    """Shifted COCG for (z_j I - H) x^j = b, all j at once.

    Seed system A = z_s I - H (z_s = z[seed]); COCG is CG with the bilinear
    form (u, v) = u^T v (no conjugation), valid for complex-symmetric A:
        rho_k = r_k^T r_k,  beta_{k-1} = rho_k / rho_{k-1},
        p_k = r_k + beta_{k-1} p_{k-1},  alpha_k = rho_k / (p_k^T A p_k),
        x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k A p_k.
    A shift j solves (A + s_j I) x^j = b with s_j = z_j - z_s.  Its residual
    is r_k / pi^j_k with pi^j_0 = pi^j_{-1} = 1 and
        pi^j_{k+1} = (1 + alpha_k s_j) pi^j_k + (alpha_k beta_{k-1} / alpha_{k-1}) (pi^j_k - pi^j_{k-1}),
    and its own coefficients are
        beta^j_{k-1} = (pi^j_{k-1} / pi^j_k)^2 beta_{k-1},  alpha^j_k = (pi^j_k / pi^j_{k+1}) alpha_k,
        p^j_k = r_k / pi^j_k + beta^j_{k-1} p^j_{k-1},  x^j_{k+1} = x^j_k + alpha^j_k p^j_k.
    The loop stops once every |r_k / pi^j_k| <= tol |b| or after maxiter
    iterations.  Returns (D[j] = conj(b)^T x^j, explicit relative residual
    |b - (z_j - H) x^j| / |b|, iterations).
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    nz = z.size
    zs = z[seed]
    s = z - zs
    bn = np.linalg.norm(b)
    x = np.zeros((nz, b.size), dtype=np.complex128)
    p = np.zeros((nz, b.size), dtype=np.complex128)
    r = b.copy()
    p_seed = np.zeros_like(b)
    pi_cur = np.ones(nz, dtype=np.complex128)
    pi_old = np.ones(nz, dtype=np.complex128)
    rho_old, alpha_old = 1.0 + 0j, 1.0 + 0j
    it = 0
    for k in range(maxiter):
        if not np.any(r):
            break
        if np.all(np.linalg.norm(r) / np.abs(pi_cur) <= tol * bn):
            break
        rho = r @ r
        beta_k = rho / rho_old if k > 0 else 0.0 + 0j
        p_seed = r + beta_k * p_seed
        Ap = zs * p_seed - _apply_complex(model, p_seed)
        alpha_k = rho / (p_seed @ Ap)
        pi_new = (1.0 + alpha_k * s) * pi_cur + (alpha_k * beta_k / alpha_old) * (pi_cur - pi_old)
        for j in range(nz):
            beta_j = (pi_old[j] / pi_cur[j]) ** 2 * beta_k
            alpha_j = (pi_cur[j] / pi_new[j]) * alpha_k
            p[j] = r / pi_cur[j] + beta_j * p[j]
            x[j] = x[j] + alpha_j * p[j]
        r = r - alpha_k * Ap
        pi_old, pi_cur = pi_cur, pi_new
        rho_old, alpha_old = rho, alpha_k
        it = k + 1
    G = np.conj(b) @ x.T
    res = np.array([np.linalg.norm(b - (z[j] * x[j] - _apply_complex(model, x[j]))) / bn for j in range(nz)])
    return G, res, it
