"""FP64 reference solvers for Eq. 5 (test infrastructure only).

MB-L2 (Eq. 5 with the Tikhonov term of Eq. 6) is solved with LSQR and MB-L1
(Eq. 5 with the L1 term of Eq. 7) with FISTA, as the paper states at the end
of "Efficient reconstruction based on scanning symmetries".  Both are written
from their published definitions (Paige & Saunders 1982, Beck & Teboulle
2009) and take the operator as two callables, so the same code runs on the
slab operator and on plain dense matrices in the tests.

Readings where the paper is silent:
* LSQR starts from x0 = 0 and runs a fixed number of iterations; Tikhonov
  weight lambda enters as damp = sqrt(lambda); an exact zero alpha or beta
  stops early.
* FISTA minimises Eq. 5 exactly as printed (no factor 1/2):
  f(H) = ||s - A H||^2 + lam ||H||_1, so grad = 2 A^T (A H - s) and the
  Lipschitz constant is L = 2 mu_max(A^T A), estimated by power iteration
  and inflated by 1 %.  Optional non-negativity turns the soft threshold
  into max(z - lam/L, 0).
"""
import math

import numpy as np


def _norm(v):
    return float(np.sqrt(np.dot(v.ravel(), v.ravel())))


def lsqr(A, AT, s, iters, damp=0.0, callback=None):
    """LSQR from x0 = 0 for min ||A x - s||^2 + damp^2 ||x||^2.

    Returns (x, info) with info = dict(iters_done, stop_reason, rnorm, arnorm,
    anorm).  stop_reason: 0 = ran ``iters`` steps, 1 = beta or alpha became 0.
    """
    s = np.asarray(s, np.float64)
    beta = _norm(s)
    x = None
    if beta == 0.0:
        v = AT(np.zeros_like(s))
        return np.zeros_like(v), dict(iters_done=0, stop_reason=1, rnorm=0.0, arnorm=0.0, anorm=0.0)
    u = s / beta
    v = AT(u)
    alpha = _norm(v)
    x = np.zeros_like(v)
    if alpha == 0.0:
        return x, dict(iters_done=0, stop_reason=1, rnorm=beta, arnorm=0.0, anorm=0.0)
    v = v / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    anorm2 = alpha * alpha
    done, reason = 0, 0
    for i in range(iters):
        # bidiagonalisation: beta u = A v - alpha u ; alpha v = A^T u - beta v
        u = A(v) - alpha * u
        beta = _norm(u)
        if beta > 0:
            u = u / beta
        anorm2 += beta * beta + damp * damp
        v = AT(u) - beta * v
        alpha = _norm(v)
        if alpha > 0:
            v = v / alpha
        anorm2 += alpha * alpha
        # plane rotation that eliminates the damping term
        if damp > 0:
            rhobar1 = math.sqrt(rhobar * rhobar + damp * damp)
            cs1, sn1 = rhobar / rhobar1, damp / rhobar1
            phibar = cs1 * phibar
        else:
            rhobar1 = rhobar
        # rotation that eliminates the sub-diagonal beta
        rho = math.sqrt(rhobar1 * rhobar1 + beta * beta)
        cs, sn = rhobar1 / rho, beta / rho
        theta = sn * alpha
        rhobar = -cs * alpha
        phi = cs * phibar
        phibar = sn * phibar
        # update x and w
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        done = i + 1
        if callback is not None:
            callback(done, x, abs(phibar))
        if beta == 0.0 or alpha == 0.0:
            reason = 1
            break
    arnorm = abs(phibar * alpha * cs) if done else 0.0
    return x, dict(iters_done=done, stop_reason=reason, rnorm=abs(phibar), arnorm=arnorm,
                   anorm=math.sqrt(anorm2))


def power_iteration(A, AT, v0, iters):
    """Largest eigenvalue of A^T A: v <- A^T A v / ||.||; mu = ||A^T A v|| / ||v||."""
    v = np.asarray(v0, np.float64)
    mu = 0.0
    for _ in range(iters):
        nv = _norm(v)
        if nv == 0.0:
            return 0.0
        w = AT(A(v))
        mu = _norm(w) / nv
        v = w / _norm(w) if _norm(w) > 0 else w
    return mu


def prox_l1(z, t, nonneg):
    """Proximal step of t ||.||_1 (optionally restricted to x >= 0)."""
    if nonneg:
        return np.maximum(z - t, 0.0)
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def lambda_from_relative(AT, s, lambda_rel):
    """lambda = lambda_rel * max |A^T s| (the relative penalty of the C1 workload)."""
    return lambda_rel * float(np.max(np.abs(AT(s))))


def fista(A, AT, s, iters, lam, L, nonneg=True, callback=None):
    """FISTA with constant step 1/L for f = ||s - A x||^2 + lam ||x||_1.

    x0 = Y1 = 0, t1 = 1; x_k = prox(Y_k - grad(Y_k)/L, lam/L);
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
    Y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}).
    """
    s = np.asarray(s, np.float64)
    Y = np.zeros_like(AT(np.zeros_like(s)))
    x_prev = Y.copy()
    t = 1.0
    x = Y
    for k in range(iters):
        g = 2.0 * AT(A(Y) - s)
        x = prox_l1(Y - g / L, lam / L, nonneg)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        Y = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev = x
        t = t_next
        if callback is not None:
            callback(k + 1, x)
    return x


def fista_objective(A, s, x, lam):
    r = A(x) - s
    return float(np.dot(r.ravel(), r.ravel()) + lam * np.abs(x).sum())


def mb_l1(A, AT, s, iters, power_iters, v0, lam=None, lambda_rel=1e-3, nonneg=True):
    """The MB-L1 pipeline: power iteration for L, relative lambda, FISTA."""
    mu = power_iteration(A, AT, v0, power_iters)
    L = 2.0 * mu * 1.01
    if lam is None or lam < 0:
        lam = lambda_from_relative(AT, s, lambda_rel)
    x = fista(A, AT, s, iters, lam, L, nonneg)
    return x, dict(L=L, lam=lam, objective=fista_objective(A, s, x, lam))
