"""Right-preconditioned Krylov solvers (FP64 oracle).

The paper's outer solvers are GMRES with restart (Section 2.1, Listings
"composition" and "params": restart M, relative tolerance tol) and
IDR(s) (s = 5 for every AMGCL variant, Section 4 Listings V1/V2 and the
solver table of Section 5) / BiCGStab(L) in Section 4 and 5; BiCGStab is the L = 1 member of
the BCGSL family PETSc uses there.  Both are written in their textbook
form (van der Vorst 1992 for BiCGStab; Saad & Schultz 1986 with Givens
rotations for GMRES), right-preconditioned so that the recurrence
residual is the residual of the original system.

Convergence reading: ||r||_2 / ||b||_2 <= tol, where a claim from the
recurrence (BiCGStab) or from the Arnoldi estimate (GMRES) is confirmed
by the true residual b - K x before it is accepted (Section 2.3 writes
the residual primitive r = f - A x and its 2-norm).  BiCGStab also
replaces its recurrence residual by the true one every
``replace_every`` iterations; when a convergence claim fails it
restarts from the true residual.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SolveInfo:
    iters: int = 0
    rel_res: float = np.inf
    converged: bool = False
    replacements: int = 0
    breakdown: bool = False
    history: list = field(default_factory=list)


def bicgstab(K, M, b, x0=None, tol=1e-8, maxiter=1000, replace_every=50):
    """Right-preconditioned BiCGStab.  K, M: callables v -> K v, v -> M^-1 v."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = SolveInfo()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        x[:] = 0.0
        info.rel_res = 0.0
        info.converged = True
        return x, info
    r = b - K(x)
    info.rel_res = np.linalg.norm(r) / nb
    if info.rel_res <= tol:
        info.converged = True
        return x, info
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    p = np.zeros(n)
    v = np.zeros(n)
    while info.iters < maxiter:
        info.iters += 1
        rho = rhat @ r
        if rho == 0.0:
            info.breakdown = True
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = M(p)
        v = K(phat)
        rv = rhat @ v
        if rv == 0.0:
            info.breakdown = True
            break
        alpha = rho / rv
        s = r - alpha * v
        shat = M(s)
        t = K(shat)
        tt = t @ t
        omega = (t @ s) / tt if tt > 0.0 else 0.0
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        res = np.linalg.norm(r) / nb
        info.history.append(res)
        claim = res <= tol
        if claim or info.iters % replace_every == 0:
            r = b - K(x)
            info.replacements += 1
            res = np.linalg.norm(r) / nb
            if res <= tol:
                info.rel_res = res
                info.converged = True
                return x, info
            if claim:
                rhat = r.copy()
                rho_old = alpha = omega = 1.0
                p = np.zeros(n)
                v = np.zeros(n)
            if omega == 0.0:
                info.breakdown = True
                break
        elif omega == 0.0:
            info.breakdown = True
            break
    info.rel_res = np.linalg.norm(b - K(x)) / nb
    info.converged = info.rel_res <= tol
    return x, info


def givens(a: float, b: float):
    """Rotation (c, s) with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def gmres(K, M, b, x0=None, m=30, tol=1e-8, maxiter=1000):
    """Right-preconditioned restarted GMRES(m), modified Gram-Schmidt."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = SolveInfo()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        x[:] = 0.0
        info.rel_res = 0.0
        info.converged = True
        return x, info
    while True:
        r = b - K(x)
        beta = np.linalg.norm(r)
        info.rel_res = beta / nb
        if info.rel_res <= tol:
            info.converged = True
            return x, info
        if info.iters >= maxiter:
            return x, info
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j = 0
        while j < m and info.iters < maxiter:
            w = K(M(V[j]))
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            info.iters += 1
            j += 1
            info.history.append(abs(g[j]) / nb)
            if abs(g[j]) / nb <= tol:
                break
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j] @ y[i + 1:j]) / H[i, i]
        x = x + M(V[:j].T @ y)


# ---------------------------------------------------------------- IDR(s)
_GOLDEN = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(counter: np.ndarray, seed: int = 0) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
    the output for counter c is the mix of seed + (c + 1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * np.uint64(_GOLDEN))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def idr_shadow_space(n: int, s: int, seed: int = 0) -> np.ndarray:
    """s orthonormal shadow vectors (rows): entry (j, i) = u - 1/2 with u the
    top 53 bits of splitmix64(j*n + i) over 2^53, then modified Gram-Schmidt."""
    c = np.arange(s * n, dtype=np.uint64)
    u = (splitmix64(c, seed) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    P = (u - 0.5).reshape(s, n)
    for j in range(s):
        for i in range(j):
            P[j] = P[j] - (P[i] @ P[j]) * P[i]
        P[j] = P[j] / np.linalg.norm(P[j])
    return P


def idrs(K, M, b, x0=None, s=5, tol=1e-8, maxiter=1000, P=None, kappa=0.7):
    """Right-preconditioned IDR(s), the bi-orthogonal variant (van Gijzen &
    Sonneveld 2011): s inner steps that keep the new residual orthogonal to
    the shadow space P, then one minimal-residual dimension-reduction step
    with the "maintaining convergence" choice of omega (kappa = 0.7).
    Iterations count applications of K; a recurrence claim is confirmed by
    the true residual, which replaces r otherwise."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = SolveInfo()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        x[:] = 0.0
        info.rel_res = 0.0
        info.converged = True
        return x, info
    if P is None:
        P = idr_shadow_space(n, s)
    r = b - K(x)
    info.rel_res = np.linalg.norm(r) / nb
    if info.rel_res <= tol:
        info.converged = True
        return x, info
    G = np.zeros((s, n))
    U = np.zeros((s, n))
    Mm = np.eye(s)
    om = 1.0

    def check(r, x):
        res = np.linalg.norm(r) / nb
        info.history.append(res)
        if res > tol:
            return r, False
        rt = b - K(x)
        info.replacements += 1
        info.rel_res = np.linalg.norm(rt) / nb
        return rt, info.rel_res <= tol

    while info.iters < maxiter:
        f = P @ r
        for k in range(s):
            c = np.zeros(s - k)
            for i in range(s - k):           # lower-triangular Mm[k:, k:] c = f[k:]
                c[i] = (f[k + i] - Mm[k + i, k:k + i] @ c[:i]) / Mm[k + i, k + i]
            v = r - c @ G[k:]
            v = M(v)
            U[k] = c @ U[k:] + om * v
            G[k] = K(U[k])
            info.iters += 1
            d = P @ G[k]
            alpha = np.zeros(k)
            for i in range(k):               # make G[k] orthogonal to P[:k]
                alpha[i] = (d[i] - Mm[i, :i] @ alpha[:i]) / Mm[i, i]
            G[k] = G[k] - alpha @ G[:k]
            U[k] = U[k] - alpha @ U[:k]
            Mm[k:, k] = d[k:] - Mm[k:, :k] @ alpha
            if Mm[k, k] == 0.0:
                info.breakdown = True
                info.rel_res = np.linalg.norm(b - K(x)) / nb
                return x, info
            beta = f[k] / Mm[k, k]
            r = r - beta * G[k]
            x = x + beta * U[k]
            r, done = check(r, x)
            if done:
                info.converged = True
                return x, info
            if info.iters >= maxiter:
                break
            f[k + 1:] = f[k + 1:] - beta * Mm[k + 1:, k]
        if info.iters >= maxiter:
            break
        v = M(r)
        t = K(v)
        info.iters += 1
        tt = t @ t
        ts = t @ r
        om = ts / tt if tt > 0.0 else 0.0
        rho = abs(ts) / (np.sqrt(tt) * np.linalg.norm(r)) if tt > 0.0 else 0.0
        if 0.0 < rho < kappa:
            om = om * kappa / rho
        if om == 0.0:
            info.breakdown = True
            break
        r = r - om * t
        x = x + om * v
        r, done = check(r, x)
        if done:
            info.converged = True
            return x, info
    info.rel_res = np.linalg.norm(b - K(x)) / nb
    info.converged = info.rel_res <= tol
    return x, info
