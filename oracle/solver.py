"""Restarted GMRES and a dense direct solve (oracle; test infrastructure only).

The paper solves A x = b with GMRES, 50 inner (restart) iterations, at most 200
outer iterations, tolerance 1e-5 (Section V), with the left preconditioner
P = M_eps G (Section IV-B): GMRES runs on P^-1 A x = P^-1 b and the tolerance
applies to the preconditioned relative residual ||P^-1 (b - A x)|| / ||P^-1 b||.

This is textbook GMRES(m) (Saad & Schultz 1986): Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix, and the least-squares
update at the end of each cycle.  Written in FP64 with NumPy.
"""

from __future__ import annotations

import numpy as np


def gmres(apply, b, tol=1e-5, restart=50, maxit=200, x0=None):
    """Solve apply(x) = b.  Vectors are complex arrays of any shape.

    Returns (x, info) with info = dict(iters, restarts, resid (final relative
    residual estimate), history (list of relative residual estimates), converged).
    """
    shape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=complex).ravel()
    history = []
    if nb == 0.0:
        return x.reshape(shape), dict(iters=0, restarts=0, resid=0.0, history=[0.0], converged=True)
    iters = 0
    for cycle in range(maxit):
        r = bv - apply(x.reshape(shape)).ravel()
        beta = np.linalg.norm(r)
        history.append(beta / nb)
        if beta / nb <= tol:
            return x.reshape(shape), dict(iters=iters, restarts=cycle, resid=beta / nb, history=history, converged=True)
        m = restart
        V = np.zeros((m + 1, bv.size), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m, dtype=complex)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            w = apply(V[j].reshape(shape)).ravel()
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            # apply the previous rotations to the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation annihilating H[j+1, j]
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            elif a == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(c) / den
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_end = j + 1
            history.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) / nb <= tol:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + V[:j_end].T @ y
        if abs(g[j_end]) / nb <= tol:
            r = bv - apply(x.reshape(shape)).ravel()
            res = np.linalg.norm(r) / nb
            return x.reshape(shape), dict(iters=iters, restarts=cycle + 1, resid=res, history=history, converged=True)
    r = bv - apply(x.reshape(shape)).ravel()
    res = np.linalg.norm(r) / nb
    return x.reshape(shape), dict(iters=iters, restarts=maxit, resid=res, history=history, converged=res <= tol)


def direct_solve(A, b):
    """Dense LU solve of A x = b (tiny grids)."""
    return np.linalg.solve(A, b.ravel()).reshape(b.shape)
