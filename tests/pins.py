"""Independent reference facts used to pin the FP64 oracle.

Nothing here imports the oracle.  Each helper is a separate route to a fact
the paper and the mathematics fix:

* ``two_point_fixed_point`` -- closed form (up to one monotone scalar root)
  of the PD fixed point for two cases joined by one edge.  Derivation: the
  fixed point minimises
      F = 1/2||x1-u1||^2 + 1/2||x2-u2||^2 + mu w ||v|| + rho sqrt(dist^2 + eps)
  (display after Eq. 3).  With m = (u1+u2)/2, delta = u1-u2 the loss is
  ||xbar-m||^2 + 1/4||Delta-delta||^2, and projecting (u1,u2,v) onto
  {v = u1-u2} gives dist^2 = ||v-delta||^2 / 3.  So m = xbar and, along
  e = Delta/||Delta||, the scalars (delta, v) minimise
      1/4 (D-delta)^2 + mu w |v| + rho sqrt((v-delta)^2/3 + eps).
  With h(e) = rho e / (3 sqrt(e^2/3 + eps)):
    unfused (v > 0):  h(v-delta) = -mu w  ->  v-delta = -c,
                      c = 3 mu w sqrt(eps) / sqrt(rho^2 - 3 mu^2 w^2),
                      delta = D - 2 mu w, valid when D - 2 mu w - c > 0;
    fused (v = 0):    1/2 (D - delta) = h(delta), a monotone root in (0, D).
  As eps -> 0 this tends to delta = D max(0, 1 - 2 mu w / D), the two-point
  solution of Eq. 1.
* ``gauss_seidel_projection`` -- the paper's own block-descent projection
  (Methods, block updates), run until the cases stop moving.
* ``projection_matrix`` -- the orthogonal projector onto
  C = {(U, V): v_ij = u_i - u_j}, formed densely from a matrix inverse.
* ``kkt_residual`` -- optimality of (U, V) for the smoothed objective F
  using that projector (subgradient of mu w ||v|| on fused edges).
* ``convex_clustering_minimizer`` -- the exact minimiser of Eq. 1 by
  accelerated projected gradient on its dual (Beck-Teboulle FISTA), with a
  duality-gap certificate.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def two_point_fixed_point(D: float, mu: float, w: float, rho: float, eps: float):
    """Return (delta, v, fused) of the two-point PD fixed point along Delta."""
    def h(e):
        return rho * e / (3.0 * np.sqrt(e * e / 3.0 + eps))

    a = mu * w
    if 3.0 * a * a < rho * rho:
        c = 3.0 * a * np.sqrt(eps) / np.sqrt(rho * rho - 3.0 * a * a)
        if D - 2.0 * a - c > 0.0:
            return D - 2.0 * a, D - 2.0 * a - c, False
    # fused: v = 0 and 1/2 (D - delta) = h(delta)
    if D == 0.0:
        return 0.0, 0.0, True
    delta = brentq(lambda t: 0.5 * (D - t) - h(t), 0.0, D, xtol=1e-15, rtol=1e-15, maxiter=500)
    assert abs(h(delta)) <= a * (1 + 1e-9)
    return delta, 0.0, True


def incidence(n, ei, ej):
    m = len(ei)
    D = np.zeros((m, n))
    for e, (i, j) in enumerate(zip(ei, ej)):
        D[e, i] = 1.0
        D[e, j] = -1.0
    return D


def gauss_seidel_projection(U, V, ei, ej, sweeps=100000, tol=1e-15):
    """The paper's block descent for the projection, cycling u_1..u_n in order.

    u_i = (u~_i + sum_{R_i} v~_ij - sum_{L_i} v~_ji + sum_{N_i} u_j) / (1 + |N_i|)
    """
    n, p = U.shape
    R = {i: [] for i in range(n)}   # j > i with edge index
    Lft = {i: [] for i in range(n)}  # j < i with edge index
    for e, (i, j) in enumerate(zip(ei, ej)):
        R[i].append((j, e))
        Lft[j].append((i, e))
    A = U.copy()
    for _ in range(sweeps):
        change = 0.0
        for i in range(n):
            num = U[i].copy()
            for j, e in R[i]:
                num += V[e] + A[j]
            for j, e in Lft[i]:
                num += -V[e] + A[j]
            new = num / (1 + len(R[i]) + len(Lft[i]))
            change = max(change, float(np.max(np.abs(new - A[i]))))
            A[i] = new
        if change <= tol * max(1.0, float(np.max(np.abs(A)))):
            break
    B = np.array([A[i] - A[j] for i, j in zip(ei, ej)]).reshape(len(ei), p)
    return A, B


def projection_matrix(n, ei, ej):
    """Dense orthogonal projector onto range([I; D]) in R^{n+m} (acts on each column)."""
    D = incidence(n, ei, ej)
    M = np.vstack([np.eye(n), D])
    return M @ np.linalg.inv(M.T @ M) @ M.T


def kkt_residual(U, V, X, mask, ei, ej, w, mu, rho, eps, fused):
    """Max violation of the optimality conditions of F at (U, V).

    grad of the smooth part: (U - X on observed, 0 elsewhere) + rho (I-P)z / sqrt(||(I-P)z||^2 + eps)
    plus mu w v/||v|| on live edges, or ||.|| <= mu w on fused edges (v = 0).
    """
    n, p = U.shape
    P = projection_matrix(n, ei, ej)
    Z = np.vstack([U, V])
    Rz = Z - P @ Z
    dF = np.sqrt(np.sum(Rz * Rz) + eps)
    G = rho * Rz / dF
    GU = G[:n] + (U - X) * (1.0 if mask is None else mask.astype(float))
    GV = G[n:]
    viol = [float(np.max(np.abs(GU)))]
    for e in range(len(ei)):
        if fused[e]:
            viol.append(max(0.0, float(np.linalg.norm(GV[e])) - mu * w[e]))
            viol.append(float(np.linalg.norm(V[e])))
        else:
            nv = np.linalg.norm(V[e])
            viol.append(float(np.max(np.abs(GV[e] + mu * w[e] * V[e] / nv))))
    return max(viol)


def convex_clustering_minimizer(X, ei, ej, w, mu, iters=400000, gap_tol=1e-13):
    """Exact minimiser of Eq. 1 via FISTA on the dual.

    Dual: max_{||lam_e|| <= mu w_e} <Lam, D X> - 1/2 ||D^T Lam||^2, U = X - D^T Lam.
    Returns (U, duality_gap).
    """
    n, p = X.shape
    D = incidence(n, ei, ej)
    Lmax = float(np.linalg.eigvalsh(D.T @ D).max()) if len(ei) else 1.0
    rad = mu * np.asarray(w, dtype=float)

    def proj(L):
        nrm = np.linalg.norm(L, axis=1)
        scale = np.where(nrm > rad, rad / np.where(nrm > 0, nrm, 1.0), 1.0)
        return L * scale[:, None]

    def primal(U):
        return 0.5 * np.sum((X - U) ** 2) + np.sum(rad * np.linalg.norm(D @ U, axis=1))

    def dual(L):
        DtL = D.T @ L
        return np.sum(L * (D @ X)) - 0.5 * np.sum(DtL * DtL)

    Lam = np.zeros((len(ei), p))
    Y = Lam.copy()
    t = 1.0
    gap = np.inf
    for k in range(iters):
        U = X - D.T @ Y
        Lnew = proj(Y + (D @ U) / Lmax)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        Y = Lnew + ((t - 1) / tn) * (Lnew - Lam)
        Lam, t = Lnew, tn
        if k % 200 == 0:
            U = X - D.T @ Lam
            gap = primal(U) - dual(Lam)
            if gap <= gap_tol * max(1.0, primal(U)):
                break
    U = X - D.T @ Lam
    return U, primal(U) - dual(Lam)
