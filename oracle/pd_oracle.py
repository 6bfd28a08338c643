"""FP64 CPU oracle: the proximal distance (PD) algorithm for convex clustering.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this module.  It
shares no code, header, table or helper with the CUDA library; the only
thing both sides share is the seeded input generator in ``synth``.

Source: G. K. Chen, E. C. Chi, J. M. O. Ranola, K. Lange, "Convex
Clustering: An Attractive Alternative to Hierarchical Clustering"
(arXiv:1409.2065).  Equations are cited by the paper's own labels, numbered
in order of appearance:

  Eq. 1  (eq_lindsten)            f_mu(U) = 1/2 sum ||x_i-u_i||^2 + mu sum_{i<j} w_ij ||u_i-u_j||
  Eq. 2  (eq_proxdist)            g_mu(U,V), splitting v_ij = u_i - u_j
  Eq. 3  (first_surrogate)        projection majorisation of dist(., C)
  Eq. 4  (sqrt_root_majorization) tangent majorisation of sqrt(t + eps)
  Eq. 5  (second_surrogate)       the separable surrogate and d_m
  Eq. 6  (eq_missing_analog)      loss over the observed set Gamma only
  Eq. 7  (eq_proxdist, 2nd copy)  g_mu with Y in place of X
  Eq. 8  (eq_weighting)           w_ij = 1{i ~_k j} exp(-phi d_ij^2)

Notation is the paper's: rows x_i of X are cases, U holds the centroids u_i,
V holds one splitting vector v_ij per edge {i,j} (i<j) with w_ij > 0, mu is
the penalty (the library calls it gamma), rho the distance penalty, eps the
smoothing constant, m the MM iteration, (A, B) = P_C(U_m, V_m) the
projection and d_m the smoothed distance.

Readings where the paper is silent (each listed in the design notes):
  * rho = rho_scale (||Y_c||_F + mu ||w||_2), eps = (eps_rel ||Y_c||_F)^2 with
    Y_c the column-centred Y_0; defaults rho_scale = 2, eps_rel = 1e-3.
  * start: U_0 = Y_0 (missing entries set to the observed column mean),
    V_0 = 0; along the mu path each solve starts from the previous one.
  * the projection is solved exactly (Cholesky of I + L); the paper's
    block descent converges to the same point.
  * an edge is fused when its prox returns exactly zero, i.e. when
    mu w_ij d_m >= rho ||b_ij||; clusters are the connected components of
    the fused edges, labelled by the rank of their smallest member.
  * the MM map is iterated to its fixed point.  To get there in a
    practical number of steps the map is applied at a Nesterov-extrapolated
    point with gradient-test restarts (``accelerate=True``); this changes
    the path to the fixed point, not the fixed point, and the literal
    iteration is available with ``accelerate=False``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

__all__ = [
    "standardize",
    "principal_axes",
    "project_path",
    "geo_distance",
    "knn_composite_weights",
    "min_connected_k",
    "EdgeGraph",
    "fill_missing",
    "pd_constants",
    "project",
    "mm_step",
    "objective",
    "GammaResult",
    "solve_gamma",
    "solve_path",
    "fused_labels",
    "knn_gaussian_weights",
    "fusion_scale",
]


# ----------------------------------------------------------------------------
# Edge set (Methods, "The Proximal Distance Algorithm": E, N_i = L_i u R_i)
# ----------------------------------------------------------------------------
class EdgeGraph:
    """Undirected weighted edge set {i, j}, i < j, w_ij > 0.

    Zero weights are dropped: the paper introduces no difference vector for
    them, since they would add work without changing the objective.  Holds the incidence matrix D (one row
    per edge, +1 at i, -1 at j), so that (D U)_e = u_i - u_j and
    (D^T V)_i = sum_{j in R_i} v_ij - sum_{j in L_i} v_ji.
    """

    def __init__(self, n: int, ei, ej, w):
        ei = np.asarray(ei, dtype=np.int64).ravel()
        ej = np.asarray(ej, dtype=np.int64).ravel()
        w = np.asarray(w, dtype=np.float64).ravel()
        if not (ei.shape == ej.shape == w.shape):
            raise ValueError("edge arrays differ in length")
        if n < 1:
            raise ValueError("n must be >= 1")
        if ei.size and (ei.min() < 0 or ej.max() >= n or np.any(ei >= ej)):
            raise ValueError("edges must satisfy 0 <= i < j < n")
        if np.any(~np.isfinite(w)) or np.any(w < 0):
            raise ValueError("weights must be finite and >= 0")
        keep = w > 0
        ei, ej, w = ei[keep], ej[keep], w[keep]
        key = ei * n + ej
        if np.unique(key).size != key.size:
            raise ValueError("duplicate edge")
        self.n, self.ei, self.ej, self.w = int(n), ei, ej, w
        m = ei.size
        rows = np.concatenate([np.arange(m), np.arange(m)])
        cols = np.concatenate([ei, ej])
        vals = np.concatenate([np.ones(m), -np.ones(m)])
        self.D = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
        self.L = (self.D.T @ self.D).toarray()
        self.deg = np.diag(self.L).copy()
        # I + L is symmetric positive definite; factor once per graph.
        self._chol = sla.cho_factor(np.eye(n) + self.L, lower=True)

    @property
    def m(self) -> int:
        return int(self.ei.size)

    def solve_I_plus_L(self, R: np.ndarray) -> np.ndarray:
        return sla.cho_solve(self._chol, R)


# ----------------------------------------------------------------------------
# Data preparation and constants
# ----------------------------------------------------------------------------
def standardize(X: np.ndarray, mask) -> np.ndarray:
    """Standardised predictors (Methods: the predictors are standardised before
    clustering), using observed entries only: each column is centred on the
    mean of its observed entries and divided by their standard deviation
    (divisor = the number of observed entries); a column whose observed
    entries are all equal is centred only, and a column with no observed
    entry is left at 0.  Missing entries are returned as 0 (their value is
    never data).  FP64 throughout."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    obs = np.ones((n, p), bool) if mask is None else np.asarray(mask).astype(bool)
    out = np.zeros((n, p))
    for c in range(p):
        vals = X[obs[:, c], c]
        if vals.size == 0:
            continue
        mean = vals.sum() / vals.size
        dev = vals - mean
        sd = np.sqrt((dev * dev).sum() / vals.size)
        out[obs[:, c], c] = dev / sd if sd > 0 else dev
    return out


def fill_missing(X: np.ndarray, mask) -> np.ndarray:
    """Y_0: X with each missing entry replaced by its column's observed mean (0 if none)."""
    X = np.asarray(X, dtype=np.float64)
    if mask is None:
        return X.copy()
    obs = np.asarray(mask).astype(bool)
    cnt = obs.sum(axis=0)
    mean = np.where(obs, X, 0.0).sum(axis=0) / np.maximum(cnt, 1)
    return np.where(obs, X, mean[None, :])


def pd_constants(Y0: np.ndarray, w: np.ndarray, mu: float,
                 rho_scale: float = 2.0, eps_rel: float = 1e-3):
    """(rho, eps) for penalty mu.

    The paper asks for rho larger than a Lipschitz constant of the loss
    (Methods, exact-penalty paragraph) and for a small eps (Eq. 4 context).
    The gradient of 1/2||Y-U||^2 over the region between Y and its centroid
    is bounded by ||Y_c||_F and that of mu sum w ||v|| by mu ||w||_2; rho is
    rho_scale times their sum.  eps is (eps_rel ||Y_c||_F)^2.  Degenerate
    data (all rows equal) falls back to rho = rho_scale, eps = eps_rel^2.
    """
    Yc = Y0 - Y0.mean(axis=0, keepdims=True)
    nyc = float(np.sqrt(np.sum(Yc * Yc)))
    nw = float(np.sqrt(np.sum(np.asarray(w, dtype=np.float64) ** 2)))
    rho = rho_scale * (nyc + mu * nw)
    if rho <= 0.0:
        rho = rho_scale
    eps = (eps_rel * nyc) ** 2
    if eps <= 0.0:
        eps = eps_rel ** 2
    return rho, eps


# ----------------------------------------------------------------------------
# One MM step of the PD algorithm
# ----------------------------------------------------------------------------
def project(U: np.ndarray, V: np.ndarray, G: EdgeGraph):
    """P_C(U, V) = (A, B), B = D A.

    The projection minimises 1/2 sum ||a_i - u_i||^2 + 1/2 sum_E ||a_i - a_j - v_ij||^2
    (Methods, block-descent paragraph); its stationarity equations are
    (I + D^T D) A = U + D^T V, solved here exactly.
    """
    A = G.solve_I_plus_L(U + G.D.T @ V)
    return A, G.D @ A


def mm_step(U, V, X, mask, G: EdgeGraph, mu: float, rho: float, eps: float):
    """Minimise the surrogate of Eq. 5 once, with Y of the missing-data rule.

    Returns (U_next, V_next, d_m, fused) where fused[e] is True when the
    block soft-threshold returned exactly zero for edge e.
    """
    A, B = project(U, V, G)
    dist2 = float(np.sum((U - A) ** 2) + np.sum((V - B) ** 2))
    d = np.sqrt(dist2 + eps)                       # d_m below Eq. 5
    if mask is None:
        Y = X
    else:                                          # Missing Data: y = x on Gamma, u_m elsewhere
        Y = np.where(np.asarray(mask).astype(bool), X, U)
    U_next = (d / (d + rho)) * Y + (rho / (d + rho)) * A       # u-update display
    nb = np.sqrt(np.sum(B * B, axis=1))
    thresh = mu * G.w * d                           # compare mu w d against rho ||b||
    fused = thresh >= rho * nb                      # includes the b = 0 case (v = 0)
    s = np.zeros_like(nb)
    live = ~fused
    s[live] = 1.0 - thresh[live] / (rho * nb[live])  # v-update display (block soft-threshold)
    V_next = s[:, None] * B
    return U_next, V_next, d, fused


def objective(U, V, X, mask, G: EdgeGraph, mu: float, rho: float, eps: float) -> float:
    """The approximate objective the MM steps drive downhill.

    1/2 sum_Gamma (x - u)^2 + mu sum_E w ||v|| + rho sqrt(dist((U,V), C)^2 + eps)
    (display after Eq. 3, with the loss of Eq. 6).
    """
    A, B = project(U, V, G)
    dist2 = float(np.sum((U - A) ** 2) + np.sum((V - B) ** 2))
    R = X - U
    if mask is not None:
        R = np.where(np.asarray(mask).astype(bool), R, 0.0)
    pen = float(np.sum(G.w * np.sqrt(np.sum(V * V, axis=1))))
    return 0.5 * float(np.sum(R * R)) + mu * pen + rho * np.sqrt(dist2 + eps)


# ----------------------------------------------------------------------------
# Fixed point of the MM map for one mu, and the mu path
# ----------------------------------------------------------------------------
@dataclass
class GammaResult:
    mu: float
    rho: float
    eps: float
    U: np.ndarray
    V: np.ndarray
    d: float
    fused: np.ndarray
    labels: np.ndarray
    iters: int
    residual: float
    converged: bool
    extra: dict = field(default_factory=dict)


def solve_gamma(X, mask, G: EdgeGraph, mu: float, rho: float, eps: float,
                U0, V0, tol: float = 1e-12, max_iter: int = 1_000_000,
                accelerate: bool = True, check_every: int = 25):
    """Iterate the MM map of ``mm_step`` to its fixed point.

    Stops when one plain step moves the iterate by at most
    tol * max(||U||_F, 1) (Frobenius norm over (U, V)).  Returns
    (U, V, d, fused, iters, residual, converged); (U, V) is the last plain
    step, d and fused are those of that step.
    """
    X = np.asarray(X, dtype=np.float64)
    U, V = np.array(U0, dtype=np.float64), np.array(V0, dtype=np.float64)
    Up, Vp = U, V
    k = 0
    it = 0
    res = np.inf
    while it < max_iter:
        it += 1
        beta = (k - 1.0) / (k + 2.0) if (accelerate and k >= 1) else 0.0
        Uy = U + beta * (U - Up)
        Vy = V + beta * (V - Vp)
        Un, Vn, _, _ = mm_step(Uy, Vy, X, mask, G, mu, rho, eps)
        # gradient-test restart (O'Donoghue & Candes): drop momentum when the
        # step opposes the previous motion
        if np.sum((Uy - Un) * (Un - U)) + np.sum((Vy - Vn) * (Vn - V)) > 0.0:
            k = 0
        else:
            k += 1
        Up, Vp, U, V = U, V, Un, Vn
        if it % check_every == 0 or it == max_iter:
            U2, V2, d2, f2 = mm_step(U, V, X, mask, G, mu, rho, eps)
            res = float(np.sqrt(np.sum((U2 - U) ** 2) + np.sum((V2 - V) ** 2)))
            scale = max(float(np.sqrt(np.sum(U * U))), 1.0)
            if res <= tol * scale:
                return U2, V2, d2, f2, it, res, True
    U2, V2, d2, f2 = mm_step(U, V, X, mask, G, mu, rho, eps)
    return U2, V2, d2, f2, it, res, False


def solve_path(X, mask, G: EdgeGraph, mus, rho_scale: float = 2.0, eps_rel: float = 1e-3,
               tol: float = 1e-12, max_iter: int = 1_000_000, accelerate: bool = True):
    """Warm-started path over the given mu grid, in the order given (Evaluation of Clusters).

    Returns a list of GammaResult, one per mu.
    """
    X = np.asarray(X, dtype=np.float64)
    Y0 = fill_missing(X, mask)
    U, V = Y0.copy(), np.zeros((G.m, X.shape[1]))
    out = []
    for mu in np.asarray(mus, dtype=np.float64):
        rho, eps = pd_constants(Y0, G.w, float(mu), rho_scale, eps_rel)
        U, V, d, fused, iters, res, ok = solve_gamma(
            X, mask, G, float(mu), rho, eps, U, V, tol=tol, max_iter=max_iter,
            accelerate=accelerate)
        out.append(GammaResult(float(mu), rho, eps, U.copy(), V.copy(), float(d), fused.copy(),
                               fused_labels(G.n, G.ei, G.ej, fused), iters, res, ok))
    return out


# ----------------------------------------------------------------------------
# Clusters: connected components of the fused edges
# ----------------------------------------------------------------------------
def fused_labels(n: int, ei, ej, fused) -> np.ndarray:
    """Label of each case = rank of the smallest index in its fused component."""
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b, f in zip(np.asarray(ei), np.asarray(ej), np.asarray(fused)):
        if f:
            ra, rb = find(int(a)), find(int(b))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    root = np.array([find(i) for i in range(n)])
    # roots are component minima (smaller root always wins), so ranking
    # the distinct roots ranks the components by smallest member
    uniq = np.unique(root)
    rank = {int(r): c for c, r in enumerate(uniq)}
    return np.array([rank[int(r)] for r in root], dtype=np.int32)


# ----------------------------------------------------------------------------
# Weights (Calibration of Weights, Eq. 8)
# ----------------------------------------------------------------------------
def knn_gaussian_weights(X, mask, k: int, phi, normalize: bool):
    """k-nearest-neighbour union graph with Gaussian-kernel weights, brute force in FP64.

    * missing entries are filled with observed column means (weights only);
    * d_ij = ||x_i - x_j||; j is a neighbour of i when it is among the k
      nearest other cases, ties going to the smaller index; i ~_k j when
      either is a neighbour of the other;
    * w_ij = exp(-phi d_ij^2); phi = "auto" takes 1 / median d_ij^2 over the
      union edges;
    * normalize=True scales the weights to sum to 1 over i < j (computed as
      exp(-phi (d^2 - min d^2)) / sum, which is the same ratio);
    * edges whose weight is exactly 0 are dropped.
    Returns (ei, ej, w, d2) with i < j sorted by (i, j).
    """
    Y = fill_missing(X, mask)
    n = Y.shape[0]
    D2 = np.empty((n, n))
    for i in range(n):                      # one row at a time keeps memory at n x p
        diff = Y - Y[i]
        D2[i] = np.einsum("jk,jk->j", diff, diff)
    kk = min(k, n - 1)
    pairs = set()
    for i in range(n):
        order = sorted((D2[i, j], j) for j in range(n) if j != i)
        for _, j in order[:kk]:
            pairs.add((min(i, j), max(i, j)))
    pairs = sorted(pairs)
    ei = np.array([a for a, _ in pairs], dtype=np.int64)
    ej = np.array([b for _, b in pairs], dtype=np.int64)
    d2 = D2[ei, ej] if ei.size else np.zeros(0)
    if isinstance(phi, str):
        if phi != "auto":
            raise ValueError("phi must be a number or 'auto'")
        med = float(np.median(d2)) if d2.size else 0.0
        phi = 1.0 / med if med > 0 else 0.0
    phi = float(phi)
    if normalize and d2.size:
        w = np.exp(-phi * (d2 - d2.min()))
        w = w / w.sum()
    else:
        w = np.exp(-phi * d2)
    keep = w > 0
    return ei[keep], ej[keep], w[keep], d2[keep], phi


def fusion_scale(X, mask, ei, ej, w) -> float:
    """Median over edges of ||x_i - x_j|| / (2 w_ij): the mu at which an isolated
    pair would fuse (two-point solution of Eq. 1)."""
    Y = fill_missing(X, mask)
    dist = np.sqrt(np.sum((Y[np.asarray(ei)] - Y[np.asarray(ej)]) ** 2, axis=1))
    return float(np.median(dist / (2.0 * np.asarray(w, dtype=np.float64))))


def min_connected_k(X, mask, k_max: int) -> int:
    """Smallest k in [1, k_max] whose k-nearest-neighbour union graph is connected
    (Calibration of Weights: i ~_k j when either is among the other's k nearest,
    distances on the rows with missing entries at observed column means, ties
    to the smaller index; complete coalescence needs a connected graph, and the
    paper proposes searching k for connectivity).  0 when no k <= k_max works.

    A plain scan over k = 1, 2, ... with union-find components; the neighbour
    order of every row is computed once in FP64.
    """
    Y = fill_missing(X, mask)
    n = Y.shape[0]
    if n < 2:
        raise ValueError("need at least two cases")
    kmax = min(int(k_max), n - 1)
    order = []
    for i in range(n):
        diff = Y - Y[i]
        d2 = np.einsum("jk,jk->j", diff, diff)
        order.append([j for _, j in sorted((d2[j], j) for j in range(n) if j != i)])
    for k in range(1, kmax + 1):
        ei = [i for i in range(n) for j in order[i][:k]]
        ej = [j for i in range(n) for j in order[i][:k]]
        if int(fused_labels(n, ei, ej, np.ones(len(ei), bool)).max()) == 0:
            return k
    return 0


def geo_distance(c1, c2, geodesic: bool) -> float:
    """Geographic distance in degrees between (latitude, longitude) pairs given in degrees.

    geodesic=False: Euclidean norm of the coordinate difference with the
    longitude difference taken modulo 360 (Calibration of Weights: the
    components of y_i - y_j are computed in modulo arithmetic);
    geodesic=True: great-circle central angle (the alternative the paper
    suggests), from the spherical case of Vincenty's formula (an atan2 of the
    cross and dot products of the two unit vectors, accurate from coincident
    points to antipodes), in degrees of arc.
    """
    lat1, lon1 = float(c1[0]), float(c1[1])
    lat2, lon2 = float(c2[0]), float(c2[1])
    if not geodesic:
        dl = math.fmod(abs(lon1 - lon2), 360.0)
        if dl > 180.0:
            dl = 360.0 - dl
        dp = lat1 - lat2
        return math.sqrt(dp * dp + dl * dl)
    r = math.pi / 180.0
    p1, p2, dl = lat1 * r, lat2 * r, (lon2 - lon1) * r
    y = math.hypot(math.cos(p2) * math.sin(dl), math.cos(p1) * math.sin(p2) - math.sin(p1) * math.cos(p2) * math.cos(dl))
    x = math.sin(p1) * math.sin(p2) + math.cos(p1) * math.cos(p2) * math.cos(dl)
    return math.atan2(y, x) / r


def knn_composite_weights(X, mask, coords, alpha: float, k: int, phi, normalize: bool, geodesic: bool = False):
    """kNN union graph and Gaussian-kernel weights on the composite distance
    d_ij = alpha ||x_i - x_j|| + (1 - alpha) g_ij (Calibration of Weights, the
    composite genetic + geographic distance), g from geo_distance; otherwise
    the rule of knn_gaussian_weights: k nearest by d (ties to the smaller
    index), union, w = exp(-phi d^2), phi "auto" = 1 / median d^2 over the
    union edges, optional normalisation over i < j, zero weights dropped.
    Returns (ei, ej, w, d2) with d2 = d^2, i < j sorted by (i, j).
    """
    Y = fill_missing(X, mask)
    C = np.asarray(coords, dtype=np.float64)
    n = Y.shape[0]
    D = np.empty((n, n))
    for i in range(n):
        diff = Y - Y[i]
        dg = np.sqrt(np.einsum("jk,jk->j", diff, diff))
        for j in range(n):
            D[i, j] = alpha * dg[j] + (1.0 - alpha) * geo_distance(C[i], C[j], geodesic)
    kk = min(k, n - 1)
    pairs = set()
    for i in range(n):
        order = sorted((D[i, j], j) for j in range(n) if j != i)
        for _, j in order[:kk]:
            pairs.add((min(i, j), max(i, j)))
    pairs = sorted(pairs)
    ei = np.array([a for a, _ in pairs], dtype=np.int64)
    ej = np.array([b for _, b in pairs], dtype=np.int64)
    d = D[ei, ej] if ei.size else np.zeros(0)
    d2 = d * d
    if isinstance(phi, str):
        med = float(np.median(d2)) if d2.size else 0.0
        phi = 1.0 / med if med > 0 else 0.0
    if normalize and d2.size:
        w = np.exp(-phi * (d2 - d2.min()))
        w = w / w.sum()
    else:
        w = np.exp(-phi * d2)
    keep = w > 0.0
    return ei[keep], ej[keep], w[keep], d2[keep], phi


def principal_axes(X, mask, q: int):
    """Leading q principal axes of Y_0 (rows are cases, missing entries at the
    observed column means; Evaluation of Clusters: the path is displayed on
    principal components of the original data), as a q x p array of unit rows
    from the SVD of the column-centred Y_0, with their variances (squared
    singular values / n).  Sign rule: the entry of largest magnitude of each
    axis is positive (the first such entry on ties).
    """
    Y = fill_missing(X, mask)
    Yc = Y - Y.mean(axis=0)
    _, s, Vt = np.linalg.svd(Yc, full_matrices=False)
    A = Vt[:q].copy()
    for c in range(A.shape[0]):
        j = int(np.argmax(np.abs(A[c])))
        if A[c, j] < 0:
            A[c] = -A[c]
    return A, (s[:q] ** 2) / Y.shape[0]


def project_path(U, X, mask, axes):
    """Scores of centroids U (n x p) on the axes: (U - column mean of Y_0) axes^T."""
    Y = fill_missing(X, mask)
    return (np.asarray(U, dtype=np.float64) - Y.mean(axis=0)) @ np.asarray(axes).T
