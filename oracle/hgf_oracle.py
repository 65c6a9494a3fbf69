"""CPU oracle for the HGF multi-label aggregation path (plain, slow, float64).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links this module: only
the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use it. It shares no
code, tables or constants with the CUDA library; it restates the paper (arXiv 1803.00005,
"Hardware-Efficient Guided Image Filtering for Multi-Label Problem") directly:

* box filter B = clipped window *sum*, A(X) = B(X) / B(G0) with G0 = ones    (Sec. 4.3, Eq. HGF_z2)
* polynomial guidance (Sec. 4.2): full monomials of degree 1..d of the input channels (default),
  or the paper's per-channel powers G_{(i-1)d+j} = I_i^j
* form A, the guided-filter ("GF") form with centred moments and an unpenalised offset (Sec. 5.1,
  Eqs. GF_linear_regression / GF_w):  a = (Sigma + eps E)^-1 cov,  b = pbar - a.mu
* multipoint aggregation q = sum_i A(a_i) G_i + A(b)                     (Sec. 4.1, Eq. HGF_z1)
* the HGF inverse by the Sherman-Morrison recursion of Prop. 1 (Sec. 3), with Eq. HGF_w3's
  combination lambda^-1 E + S alpha
* form B, the paper's own HGF (Sec. 4.1, Eq. HGF_linear_regression): G0 = 1, uncentred box sums,
  all n+1 coefficients penalised by lambda in sum units, Z by Eq. HGF_z2
* WTA label selection (Sec. 1): argmin over labels, lowest label on ties, NaN treated as +inf
* post-WTA refinement (Sec. 6 names the framework's post processing): left-right consistency
  and hole filling, a reading (see refine_lr)
* the cost volume V(x, y, l) of a stereo pair (Sec. 1; the cost computation step of the
  cost-volume filtering framework of Sec. 6, whose formula the paper does not print: the reading
  is a truncated colour + gradient difference, see cost_volume)

Readings of the paper used here (where it is silent, ambiguous or garbled):
* Prop. 1's base case is alpha^0_00 = -1/(lambda (lambda + G_00)); the printed -(lambda+G_00)^-1
  holds only for lambda = 1. Starting the recursion at kappa = 0 with an empty alpha gives it.
* Eq. alpha's first case lacks the factor gamma^kappa that Prop. 1 has; gamma F + alpha is used.
* Eq. HGF_w4's index kappa is read as k: W_k = lambda^-1 G_{k,n+1} + sum_ij alpha_ij G_ki G_j,n+1.
* Windows are clipped at the image border (no padding); N(x) = B(ones) varies near borders.

Every function is pinned in tests/test_oracle_pins.py against closed forms, brute force, library
routines and invariants (see each test's docstring for what it pins).
"""
from __future__ import annotations

import itertools
import numpy as np

__all__ = [
    "box_sum", "window_count", "box_mean", "monomial_exponents", "polynomial_guidance",
    "n_channels", "cholesky_solve", "hgf_alpha", "hgf_inverse", "guidance_moments",
    "centred_filter", "centred_filter_hgf", "paper_filter", "wta", "filter_at", "filter_region",
]


# --------------------------------------------------------------------------------------------
# Box filtering (Sec. 4.3: B is a window sum; Prop. 2: Gram entries are box sums)
# --------------------------------------------------------------------------------------------
def box_sum(X: np.ndarray, r: int) -> np.ndarray:
    """Clipped (2r+1)x(2r+1) window sums over the last two axes, by direct summation.

    out[..., y, x] = sum of X[..., y', x'] over |y'-y| <= r, |x'-x| <= r inside the image.
    Computed separably (rows, then columns), adding one shifted copy per offset."""
    X = np.asarray(X, dtype=np.float64)
    H, W = X.shape[-2:]
    tmp = np.zeros_like(X)
    for dx in range(-r, r + 1):
        lo, hi = max(0, -dx), min(W, W - dx)
        if lo < hi:
            tmp[..., :, lo:hi] += X[..., :, lo + dx:hi + dx]
    out = np.zeros_like(X)
    for dy in range(-r, r + 1):
        lo, hi = max(0, -dy), min(H, H - dy)
        if lo < hi:
            out[..., lo:hi, :] += tmp[..., lo + dy:hi + dy, :]
    return out


def window_count(H: int, W: int, r: int) -> np.ndarray:
    """N(x, y) = B(G0)(x, y): number of pixels in the clipped window."""
    return box_sum(np.ones((H, W)), r)


def box_mean(X: np.ndarray, r: int, N: np.ndarray | None = None) -> np.ndarray:
    """A(X) = B(X) / B(G0) (the average operator of Eq. HGF_z2)."""
    X = np.asarray(X, dtype=np.float64)
    if N is None:
        N = window_count(X.shape[-2], X.shape[-1], r)
    return box_sum(X, r) / N


# --------------------------------------------------------------------------------------------
# Polynomial guidance (Sec. 4.2)
# --------------------------------------------------------------------------------------------
def monomial_exponents(C: int, degree: int, basis: str = "monomial"):
    """Channel multisets defining G_1..G_n.

    monomial: every monomial of degree 1..d, degree-major, then lexicographic multisets
              (R, G, B, RR, RG, RB, GG, GB, BB, RRR, ...); n = C(C+d, d) - 1.
    powers:   the paper's G_{(i-1)d+j} = I_i^j, channel-major then power; n = C d."""
    if basis == "monomial":
        out = []
        for deg in range(1, degree + 1):
            out.extend(itertools.combinations_with_replacement(range(C), deg))
        return out
    if basis == "powers":
        return [tuple([i] * j) for i in range(C) for j in range(1, degree + 1)]
    raise ValueError(basis)


def n_channels(C: int, degree: int, basis: str = "monomial") -> int:
    return len(monomial_exponents(C, degree, basis))


def polynomial_guidance(I: np.ndarray, degree: int, basis: str = "monomial") -> np.ndarray:
    """(n, H, W) float64 guidance channels G_1..G_n from the (C, H, W) input image."""
    I = np.asarray(I, dtype=np.float64)
    chans = []
    for ms in monomial_exponents(I.shape[0], degree, basis):
        g = np.ones(I.shape[1:])
        for c in ms:
            g = g * I[c]
        chans.append(g)
    return np.stack(chans)


# --------------------------------------------------------------------------------------------
# Per-pixel linear algebra, vectorised over the trailing pixel axes
# --------------------------------------------------------------------------------------------
def cholesky_solve(M: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solve M a = c per pixel with a textbook Cholesky factorisation M = L L^T.

    M: (n, n, *P) symmetric positive definite; c: (n, *P) or (K, n, *P). Returns a like c."""
    n = M.shape[0]
    L = np.zeros_like(M)
    for j in range(n):
        s = M[j, j] - sum(L[j, k] * L[j, k] for k in range(j))
        L[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (M[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    batched = c.ndim == M.ndim  # (K, n, *P)
    cc = c if batched else c[None]
    y = np.zeros_like(cc)
    for i in range(n):  # forward substitution L y = c
        y[:, i] = (cc[:, i] - sum(L[i, k] * y[:, k] for k in range(i))) / L[i, i]
    a = np.zeros_like(cc)
    for i in reversed(range(n)):  # back substitution L^T a = y
        a[:, i] = (y[:, i] - sum(L[k, i] * a[:, k] for k in range(i + 1, n))) / L[i, i]
    return a if batched else a[0]


def hgf_alpha(S: np.ndarray, lam: float) -> np.ndarray:
    """alpha = alpha^n of Prop. 1 (Sec. 3) for the Gram matrix S (m, m, *P) and lambda.

    Sherman-Morrison over kappa = 0..m-1, starting from an empty alpha:
      u_i    = sum_{j<kappa} alpha_ij S_{j kappa}
      gamma  = -(1 + S_kk / lambda + sum_{i<kappa} S_{kappa i} u_i)^-1
      alpha_ij += gamma u_i u_j           (i, j < kappa; gamma F^kappa_ij, F_ij = u_i u_j)
      alpha_{i kappa} = alpha_{kappa i} = gamma u_i / lambda
      alpha_{kappa kappa} = gamma / lambda^2"""
    m = S.shape[0]
    alpha = np.zeros_like(S, dtype=np.float64)
    for k in range(m):
        u = [sum(alpha[i, j] * S[j, k] for j in range(k)) for i in range(k)]
        den = 1.0 + S[k, k] / lam + sum(S[k, i] * u[i] for i in range(k))
        gamma = -1.0 / den
        for i in range(k):
            for j in range(k):
                alpha[i, j] = alpha[i, j] + gamma * u[i] * u[j]
            alpha[i, k] = gamma * u[i] / lam
            alpha[k, i] = gamma * u[i] / lam
        alpha[k, k] = gamma / (lam * lam)
    return alpha


def hgf_inverse(S: np.ndarray, lam: float) -> np.ndarray:
    """(lambda E + S)^-1 = lambda^-1 E + S alpha (Prop. 1 combined as in Eq. HGF_w3)."""
    m = S.shape[0]
    alpha = hgf_alpha(S, lam)
    Sa = np.einsum("ij...,jk...->ik...", S, alpha)
    eye = np.eye(m).reshape((m, m) + (1,) * (S.ndim - 2))
    return eye / lam + Sa


# --------------------------------------------------------------------------------------------
# Form A: centred guided-filter form (Sec. 5.1) with multipoint aggregation (Sec. 4.1)
# --------------------------------------------------------------------------------------------
def guidance_moments(I, r, eps, degree, basis="monomial"):
    """Guidance-only part (once per guidance, Sec. 5.3 precompute): G, N, mu = A(G),
    and M = Sigma + eps E with Sigma_ij = A(G_i G_j) - mu_i mu_j."""
    G = polynomial_guidance(I, degree, basis)
    n, H, W = G.shape
    N = window_count(H, W, r)
    mu = box_sum(G, r) / N
    M = np.empty((n, n, H, W))
    for i in range(n):
        for j in range(i, n):
            s = box_sum(G[i] * G[j], r) / N - mu[i] * mu[j]
            M[i, j] = s
            M[j, i] = s
    for i in range(n):
        M[i, i] += eps
    return G, N, mu, M


def _coefficients(P, G, N, mu, r, solve):
    """a = (Sigma + eps E)^-1 cov, b = pbar - a.mu for a stack of slices P (K, H, W)."""
    pbar = box_sum(P, r) / N                                       # (K, H, W)
    cov = box_sum(G[None] * P[:, None], r) / N - mu[None] * pbar[:, None]   # (K, n, H, W)
    a = solve(cov)
    b = pbar - np.einsum("kihw,ihw->khw", a, mu)
    return a, b


def _aggregate(a, b, G, N, r):
    """q = sum_i A(a_i) G_i + A(b) (Eq. HGF_z1 / HGF_z2)."""
    abar = box_sum(a, r) / N
    bbar = box_sum(b, r) / N
    return np.einsum("kihw,ihw->khw", abar, G) + bbar


def centred_filter(I, P, r, eps, degree, basis="monomial", labels_per_chunk=8):
    """Form A filtered slices q (K, H, W) for cost slices P (K, H, W), Cholesky solve."""
    P = np.asarray(P, dtype=np.float64)
    if P.ndim == 2:
        return centred_filter(I, P[None], r, eps, degree, basis, labels_per_chunk)[0]
    G, N, mu, M = guidance_moments(I, r, eps, degree, basis)
    out = np.empty_like(P)
    for k0 in range(0, P.shape[0], labels_per_chunk):
        chunk = P[k0:k0 + labels_per_chunk]
        a, b = _coefficients(chunk, G, N, mu, r, lambda cov: cholesky_solve(M, cov))
        out[k0:k0 + labels_per_chunk] = _aggregate(a, b, G, N, r)
    return out


def centred_filter_hgf(I, P, r, eps, degree, basis="monomial", labels_per_chunk=8):
    """Form A with the per-pixel inverse taken from the HGF recursion (Prop. 1, lambda = eps,
    S = Sigma), combined as lambda^-1 E + S alpha (Eq. HGF_w3)."""
    P = np.asarray(P, dtype=np.float64)
    if P.ndim == 2:
        return centred_filter_hgf(I, P[None], r, eps, degree, basis, labels_per_chunk)[0]
    G, N, mu, M = guidance_moments(I, r, eps, degree, basis)
    n = G.shape[0]
    Sigma = M - eps * np.eye(n)[:, :, None, None]
    Minv = hgf_inverse(Sigma, eps)
    out = np.empty_like(P)
    for k0 in range(0, P.shape[0], labels_per_chunk):
        chunk = P[k0:k0 + labels_per_chunk]
        a, b = _coefficients(chunk, G, N, mu, r,
                             lambda cov: np.einsum("ijhw,kjhw->kihw", Minv, cov))
        out[k0:k0 + labels_per_chunk] = _aggregate(a, b, G, N, r)
    return out


# --------------------------------------------------------------------------------------------
# Form B: the paper's HGF (Sec. 4.1 / 4.3): G0 = 1, penalised w(0), uncentred box sums
# --------------------------------------------------------------------------------------------
def paper_filter(I, P, r, lam, degree, basis="powers", solver="hgf"):
    """Z = sum_{i>=1} A(W_i) G_i + A(W_0) with w = (lambda E + G)^-1 b per pixel, where
    G_ij = B(G_i G_j) (i, j = 0..n, G_0 = 1) and b_k = B(G_k Y) (Eqs. HGF_Iij, HGF_w3, HGF_z2).
    solver="hgf": w = (lambda^-1 E + G alpha) b (Prop. 1); "cholesky": textbook solve."""
    P = np.asarray(P, dtype=np.float64)
    single = P.ndim == 2
    P = P[None] if single else P
    Gn = polynomial_guidance(I, degree, basis)
    n, H, W = Gn.shape
    G = np.concatenate([np.ones((1, H, W)), Gn])
    N = window_count(H, W, r)
    Gram = np.empty((n + 1, n + 1, H, W))
    for i in range(n + 1):
        for j in range(i, n + 1):
            s = box_sum(G[i] * G[j], r)
            Gram[i, j] = s
            Gram[j, i] = s
    bvec = box_sum(G[None] * P[:, None], r)                   # (K, n+1, H, W)
    if solver == "hgf":
        Minv = hgf_inverse(Gram, lam)
        w = np.einsum("ijhw,kjhw->kihw", Minv, bvec)
    else:
        M = Gram + lam * np.eye(n + 1)[:, :, None, None]
        w = cholesky_solve(M, bvec)
    wa = box_sum(w, r) / N
    Z = np.einsum("kihw,ihw->khw", wa[:, 1:], Gn) + wa[:, 0]
    return Z[0] if single else Z


# --------------------------------------------------------------------------------------------
# Cost volume of a stereo pair (Sec. 1; reading of the framework's cost computation, Sec. 6)
# --------------------------------------------------------------------------------------------
def cost_volume(ref, other, L, alpha=0.9, tau_color=0.028, tau_grad=0.008, direction=1):
    """V(x, y, l) = alpha min(mean_c |I_c(x,y) - J_c(x',y)|, tau_color)
                  + (1 - alpha) min(|dI(x,y) - dJ(x',y)|, tau_grad),
    x' = clamp(x - direction * l, 0, W-1), I = ref, J = other (C x H x W), dI the central
    difference along x of the channel mean with clamped neighbours, 0.5 (g(x+1) - g(x-1)).
    direction = 1: the reference is the left view (matches lie to the left in the right view);
    -1: the reference is the right view. Returns float64 (L, H, W). One label at a time, plain
    numpy."""
    I = np.asarray(ref, dtype=np.float64)
    J = np.asarray(other, dtype=np.float64)
    C, H, W = I.shape
    x = np.arange(W)
    xp, xm = np.minimum(x + 1, W - 1), np.maximum(x - 1, 0)

    def grad(img):
        g = img.mean(axis=0)
        return 0.5 * (g[:, xp] - g[:, xm])

    dI, dJ = grad(I), grad(J)
    V = np.empty((L, H, W))
    for l in range(L):
        xs = np.clip(x - direction * l, 0, W - 1)
        col = np.abs(I - J[:, :, xs]).mean(axis=0)
        grd = np.abs(dI - dJ[:, xs])
        V[l] = alpha * np.minimum(col, tau_color) + (1.0 - alpha) * np.minimum(grd, tau_grad)
    return V


# --------------------------------------------------------------------------------------------
# Post-WTA refinement (reading of the framework's post processing, Sec. 6)
# --------------------------------------------------------------------------------------------
def refine_lr(DL, DR, threshold=1):
    """Left-right consistency check and hole filling, one pixel at a time.
    keep(x, y): d = DL(x, y) >= 0, x - d >= 0 and |d - DR(x - d, y)| <= threshold.
    Pixels not kept take min(nearest kept DL to the left, nearest kept DL to the right) on their
    row; one side only: that one; none: their own DL. Returns (out, keep)."""
    DL = np.asarray(DL)
    DR = np.asarray(DR)
    H, W = DL.shape
    keep = np.zeros((H, W), dtype=bool)
    for y in range(H):
        for x in range(W):
            d = int(DL[y, x])
            keep[y, x] = d >= 0 and x - d >= 0 and abs(d - int(DR[y, x - d])) <= threshold
    out = DL.copy()
    for y in range(H):
        for x in range(W):
            if keep[y, x]:
                continue
            left = [int(DL[y, i]) for i in range(x - 1, -1, -1) if keep[y, i]][:1]
            right = [int(DL[y, i]) for i in range(x + 1, W) if keep[y, i]][:1]
            cand = left + right
            out[y, x] = min(cand) if cand else DL[y, x]
    return out, keep


# --------------------------------------------------------------------------------------------
# WTA (Sec. 1)
# --------------------------------------------------------------------------------------------
def wta(Q: np.ndarray):
    """labels = argmin_l Q[l] (lowest l on ties, NaN as +inf); best; margin = second - best."""
    Q = np.where(np.isnan(Q), np.inf, np.asarray(Q, dtype=np.float64))
    labels = np.argmin(Q, axis=0).astype(np.int32)
    best = np.take_along_axis(Q, labels[None].astype(np.int64), axis=0)[0]
    if Q.shape[0] > 1:
        part = np.partition(Q, 1, axis=0)
        margin = part[1] - part[0]
    else:
        margin = np.full(best.shape, np.inf)
    return labels, best, margin


def filter_at(I, P, r, eps, degree, points, basis="monomial"):
    """Form A output at selected pixels (y, x) of a large image, computed on the smallest crop
    that holds every input the output depends on: q(x) reads coefficients in its window, each of
    which reads its own window, so inputs within distance 2r suffice. Windows that touch the
    image border are clipped by the same border inside the crop, so the result is exact.
    Returns (K, len(points))."""
    P = np.asarray(P)
    H, W = P.shape[-2:]
    out = np.empty((P.shape[0], len(points)))
    for t, (y, x) in enumerate(points):
        y0, y1 = max(0, y - 2 * r), min(H, y + 2 * r + 1)
        x0, x1 = max(0, x - 2 * r), min(W, x + 2 * r + 1)
        q = centred_filter(np.asarray(I)[:, y0:y1, x0:x1],
                           np.asarray(P[:, y0:y1, x0:x1], dtype=np.float64),
                           r, eps, degree, basis)
        out[:, t] = q[:, y - y0, x - x0]
    return out


def filter_region(I, P, r, eps, degree, y0, y1, x0, x1, basis="monomial"):
    """Form A output on the rectangle [y0, y1) x [x0, x1) of a large image, computed, as in
    filter_at, on the smallest crop that holds every input it depends on (the rectangle grown by
    2r on each side and clipped to the image): exact, because windows that touch the image border
    are clipped by the same border inside the crop. Returns (K, y1 - y0, x1 - x0)."""
    P = np.asarray(P)
    H, W = P.shape[-2:]
    cy0, cy1 = max(0, y0 - 2 * r), min(H, y1 + 2 * r)
    cx0, cx1 = max(0, x0 - 2 * r), min(W, x1 + 2 * r)
    q = centred_filter(np.asarray(I)[:, cy0:cy1, cx0:cx1],
                       np.asarray(P[:, cy0:cy1, cx0:cx1], dtype=np.float64), r, eps, degree, basis)
    return q[:, y0 - cy0:y1 - cy0, x0 - cx0:x1 - cx0]
