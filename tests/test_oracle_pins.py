"""Pins for the CPU oracle: each test ties one oracle function to something other than itself
(brute force, a closed form, a library routine, an invariant or a hand-worked example), chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails at least one of them."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import hgf_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------------------------ box sums
def brute_box(X, r):
    H, W = X.shape
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            s = 0.0
            for yy in range(H):
                for xx in range(W):
                    if abs(yy - y) <= r and abs(xx - x) <= r:
                        s += X[yy, xx]
            out[y, x] = s
    return out


@pytest.mark.parametrize("H,W,r", [(1, 1, 0), (1, 7, 2), (5, 1, 3), (6, 9, 1), (12, 5, 4),
                                   (7, 8, 6), (3, 4, 9), (12, 12, 0), (10, 11, 3)])
def test_box_sum_brute_force(H, W, r):
    """B = window sum over the clipped (2r+1)^2 window (Sec. 4.3), including r >= size."""
    X = rng(H * 100 + W * 10 + r).normal(size=(H, W))
    np.testing.assert_allclose(O.box_sum(X, r), brute_box(X, r), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("H,W,r", [(1, 1, 0), (9, 4, 2), (13, 17, 5), (6, 6, 8)])
def test_window_count_closed_form(H, W, r):
    """N(x,y) = (min(x+r,W-1) - max(x-r,0) + 1)(min(y+r,H-1) - max(y-r,0) + 1)."""
    ys, xs = np.mgrid[0:H, 0:W]
    N = ((np.minimum(xs + r, W - 1) - np.maximum(xs - r, 0) + 1)
         * (np.minimum(ys + r, H - 1) - np.maximum(ys - r, 0) + 1))
    np.testing.assert_array_equal(O.window_count(H, W, r), N)


# ------------------------------------------------------------------------------------ guidance
def test_monomial_basis_counts_and_order():
    """n = C(C+d, d) - 1 for the full monomial basis; canonical degree-major lexicographic order;
    the paper's powers basis has n = C d (Sec. 4.2)."""
    assert [O.n_channels(3, d) for d in (1, 2, 3)] == [3, 9, 19]
    assert O.monomial_exponents(3, 2) == [(0,), (1,), (2,), (0, 0), (0, 1), (0, 2), (1, 1),
                                          (1, 2), (2, 2)]
    assert O.monomial_exponents(3, 2, "powers") == [(0,), (0, 0), (1,), (1, 1), (2,), (2, 2)]
    assert [O.n_channels(1, d) for d in (1, 2, 3)] == [1, 2, 3]
    I = rng(1).uniform(size=(3, 4, 5))
    G = O.polynomial_guidance(I, 3)
    np.testing.assert_allclose(G[4], I[0] * I[1])
    np.testing.assert_allclose(G[18], I[2] ** 3)
    np.testing.assert_allclose(G[10], I[0] * I[0] * I[1])
    Gp = O.polynomial_guidance(I, 2, "powers")
    np.testing.assert_allclose(Gp[3], I[1] ** 2)


# ------------------------------------------------------------------------------------ inverse
def random_gram(m, n_samples, seed, scale=1.0):
    X = rng(seed).normal(size=(n_samples, m)) * scale
    return X.T @ X, X


def test_prop1_hand_worked_m2():
    """Prop. 1 at m = 2 against exact rationals worked by hand (tests/golden/prop1_m2.txt)."""
    want = {}
    with open(os.path.join(GOLDEN, "prop1_m2.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, i, j, num, den = line.split()
            want[(name, int(i), int(j))] = Fraction(int(num), int(den))
    S = np.array([[2.0, 1.0], [1.0, 3.0]])
    al = O.hgf_alpha(S, 1.0)
    inv = O.hgf_inverse(S, 1.0)
    S2 = np.array([[4.0, 0.0], [0.0, 1.0]])
    al2 = O.hgf_alpha(S2, 2.0)
    for i in range(2):
        for j in range(2):
            assert al[i, j] == pytest.approx(float(want[("alpha", i, j)]), abs=1e-15)
            assert inv[i, j] == pytest.approx(float(want[("inverse", i, j)]), abs=1e-15)
            assert al2[i, j] == pytest.approx(float(want[("alpha2", i, j)]), abs=1e-15)


@pytest.mark.parametrize("lam", [1.0, 0.3, 1e-4])
def test_prop1_closed_forms(lam):
    """m = 1: alpha = -1/(lambda (lambda + s)); diagonal S: alpha_kk = -1/(lambda (lambda+s_k)),
    off-diagonal 0 (base case of Prop. 1 as corrected)."""
    s = 2.5
    a1 = O.hgf_alpha(np.array([[s]]), lam)
    assert a1[0, 0] == pytest.approx(-1.0 / (lam * (lam + s)), rel=1e-13)
    d = np.array([0.5, 3.0, 0.0, 7.0])
    a = O.hgf_alpha(np.diag(d), lam)
    np.testing.assert_allclose(np.diag(a), -1.0 / (lam * (lam + d)), rtol=1e-13)
    np.testing.assert_array_equal(a - np.diag(np.diag(a)), 0.0)


@pytest.mark.parametrize("m", [1, 2, 3, 5, 9, 13, 19])
@pytest.mark.parametrize("lam", [1.0, 1e-2, 1e-4, 1e-8])
def test_hgf_inverse_vs_lapack(m, lam):
    """Prop. 1 + Eq. HGF_w3 give (lambda E + S)^-1 for random SPD Gram matrices; alpha itself
    equals -lambda^-1 (lambda E + S)^-1. Bound: the combination lambda^-1 E + S alpha cancels
    lambda^-1 against lambda^-1 - 1/(lambda + s), losing log10(1 + |S|/lambda) digits."""
    S, _ = random_gram(m, 40, seed=m * 7 + int(-np.log10(lam)))
    ref = np.linalg.inv(lam * np.eye(m) + S)
    cond = np.linalg.cond(lam * np.eye(m) + S)
    normS = np.linalg.norm(S, 2)
    eps64 = np.finfo(np.float64).eps
    alpha = O.hgf_alpha(S, lam)
    err_a = np.linalg.norm(alpha + ref / lam) / np.linalg.norm(ref / lam)
    assert err_a <= 50 * m * eps64 * cond
    inv = O.hgf_inverse(S, lam)
    err = np.linalg.norm(inv - ref) / np.linalg.norm(ref)
    assert err <= 50 * m * eps64 * cond * (1 + normS / lam)


def test_hgf_alpha_vectorised_over_pixels():
    """The per-pixel vectorisation equals pixel-by-pixel evaluation."""
    ms = [random_gram(4, 10, seed=s)[0] for s in range(6)]
    S = np.stack(ms, axis=-1).reshape(4, 4, 2, 3)
    a = O.hgf_alpha(S, 0.1)
    for k in range(6):
        np.testing.assert_allclose(a.reshape(4, 4, 6)[:, :, k], O.hgf_alpha(ms[k], 0.1),
                                   rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m", [1, 3, 9, 19])
def test_cholesky_solve_vs_lapack(m):
    """Textbook Cholesky solve equals LAPACK's LU solve (numpy.linalg.solve)."""
    S, _ = random_gram(m, 60, seed=m)
    M = S + 1e-3 * np.eye(m)
    c = rng(m + 1).normal(size=(m,))
    a = O.cholesky_solve(M[:, :, None], c[:, None])[:, 0]
    np.testing.assert_allclose(a, np.linalg.solve(M, c), rtol=1e-9 * np.linalg.cond(M) ** 0.5)
    # batched right-hand sides
    cK = rng(m + 2).normal(size=(3, m, 1))
    aK = O.cholesky_solve(M[:, :, None], cK)
    for k in range(3):
        np.testing.assert_allclose(aK[k, :, 0], np.linalg.solve(M, cK[k, :, 0]),
                                   rtol=1e-9 * np.linalg.cond(M) ** 0.5)


@pytest.mark.parametrize("n_omega,m", [(9, 3), (25, 4), (6, 6), (4, 7)])
def test_prop1_in_window_space(n_omega, m):
    """Prop. 1 as stated: (lambda E + sum_i c_i c_i^T)^-1 = lambda^-1 E + sum_ij alpha_ij c_i c_j^T
    with |Omega|-dimensional vectors c_i (also when m > |Omega|, where the c_i are dependent),
    and the push-through identity behind Eq. HGF_w2."""
    lam = 0.37
    X = rng(n_omega * m).normal(size=(n_omega, m))          # columns c_0..c_{m-1}
    alpha = O.hgf_alpha(X.T @ X, lam)
    lhs = np.linalg.inv(lam * np.eye(n_omega) + X @ X.T)
    rhs = np.eye(n_omega) / lam + X @ alpha @ X.T
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-10)
    y = rng(1).normal(size=n_omega)
    w1 = np.linalg.solve(lam * np.eye(m) + X.T @ X, X.T @ y)     # Eq. HGF_w1
    w2 = X.T @ np.linalg.solve(lam * np.eye(n_omega) + X @ X.T, y)  # Eq. HGF_w2
    w3 = O.hgf_inverse(X.T @ X, lam) @ (X.T @ y)                 # Eq. HGF_w3
    np.testing.assert_allclose(w1, w2, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(w1, w3, rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------------------------ filters
def brute_centred(I, p, r, eps, degree, basis="monomial"):
    """Form A by explicit per-window ridge least squares (Sec. 5.1) and Eq. HGF_z1's average of
    the multipoint estimates, via numpy.linalg.lstsq; shares only polynomial_guidance."""
    G = O.polynomial_guidance(I, degree, basis)
    n, H, W = G.shape
    coef = np.empty((H, W, n + 1))
    for y in range(H):
        for x in range(W):
            ys = range(max(0, y - r), min(H, y + r + 1))
            xs = range(max(0, x - r), min(W, x + r + 1))
            rows = [(yy, xx) for yy in ys for xx in xs]
            N = len(rows)
            X = np.array([[G[i, yy, xx] for i in range(n)] + [1.0] for yy, xx in rows])
            t = np.array([p[yy, xx] for yy, xx in rows])
            # minimise sum_q (t - X w)^2 + N eps |a|^2 (offset unpenalised)
            pen = np.hstack([np.sqrt(N * eps) * np.eye(n), np.zeros((n, 1))])
            w, *_ = np.linalg.lstsq(np.vstack([X, pen]), np.concatenate([t, np.zeros(n)]),
                                    rcond=None)
            coef[y, x] = w
    q = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            vals = []
            for yy in range(max(0, y - r), min(H, y + r + 1)):
                for xx in range(max(0, x - r), min(W, x + r + 1)):
                    vals.append(coef[yy, xx, :n] @ G[:, y, x] + coef[yy, xx, n])
            q[y, x] = np.mean(vals)
    return q


def brute_paper(I, p, r, lam, degree, basis="powers"):
    """Form B (Eq. HGF_linear_regression) by per-window ridge least squares with every
    coefficient penalised, and Eq. HGF_z1's average."""
    G = O.polynomial_guidance(I, degree, basis)
    n, H, W = G.shape
    coef = np.empty((H, W, n + 1))
    for y in range(H):
        for x in range(W):
            rows = [(yy, xx) for yy in range(max(0, y - r), min(H, y + r + 1))
                    for xx in range(max(0, x - r), min(W, x + r + 1))]
            X = np.array([[1.0] + [G[i, yy, xx] for i in range(n)] for yy, xx in rows])
            t = np.array([p[yy, xx] for yy, xx in rows])
            A = np.vstack([X, np.sqrt(lam) * np.eye(n + 1)])
            w, *_ = np.linalg.lstsq(A, np.concatenate([t, np.zeros(n + 1)]), rcond=None)
            coef[y, x] = w
    Z = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            vals = [coef[yy, xx, 1:] @ G[:, y, x] + coef[yy, xx, 0]
                    for yy in range(max(0, y - r), min(H, y + r + 1))
                    for xx in range(max(0, x - r), min(W, x + r + 1))]
            Z[y, x] = np.mean(vals)
    return Z


@pytest.mark.parametrize("H,W,r,degree,eps", [(9, 11, 2, 1, 1e-3), (8, 7, 1, 2, 1e-2),
                                              (6, 10, 3, 2, 1e-4), (5, 5, 4, 1, 1e-3),
                                              (7, 4, 1, 3, 1e-2)])
def test_centred_filter_vs_brute_lstsq(H, W, r, degree, eps):
    g = rng(H * W + r)
    I = g.uniform(size=(3, H, W))
    p = g.uniform(size=(H, W)) * 0.03
    ref = brute_centred(I, p, r, eps, degree)
    np.testing.assert_allclose(O.centred_filter(I, p, r, eps, degree), ref, rtol=1e-8, atol=1e-11)
    np.testing.assert_allclose(O.centred_filter_hgf(I, p, r, eps, degree), ref, rtol=1e-6,
                               atol=1e-9)


@pytest.mark.parametrize("H,W,r,degree,lam,C", [(8, 9, 2, 2, 0.05, 3), (6, 7, 1, 3, 0.5, 1),
                                                (7, 5, 2, 1, 0.01, 3)])
def test_paper_filter_vs_brute_lstsq(H, W, r, degree, lam, C):
    g = rng(H + W + r + C)
    I = g.uniform(size=(C, H, W))
    p = g.uniform(size=(H, W))
    ref = brute_paper(I, p, r, lam, degree)
    np.testing.assert_allclose(O.paper_filter(I, p, r, lam, degree, solver="cholesky"), ref,
                               rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(O.paper_filter(I, p, r, lam, degree, solver="hgf"), ref,
                               rtol=1e-6, atol=1e-8)


def test_paper_filter_constant_guidance_closed_form():
    """Form B with constant guidance g (one channel, degree 1): per window the 2x2 ridge system
    [[lam + N, N g], [N g, lam + N g^2]] w = [S, g S] (S = window sum of Y)."""
    H, W, r, lam, g0 = 6, 7, 2, 0.3, 0.6
    I = np.full((1, H, W), g0)
    Y = rng(3).uniform(size=(H, W))
    N = O.window_count(H, W, r)
    S = O.box_sum(Y, r)
    det = (lam + N) * (lam + N * g0 * g0) - (N * g0) ** 2
    w0 = ((lam + N * g0 * g0) * S - N * g0 * g0 * S) / det
    w1 = ((lam + N) * g0 * S - N * g0 * S) / det
    Z = (O.box_sum(w1, r) / N) * g0 + O.box_sum(w0, r) / N
    np.testing.assert_allclose(O.paper_filter(I, Y, r, lam, 1, solver="hgf"), Z, rtol=1e-10)


def test_constant_guidance_reduces_to_double_mean():
    """Constant guidance: Sigma = 0, cov = 0, a = 0, so q = A(A(p))."""
    H, W, r = 10, 13, 3
    I = np.full((3, H, W), 0.4)
    p = rng(4).uniform(size=(H, W))
    N = O.window_count(H, W, r)
    want = O.box_sum(O.box_sum(p, r) / N, r) / N
    np.testing.assert_allclose(O.centred_filter(I, p, r, 1e-4, 2), want, rtol=1e-10, atol=1e-13)


def test_constant_slice_is_reproduced():
    H, W, r = 9, 11, 2
    I = rng(5).uniform(size=(3, H, W))
    q = O.centred_filter(I, np.full((H, W), 0.0173), r, 1e-4, 2)
    np.testing.assert_allclose(q, 0.0173, rtol=1e-9)


def test_linear_in_slice_and_shift_invariant():
    H, W, r = 9, 10, 2
    g = rng(6)
    I = g.uniform(size=(3, H, W))
    p1, p2 = g.uniform(size=(2, H, W))
    q1 = O.centred_filter(I, p1, r, 1e-3, 2)
    q2 = O.centred_filter(I, p2, r, 1e-3, 2)
    np.testing.assert_allclose(O.centred_filter(I, 2.0 * p1 - 0.5 * p2, r, 1e-3, 2),
                               2.0 * q1 - 0.5 * q2, rtol=1e-9, atol=1e-12)
    # degree-1 channels are the inputs themselves: G_i -> G_i + c_i leaves form A unchanged
    q = O.centred_filter(I, p1, r, 1e-3, 1)
    qs = O.centred_filter(I + np.array([0.3, -0.2, 0.7])[:, None, None], p1, r, 1e-3, 1)
    np.testing.assert_allclose(qs, q, rtol=1e-9, atol=1e-12)


def test_transpose_equivariance():
    H, W, r = 7, 12, 2
    g = rng(7)
    I = g.uniform(size=(3, H, W))
    p = g.uniform(size=(H, W))
    q = O.centred_filter(I, p, r, 1e-3, 2)
    qt = O.centred_filter(I.transpose(0, 2, 1), p.T, r, 1e-3, 2)
    np.testing.assert_allclose(qt, q.T, rtol=1e-9, atol=1e-12)


def test_affine_slice_reproduced_as_eps_vanishes():
    """p = sum_i c_i G_i + c_0 is fitted exactly by every window as eps -> 0 (noise guidance so
    that every window is non-degenerate)."""
    H, W, r = 12, 12, 2
    g = rng(8)
    I = g.uniform(size=(3, H, W))
    G = O.polynomial_guidance(I, 2)
    c = g.normal(size=9)
    p = np.einsum("i,ihw->hw", c, G) + 0.2
    q = O.centred_filter(I, p, r, 1e-10, 2)
    assert np.max(np.abs(q - p)) < 1e-5 * np.max(np.abs(p))


def test_quadratic_slice_needs_degree_two():
    """A slice quadratic in RGB is reproduced by the degree-2 monomial guidance, not by the
    degree-1 (linear GF) guidance (the nonlinearity claim of Sec. 6)."""
    H, W, r = 14, 14, 3
    g = rng(9)
    I = g.uniform(size=(3, H, W))
    p = 0.5 * I[0] ** 2 - 0.8 * I[1] * I[2] + 0.3 * I[2]
    e2 = np.max(np.abs(O.centred_filter(I, p, r, 1e-9, 2) - p))
    e1 = np.max(np.abs(O.centred_filter(I, p, r, 1e-9, 1) - p))
    assert e2 < 1e-5
    assert e1 > 1e-2


def test_wta_ties_nan_and_permutation():
    Q = np.array([[[1.0, 2.0]], [[1.0, np.nan]], [[0.5, 2.0]]])    # (L=3, H=1, W=2)
    labels, best, margin = O.wta(Q)
    assert labels.tolist() == [[2, 0]]      # tie 2.0 vs 2.0 at pixel 1: lowest label; NaN = inf
    assert best.tolist() == [[0.5, 2.0]]
    assert margin.tolist() == [[0.5, 0.0]]
    g = rng(10)
    Q = g.uniform(size=(6, 5, 4))
    perm = g.permutation(6)
    l0, _, _ = O.wta(Q)
    l1, _, _ = O.wta(Q[perm])
    np.testing.assert_array_equal(perm[l1], l0)


def test_filter_at_matches_full_image():
    H, W, r = 30, 34, 3
    g = rng(11)
    I = g.uniform(size=(3, H, W)).astype(np.float32)
    P = (g.uniform(size=(3, H, W)) * 0.03).astype(np.float32)
    q = O.centred_filter(I, P, r, 1e-4, 2)
    pts = [(0, 0), (H - 1, W - 1), (15, 17), (2, 30), (29, 5), (6, 6)]
    got = O.filter_at(I, P, r, 1e-4, 2, pts)
    for t, (y, x) in enumerate(pts):
        np.testing.assert_allclose(got[:, t], q[:, y, x], rtol=1e-12, atol=1e-15)


def test_filter_region_matches_full_image():
    """filter_region on rectangles at the corners, the edges and the interior (and one wider than
    the crop margin) equals the full-image filter there."""
    H, W, r = 31, 37, 3
    g = rng(12)
    I = g.uniform(size=(3, H, W)).astype(np.float32)
    P = (g.uniform(size=(3, H, W)) * 0.03).astype(np.float32)
    q = O.centred_filter(I, P, r, 1e-4, 2)
    for y0, y1, x0, x1 in ((0, 5, 0, 4), (26, 31, 30, 37), (10, 17, 12, 25), (0, 31, 35, 37),
                           (3, 4, 0, 37)):
        got = O.filter_region(I, P, r, 1e-4, 2, y0, y1, x0, x1)
        np.testing.assert_allclose(got, q[:, y0:y1, x0:x1], rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------------------- cost volume
def test_cost_volume_zero_at_the_true_shift():
    """A scene point at left x seen at right x - d (right(x') = left(x' + d)): the
    left-reference cost is exactly 0 at label d wherever x - d and the gradient neighbours are
    inside both views (d + 1 <= x <= W - 2) and positive at the other labels there; identical
    views cost 0 at label 0; the right-reference cost (direction -1) of the same pair is 0 at
    label d for 1 <= x <= W - d - 2."""
    rng = np.random.Generator(np.random.PCG64(3))
    H, W, d = 5, 23, 4
    base = rng.uniform(0, 1, (3, H, W + d))
    left, right = base[:, :, :W], base[:, :, d:d + W]
    V = O.cost_volume(left, right, 8)
    assert np.all(V[d][:, d + 1:W - 1] == 0.0)
    others = np.delete(V[:, :, d + 1:W - 1], d, axis=0)
    assert np.all(others > 0.0)
    assert np.all(O.cost_volume(left, left, 1) == 0.0)
    VR = O.cost_volume(right, left, 8, direction=-1)
    assert np.all(VR[d][:, 1:W - d - 1] == 0.0)


def test_cost_volume_constant_offset_closed_form():
    """Constant views with per-channel offsets delta_c: gradients vanish, so
    V = alpha min(mean_c |delta_c|, tau_color) for every label and pixel (truncation and the
    alpha weight are pinned by choosing offsets on both sides of tau_color)."""
    for delta, alpha in (((0.01, -0.02, 0.005), 0.9), ((0.1, 0.2, -0.3), 0.6)):
        I = np.full((3, 4, 9), 0.5)
        J = I + np.array(delta)[:, None, None]
        V = O.cost_volume(I, J, 5, alpha=alpha, tau_color=0.028, tau_grad=0.008)
        want = alpha * min(np.mean(np.abs(delta)), 0.028)
        np.testing.assert_allclose(V, want, rtol=1e-15, atol=0)


def test_cost_volume_ramp_gradient_and_border_clamp():
    """Identical horizontal ramps I_c = J_c = a x: the colour term is alpha min(a l, tau_color)
    wherever x - l >= 0, the gradient term vanishes in the interior (both slopes a) and at the
    clamped border the match column is x' = 0, so V(x, l) for x < l equals the cost at
    x' = 0: alpha min(a x, tau_color) + (1 - alpha) min(|dI(x) - dJ(0)|, tau_grad) with
    dJ(0) = a / 2 (one-sided neighbour) and dI(x) = a inside."""
    a, W, L, alpha = 0.004, 16, 6, 0.9
    I = np.tile(a * np.arange(W, dtype=np.float64), (3, 2, 1))
    V = O.cost_volume(I, I, L, alpha=alpha, tau_color=0.015, tau_grad=0.008)
    for l in range(L):
        for x in range(W):
            xs = max(x - l, 0)
            col = alpha * min(a * (x - xs), 0.015)
            dI = a if 0 < x < W - 1 else a / 2
            dJ = a if 0 < xs < W - 1 else a / 2
            want = col + (1 - alpha) * min(abs(dI - dJ), 0.008)
            assert abs(V[l, 0, x] - want) < 1e-15, (l, x)


# ------------------------------------------------------------------------- post-WTA refinement
def test_refine_lr_hand_worked_rows():
    """Hand-worked rows (threshold 1). Row 0: DL = DR warped consistently except an occlusion
    band at x = 3, 4 (disparities 5 pointing outside, 0 inconsistent): filled with the smaller
    neighbour 1. Row 1: nothing consistent: DL unchanged. Row 2: kept pixels on the right only:
    the nearest one to the right fills."""
    DL = np.array([[0, 1, 1, 5, 0, 2, 2, 2],
                   [7, 7, 7, 7, 7, 7, 7, 7],
                   [9, 9, 9, 0, 0, 1, 1, 1]])
    DR = np.array([[0, 1, 1, 1, 2, 2, 2, 2],
                   [0, 0, 0, 0, 0, 0, 0, 0],
                   [0, 0, 0, 0, 1, 1, 1, 1]])
    out, keep = O.refine_lr(DL, DR, 1)
    # row 0: x=3: d=5 -> x-d<0 drop; x=4: d=0 -> DR(4)=2, |0-2|>1 drop; others consistent
    assert keep[0].tolist() == [True, True, True, False, False, True, True, True]
    assert out[0].tolist() == [0, 1, 1, 1, 1, 2, 2, 2]
    assert not keep[1].any() and out[1].tolist() == DL[1].tolist()
    # row 2: x<3: d=9 outside; x=3,4: d=0 -> DR=0 at 3 (kept), DR(4)=1 (|0-1|<=1 kept)
    assert keep[2].tolist() == [False, False, False, True, True, True, True, True]
    assert out[2].tolist() == [0, 0, 0, 0, 0, 1, 1, 1]


def test_refine_lr_consistent_maps_unchanged():
    """Maps from a fronto-parallel plane at disparity d (DL = DR = d) are consistent wherever
    x >= d; the left border x < d is filled from the first kept pixel (d)."""
    DL = np.full((3, 10), 3)
    out, keep = O.refine_lr(DL, DL, 0)
    assert keep[:, 3:].all() and not keep[:, :3].any()
    assert (out == 3).all()
