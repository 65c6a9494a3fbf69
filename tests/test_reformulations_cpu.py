"""CPU checks of the exact reformulations the CUDA kernels use, emulated in numpy against the
oracle (float64): each is algebraically exact, so it must agree to rounding.

* Paper form in image-mean-shifted coordinates (k_inverse_paper + k_coef): with [1, G] = T [1, Gs],
  Gram = T Gram_s T^T is rebuilt from the shifted sums, Mt = T^T (lambda E + Gram)^-1 T multiplies
  the shifted slice sums, and A(v_0) + sum_i A(v_i) Gs_i equals the paper's output.
* Centred form in window-sum units (k_inverse): T = N Sigma, lambda' = N eps and
  (Sigma + eps E)^-1 = N (lambda' E + T)^-1 = -N lambda' alpha'.
* The Newton reciprocal of the recursion's denominators: two steps from the float32 reciprocal
  reach float64 accuracy.
* The double-float building blocks: two_sum and two_prod are error-free in float32.
"""
import numpy as np

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth


def test_paper_form_in_shifted_coordinates():
    sc = synth.make_case(40, 30, 3, 5, "f32")
    I = sc.guidance.astype(np.float64)
    P = sc.cost.astype(np.float64)
    r, lam, deg = 3, 0.05, 2
    ref = O.paper_filter(I, P, r, lam, deg, basis="monomial")
    G = O.polynomial_guidance(I, deg, "monomial")
    n, H, W = G.shape
    c = G.mean(axis=(1, 2))
    Gs = G - c[:, None, None]
    N = O.window_count(H, W, r)
    sg = np.stack([O.box_sum(Gs[i], r) for i in range(n)])
    M = n + 1
    Gram = np.zeros((M, M, H, W))
    Gram[0, 0] = N
    for i in range(n):
        Gram[0, i + 1] = Gram[i + 1, 0] = sg[i] + c[i] * N
        for j in range(i, n):
            sgg = O.box_sum(Gs[i] * Gs[j], r)
            Gram[i + 1, j + 1] = Gram[j + 1, i + 1] = sgg + c[i] * sg[j] + c[j] * sg[i] + c[i] * c[j] * N
    T = np.eye(M)
    T[1:, 0] = c
    Mt = np.einsum("ji,jkhw,kl->ilhw", T, O.hgf_inverse(Gram, lam), T)
    out = np.empty_like(ref)
    for l in range(P.shape[0]):
        bs = np.stack([O.box_sum(P[l], r)] + [O.box_sum(Gs[i] * P[l], r) for i in range(n)])
        v = np.einsum("ijhw,jhw->ihw", Mt, bs)
        va = np.stack([O.box_sum(v[i], r) for i in range(M)]) / N
        out[l] = va[0] + np.einsum("ihw,ihw->hw", va[1:], Gs)
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-8


def test_centred_inverse_in_window_sum_units():
    sc = synth.make_case(30, 20, 1, 9, "f32")
    G = O.polynomial_guidance(sc.guidance.astype(np.float64), 2, "monomial")
    n, H, W = G.shape
    r, eps = 4, 1e-4
    N = O.window_count(H, W, r)
    s = np.stack([O.box_sum(G[i], r) for i in range(n)])
    Sigma = np.empty((n, n, H, W))
    Tm = np.empty((n, n, H, W))
    for i in range(n):
        for j in range(n):
            sij = O.box_sum(G[i] * G[j], r)
            Sigma[i, j] = sij / N - (s[i] / N) * (s[j] / N)
            Tm[i, j] = sij - (s[i] / N) * s[j]
    want = O.hgf_inverse(Sigma, eps)                      # (Sigma + eps E)^-1 by Prop. 1
    got = np.empty_like(want)
    for y in range(H):
        for x in range(W):
            lam_p = N[y, x] * eps
            a = O.hgf_alpha(Tm[:, :, y, x], lam_p)
            got[:, :, y, x] = -N[y, x] * lam_p * a
    assert np.max(np.abs(got - want) / np.max(np.abs(want), axis=(0, 1))) < 1e-8


def test_newton_reciprocal_from_float32_seed():
    rng = np.random.Generator(np.random.PCG64(4))
    d = np.concatenate([1.0 + rng.uniform(0, 1e6, 1000), np.exp(rng.uniform(0, 20, 1000))])
    r = (np.float32(1.0) / d.astype(np.float32)).astype(np.float64)
    for _ in range(2):
        r = r + r * (1.0 - d * r)
    assert np.max(np.abs(r * d - 1.0)) < 4e-16


def test_double_float_error_free_transformations():
    rng = np.random.Generator(np.random.PCG64(6))
    a = rng.standard_normal(10000).astype(np.float32) * np.float32(1e3)
    b = rng.standard_normal(10000).astype(np.float32)
    with np.errstate(over="ignore"):
        s = a + b                                          # two_sum (Knuth)
        bb = s - a
        e = (a - (s - bb)) + (b - bb)
    assert np.array_equal(s.astype(np.float64) + e.astype(np.float64),
                          a.astype(np.float64) + b.astype(np.float64))
    p = a * b                                              # two_prod via an exact float64 FMA
    err = (a.astype(np.float64) * b.astype(np.float64) - p.astype(np.float64)).astype(np.float32)
    assert np.array_equal(p.astype(np.float64) + err.astype(np.float64),
                          a.astype(np.float64) * b.astype(np.float64))
