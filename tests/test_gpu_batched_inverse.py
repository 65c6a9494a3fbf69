"""Batched (lambda E + S_i)^-1 on the GPU (hgf_batched_inverse): Prop. 1's recursion and the
per-matrix Cholesky route against the oracle's Prop. 1 inverse (float64, pinned against LU /
Cholesky solves on CPU), on seeded Gram matrices S_i = sum_k x_k x_k^T of 25 samples
x_k ~ U[0,1]^n.

Bound per matrix: max|X - X*| / max|X*| <= 10 n u (1 + ||S||/lambda) cond(lambda E + S), with u
the unit roundoff of the arithmetic (2^-53 for float64, 2^-47 for double-float pairs of float32,
2^-24 for float32): the recursion's error
grows with ||S||/lambda (its gamma denominators) times the conditioning of the solve."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


@pytest.mark.parametrize("n", [1, 3, 9, 19])
@pytest.mark.parametrize("lam", [1e-2, 1.0])
def test_batched_inverse_parity(ctx, n, lam, capsys):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    count = 3001  # ragged last block
    S = synth.gram_batch(count, n, seed=100 + n)
    ref = O.hgf_inverse(np.moveaxis(S, 0, -1), lam)          # (n, n, count)
    ref = np.moveaxis(ref, -1, 0)
    A = S + lam * np.eye(n)[None]
    ev = np.linalg.eigvalsh(A)
    cond = ev[:, -1] / ev[:, 0]
    growth = 1.0 + np.linalg.norm(S, 2, axis=(1, 2)) / lam
    Sd = torch.from_numpy(synth.pack_upper(S)).cuda()
    rows, cols = np.triu_indices(n)
    for method in ("prop1", "cholesky"):
        for prec, u in (("f64", 2.0 ** -53), ("df64", 2.0 ** -47), ("f32", 2.0 ** -24)):
            out = hgf.hgf_batched_inverse(ctx, Sd, n, lam, method=method, precision=prec)
            torch.cuda.synchronize()
            got = out.cpu().numpy()                            # (P, count)
            want = ref[:, rows, cols].T
            err = np.max(np.abs(got - want), axis=0) / np.max(np.abs(want), axis=0)
            bound = 10 * n * u * growth * cond
            assert np.all(np.isfinite(got)), (method, prec)
            with capsys.disabled():
                print(f"\nn={n} lambda={lam} {method} {prec}: max err {err.max():.2e}, "
                      f"max err/bound {np.max(err / bound):.2e}")
            if prec == "f64" or np.all(bound < 1e-1):
                assert np.all(err <= bound), (method, prec, float(np.max(err / bound)))


def test_batched_inverse_closed_forms(ctx):
    """n = 1: 1/(lambda + s); diagonal S: 1/(lambda + s_k) on the diagonal, 0 elsewhere."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    s = np.array([0.0, 0.5, 3.0, 100.0])
    S1 = torch.from_numpy(s[None].copy()).cuda()
    for method in ("prop1", "cholesky"):
        got = hgf.hgf_batched_inverse(ctx, S1, 1, 0.25, method=method).cpu().numpy()[0]
        np.testing.assert_allclose(got, 1.0 / (0.25 + s), rtol=1e-15)
    d = np.diag([0.0, 1.0, 2.0, 7.5])[None]
    Sd = torch.from_numpy(synth.pack_upper(d)).cuda()
    for method in ("prop1", "cholesky"):
        got = hgf.hgf_batched_inverse(ctx, Sd, 4, 0.5, method=method).cpu().numpy()[:, 0]
        want = synth.pack_upper(np.diag(1.0 / (0.5 + np.diag(d[0])))[None])[:, 0]
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-16)


def test_batched_inverse_argument_errors(ctx):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    S = torch.zeros((6, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(hgf.HGFError) as ei:
        hgf.hgf_batched_inverse(ctx, S, 3, 0.0)
    assert ei.value.status == hgf.HGF_EINVAL
    S11 = torch.zeros((66, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(hgf.HGFError) as ei:
        hgf.hgf_batched_inverse(ctx, S11, 11, 1.0)
    assert ei.value.status == hgf.HGF_EUNSUPPORTED
