"""GPU parity of the multiple-level sketch (Algorithm 2, Section 4).

Z2 = Z1 S2^T with the SRHT S2 = s2^-1/2 P H D, then Z3 = s3^-1/2 Z2 G^T.
The transform runs in FP32 (log2 m butterfly passes, each adding at most one
rounding of the running sums: |error| <= log2(m) 2^-24 sum_j |z1_j| / sqrt(s2)
per entry); the projection runs on the tensor cores from split BF16 operands
(2^-16 of sum |z2||g| per entry, relative).  With G = sqrt(s3) I the
projection is the identity, which isolates the transform.
"""
import math

import numpy as np
import pytest

import krr_synth as ks
from oracle import krr_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr
    return _krr


@pytest.fixture()
def h(K):
    hh = K.Handle()
    yield hh
    torch.cuda.synchronize()
    hh.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,s1,m,s2", [(1000, 300, 512, 256), (333, 1024, 1024, 64)])
def test_srht_isolated_matches_oracle(K, h, n, s1, m, s2):
    P = ks.make_config(2, n=n, s=s1)
    Z1 = O.rff_features(P.X, P.W, P.b).astype(np.float32)
    signs, rows = ks.srht_draw(n + m, m, s2)
    G = (math.sqrt(s2) * np.eye(s2)).astype(np.float32)   # exact in BF16 for s2 = 4^j
    Z3 = torch.full((n, s2), float("nan"), dtype=torch.float32, device="cuda")
    K.krr_multilevel_features(h, dev(Z1), signs, rows, dev(G), Z3)
    ref = O.srht_apply(Z1, signs, rows)
    bound = (2.0 ** -16 * np.abs(ref)
             + math.log2(m) * 2.0 ** -23 * np.abs(Z1).sum(axis=1, keepdims=True) / math.sqrt(s2))
    err = np.abs(Z3.cpu().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("n,s1,m,s2,s3", [(1500, 256, 256, 192, 100), (700, 700, 1024, 512, 333)])
def test_multilevel_features_match_oracle(K, h, n, s1, m, s2, s3):
    P = ks.make_config(1, n=n, s=s1)
    Z1 = O.rff_features(P.X, P.W, P.b).astype(np.float32)
    signs, rows = ks.srht_draw(3 * n, m, s2)
    G = ks.gaussian_draw(5 * n, s3, s2)
    Z3 = torch.full((n, s3), float("nan"), dtype=torch.float32, device="cuda")
    K.krr_multilevel_features(h, dev(Z1), signs, rows, dev(G), Z3)
    Z2 = O.srht_apply(Z1, signs, rows)
    ref = O.gaussian_projection(Z2, G)
    G64 = np.abs(G.astype(np.float64))
    e2 = math.log2(m) * 2.0 ** -23 * np.abs(Z1).sum(axis=1, keepdims=True) / math.sqrt(s2)
    bound = (2.0 ** -15 * (np.abs(Z2) @ G64.T) + e2 * G64.sum(axis=1)[None, :]) / math.sqrt(s3)
    err = np.abs(Z3.cpu().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_multilevel_arguments_checked(K, h):
    Z1 = dev(np.zeros((10, 6), np.float32))
    G = dev(np.ones((2, 4), np.float32))
    Z3 = torch.empty((10, 2), dtype=torch.float32, device="cuda")
    signs, rows = ks.srht_draw(1, 8, 4)
    bad_rows = rows.copy()
    bad_rows[0] = 8
    with pytest.raises(K.KrrError):
        K.krr_multilevel_features(h, Z1, signs, bad_rows, G, Z3)
    bad_signs = signs.copy()
    bad_signs[3] = 2
    with pytest.raises(K.KrrError):
        K.krr_multilevel_features(h, Z1, bad_signs, rows, G, Z3)
    s12, r12 = np.ones(12, np.int8), np.arange(4, dtype=np.int32)
    with pytest.raises(K.KrrError):      # m not a power of two
        K.krr_multilevel_features(h, Z1, s12, r12, G, Z3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_algorithm2_solve(K, h, precision):
    """Algorithm 2 end to end: RFF features (s1), SRHT (s2), Gaussian projection
    (s3), the Woodbury preconditioner from Z3 and PCG with it (precond = 2)."""
    P = ks.make_config(1, n=2000, s=512)
    s2, s3 = 256, 192
    signs, rows = ks.srht_draw(21, 512, s2)
    G = ks.gaussian_draw(22, s3, s2)
    Xd = dev(P.X)
    Z1 = torch.empty((P.n, 512), dtype=torch.float32, device="cuda")
    K.krr_rff_features(h, Xd, dev(P.W), dev(P.b), Z1)
    Z3 = torch.empty((P.n, s3), dtype=torch.float32, device="cuda")
    K.krr_multilevel_features(h, Z1, signs, rows, dev(G), Z3)
    K.krr_precond_setup(h, Z3, P.lam, "zl",
                        z_format="fixed" if precision == "mixed" else "fp32")
    C = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
    tol = 1e-8 if precision == "fp64" else 1e-6
    o = K.default_opts(tol=tol, precision=precision, precond=2, max_iter=6000)
    rep = K.krr_pcg_solve(h, Xd, P.sigma, P.lam, None, None, dev(P.Y), C, o)
    assert rep["status"] == "KRR_OK"
    assert O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, P.lam)[0] <= tol
    if precision == "fp64":
        ref = O.krr_multilevel_pcg_solve(P.X, P.Y, P.sigma, P.lam, P.W, P.b, signs, rows, G,
                                         tol=tol, max_iter=6000)
        it, it_ref = rep["iters"][0], int(ref["iters"][0])
        assert abs(it - it_ref) <= max(3, 0.05 * it_ref), (it, it_ref)


def test_precond_keep_needs_a_matching_setup(K, h):
    P = ks.make_config(1, n=300, s=32)
    C = torch.zeros((300, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-8, precision="fp64", precond=2)
    with pytest.raises(K.KrrError):
        K.krr_pcg_solve(h, dev(P.X), P.sigma, P.lam, None, None, dev(P.Y), C, o)
