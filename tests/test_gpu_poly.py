"""GPU parity of the polynomial-kernel path (Section 6's kernel
k(x, z) = (gamma x^T z + c)^q with the TensorSketch features of Section 2.2).

* Features: on points with small integer coordinates (gamma = c = 1) every
  product and sum is an integer below 2^24, so the CUDA sketch must equal the
  oracle's enumeration of the d~^q monomials exactly -- this pins the hash
  and sign indexing (which bucket, which sign, mod s).  On Gaussian points the
  FP32 sums are compared within 1e-5 of the sum of the absolute terms.
* Products: FP64 against the oracle's explicit kernel (1e-12 of
  sum_j |P_ij||v_j|); the tensor-core product against the kernel of the
  rounded points (FP16 / BF16 / split BF16), FP32 epilogue.
* Solves: Algorithm 1 with the TensorSketch preconditioner against the
  oracle's, and the mixed-precision solve to the FP64 target.
"""
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


def tables(seed, d, q, s, c):
    return ks.tensorsketch_draw(seed, d + (1 if c > 0 else 0), q, s)


@pytest.mark.parametrize("n,d,q,s,c", [(300, 8, 2, 64, 1.0), (200, 6, 3, 50, 1.0),
                                       (150, 9, 2, 37, 0.0), (100, 5, 1, 16, 1.0)])
def test_tensorsketch_exact_on_integer_points(K, h, n, d, q, s, c):
    rng = np.random.default_rng(n + d + q)
    X = rng.integers(-3, 4, size=(n, d)).astype(np.float32)
    hs, g = tables(10 + q, d, q, s, c)
    Z = torch.full((n, s), float("nan"), dtype=torch.float32, device="cuda")
    K.krr_tensorsketch_features(h, dev(X), hs, g, s, 1.0, c, Z)
    ref = O.tensorsketch_features(X, hs, g, s, 1.0, c)
    assert np.array_equal(Z.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("n,d,q,s,gamma,c", [(500, 16, 2, 128, 0.0625, 1.0),
                                             (300, 6, 3, 64, 0.5, 2.0)])
def test_tensorsketch_matches_oracle_fp32(K, h, n, d, q, s, gamma, c):
    rng = np.random.default_rng(3 * n + d)
    X = rng.standard_normal((n, d)).astype(np.float32)
    hs, g = tables(20 + q, d, q, s, c)
    Z = torch.empty((n, s), dtype=torch.float32, device="cuda")
    K.krr_tensorsketch_features(h, dev(X), hs, g, s, gamma, c, Z)
    ref = O.tensorsketch_features(X, hs, g, s, gamma, c)
    scale = O.tensorsketch_features(np.abs(X), hs, np.ones_like(g), s, gamma, c)
    err = np.abs(Z.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float(np.max(err / (scale + 1e-30)))


def test_tensorsketch_rejects_bad_tables(K, h):
    X = dev(np.zeros((4, 3), np.float32))
    hs, g = tables(1, 3, 2, 8, 0.0)
    Z = torch.empty((4, 8), dtype=torch.float32, device="cuda")
    bad = hs.copy()
    bad[1, 2] = 8
    with pytest.raises(K.KrrError):
        K.krr_tensorsketch_features(h, X, bad, g, 8, 1.0, 0.0, Z)
    sg = g.copy()
    sg[0, 0] = 0
    with pytest.raises(K.KrrError):
        K.krr_tensorsketch_features(h, X, hs, sg, 8, 1.0, 0.0, Z)


@pytest.mark.parametrize("nr,nc,d,q,k,shift", [(700, 700, 16, 2, 1, 1e-3), (300, 517, 10, 3, 4, 0.0)])
def test_poly_product_fp64(K, h, nr, nc, d, q, k, shift):
    rng = np.random.default_rng(nr + nc + q)
    Xc = rng.standard_normal((nc, d)).astype(np.float32)
    Xr = Xc if nr == nc else rng.standard_normal((nr, d)).astype(np.float32)
    V = rng.standard_normal((nc, k))
    gamma, c = 1.0 / d, 1.0
    Q = torch.empty((nr, k), dtype=torch.float64, device="cuda")
    Xc_d = dev(Xc)
    K.krr_kernel_matvec_poly(h, Xc_d if nr == nc else dev(Xr), Xc_d, gamma, c, q, shift, dev(V), Q,
                             "fp64")
    P = O.poly_kernel(Xr, Xc, gamma, c, q)
    ref = P @ V + (shift * V if shift else 0.0)
    scale = np.abs(P) @ np.abs(V) + (shift * np.abs(V) if shift else 0.0)
    err = np.abs(Q.cpu().numpy() - ref)
    assert np.all(err <= 1e-12 * scale), float(np.max(err / scale))


def rounded(X, prec):
    t = torch.from_numpy(X.astype(np.float32))
    if prec == "bf16x3":
        hi = t.to(torch.bfloat16).double()
        lo = (t.double() - hi).float().to(torch.bfloat16).double()
        return hi.numpy(), lo.numpy()
    return t.to(torch.float16 if prec == "fp16" else torch.bfloat16).double().numpy()


@pytest.mark.parametrize("prec,n,d,q,k", [("fp16", 1000, 16, 2, 1), ("bf16", 777, 64, 3, 3),
                                          ("bf16x3", 900, 32, 2, 10), ("fp16", 3000, 100, 2, 1)])
def test_poly_product_tensor_core(K, h, prec, n, d, q, k):
    rng = np.random.default_rng(n + d + k)
    X = rng.standard_normal((n, d)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    gamma, c = 1.0 / d, 1.0
    Q = torch.full((n, k), float("nan"), dtype=torch.float32, device="cuda")
    Xd = dev(X)
    K.krr_kernel_matvec_poly(h, Xd, Xd, gamma, c, q, 0.25, dev(V), Q, prec)
    if prec == "bf16x3":
        hi, lo = rounded(X, prec)
        S = hi @ hi.T + lo @ hi.T + hi @ lo.T
        A = np.abs(hi + lo)
    else:
        Xh = rounded(X, prec)
        S = Xh @ Xh.T
        A = np.abs(Xh)
    V64 = V.astype(np.float64)
    P = (gamma * S + c) ** q
    ref = P @ V64 + 0.25 * V64
    scale = ((gamma * (A @ A.T) + c) ** q) @ np.abs(V64) + 0.25 * np.abs(V64)
    err = np.abs(Q.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 1e-5 * scale), float(np.max(err / scale))


def poly_problem(n, d, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    w = rng.standard_normal(d)
    y = np.sin(X.astype(np.float64) @ w / np.sqrt(d)) + 0.1 * rng.standard_normal(n)
    return X, y.reshape(n, 1)


def test_poly_pcg_fp64_matches_oracle(K, h):
    n, d, q, s, lam = 800, 8, 2, 96, 1e-3
    gamma, c = 1.0 / d, 1.0
    X, Y = poly_problem(n, d, 5)
    hs, g = tables(77, d, q, s, c)
    C = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-8, precision="fp64", max_iter=2000)
    rep = K.krr_poly_pcg_solve(h, dev(X), gamma, c, q, lam, hs, g, s, dev(Y), C, o)
    assert rep["status"] == "KRR_OK", rep
    ref = O.krr_poly_pcg_solve(X, Y, gamma, c, q, lam, hs, g, s, tol=1e-8, max_iter=2000)
    assert abs(rep["iters"][0] - int(ref["iters"][0])) <= 3, (rep["iters"], ref["iters"])
    A = O.poly_kernel(X, X, gamma, c, q) + lam * np.eye(n)
    Cx = np.linalg.solve(A, Y)
    got = C.cpu().numpy()
    res = np.linalg.norm(Y - A @ got) / np.linalg.norm(Y)
    assert res <= 1e-8
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(got - Cx) <= 10 * kappa * 1e-8 * np.linalg.norm(Cx)


@pytest.mark.parametrize("inner", ["fp16", "bf16"])
def test_poly_pcg_mixed_reaches_fp64_target(K, h, inner):
    n, d, q, s, lam = 4096, 16, 2, 256, 1e-4
    gamma, c = 1.0 / d, 1.0
    X, Y = poly_problem(n, d, 9)
    hs, g = tables(78, d, q, s, c)
    C = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-6, precision="mixed", max_iter=6000, inner_precision=inner)
    rep = K.krr_poly_pcg_solve(h, dev(X), gamma, c, q, lam, hs, g, s, dev(Y), C, o, check=False)
    assert rep["status"] == "KRR_OK", rep
    P = O.poly_kernel(X, X, gamma, c, q)
    got = C.cpu().numpy()
    res = np.linalg.norm(Y - P @ got - lam * got) / np.linalg.norm(Y)
    assert res <= 1e-6, (res, rep)


def test_poly_plain_cg_and_gaussian_state_untouched(K, h):
    """A polynomial solve without preconditioner (plain CG), then a Gaussian
    product on the same handle: the handle's kernel goes back to the Gaussian."""
    n, d, q, lam = 500, 6, 3, 1e-2
    X, Y = poly_problem(n, d, 11)
    C = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-8, precision="fp64", precond=0, max_iter=3000)
    rep = K.krr_poly_pcg_solve(h, dev(X), 1.0 / d, 1.0, q, lam, None, None, 0, dev(Y), C, o)
    assert rep["status"] == "KRR_OK"
    A = O.poly_kernel(X, X, 1.0 / d, 1.0, q) + lam * np.eye(n)
    assert np.linalg.norm(Y - A @ C.cpu().numpy()) <= 1e-8 * np.linalg.norm(Y)
    V = np.random.default_rng(1).standard_normal((n, 1))
    Q = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    Xd = dev(X)
    K.krr_kernel_matvec(h, Xd, Xd, 2.0, 0.0, dev(V), Q, "fp64")
    ref = O.gaussian_kernel(X, X, 2.0) @ V
    assert np.allclose(Q.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
