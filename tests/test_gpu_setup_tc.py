"""GPU parity of the tensor-core set-up of the preconditioner (KRR_Z_FIXED).

Features.  The fixed-point feature map stores the 8-bit codes
q = clamp(rint(z 2^(7-e)), -127, 127), 2^e the smallest power of two
>= sqrt(2/s), so Z ~= 2^e Zs with Zs = q / 128.  Against the oracle's FP64 features z
(Section 2.2) each entry may differ by the rounding to the grid, 2^(e-8)
(2^(e-7) where the clamp acts, |z| near 2^e), plus the error of the cosine's
argument: split BF16 operands give dot products to about 2^-16 of
sum_t |x_t||w_t|, and the FP32 sum with b adds a few ulps of |xw + b|.

Gram.  With caller features the rounding decision is rint(z 2^(7-e)) of the
FP32 input, which numpy reproduces exactly, so the quantised features Zt are
known exactly on the host and the set-up must invert Zt Zt^T + lambda_p I to
FP64 accuracy (the Gram matrix is an exact integer sum).
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


def grid_exponent(maxabs: float) -> int:
    """Smallest e with maxabs <= 2^e."""
    m, E = math.frexp(maxabs)
    return E - 1 if m == 0.5 else E


def quantise(Z32: np.ndarray):
    """Host copy of the fixed-point rounding of FP32 features: (Zt, e)."""
    e = grid_exponent(float(np.max(np.abs(Z32))))
    q = np.clip(np.rint(Z32.astype(np.float32) * np.float32(2.0 ** (7 - e))), -127, 127)
    return q.astype(np.float64) * 2.0 ** (e - 7), e


@pytest.mark.parametrize("cfg,n,s", [(1, 1000, 200), (2, 3000, 2048), (3, 700, 300),
                                     (5, 1333, 257)])
def test_fixed_features_match_oracle(K, h, cfg, n, s):
    P = ks.make_config(cfg, n=n, s=s)
    Zq = torch.full((n, s), -128, dtype=torch.int8, device="cuda")
    e = K.krr_rff_features_fixed(h, dev(P.X), dev(P.W), dev(P.b), Zq)
    assert e == grid_exponent(float(np.float32(math.sqrt(2.0 / s))))
    q = Zq.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(q) <= 127)     # every entry written (-128 is never a code)
    zs = q / 128.0
    z = O.rff_features(P.X, P.W, P.b)
    X64, W64 = P.X.astype(np.float64), P.W.astype(np.float64)
    arg = X64 @ W64 + P.b.astype(np.float64)
    arg_err = 2.0 ** -15 * (np.abs(X64) @ np.abs(W64)) + 1e-6 * (np.abs(arg) + 1.0)
    step = 2.0 ** e
    grid = np.where(np.abs(z) >= step * (127.5 / 128.0) - math.sqrt(2.0 / s) * arg_err,
                    step / 128.0, step / 256.0)
    err = np.abs(step * zs - z)
    bound = grid + math.sqrt(2.0 / s) * arg_err + 1e-12
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("n,s,form", [(1000, 128, "zl"), (4100, 384, "u"), (9000, 2048, "zl"),
                                      (777, 100, "zl"), (500, 40, "u")])
def test_fixed_gram_inverts_the_quantised_operator(K, h, n, s, form):
    """Caller features through KRR_Z_FIXED: the apply inverts Zt Zt^T + lambda_p I
    for the host-quantised Zt (exact Gram; FP64 Cholesky and inverse)."""
    P = ks.make_config(2, n=n, s=s)
    Z = O.rff_features(P.X, P.W, P.b).astype(np.float32)
    Zt, _ = quantise(Z)
    lam_p = 1e-4
    K.krr_precond_setup(h, dev(Z), lam_p, form, z_format="fixed")
    rng = np.random.default_rng(n + s)
    V = rng.standard_normal((n, 2))
    Mv = Zt @ (Zt.T @ V) + lam_p * V
    out = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    K.krr_precond_apply(h, dev(Mv), out)
    got = out.cpu().numpy()
    # The U form stores U = L^-1 Zs^T in FP32: U^T U carries about 2 eps_32
    # relative error, and the apply divides r - U^T U r by lambda_p with
    # ||r|| <= (||Zt||^2 + lambda_p) ||v||.
    # The ZL form is FP64 throughout: its error grows with cond(G) = (||Zt||^2 +
    # lambda_p) / lambda_p at most.
    znorm2 = np.linalg.norm(Zt, 2) ** 2
    kappa = (znorm2 + lam_p) / lam_p
    tol = max(1e-9, 100 * 2.0 ** -53 * kappa) if form == "zl" else 4 * 2.0 ** -24 * kappa
    assert np.linalg.norm(got - V) <= tol * np.linalg.norm(V), \
        float(np.linalg.norm(got - V) / np.linalg.norm(V))
    ref = O.precond_apply(O.precond_setup(Zt, lam_p), Mv)
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_fixed_gram_full_size(K, h):
    """The benched shape (n = 65,536, s = 2,048): several K ranges per tile pair."""
    P = ks.make_config(2, s=2048)
    Z = O.rff_features(P.X, P.W, P.b).astype(np.float32)
    Zt, _ = quantise(Z)
    lam_p = P.lam
    K.krr_precond_setup(h, dev(Z), lam_p, "zl", z_format="fixed")
    rng = np.random.default_rng(65536)
    V = rng.standard_normal((P.n, 1))
    Mv = Zt @ (Zt.T @ V) + lam_p * V
    out = torch.empty_like(dev(V))
    K.krr_precond_apply(h, dev(Mv), out)
    got = out.cpu().numpy()
    kappa = (np.linalg.norm(Zt, 2) ** 2 + lam_p) / lam_p
    tol = max(1e-9, 100 * 2.0 ** -53 * kappa)
    assert np.linalg.norm(got - V) <= tol * np.linalg.norm(V), \
        float(np.linalg.norm(got - V) / np.linalg.norm(V))


def test_fixed_features_full_size_sampled(K, h):
    P = ks.make_config(2, s=2048)
    Zq = torch.full((P.n, P.s), -128, dtype=torch.int8, device="cuda")
    e = K.krr_rff_features_fixed(h, dev(P.X), dev(P.W), dev(P.b), Zq)
    rows = np.unique(np.r_[np.arange(0, P.n, 257), P.n - 1])
    q = Zq.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(q) <= 127)
    zs = q[rows] / 128.0
    z = O.rff_features(P.X[rows], P.W, P.b)
    X64, W64 = P.X[rows].astype(np.float64), P.W.astype(np.float64)
    arg = X64 @ W64 + P.b.astype(np.float64)
    arg_err = 2.0 ** -15 * (np.abs(X64) @ np.abs(W64)) + 1e-6 * (np.abs(arg) + 1.0)
    bound = 2.0 ** (e - 7) + math.sqrt(2.0 / P.s) * arg_err
    assert np.all(np.abs(2.0 ** e * zs - z) <= bound)


def test_mixed_solve_with_each_feature_format(K, h):
    """The mixed solve reaches the FP64 target with fixed-point (default), BF16 and
    FP32 features; the oracle recomputes the residual."""
    P = ks.make_config(2, n=4096, s=256)
    for zf in (-1, 1, 0):
        C = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
        o = K.default_opts(tol=1e-6, precision="mixed", max_iter=6000, z_format=zf)
        rep = K.krr_pcg_solve(h, dev(P.X), P.sigma, P.lam, dev(P.W), dev(P.b), dev(P.Y), C, o,
                              check=False)
        assert rep["status"] == "KRR_OK", (zf, rep)
        assert O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, P.lam)[0] <= 1e-6
