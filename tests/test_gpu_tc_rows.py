"""Tensor-core products with a row set other than the columns: prediction
f = K(X_te, X) c (Section 1) and the derivative product (D o K) V of the
hyper-parameter gradient, on FP16, BF16 and split-BF16 points.

Both sides are rounded with the training set's mean and scale:
xh = round(sqrt(log2 e)/sigma (x - mean_train)), so the product is the
Gaussian kernel exp2(-||xh_i - xh_j||^2 / 2) of the rounded points; the
oracle evaluates exactly that (and D o K = -2 ln 2 log2(K) K of it) in FP64.
The device arithmetic is the fused product's: FP32 accumulation of exact
products, ex2.approx, FP32 tile sums merged in FP64 (bound 1e-5 of
sum_j |K_ij||v_j|).  The derivative contracts exp2(S) S and exp2(S) in FP32
and subtracts the row and column terms afterwards, so its rounding scales with
sum_j K_ij (|S_ij| + nh_i/2 + nh_j/2) |v_j| instead.
"""
import math

import numpy as np
import pytest

import krr_synth as ks
from oracle import krr_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOG2E = 1.0 / math.log(2.0)
SIG_H = 1.0 / math.sqrt(math.log(2.0))


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


def to_dtype(u, dtype):
    return torch.from_numpy(u.astype(np.float32)).to(dtype).double().numpy()


def rounded_pair(Xr, Xc, sigma, prec):
    """Rounded rows and columns in FP64 (split points as (hi, lo) pairs)."""
    mu = Xc.astype(np.float64).mean(axis=0)
    sc = math.sqrt(LOG2E) / sigma
    ur = sc * (Xr.astype(np.float64) - mu)
    uc = sc * (Xc.astype(np.float64) - mu)
    if prec == "bf16x3":
        hr = to_dtype(ur, torch.bfloat16)
        hc = to_dtype(uc, torch.bfloat16)
        return (hr, to_dtype(ur - hr, torch.bfloat16)), (hc, to_dtype(uc - hc, torch.bfloat16))
    dt = torch.float16 if prec == "fp16" else torch.bfloat16
    return to_dtype(ur, dt), to_dtype(uc, dt)


def log2_kernel(R, Cc, prec):
    """log2 K_ij = S_ij - nh_i/2 - nh_j/2 and S of the device's arithmetic, in FP64."""
    if prec == "bf16x3":
        (hr, lr), (hc, lc) = R, Cc
        S = hr @ hc.T + lr @ hc.T + hr @ lc.T
        nr = np.sum((hr + lr) ** 2, axis=1)
        nc = np.sum((hc + lc) ** 2, axis=1)
    else:
        S = R @ Cc.T
        nr = np.sum(R * R, axis=1)
        nc = np.sum(Cc * Cc, axis=1)
    return S - 0.5 * nr[:, None] - 0.5 * nc[None, :], S, nr, nc


CASES = [("fp16", 5, 700, 333, 1), ("bf16", 2, 1300, 517, 3), ("bf16x3", 2, 1100, 260, 2),
         ("fp16", 3, 600, 129, 10)]


@pytest.mark.parametrize("prec,cfg,n,m,k", CASES)
def test_predict_tensor_core_rows(K, h, prec, cfg, n, m, k):
    P = ks.make_config(cfg, n=n, m=m, s=16) if cfg != 3 else ks.make_config(3, n=n, s=16)
    Xte = P.Xte if P.Xte is not None else ks.make_config(3, n=m, s=16).X
    rng = np.random.default_rng(n + m + k)
    Cc = rng.standard_normal((n, k))
    F = torch.full((Xte.shape[0], k), float("nan"), dtype=torch.float64, device="cuda")
    K.krr_predict(h, dev(P.X), dev(Xte), P.sigma, dev(Cc), F, prec)
    R, Cp = rounded_pair(Xte, P.X, P.sigma, prec)
    L, _, _, _ = log2_kernel(R, Cp, prec)
    Kt = np.exp2(L)
    ref = Kt @ Cc
    scale = Kt @ np.abs(Cc)
    err = np.abs(F.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * scale + 1e-30), float(np.max(err / scale))
    # and the rounded kernel stays close to the exact one
    exact = O.predict(P.X, Xte, Cc, P.sigma)
    assert np.all(np.abs(F.cpu().numpy() - exact) <= 5e-2 * scale)


@pytest.mark.parametrize("prec,cfg,n,m,k", CASES + [("fp16", 5, 500, 500, 7)])
def test_dsigma_tensor_core_rows(K, h, prec, cfg, n, m, k):
    P = ks.make_config(cfg, n=n, m=m, s=16) if cfg != 3 else ks.make_config(3, n=n, s=16)
    same = (n == m)
    Xr = P.X if same else (P.Xte if P.Xte is not None else ks.make_config(3, n=m, s=16).X)
    rng = np.random.default_rng(2 * n + m + k)
    V = rng.standard_normal((n, k))
    Q = torch.full((Xr.shape[0], k), float("nan"), dtype=torch.float64, device="cuda")
    Xc_d = dev(P.X)
    K.krr_kernel_dsigma_matvec(h, Xc_d if same else dev(Xr), Xc_d, P.sigma, dev(V), Q,
                               precision=prec)
    R, Cp = rounded_pair(Xr, P.X, P.sigma, prec)
    L, S, nr, nc = log2_kernel(R, Cp, prec)
    Kt = np.exp2(L)
    DK = -2.0 * math.log(2.0) * L * Kt
    ref = DK @ V
    scale = (Kt * (np.abs(S) + 0.5 * nr[:, None] + 0.5 * nc[None, :] + 1.0)) @ np.abs(V)
    err = np.abs(Q.cpu().numpy() - ref)
    assert np.all(err <= 1e-5 * scale), float(np.max(err / scale))
    if prec != "bf16x3":
        # the same as the oracle's D o K evaluated on the rounded points
        Xh_r, Xh_c = R, Cp
        G = O.kernel_dlogsigma(Xh_r, Xh_c, SIG_H)
        assert np.all(np.abs(Q.cpu().numpy() - G @ V) <= 1e-5 * scale)
