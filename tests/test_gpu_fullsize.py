"""Element-wise parity of the tensor-core products at the benched sizes.

The small parity tests (n <= 3000) never leave the first work item of a CTA:
with 152 persistent CTAs each takes at most one (row tile, column chunk)
item, the TMA ring never wraps and neither TMEM accumulator is reused.  At
n = 32,768 - 65,536 each CTA takes several items of tens of 256-column tiles,
so the ring wraps many times and both accumulators alternate.  These tests
run the products in exactly the launch configuration the solvers use (the
fixed wave-balance plan, or the symmetric plan) on workload-2-shaped points
(the 64-dimensional Gaussian mixture, sigma = 8) and compare a few hundred
sampled rows, spread over every row tile and including the ragged last tile,
element by element with the FP64 oracle evaluated on those rows only:

* FP16 / BF16 points: the Gaussian kernel of the rounded points
  xh = round(sqrt(log2 e)/sigma (x - mean)), bound 1e-5 of sum_j |K_ij||v_j|
  (FP32 accumulation of exact products, ex2.approx, FP32 tile sums);
* split points (hi + lo, three MMAs): emulated in FP64, same bound;
* the digit-sliced HP product: the exact kernel of the FP32 points, bound
  2e-12 of sum_j |K_ij||v_j|.
"""
import math

import numpy as np
import pytest

import krr_synth as ks
from oracle import krr_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOG2E = 1.0 / math.log(2.0)
SIG_H = 1.0 / math.sqrt(math.log(2.0))   # exp2(-|d|^2/2) = exp(-|d|^2 / (2 SIG_H^2))


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


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct rows: one per 128-row tile first, then random ones, and
    always the first and last row."""
    rng = np.random.default_rng(seed)
    tiles = np.arange(0, n, 128)
    per_tile = tiles + rng.integers(0, 128, size=tiles.size)
    per_tile = per_tile[per_tile < n]
    pick = set(per_tile[rng.permutation(per_tile.size)[: max(count - 2, 0)]].tolist())
    pick.update({0, n - 1})
    while len(pick) < count:
        pick.add(int(rng.integers(0, n)))
    return np.array(sorted(pick))


def rounded(X, sigma, dtype):
    X64 = X.astype(np.float64)
    u = (math.sqrt(LOG2E) / sigma) * (X64 - X64.mean(axis=0))
    return torch.from_numpy(u.astype(np.float32)).to(dtype).to(torch.float64).numpy()


def run_product(K, h, X, V, sigma, shift, prec, dtype=torch.float32, plan=0):
    Xd = torch.from_numpy(X).cuda()
    Vd = torch.from_numpy(V).cuda()
    Q = torch.full(V.shape, float("nan"), dtype=dtype, device="cuda")
    h.set_autotune(plan)
    try:
        K.krr_kernel_matvec(h, Xd, Xd, sigma, shift, Vd, Q, prec)
    finally:
        h.set_autotune(0)
    torch.cuda.synchronize()
    return Q.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,k,prec,plan", [
    (65536, 1, "fp16", 0),        # the benched product, headline size
    (65536, 1, "fp16", 2),        # the symmetric plan at the headline size
    (65536, 1, "fp16", 3),        # the symmetric plan, 8 epilogue warps
    (40000, 10, "fp16", 0),       # multi-RHS, ragged last tile
    (32768, 1, "bf16", 0),
    (33000, 10, "bf16", 0),
])
def test_rounded_point_product_full_size(K, h, n, k, prec, plan):
    P = ks.make_config(2, n=n, s=8)
    rng = np.random.default_rng(n + k + plan)
    V = rng.standard_normal((n, k)).astype(np.float32)
    shift = P.lam
    got = run_product(K, h, P.X, V, P.sigma, shift, prec, plan=plan)
    rows = sample_rows(n, 256, n + k)
    Xh = rounded(P.X, P.sigma, torch.float16 if prec == "fp16" else torch.bfloat16)
    V64 = V.astype(np.float64)
    ref = O.kernel_matvec_blocked(Xh[rows], Xh, V64, SIG_H) + shift * V64[rows]
    scale = O.kernel_matvec_blocked(Xh[rows], Xh, np.abs(V64), SIG_H) + shift * np.abs(V64[rows])
    err = np.abs(got[rows] - ref)
    assert np.all(np.isfinite(got)), "rows left unwritten"
    assert np.all(err <= 1e-5 * scale), float(np.max(err / scale))


@pytest.mark.parametrize("n,k", [(32768, 1), (36000, 10)])
def test_split_point_product_full_size(K, h, n, k):
    P = ks.make_config(2, n=n, s=8)
    rng = np.random.default_rng(3 * n + k)
    V = rng.standard_normal((n, k)).astype(np.float32)
    got = run_product(K, h, P.X, V, P.sigma, 0.0, "bf16x3")
    rows = sample_rows(n, 256, 7 * n + k)
    X64 = P.X.astype(np.float64)
    u = (math.sqrt(LOG2E) / P.sigma) * (X64 - X64.mean(axis=0))
    to_bf16 = lambda a: torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    hi = to_bf16(u)
    lo = to_bf16(u - hi)
    xs = hi + lo
    nh = np.sum(xs * xs, axis=1)
    S = hi[rows] @ hi.T + lo[rows] @ hi.T + hi[rows] @ lo.T
    Kt = np.exp2(S - 0.5 * nh[rows, None] - 0.5 * nh[None, :])
    V64 = V.astype(np.float64)
    ref, scale = Kt @ V64, Kt @ np.abs(V64)
    err = np.abs(got[rows] - ref)
    assert np.all(np.isfinite(got))
    assert np.all(err <= 1e-5 * scale), float(np.max(err / scale))


@pytest.mark.parametrize("n,k", [(32768, 1), (34000, 3)])
def test_hp_product_full_size(K, h, n, k):
    P = ks.make_config(2, n=n, s=8)
    rng = np.random.default_rng(5 * n + k)
    V = rng.standard_normal((n, k))
    got = run_product(K, h, P.X, V, P.sigma, P.lam, "hp", dtype=torch.float64)
    rows = sample_rows(n, 256, 11 * n + k)
    ref = O.kernel_matvec_blocked(P.X[rows], P.X, V, P.sigma) + P.lam * V[rows]
    scale = O.kernel_matvec_blocked(P.X[rows], P.X, np.abs(V), P.sigma) + P.lam * np.abs(V[rows])
    err = np.abs(got[rows] - ref)
    assert np.all(np.isfinite(got))
    assert np.all(err <= 2e-12 * scale), float(np.max(err / scale))
