"""GPU parity of the tcgen05 fused kernel product and the mixed-precision solve.

The BF16 product (and, with 11-bit significands, the FP16 one) evaluates the
Gaussian kernel of the BF16-rounded, centred,
scaled points xh = bf16(sqrt(log2(e))/sigma (x - mean)), i.e.
K_ij = exp2(-||xh_i - xh_j||^2 / 2).  The oracle evaluates exactly that kernel
on the same rounded points (rounding done on the CPU by torch, round to
nearest even like the device), so the comparison isolates the tensor-core
arithmetic: FP32 accumulation of exact BF16 products, ex2.approx (rel. error
~2^-22) and FP32 sums of at most 256 terms per tile before FP64 chunk sums.
"""
import math

import numpy as np
import pytest

import krr_synth as ks
from oracle import krr_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOG2E = 1.0 / math.log(2.0)


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


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def rounded_points(X, sigma, dtype=None):
    """xh = bf16(sqrt(log2 e)/sigma * (x - mean)) in FP64 (mean in FP64); fp16 with
    ``dtype=torch.float16``."""
    X64 = X.astype(np.float64)
    mu = X64.mean(axis=0)
    scale = math.sqrt(LOG2E) / sigma
    xf = (scale * (X64 - mu)).astype(np.float32)
    return torch.from_numpy(xf).to(dtype or torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("n,d,k", [(1000, 37, 1), (777, 64, 3), (1300, 100, 10), (300, 8, 16),
                                   (520, 64, 2)])
def test_matvec_bf16_matches_rounded_oracle(K, h, n, d, k):
    rng = np.random.default_rng(n + d + k)
    X = rng.standard_normal((n, d)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    sigma = math.sqrt(d)
    Q = torch.empty((n, k), dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.0, torch.from_numpy(V).cuda(), Q, "bf16")
    Xh = rounded_points(X, sigma)
    sig_h = 1.0 / math.sqrt(math.log(2.0))   # exp2(-|d|^2/2) = exp(-|d|^2 / (2 sig_h^2))
    Kh = O.gaussian_kernel(Xh, Xh, sig_h)
    ref = Kh @ V.astype(np.float64)
    scale = Kh @ np.abs(V.astype(np.float64))
    got = Q.cpu().numpy().astype(np.float64)
    # FP32 exponentials contracted in FP32
    assert np.all(np.abs(got - ref) <= 1e-5 * scale), np.max(np.abs(got - ref) / scale)
    # and against the exact kernel of the unrounded points: the BF16 rounding of x
    # moves -||x_i - x_j||^2/(2 sigma^2) by about 2^-8 of its size
    exact = O.gaussian_kernel(X, X, sigma) @ V.astype(np.float64)
    assert np.all(np.abs(got - exact) <= 3e-2 * scale)


@pytest.mark.parametrize("n,d,k", [(1000, 37, 1), (777, 64, 3), (1300, 100, 10), (300, 8, 16)])
def test_matvec_fp16_matches_rounded_oracle(K, h, n, d, k):
    """KRR_FP16: the same product on FP16-rounded points (11-bit significands)."""
    rng = np.random.default_rng(7 * n + d + k)
    X = rng.standard_normal((n, d)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    sigma = math.sqrt(d)
    Q = torch.empty((n, k), dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.0, torch.from_numpy(V).cuda(), Q, "fp16")
    Xh = rounded_points(X, sigma, torch.float16)
    sig_h = 1.0 / math.sqrt(math.log(2.0))
    Kh = O.gaussian_kernel(Xh, Xh, sig_h)
    ref = Kh @ V.astype(np.float64)
    scale = Kh @ np.abs(V.astype(np.float64))
    got = Q.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * scale), np.max(np.abs(got - ref) / scale)
    # eight times finer point rounding than BF16 (2^-11 against 2^-8 relative)
    exact = O.gaussian_kernel(X, X, sigma) @ V.astype(np.float64)
    err16 = np.max(np.abs(got - exact) / scale)
    Qb = torch.empty_like(Q)
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.0, torch.from_numpy(V).cuda(), Qb, "bf16")
    err_b = np.max(np.abs(Qb.cpu().numpy().astype(np.float64) - exact) / scale)
    assert err16 <= 5e-3 and err16 < err_b / 3, (err16, err_b)


@pytest.mark.parametrize("n,d,k", [(777, 64, 3), (300, 8, 16), (2000, 784, 10), (400, 64, 1)])
def test_matvec_bf16p_matches_emulated_roundings(K, h, n, d, k):
    """Two-GEMM variant: P = bf16(exp2(xh_i.xh_j)) and Vt = bf16(ra_j v_j) on the
    tensor cores; both roundings emulated in FP64 (round to nearest even)."""
    rng = np.random.default_rng(n + d + k + 3)
    X = rng.standard_normal((n, d)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    sigma = math.sqrt(d)
    Q = torch.empty((n, k), dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.0, torch.from_numpy(V).cuda(), Q, "bf16p")
    got = Q.cpu().numpy().astype(np.float64)
    Xh = rounded_points(X, sigma)
    S = Xh @ Xh.T
    P = bf16_round(np.exp2(S))
    ra = np.exp2(-0.5 * np.sum(Xh * Xh, axis=1)).astype(np.float32).astype(np.float64)
    Vt = bf16_round((ra[:, None] * V.astype(np.float64)).astype(np.float32))
    emul = ra[:, None] * (P @ Vt)
    Kh = O.gaussian_kernel(Xh, Xh, 1.0 / math.sqrt(math.log(2.0)))
    scale = Kh @ np.abs(V.astype(np.float64))
    assert np.all(np.abs(got - emul) <= 1e-3 * scale), np.max(np.abs(got - emul) / scale)
    # each term carries two BF16 roundings of at most 2^-9 relative
    ref = Kh @ V.astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2 ** -8 * scale), np.max(np.abs(got - ref) / scale)


def split_points(X, sigma):
    """hi = bf16(u), lo = bf16(u - hi) for u = sqrt(log2 e)/sigma (x - mean), in FP64."""
    X64 = X.astype(np.float64)
    u = (math.sqrt(LOG2E) / sigma) * (X64 - X64.mean(axis=0))
    hi = bf16_round(u.astype(np.float32))
    lo = bf16_round((u - hi).astype(np.float32))
    return hi, lo


@pytest.mark.parametrize("n,d,k", [(1000, 37, 1), (600, 64, 2), (777, 54, 4), (300, 8, 16)])
def test_matvec_bf16x3_matches_split_oracle(K, h, n, d, k):
    """Split points xh = hi + lo: S = hi.hi + lo.hi + hi.lo on the tensor cores
    (lo.lo dropped), norms of hi + lo.  Emulated in FP64."""
    rng = np.random.default_rng(n + d + k + 7)
    X = (rng.standard_normal((n, d)) * np.linspace(0.5, 2.0, d)).astype(np.float32)
    V = rng.standard_normal((n, k)).astype(np.float32)
    sigma = 0.7 * math.sqrt(d)
    Q = torch.empty((n, k), dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.0, torch.from_numpy(V).cuda(), Q, "bf16x3")
    got = Q.cpu().numpy().astype(np.float64)
    hi, lo = split_points(X, sigma)
    xs = hi + lo
    S = hi @ hi.T + lo @ hi.T + hi @ lo.T
    nh = np.sum(xs * xs, axis=1)
    Kt = np.exp2(S - 0.5 * nh[:, None] - 0.5 * nh[None, :])
    V64 = V.astype(np.float64)
    scale = Kt @ np.abs(V64)
    exact = O.gaussian_kernel(X, X, sigma) @ V64
    assert np.all(np.abs(got - Kt @ V64) <= 1e-5 * scale), np.max(np.abs(got - Kt @ V64) / scale)
    # 16-bit points: the kernel moves by about 2^-16 of -log2 K
    assert np.all(np.abs(got - exact) <= 2e-4 * scale), np.max(np.abs(got - exact) / scale)


@pytest.mark.parametrize("n,d,k,shift", [(1000, 37, 1, 0.0), (777, 64, 3, 1e-4), (300, 8, 16, 0.0),
                                         (2048, 54, 2, 1e-3)])
def test_matvec_hp_matches_oracle(K, h, n, d, k, shift):
    """High-precision tensor-core product: the kernel of points truncated to 45
    fixed-point bits per coordinate (error <= 2^-45 relative to the row maximum),
    exact integer level sums, float-float exp2 and accumulation.  Each K_ij
    carries ~1e-13 relative error; bound 2e-12 of sum_j |K_ij| |V_j|."""
    rng = np.random.default_rng(n + d + k)
    X = (rng.standard_normal((n, d)) * 2 + 1).astype(np.float32)
    V = rng.standard_normal((n, k))
    sigma = 0.8 * math.sqrt(d)
    Q = torch.empty((n, k), dtype=torch.float64, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, sigma, shift, torch.from_numpy(V).cuda(), Q, "hp")
    ref = O.kernel_matvec_blocked(X, X, V, sigma) + shift * V
    scale = O.kernel_matvec_blocked(X, X, np.abs(V), sigma) + shift * np.abs(V)
    err = np.abs(Q.cpu().numpy() - ref)
    assert np.all(err <= 2e-12 * scale), float(np.max(err / scale))


@pytest.mark.parametrize("nr,nc,d,k,shift", [(700, 700, 100, 1, 1e-3), (257, 1030, 54, 3, 0.0),
                                               (500, 500, 784, 10, 0.0), (130, 65, 7, 16, 0.0)])
def test_matvec_hp_simt_matches_oracle(K, h, nr, nc, d, k, shift):
    """HP product for any d and for distinct row and column sets: float-float
    norm-expansion distances of the FP32 inputs, float-float exp2 and sums."""
    rng = np.random.default_rng(nr + nc + d + k)
    Xc = (rng.random((nc, d)) * (rng.random((nc, d)) < 0.3)).astype(np.float32) if d == 784 \
        else (rng.standard_normal((nc, d)) * 1.5 + 0.5).astype(np.float32)
    Xr = Xc[:nr].copy() if nr == nc else (rng.standard_normal((nr, d)) + 0.5).astype(np.float32)
    V = rng.standard_normal((nc, k))
    sigma = 0.9 * math.sqrt(d) if d != 784 else 8.0
    Xcd = torch.from_numpy(Xc).cuda()
    Xrd = Xcd if nr == nc else torch.from_numpy(Xr).cuda()
    Q = torch.empty((nr, k), dtype=torch.float64, device="cuda")
    K.krr_kernel_matvec(h, Xrd, Xcd, sigma, shift, torch.from_numpy(V).cuda(), Q, "hp")
    Kx = O.gaussian_kernel(Xr, Xc, sigma)
    ref = Kx @ V + (shift * V if shift else 0.0)
    scale = Kx @ np.abs(V) + (shift * np.abs(V) if shift else 0.0)
    err = np.abs(Q.cpu().numpy() - ref)
    assert np.all(err <= 2e-12 * scale), float(np.max(err / scale))


def test_dsigma_hp_matches_oracle(K, h):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((400, 54)).astype(np.float32)
    V = rng.standard_normal((400, 2))
    sigma = 4.0
    Xd = torch.from_numpy(X).cuda()
    Q = torch.empty((400, 2), dtype=torch.float64, device="cuda")
    K.krr_kernel_dsigma_matvec(h, Xd, Xd, sigma, torch.from_numpy(V).cuda(), Q, precision="hp")
    G = O.kernel_dlogsigma(X, X, sigma)
    err = np.abs(Q.cpu().numpy() - G @ V)
    assert np.all(err <= 2e-12 * (G @ np.abs(V))), float(np.max(err / (G @ np.abs(V))))


def test_matvec_bf16_shift(K, h):
    P = ks.make_config(2, n=700)
    rng = np.random.default_rng(2)
    V = rng.standard_normal((700, 2)).astype(np.float32)
    Xd = torch.from_numpy(P.X).cuda()
    Q0 = torch.empty((700, 2), dtype=torch.float32, device="cuda")
    Q1 = torch.empty_like(Q0)
    Vd = torch.from_numpy(V).cuda()
    K.krr_kernel_matvec(h, Xd, Xd, P.sigma, 0.0, Vd, Q0, "bf16")
    K.krr_kernel_matvec(h, Xd, Xd, P.sigma, 0.25, Vd, Q1, "bf16")
    np.testing.assert_allclose((Q1 - Q0).cpu().numpy(), 0.25 * V, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("cfg,n,s,tol,inner", [(2, 4096, 128, 1e-6, "fp16"),
                                               (2, 4096, 128, 1e-6, "bf16"),
                                               (5, 3000, 256, 1e-6, "fp16"),
                                               (5, 8192, 512, 1e-6, "fp16"),
                                               (5, 8192, 512, 1e-6, "bf16"),
                                               (1, 2000, 200, 1e-8, "fp16")])
def test_pcg_mixed_reaches_tolerance(K, h, cfg, n, s, tol, inner):
    """FP16 (or BF16) inner PCG + refinement with an FP64 residual reaches the FP64 target.

    The oracle recomputes ||y - (K + lambda I) c|| / ||y|| of the returned c.
    Workload 1's weak preconditioner needs ~1800 iterations in all (cap 6000)."""
    P = ks.make_config(cfg, n=n, s=s)
    C = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=tol, precision="mixed", max_iter=6000, inner_precision=inner)
    rep = K.krr_pcg_solve(h, torch.from_numpy(P.X).cuda(), P.sigma, P.lam,
                          torch.from_numpy(P.W).cuda(), torch.from_numpy(P.b).cuda(),
                          torch.from_numpy(P.Y).cuda(), C, o, check=False)
    assert rep["status"] == "KRR_OK", rep
    res = O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, P.lam)[0]
    assert res <= tol, (res, rep)
    assert rep["outer_steps"] >= 1


@pytest.mark.parametrize("n,d,k,prec", [(3000, 64, 1, "fp16"), (2000, 100, 10, "bf16"),
                                        (2500, 40, 3, "bf16x3")])
def test_autotuned_plan_computes_the_same_product(K, h, n, d, k, prec):
    """The tuner only changes how the column tiles are split into chunks and the
    TMA ring depth: the product matches the default plan's up to FP32 summation
    order, and the shape lands in the tuner's table."""
    rng = np.random.default_rng(n + 3 * d + k)
    X = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).cuda()
    V = torch.from_numpy(rng.standard_normal((n, k)).astype(np.float32)).cuda()
    sigma = math.sqrt(d)
    Q0 = torch.empty((n, k), dtype=torch.float32, device="cuda")
    Q1 = torch.empty_like(Q0)
    K.krr_kernel_matvec(h, X, X, sigma, 0.0, V, Q0, prec)
    before = h.set_autotune(True)
    K.krr_kernel_matvec(h, X, X, sigma, 0.0, V, Q1, prec)
    after = h.set_autotune(False)
    assert after >= before + (0 if before else 1)
    scale = (torch.from_numpy(O.gaussian_kernel(X.cpu().numpy(), X.cpu().numpy(), sigma)).cuda()
             @ V.abs().double()).float()
    assert torch.all((Q1 - Q0).abs() <= 1e-5 * scale), float(((Q1 - Q0).abs() / scale).max())


def test_mixed_solve_with_autotuning(K, h):
    """A mixed solve on an autotuning handle still reaches the FP64 target."""
    P = ks.make_config(2, n=4096, s=128)
    h.set_autotune(True)
    C = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-6, precision="mixed", max_iter=6000)
    rep = K.krr_pcg_solve(h, torch.from_numpy(P.X).cuda(), P.sigma, P.lam,
                          torch.from_numpy(P.W).cuda(), torch.from_numpy(P.b).cuda(),
                          torch.from_numpy(P.Y).cuda(), C, o, check=False)
    h.set_autotune(False)
    assert rep["status"] == "KRR_OK", rep
    assert O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, P.lam)[0] <= 1e-6


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n,d,prec", [(3000, 64, "fp16"), (1000, 37, "bf16"), (517, 8, "fp16")])
def test_symmetric_product_matches_rounded_oracle(K, h, n, d, prec, mode):
    """The symmetric product (tiles I <= J only, each exponential used for K_ij
    and K_ji) is the same kernel of the rounded points as the full product."""
    rng = np.random.default_rng(11 * n + d)
    X = rng.standard_normal((n, d)).astype(np.float32)
    V = rng.standard_normal((n, 1)).astype(np.float32)
    sigma = math.sqrt(d)
    Xd, Vd = torch.from_numpy(X).cuda(), torch.from_numpy(V).cuda()
    Qs = torch.empty((n, 1), dtype=torch.float32, device="cuda")
    Qf = torch.empty_like(Qs)
    h.set_autotune(mode)
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.5, Vd, Qs, prec)
    h.set_autotune(0)
    K.krr_kernel_matvec(h, Xd, Xd, sigma, 0.5, Vd, Qf, prec)
    Xh = rounded_points(X, sigma, torch.float16 if prec == "fp16" else None)
    Kh = O.gaussian_kernel(Xh, Xh, 1.0 / math.sqrt(math.log(2.0)))
    ref = Kh @ V.astype(np.float64) + 0.5 * V.astype(np.float64)
    scale = Kh @ np.abs(V.astype(np.float64)) + 0.5 * np.abs(V.astype(np.float64))
    gs = Qs.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gs - ref) <= 1e-5 * scale), np.max(np.abs(gs - ref) / scale)
    assert np.all(np.abs(gs - Qf.cpu().numpy()) <= 1e-5 * scale)


def test_set_autotune_rejects_bad_mode(K, h):
    with pytest.raises(K.KrrError):
        h.set_autotune(4)


def test_mixed_solve_keeping_the_search_direction(K, h):
    """keep_direction = 1 (residual replacement instead of a fresh restart) still
    reaches the FP64 target."""
    P = ks.make_config(2, n=4096, s=128)
    C = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-6, precision="mixed", max_iter=6000, keep_direction=1)
    rep = K.krr_pcg_solve(h, torch.from_numpy(P.X).cuda(), P.sigma, P.lam,
                          torch.from_numpy(P.W).cuda(), torch.from_numpy(P.b).cuda(),
                          torch.from_numpy(P.Y).cuda(), C, o, check=False)
    assert rep["status"] == "KRR_OK", rep
    assert rep["outer_steps"] >= 2
    assert O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, P.lam)[0] <= 1e-6
