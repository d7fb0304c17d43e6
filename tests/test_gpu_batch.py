"""GPU parity of the uneven batch: independent problems solved in lockstep.

Each problem of ``krr_synth.make_uneven`` (log-uniform n, d in {16, 32, 64,
128}, log-uniform lambda, s = min(n/8, 4096), its own RFF draw) is checked
against the FP64 oracle: the true relative residual of Eq. (1) recomputed by
the oracle must meet the tolerance, and the FP64 batch must take the
oracle's PCG iteration counts (5% band; the recurrences agree up to
rounding) and match the oracle's direct solution.
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(K, h, probs, opts, device=True):
    items, outs = [], []
    for P in probs:
        Cout = (torch.zeros((P.n, P.k), dtype=torch.float64, device="cuda") if device
                else np.zeros((P.n, P.k)))
        outs.append(Cout)
        if device:
            items.append((cuda(P.X), P.sigma, P.lam, cuda(P.W), cuda(P.b), cuda(P.Y), Cout))
        else:
            items.append((P.X, P.sigma, P.lam, P.W, P.b, np.ascontiguousarray(P.Y), Cout))
    reps = K.krr_pcg_solve_batched(h, items, opts, check=False)
    Cs = [c.cpu().numpy() if device else c for c in outs]
    return reps, Cs


def test_batched_fp64_matches_oracle(K, h):
    probs = ks.make_uneven(nprob=7, scale=0.05)
    opts = K.default_opts(tol=1e-8, max_iter=20000)
    reps, Cs = _run(K, h, probs, opts)
    for P, r, C in zip(probs, reps, Cs):
        assert r["status_code"] == K.KRR_OK, (P.name, r)
        res = O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)
        assert np.all(res <= 1e-8), (P.name, res)
        ref = O.krr_pcg_solve(P.X, P.Y, P.sigma, P.lam, P.W, P.b, tol=1e-8, max_iter=20000)
        it_o, it_g = ref["iters"][0], r["iters"][0]
        assert abs(it_g - it_o) <= max(3, 0.05 * it_o), (P.name, it_g, it_o)
        C0 = O.direct_solve(P.X, P.Y, P.sigma, P.lam)
        # the residual bound times the condition number bounds the error
        assert np.linalg.norm(C - C0) <= 1e-3 * np.linalg.norm(C0), P.name


def test_batched_fp64_equals_single_solves(K, h):
    """The lockstep graph runs each problem's own kernels in the same order
    as the single-problem solve, so the coefficients agree bit for bit."""
    probs = ks.make_uneven(nprob=4, scale=0.03)
    opts = K.default_opts(tol=1e-8, max_iter=20000)
    reps, Cs = _run(K, h, probs, opts)
    for P, r, C in zip(probs, reps, Cs):
        C1 = torch.zeros((P.n, P.k), dtype=torch.float64, device="cuda")
        r1 = K.krr_pcg_solve(h, cuda(P.X), P.sigma, P.lam, cuda(P.W), cuda(P.b), cuda(P.Y), C1,
                             opts)
        assert r1["iters"] == r["iters"]
        np.testing.assert_array_equal(C1.cpu().numpy(), C)


def test_batched_mixed_reaches_tolerance(K, h):
    """BF16 tensor-core inner loops in lockstep, HP (d <= 64) or FP64 (d = 128)
    residuals per problem; n from 160 to 5000.

    The solve certifies ||y - A c|| <= tol ||y|| with the HP product, whose
    entries carry at most 2e-12 relative error; the FP64 residual may exceed
    tol by that error, 2e-12 ||(K + lambda I)|c||| / ||y||, which matters only
    when lambda is tiny and |c| >> |y|."""
    probs = ks.make_uneven(nprob=10, scale=0.16)
    opts = K.default_opts(tol=1e-6, max_iter=60000, precision="mixed", max_outer=60)
    reps, Cs = _run(K, h, probs, opts)
    for P, r, C in zip(probs, reps, Cs):
        assert r["status_code"] == K.KRR_OK, (P.name, P.n, P.d, r)
        res = O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)
        hp_err = 0.0
        if P.d <= 64:
            scale = O.kernel_matvec_blocked(P.X, P.X, np.abs(C), P.sigma) + P.lam * np.abs(C)
            hp_err = 2e-12 * np.linalg.norm(scale, axis=0) / np.linalg.norm(P.Y, axis=0)
        assert np.all(res <= 1e-6 + hp_err), (P.name, res, hp_err)


def test_batched_fp32_and_host_buffers(K, h):
    probs = ks.make_uneven(nprob=2, scale=0.03)
    # FP32 kernel entries (norm expansion) floor these residuals near 1e-5
    opts = K.default_opts(tol=1e-4, max_iter=20000, precision="fp32")
    reps, Cs = _run(K, h, probs, opts, device=False)
    for P, r, C in zip(probs, reps, Cs):
        assert r["status_code"] == K.KRR_OK, (P.name, r)
        res = O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)
        assert np.all(res <= 1e-4), (P.name, res)


def test_batched_degenerate_cases(K, h):
    """A zero right-hand side converges at once (c = 0); a one-problem batch
    and a problem without preconditioner go through the same graph."""
    probs = ks.make_uneven(nprob=2, scale=0.03)
    Z = probs[1]
    Z.Y = np.zeros_like(Z.Y)
    opts = K.default_opts(tol=1e-8, max_iter=20000)
    reps, Cs = _run(K, h, probs, opts)
    assert all(r["status_code"] == K.KRR_OK for r in reps)
    assert reps[1]["iters"] == [0] and np.all(Cs[1] == 0.0)
    reps, Cs = _run(K, h, probs[:1], K.default_opts(tol=1e-8, max_iter=20000, precond=0))
    assert reps[0]["status_code"] == K.KRR_OK
    res = O.true_rel_residual(probs[0].X, probs[0].Y, Cs[0], probs[0].sigma, probs[0].lam)
    assert res[0] <= 1e-8


def test_batched_rejects_bad_arguments(K, h):
    probs = ks.make_uneven(nprob=2, scale=0.03)

    def items(ps):
        return [(cuda(P.X), P.sigma, P.lam, cuda(P.W), cuda(P.b), cuda(P.Y),
                 torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")) for P in ps]

    with pytest.raises(K.KrrError):
        K.krr_pcg_solve_batched(h, items(probs), K.default_opts(warm_start=1))
    with pytest.raises(K.KrrError):
        K.krr_pcg_solve_batched(h, [], K.default_opts())
    probs[1].lam = -1.0
    with pytest.raises(K.KrrError):
        K.krr_pcg_solve_batched(h, items(probs), K.default_opts())


def test_batched_mixed_one_launch_product(K, h):
    """The FP16-point products of all low-level solves run as one persistent
    launch per iteration (batch_product = 1, the default) instead of one
    launch sequence per problem: the same solutions to the same tolerance,
    iteration counts within the rounding noise of the FP32 inner loops."""
    probs = ks.make_uneven(nprob=12, scale=0.2)
    res_runs = {}
    for bp in (0, 1):
        opts = K.default_opts(tol=1e-6, max_iter=60000, precision="mixed", max_outer=60,
                              batch_product=bp)
        reps, Cs = _run(K, h, probs, opts)
        res_runs[bp] = (reps, Cs)
        for P, r, C in zip(probs, reps, Cs):
            assert r["status_code"] == K.KRR_OK, (bp, P.name, P.n, P.d, r)
            res = O.true_rel_residual(P.X, P.Y, C, P.sigma, P.lam)
            hp_err = 0.0
            if P.d <= 64:
                scale = O.kernel_matvec_blocked(P.X, P.X, np.abs(C), P.sigma) + P.lam * np.abs(C)
                hp_err = 2e-12 * np.linalg.norm(scale, axis=0) / np.linalg.norm(P.Y, axis=0)
            assert np.all(res <= 1e-6 + hp_err), (bp, P.name, res, hp_err)
    for r0, r1 in zip(res_runs[0][0], res_runs[1][0]):
        a, b = r0["iters"][0], r1["iters"][0]
        assert abs(a - b) <= 0.15 * max(a, b) + 10, (a, b)


def test_batched_product_matches_single_products(K, h):
    """The one-launch product of many problems (d = 16 ... 128, n from a few
    hundred to a few thousand, ragged tiles) equals each problem's own FP16
    product up to FP32 summation order (1e-5 of sum_j |K_ij||v_j|)."""
    probs = ks.make_uneven(nprob=20, scale=0.15)
    rng = np.random.default_rng(20)
    items, Vs, Qs = [], [], []
    for P in probs:
        V = torch.from_numpy(rng.standard_normal((P.n, 1)).astype(np.float32)).cuda()
        Q = torch.full((P.n, 1), float("nan"), dtype=torch.float32, device="cuda")
        items.append((cuda(P.X), P.sigma, P.lam, V, Q))
        Vs.append(V)
        Qs.append(Q)
    K.krr_kernel_matvec_batched(h, items)
    torch.cuda.synchronize()
    for P, (X, sigma, lam, V, Q) in zip(probs, items):
        Q1 = torch.empty_like(Q)
        K.krr_kernel_matvec(h, X, X, sigma, lam, V, Q1, "fp16")
        scale = (torch.from_numpy(O.gaussian_kernel(P.X, P.X, sigma)).cuda()
                 @ V.abs().double()).float() + lam * V.abs()
        assert torch.all(torch.isfinite(Q))
        assert torch.all((Q - Q1).abs() <= 1e-5 * scale), (P.name, P.n, P.d,
                                                           float(((Q - Q1).abs() / scale).max()))


@pytest.mark.parametrize("picks", [(37, 43, 61, 3, 59), (43,)])
def test_batched_product_full_size(K, h, picks):
    """The one-launch product at the uneven batch's full sizes (n = 20,284 ...
    30,402 with d = 32, next to small problems): every problem's result equals
    its own FP16 product to 1e-5 of sum_j |K_ij||v_j| (that scale from the FP64
    product of |v|), over many items per CTA and chunks of eight column tiles."""
    allp = ks.make_uneven()
    probs = [allp[i] for i in picks]
    rng = np.random.default_rng(sum(picks))
    items = []
    for P in probs:
        V = torch.from_numpy(rng.standard_normal((P.n, 1)).astype(np.float32)).cuda()
        Q = torch.full((P.n, 1), float("nan"), dtype=torch.float32, device="cuda")
        items.append((cuda(P.X), P.sigma, P.lam, V, Q))
    K.krr_kernel_matvec_batched(h, items)
    torch.cuda.synchronize()
    for P, (X, sigma, lam, V, Q) in zip(probs, items):
        Q1 = torch.empty_like(Q)
        K.krr_kernel_matvec(h, X, X, sigma, lam, V, Q1, "fp16")
        S = torch.empty((P.n, 1), dtype=torch.float64, device="cuda")
        K.krr_kernel_matvec(h, X, X, sigma, lam, V.abs().double(), S, "fp64")
        torch.cuda.synchronize()
        err = (Q.double() - Q1.double()).abs()
        assert torch.all(torch.isfinite(Q)), P.name
        assert torch.all(err <= 1e-5 * S), (P.name, P.n, P.d, float((err / S).max()))
