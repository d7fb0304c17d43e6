"""The fused PCG iteration of the mixed solve's FP32 inner loop (Algorithm 1).

With ``fuse_step = 1`` (the default) an inner iteration runs as 8 launches:
the product kernel, its chunk sums with p.q and alpha, the apply's Z^T pass
with the x, r update and ||r||^2, the slab sums, the two triangular products,
the apply's Z w pass with r.z, beta and the loop test, and p = z + beta p with
the next product weights.  ``fuse_step = 0`` runs the separate CG kernels (13
launches).  The element-wise arithmetic is the same; only the partition of the
||r||^2 and r.z reductions over CTAs differs, so the two loops agree to the
FP32 rounding of those two scalars.
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


def problem(n, s, k):
    P = ks.make_config(2, n=n, s=s)
    Y = P.Y
    if k > 1:
        rng = np.random.default_rng(n + 7 * k)
        Y = np.concatenate([P.Y, rng.standard_normal((n, k - 1))], axis=1)
    return P, Y


def solve(K, h, P, Y, dv=None, **kw):
    """One mixed solve; ``dv`` = (X, W, b, Y) device tensors to reuse (the
    handle caches operands prepared from the same X, so repeated solves on
    the same tensors launch the same set-up kernels)."""
    C = torch.zeros((P.n, Y.shape[1]), dtype=torch.float64, device="cuda")
    o = K.default_opts(precision="mixed", **kw)
    Xd, Wd, bd, Yd = dv if dv is not None else (dev(P.X), dev(P.W), dev(P.b), dev(Y))
    l0 = K._lib.krr_launch_count()
    rep = K.krr_pcg_solve(h, Xd, P.sigma, P.lam, Wd, bd, Yd, C, o, check=False)
    torch.cuda.synchronize()
    return rep, C.cpu().numpy(), K._lib.krr_launch_count() - l0


@pytest.mark.parametrize("n,s,k,inner,graph", [
    (4096, 128, 1, "fp16", 1),
    (3001, 256, 1, "bf16", 0),     # ragged last tile, host-driven loop
    (2500, 128, 3, "fp16", 1),     # several right-hand sides
    (2000, 64, 1, "bf16x3", 1),    # split points
])
def test_fused_iterations_match_separate_kernels(K, h, n, s, k, inner, graph):
    """A few inner iterations: the iterates of the two loops agree to the
    rounding of the two reductions whose CTA partition differs."""
    P, Y = problem(n, s, k)
    kw = dict(tol=1e-14, inner_tol=1e-12, max_iter=6, max_outer=1, inner_precision=inner,
              use_graph=graph)
    r1, C1, _ = solve(K, h, P, Y, fuse_step=1, **kw)
    r0, C0, _ = solve(K, h, P, Y, fuse_step=0, **kw)
    assert r1["iters"][:k] == r0["iters"][:k] == [6] * k, (r1["iters"], r0["iters"])
    # the inner loops' recursive residuals (reported whether or not the outer
    # step keeps the correction) and the corrections kept
    rec1, rec0 = np.array(r1["rel_res_rec"][:k]), np.array(r0["rel_res_rec"][:k])
    assert np.all(rec0 > 0) and np.all(np.abs(rec1 - rec0) <= 1e-4 * rec0), (rec1, rec0)
    assert np.all(np.isfinite(C1))
    n0 = np.linalg.norm(C0, axis=0)
    assert np.all(np.linalg.norm(C1 - C0, axis=0) <= 1e-4 * n0), (C1 - C0, n0)


@pytest.mark.parametrize("k", [1, 3])
def test_fused_mixed_solve_reaches_oracle_residual(K, h, k):
    P, Y = problem(4096, 128, k)
    r1, C1, _ = solve(K, h, P, Y, tol=1e-6, max_iter=8000, fuse_step=1)
    r0, C0, _ = solve(K, h, P, Y, tol=1e-6, max_iter=8000, fuse_step=0)
    assert r1["status"] == "KRR_OK" and r0["status"] == "KRR_OK", (r1, r0)
    res = O.true_rel_residual(P.X, Y, C1, P.sigma, P.lam)
    assert np.all(np.asarray(res) <= 1e-6), res
    # the two loops follow the same iteration up to FP32 reduction order
    for c in range(k):
        assert abs(r1["iters"][c] - r0["iters"][c]) <= 0.1 * r0["iters"][c] + 5


@pytest.mark.parametrize("s,fused_launches", [(128, 8), (200, 13)])
def test_fused_body_launch_count(K, h, s, fused_launches):
    """Launches per inner iteration, from two runs that differ only in their
    iteration cap: 8 with the fused body; 13 where the streamed apply cannot
    serve the shape (8-bit rows of 200 bytes are not 16-byte aligned) and the
    loop falls back to the separate kernels."""
    P, Y = problem(3000, s, 1)
    dv = (dev(P.X), dev(P.W), dev(P.b), dev(Y))
    kw = dict(tol=1e-14, inner_tol=1e-12, max_outer=1, use_graph=1, dv=dv)
    solve(K, h, P, Y, max_iter=5, **kw)   # operands prepared once
    for fuse, per_iter in ((1, fused_launches), (0, 13)):
        ra, _, la = solve(K, h, P, Y, max_iter=10, fuse_step=fuse, **kw)
        rb, _, lb = solve(K, h, P, Y, max_iter=30, fuse_step=fuse, **kw)
        ia, ib = ra["iters"][0], rb["iters"][0]
        assert ia == 10 and ib > ia, (ia, ib)
        assert lb - la == per_iter * (ib - ia), (fuse, la, lb, ia, ib)
