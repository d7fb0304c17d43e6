"""GPU parity of the hyper-parameter gradient (the held-out-MSE workload, d = 54).

The paper keeps sigma and lambda fixed; the gradient of
L = (1/m) ||K(Xte, X) (K + lambda I)^-1 y - yte||^2 with respect to log sigma
and log lambda is derived by implicit differentiation of Eq. (1).  The CUDA
path (adjoint PCG solve plus the (D o K) products, all through the C ABI) is
compared with the FP64 oracle's closed form and with central differences of
the CUDA forward pass, at n = 2000 as the workload's gradient check asks,
within 1e-4 relative.
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


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("nr,nc,d,k", [(300, 300, 54, 1), (257, 1030, 54, 3), (129, 77, 7, 16)])
def test_dsigma_matvec_matches_oracle(K, h, nr, nc, d, k):
    rng = np.random.default_rng(nr * 7 + nc + k)
    Xc = rng.standard_normal((nc, d)).astype(np.float32)
    Xr = Xc[:nr].copy() if nr == nc else rng.standard_normal((nr, d)).astype(np.float32)
    V = rng.standard_normal((nc, k))
    sigma = 0.6 * math.sqrt(d)
    Xcd = cuda(Xc)
    Xrd = Xcd if nr == nc else cuda(Xr)
    Q = torch.empty((nr, k), dtype=torch.float64, device="cuda")
    K.krr_kernel_dsigma_matvec(h, Xrd, Xcd, sigma, cuda(V), Q)
    ref = O.kernel_dlogsigma(Xr.astype(np.float64), Xc.astype(np.float64), sigma) @ V
    scale = np.abs(O.kernel_dlogsigma(Xr.astype(np.float64), Xc.astype(np.float64), sigma)) @ np.abs(V)
    err = np.abs(Q.cpu().numpy() - ref) / scale
    assert err.max() < 1e-12


def _problem(n=2000, m=500, s=200, k=1):
    P = ks.make_config(5, n=n, m=m, s=s)
    Y, Yte = P.Y, P.Yte
    if k > 1:
        # a second target: the first column scaled and shifted (same structure)
        Y = np.concatenate([Y, 0.5 * Y + 0.25], axis=1)
        Yte = np.concatenate([Yte, 0.5 * Yte + 0.25], axis=1)
    return P, Y, Yte


@pytest.fixture(scope="module")
def oracle_grads():
    out = {}
    for k in (1, 2):
        P, Y, Yte = _problem(k=k)
        out[k] = O.hypergrad(P.X, Y, P.Xte, Yte, P.sigma, P.lam)
    return out


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hypergrad_matches_oracle(K, h, oracle_grads, k, precision):
    P, Y, Yte = _problem(k=k)
    ref = oracle_grads[k]
    # the mixed solve's residual is computed by the HP product (about 1e-13
    # relative per kernel entry); its FP16 inner solves need more refinement
    # steps for a tight tolerance
    tol, rel = (1e-10, 1e-6) if precision == "fp64" else (1e-9, 1e-5)
    opts = K.default_opts(tol=tol, max_iter=20000, precision=precision, max_outer=80)
    C = cuda(ref["c"])  # the exact forward solution, so only the backward is compared
    m = P.Xte.shape[0]
    F = O.predict(P.X, P.Xte, ref["c"], P.sigma)
    GF = (2.0 / m) * (F - Yte)
    Wadj = torch.empty_like(C)
    (dls, dll), rep = K.krr_hypergrad(h, cuda(P.X), cuda(P.Xte), P.sigma, P.lam, cuda(P.W),
                                      cuda(P.b), C, cuda(GF), opts, Wadj=Wadj)
    assert rep["status_code"] == K.KRR_OK
    assert dls == pytest.approx(ref["dlogsigma"], rel=rel)
    assert dll == pytest.approx(ref["dloglambda"], rel=rel)
    w = Wadj.cpu().numpy()
    assert np.linalg.norm(w - ref["w"]) <= 100 * rel * np.linalg.norm(ref["w"])


def test_hypergrad_host_buffers(K, h, oracle_grads):
    P, Y, Yte = _problem(k=1)
    ref = oracle_grads[1]
    m = P.Xte.shape[0]
    GF = (2.0 / m) * (O.predict(P.X, P.Xte, ref["c"], P.sigma) - Yte)
    opts = K.default_opts(tol=1e-10, max_iter=20000)
    (dls, dll), _ = K.krr_hypergrad(h, P.X, P.Xte, P.sigma, P.lam, P.W, P.b,
                                    np.ascontiguousarray(ref["c"]), np.ascontiguousarray(GF), opts)
    assert dls == pytest.approx(ref["dlogsigma"], rel=1e-6)
    assert dll == pytest.approx(ref["dloglambda"], rel=1e-6)


def _loss_and_grad(K, h, P, Y, Yte, ls, ll, opts):
    from paper_1611_03220_gb300.autograd import krr_predict_fn
    X, Xte = cuda(P.X), cuda(P.Xte)
    log_s = torch.tensor(ls, dtype=torch.float64, requires_grad=True)
    log_l = torch.tensor(ll, dtype=torch.float64, requires_grad=True)
    F = krr_predict_fn(log_s, log_l, X, cuda(Y), Xte, cuda(P.W), cuda(P.b), handle=h, opts=opts)
    loss = ((F - cuda(Yte)) ** 2).sum() / F.shape[0]
    loss.backward()
    return float(loss.detach()), float(log_s.grad), float(log_l.grad)


def test_autograd_matches_oracle_and_central_differences(K, h, oracle_grads):
    # more features than the other cases: the solution is the same, the 9
    # FP64 solves take about a third of the iterations
    P, Y, Yte = _problem(k=1, s=1000)
    ref = oracle_grads[1]
    opts = K.default_opts(tol=1e-11, max_iter=20000)
    ls0, ll0 = math.log(P.sigma), math.log(P.lam)
    loss, gs, gl = _loss_and_grad(K, h, P, Y, Yte, ls0, ll0, opts)
    assert loss == pytest.approx(ref["loss"], rel=1e-8)
    assert gs == pytest.approx(ref["dlogsigma"], rel=1e-4)
    assert gl == pytest.approx(ref["dloglambda"], rel=1e-4)

    # central differences of the CUDA forward pass (Richardson over two steps)
    def fwd(ls, ll):
        from paper_1611_03220_gb300.autograd import krr_predict_fn
        with torch.no_grad():
            F = krr_predict_fn(torch.tensor(ls, dtype=torch.float64),
                               torch.tensor(ll, dtype=torch.float64), cuda(P.X), cuda(Y),
                               cuda(P.Xte), cuda(P.W), cuda(P.b), handle=h, opts=opts)
        return float(((F - cuda(Yte)) ** 2).sum()) / F.shape[0]

    for which, g in (("s", gs), ("l", gl)):
        fd = []
        for step in (2e-3, 1e-3):
            if which == "s":
                fd.append((fwd(ls0 + step, ll0) - fwd(ls0 - step, ll0)) / (2 * step))
            else:
                fd.append((fwd(ls0, ll0 + step) - fwd(ls0, ll0 - step)) / (2 * step))
        rich = (4 * fd[1] - fd[0]) / 3
        assert g == pytest.approx(rich, rel=1e-4)


def test_autograd_mixed_precision(K, h, oracle_grads):
    """BF16 tensor-core solves with HP refinement, forward and adjoint."""
    P, Y, Yte = _problem(k=1)
    ref = oracle_grads[1]
    opts = K.default_opts(tol=1e-8, max_iter=20000, precision="mixed", max_outer=80)
    loss, gs, gl = _loss_and_grad(K, h, P, Y, Yte, math.log(P.sigma), math.log(P.lam), opts)
    assert loss == pytest.approx(ref["loss"], rel=1e-6)
    assert gs == pytest.approx(ref["dlogsigma"], rel=1e-4)
    assert gl == pytest.approx(ref["dloglambda"], rel=1e-4)


def test_hypergrad_rejects_bad_arguments(K, h):
    P, Y, Yte = _problem(n=300, m=50, s=32)
    C = torch.zeros((300, 1), dtype=torch.float64, device="cuda")
    GF = torch.zeros((50, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KrrError):
        K.krr_hypergrad(h, cuda(P.X), cuda(P.Xte), -1.0, P.lam, cuda(P.W), cuda(P.b), C, GF)
    with pytest.raises(K.KrrError):
        K.krr_hypergrad(h, cuda(P.X), cuda(P.Xte), P.sigma, P.lam, cuda(P.W), cuda(P.b), C, GF,
                        K.default_opts(warm_start=1))
    Q = torch.empty((300, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KrrError):
        K.krr_kernel_dsigma_matvec(h, cuda(P.X), cuda(P.X), P.sigma, C, Q, precision="fp32")
