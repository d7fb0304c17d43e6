"""GPU parity of the adaptive sketch size (Section 5, Theorem 4).

The device doubles s from s0 until the power-iteration estimate of
||(I - P) K (I - P)|| falls to 0.1 lambda, exactly as the oracle's
``adaptive_sketch_size`` does from the same start vector.  Its projection P
comes from a Newton-Schulz sign iteration on the s x s Gram matrix and a
regularised inverse (relative change of P's eigenvalues <= 1e-3 * tau / t on
its range), so the estimates agree with the oracle's exact projection to a
few parts in 1e6 unless an eigenvalue of Z Z^T sits within about 1 % of the
threshold; the tests take seeds whose spectra do not.
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


@pytest.mark.parametrize("lam,s0", [(1e-1, 16), (3e-2, 8)])
def test_adaptive_size_matches_oracle(K, h, lam, s0):
    P = ks.make_config(1, n=300)
    W, b = ks.rff_draw(77, P.d, 256, P.sigma)
    x0 = np.random.default_rng(1).standard_normal(300)
    ref = O.adaptive_sketch_size(P.X, P.sigma, lam, W, b, s0, x0, iters=60)
    out = K.krr_precond_setup_adaptive(h, dev(P.X), P.sigma, lam, dev(W), dev(b), s0, dev(x0),
                                       power_iters=60, precision="fp64")
    assert out["s"] == ref["s"], (out, ref["history"])
    est_ref = [e for _, e in ref["history"]]
    assert out["tests"] == len(est_ref)
    np.testing.assert_allclose(out["estimates"], est_ref, rtol=1e-4, atol=1e-9 * lam)


def test_adaptive_then_solve(K, h):
    """The chosen features become the handle's preconditioner; PCG with it
    (precond = 2) reaches the oracle-checked residual."""
    P = ks.make_config(2, n=4096)
    W, b = ks.rff_draw(2002, P.d, 1024, P.sigma)
    x0 = np.random.default_rng(2).standard_normal(P.n)
    lam = 1e-2
    out = K.krr_precond_setup_adaptive(h, dev(P.X), P.sigma, lam, dev(W), dev(b), 64, dev(x0),
                                       power_iters=20, precision="fp16")
    assert out["s"] in (64, 128, 256, 512, 1024)
    assert out["tests"] == int(np.log2(out["s"] // 64)) + 1
    est = out["estimates"]
    assert est[-1] <= 0.1 * lam or out["s"] == 1024
    assert all(e > 0.1 * lam for e in est[:-1])
    C = torch.zeros((P.n, 1), dtype=torch.float64, device="cuda")
    o = K.default_opts(tol=1e-8, precision="fp64", precond=2, max_iter=5000)
    rep = K.krr_pcg_solve(h, dev(P.X), P.sigma, lam, None, None, dev(P.Y), C, o)
    assert rep["status"] == "KRR_OK"
    assert O.true_rel_residual(P.X, P.Y, C.cpu().numpy(), P.sigma, lam)[0] <= 1e-8


def test_adaptive_rejects_bad_sizes(K, h):
    P = ks.make_config(1, n=100)
    W, b = ks.rff_draw(3, P.d, 64, P.sigma)
    x0 = np.ones(100)
    with pytest.raises(K.KrrError):
        K.krr_precond_setup_adaptive(h, dev(P.X), P.sigma, 1e-2, dev(W), dev(b), 128, dev(x0))
