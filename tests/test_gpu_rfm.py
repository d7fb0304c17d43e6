"""GPU parity of the random-features method (krr_rfm_fit / krr_rfm_predict).

The device computes the features in FP32 (|Z_ij - Z*_ij| of order 2^-23 times
the argument), then the Gram matrix, Cholesky and triangular solves in FP64.
A relative perturbation e of Z moves the ridge solution by at most about
kappa e with kappa = (||Z||^2 + lambda) / lambda, and ||Z||^2 <= sum_i ||z_i||^2,
which is about n because every feature row has squared norm close to 1.  The
cases keep kappa e below 1e-3 and test at that level; the predictor alone
(given the oracle's w) is checked at 1e-5 of sum |phi| |w|.
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


@pytest.mark.parametrize("n,s,lam,k", [(1000, 64, 1.5, 1), (1500, 200, 3.0, 3), (777, 40, 1.0, 2)])
def test_rfm_fit_matches_oracle(K, h, n, s, lam, k):
    P = ks.make_config(1, n=n, s=s)
    Y = np.ascontiguousarray(np.repeat(P.Y, k, axis=1) * np.arange(1, k + 1))
    Wf = torch.empty((s, k), dtype=torch.float64, device="cuda")
    K.krr_rfm_fit(h, cuda(P.X), cuda(P.W), cuda(P.b), lam, cuda(Y), Wf)
    ref = O.rfm_fit(P.X, P.W, P.b, lam, Y)
    got = Wf.cpu().numpy()
    kappa = (n + lam) / lam
    assert kappa * 1e-6 <= 1e-3
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert np.all(err <= 1e-3), err
    # the fitted values at the training points, through the device predictor
    F = torch.empty((n, k), dtype=torch.float64, device="cuda")
    K.krr_rfm_predict(h, cuda(P.X), cuda(P.W), cuda(P.b), Wf, F)
    fref = O.rfm_predict(P.X, P.W, P.b, ref)
    ferr = np.linalg.norm(F.cpu().numpy() - fref, axis=0) / np.linalg.norm(fref, axis=0)
    assert np.all(ferr <= 1e-3), ferr


@pytest.mark.parametrize("m,s,k", [(333, 128, 1), (2048, 512, 4)])
def test_rfm_predict_matches_oracle(K, h, m, s, k):
    """The predictor alone, on the oracle's own w."""
    P = ks.make_config(1, n=500, s=s)
    rng = np.random.default_rng(m + s)
    Xte = rng.standard_normal((m, P.X.shape[1])).astype(np.float32)
    w = rng.standard_normal((s, k))
    F = torch.empty((m, k), dtype=torch.float64, device="cuda")
    K.krr_rfm_predict(h, cuda(Xte), cuda(P.W), cuda(P.b), cuda(w), F)
    Zte = O.rff_features(Xte, P.W, P.b)
    ref = Zte @ w
    scale = np.abs(Zte) @ np.abs(w)
    assert np.all(np.abs(F.cpu().numpy() - ref) <= 1e-5 * scale)


def test_rfm_host_buffers(K, h):
    """Host (numpy) inputs and outputs give the device-buffer result."""
    P = ks.make_config(1, n=600, s=48)
    Wf_h = np.zeros((48, 1))
    K.krr_rfm_fit(h, P.X, P.W, P.b, 1.0, P.Y, Wf_h)
    Wf_d = torch.empty((48, 1), dtype=torch.float64, device="cuda")
    K.krr_rfm_fit(h, cuda(P.X), cuda(P.W), cuda(P.b), 1.0, cuda(P.Y), Wf_d)
    np.testing.assert_array_equal(Wf_h, Wf_d.cpu().numpy())
    F_h = np.zeros((600, 1))
    K.krr_rfm_predict(h, P.X, P.W, P.b, Wf_h, F_h)
    assert np.all(np.isfinite(F_h)) and np.linalg.norm(F_h) > 0


def test_rfm_rejects_bad_arguments(K, h):
    P = ks.make_config(1, n=100, s=16)
    Wf = torch.empty((16, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KrrError):
        K.krr_rfm_fit(h, cuda(P.X), cuda(P.W), cuda(P.b), 0.0, cuda(P.Y), Wf)
    with pytest.raises(K.KrrError):
        K.krr_rfm_fit(h, cuda(P.X), cuda(P.W), cuda(P.b), -1.0, cuda(P.Y), Wf)
    # more features than points: refused before any launch
    Q = ks.make_config(1, n=100, s=128)
    Wq = torch.empty((128, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KrrError):
        K.krr_rfm_fit(h, cuda(Q.X), cuda(Q.W), cuda(Q.b), 1.0, cuda(Q.Y), Wq)
