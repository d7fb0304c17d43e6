"""The kernel product that allocates nothing gives the regular product's answer.

``krr_kernel_matvec_fp64_noalloc`` exists for callers that cannot call
cudaMalloc when they need a product (graph capture in progress, a framework
allocator that owns the GPU's memory, loops that must not synchronise).  It
keeps its partial sums in a fixed device array shared by every call, so the
test runs it twice in a row on different inputs -- the second call must not
see anything of the first -- and checks each result against the regular
handle-based FP64 entry point on the same inputs, with the FP64 product's
tolerance (1e-12 of sum_j |K_ij| |V_j|).  One case fills the scratch array
exactly, which forces the product down to a single column split.  This file
is collected last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_product_matches_regular_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr as K
    from oracle import krr_oracle as O

    rng = np.random.default_rng(2024)
    # the last case fills the scratch exactly (nr * k = 2^20 doubles), so the
    # column split is cut to one partial per row and RHS
    cases = [(1000, 777, 37, 3, 0.0), (640, 640, 64, 1, 0.125), (65536, 512, 4, 16, 0.0)]
    with K.Handle() as h:
        for nr, nc, d, k, shift in cases:
            Xr = rng.standard_normal((nr, d)).astype(np.float32)
            Xc = Xr if shift else rng.standard_normal((nc, d)).astype(np.float32)
            V = rng.standard_normal((nc, k))
            sigma = 0.9 * math.sqrt(d)
            Xr_d, Xc_d, V_d = (torch.from_numpy(a).cuda() for a in (Xr, Xc, V))
            Q_reg = torch.empty((nr, k), dtype=torch.float64, device="cuda")
            Q_na = torch.full((nr, k), float("nan"), dtype=torch.float64, device="cuda")
            K.krr_kernel_matvec(h, Xr_d, Xc_d, sigma, shift, V_d, Q_reg, "fp64")
            st = K.krr_kernel_matvec_fp64_noalloc(Xr_d, Xc_d, sigma, shift, V_d, Q_na)
            assert st == K.KRR_OK
            torch.cuda.synchronize()
            scale = O.gaussian_kernel(Xr, Xc, sigma) @ np.abs(V)
            if shift:
                scale = scale + abs(shift) * np.abs(V)
            diff = np.abs(Q_na.cpu().numpy() - Q_reg.cpu().numpy())
            assert np.all(diff <= 1e-12 * scale), float(np.max(diff / scale))


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03220_gb300 import build
    build()
    from paper_1611_03220_gb300 import _krr as K
    nr, k = (1 << 20) // 4 + 1, 4      # nr * k just above 2^20 doubles
    X = torch.zeros((nr, 2), dtype=torch.float32, device="cuda")
    V = torch.zeros((nr, k), dtype=torch.float64, device="cuda")
    Q = torch.zeros_like(V)
    assert K.krr_kernel_matvec_fp64_noalloc(X, X, 1.0, 0.0, V, Q) == K.KRR_EINVAL
