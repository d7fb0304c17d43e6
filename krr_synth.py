"""Seeded synthetic inputs for the kernel ridge regression workloads.

This module only draws random numbers: it holds none of the method's
arithmetic (no kernel, no feature map, no solver).  Both the FP64 oracle
(``oracle/``) and the CUDA path receive exactly the arrays made here, so the
two sides see bit-identical inputs.

The five workloads mirror the shapes of the datasets the paper experiments
on (Section 5, Table 1: MNIST n=60000 d=780, COVTYPE d=54), none of which is
available here; they are stand-ins with the stated recipes:

  1. "plain"      n=2000, d=8, X~N(0,I), y=sin(sum x)+0.1 eps, sigma=1,
                  lambda=1e-3, s=200, tol 1e-8 (FP64 path).
  2. "precision"  n=65536, d=64, 10-component Gaussian mixture (centres
                  N(0,4I), unit spread), y = a_c.x + b_c + 0.1 eps,
                  sigma=sqrt(d)=8, lambda=1e-4, s=2048, tol 1e-6.
  3. "multirhs"   n=60000, d=784, pixel-like [0,1] features with ~19%
                  nonzeros (uniform intensities), 10 one-hot RHS, sigma=8,
                  lambda=1e-3, s=8192.
  4. "uneven"     64 independent problems, n log-uniform in [1000, 32768],
                  d uniform in {16,32,64,128}, X~N(0,I), sigma=sqrt(d),
                  lambda log-uniform in [1e-5, 1e-2], s=min(n/8, 4096).
  5. "grad"       n=131072 train + 16384 held-out, d=54 (10 N(0,1) columns,
                  44 Bernoulli(0.1) columns), y=sign(w.x - median(w.x)),
                  sigma=4, lambda=1e-3, s=4096.

Random Fourier feature draws (the paper, Section 2.2: w ~ p, b ~ U[0, 2pi])
are inputs too: ``W = Omega / sigma`` with ``Omega ~ N(0, I)`` (d x s) and
``b ~ U[0, 2pi)``.  Seeds: data ``1000+i``, features ``2000+i``.

Every function takes an optional ``n`` so tests can draw a smaller instance
of the same recipe.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Problem", "make_config", "make_uneven", "rff_draw", "tensorsketch_draw",
           "srht_draw", "gaussian_draw", "CONFIGS"]


@dataclasses.dataclass
class Problem:
    """One KRR instance: training points, right-hand sides and parameters."""

    name: str
    X: np.ndarray            # n x d float32, row-major
    Y: np.ndarray            # n x k float64
    sigma: float
    lam: float
    s: int
    tol: float
    W: np.ndarray            # d x s float32 (RFF frequencies, already / sigma)
    b: np.ndarray            # s float32 (RFF phases)
    Xte: np.ndarray | None = None   # m x d float32 held-out points
    Yte: np.ndarray | None = None   # m x k float64 held-out targets

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def k(self) -> int:
        return self.Y.shape[1]


def rff_draw(seed: int, d: int, s: int, sigma: float) -> tuple[np.ndarray, np.ndarray]:
    """Draw the random Fourier feature sample (W d x s, b length s) as float32.

    W has i.i.d. N(0, sigma^-2) entries and b is U[0, 2 pi).  Both are rounded
    to float32 once so the oracle and the device see the same values.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    omega = rng.standard_normal((d, s))
    W = (omega / sigma).astype(np.float32)
    b = rng.uniform(0.0, 2.0 * math.pi, size=s).astype(np.float32)
    return W, b


def tensorsketch_draw(seed: int, d: int, q: int, s: int) -> tuple[np.ndarray, np.ndarray]:
    """Draw the hash and sign tables of a degree-q TensorSketch (Section 2.2).

    Returns ``h`` (q x d int32, entries uniform on [0, s)) and ``g`` (q x d int8,
    entries uniform on {-1, +1}).  Fully random tables are k-wise independent
    for every k, so they meet the 3-wise (hashes) and 4-wise (signs)
    requirements.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.integers(0, s, size=(q, d)).astype(np.int32)
    g = (2 * rng.integers(0, 2, size=(q, d)) - 1).astype(np.int8)
    return h, g


def srht_draw(seed: int, m: int, s2: int) -> tuple[np.ndarray, np.ndarray]:
    """Draw a subsampled randomized Hadamard transform of size s2 x m (Section 4):
    the diagonal of random signs D (m int8 in {-1, +1}) and the sampled rows of
    P (s2 distinct int32 indices, uniform without replacement, sorted)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    signs = (2 * rng.integers(0, 2, size=m) - 1).astype(np.int8)
    rows = np.sort(rng.choice(m, size=s2, replace=False)).astype(np.int32)
    return signs, rows


def gaussian_draw(seed: int, s3: int, s2: int) -> np.ndarray:
    """An s3 x s2 matrix of independent standard normal entries (the dense
    projection of Algorithm 2), rounded to float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((s3, s2)).astype(np.float32)


def _cfg1(n: int, s: int | None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(1001))
    d = 8
    X = rng.standard_normal((n, d))
    y = np.sin(X.sum(axis=1)) + 0.1 * rng.standard_normal(n)
    s = 200 if s is None else s
    W, b = rff_draw(2001, d, s, 1.0)
    return Problem("plain", X.astype(np.float32), y[:, None].astype(np.float64),
                   1.0, 1e-3, s, 1e-8, W, b)


def _cfg2(n: int, s: int | None, m: int | None = None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(1002))
    d, ncent = 64, 10
    centres = 2.0 * rng.standard_normal((ncent, d))             # N(0, 4I)
    labels = rng.integers(0, ncent, size=n)
    X = centres[labels] + rng.standard_normal((n, d))
    a = rng.standard_normal((ncent, d)) / math.sqrt(d)          # a_c ~ N(0, I/d)
    bc = rng.standard_normal(ncent)                             # b_c ~ N(0, 1)
    y = np.einsum("ij,ij->i", X, a[labels]) + bc[labels] + 0.1 * rng.standard_normal(n)
    sigma = math.sqrt(d)
    s = 2048 if s is None else s
    W, b = rff_draw(2002, d, s, sigma)
    P = Problem("precision", X.astype(np.float32), y[:, None].astype(np.float64),
                sigma, 1e-4, s, 1e-6, W, b)
    if m:
        # held-out points from the same mixture, drawn after every training draw
        lt = rng.integers(0, ncent, size=m)
        Xt = centres[lt] + rng.standard_normal((m, d))
        yt = np.einsum("ij,ij->i", Xt, a[lt]) + bc[lt] + 0.1 * rng.standard_normal(m)
        P.Xte, P.Yte = Xt.astype(np.float32), yt[:, None].astype(np.float64)
    return P


def _cfg3(n: int, s: int | None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(1003))
    d, ncls = 784, 10
    mask = rng.random((n, d)) < 0.19
    inten = 1.0 - rng.random((n, d))                            # U(0, 1]
    X = np.where(mask, inten, 0.0)
    labels = rng.integers(0, ncls, size=n)
    Y = np.zeros((n, ncls))
    Y[np.arange(n), labels] = 1.0
    s = 8192 if s is None else s
    W, b = rff_draw(2003, d, s, 8.0)
    return Problem("multirhs", X.astype(np.float32), Y, 8.0, 1e-3, s, 1e-6, W, b)


def _cfg5(n: int, s: int | None, m: int | None) -> Problem:
    rng = np.random.Generator(np.random.PCG64(1005))
    d = 54
    m = 16384 if m is None else m
    tot = n + m
    cont = rng.standard_normal((tot, 10))
    binf = (rng.random((tot, 44)) < 0.1).astype(np.float64)
    Xall = np.concatenate([cont, binf], axis=1)
    w = rng.standard_normal(d)
    proj = Xall @ w
    yall = np.where(proj - np.median(proj) >= 0.0, 1.0, -1.0)
    s = 4096 if s is None else s
    W, b = rff_draw(2005, d, s, 4.0)
    return Problem("grad", Xall[:n].astype(np.float32), yall[:n, None].copy(),
                   4.0, 1e-3, s, 1e-6, W, b,
                   Xte=Xall[n:].astype(np.float32), Yte=yall[n:, None].copy())


CONFIGS = {1: 2000, 2: 65536, 3: 60000, 5: 131072}


def make_config(i: int, n: int | None = None, s: int | None = None,
                m: int | None = None) -> Problem:
    """Draw workload ``i`` (1, 2, 3 or 5) at its full size or at ``n`` points.

    ``s`` overrides the feature count (smaller instances usually want fewer
    features); ``m`` overrides the held-out size of workload 5.
    """
    if i not in CONFIGS:
        raise ValueError(f"no single-problem workload {i}; use make_uneven for 4")
    n = CONFIGS[i] if n is None else int(n)
    if i == 1:
        return _cfg1(n, s)
    if i == 2:
        return _cfg2(n, s, m)
    if i == 3:
        return _cfg3(n, s)
    return _cfg5(n, s, m)


def make_uneven(nprob: int = 64, nmin: int = 1000, nmax: int = 32768,
                scale: float = 1.0) -> list[Problem]:
    """Draw the uneven batch: ``nprob`` independent problems of log-uniform size.

    ``scale`` shrinks every n (and s with it) for small test instances while
    keeping the same per-problem seeds and draws.
    """
    seqs = np.random.SeedSequence(1004).spawn(nprob)
    out = []
    for p, ss in enumerate(seqs):
        rng = np.random.Generator(np.random.PCG64(ss))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        d = int(rng.choice([16, 32, 64, 128]))
        lam = 10.0 ** rng.uniform(-5.0, -2.0)
        n = max(8, int(round(n * scale)))
        s = max(4, min(n // 8, 4096))
        X = rng.standard_normal((n, d))
        y = np.sin(X.sum(axis=1)) + 0.1 * rng.standard_normal(n)
        sigma = math.sqrt(d)
        fseed = int(ss.generate_state(1)[0])
        W, b = rff_draw(fseed, d, s, sigma)
        out.append(Problem(f"uneven{p}", X.astype(np.float32), y[:, None].astype(np.float64),
                           sigma, lam, s, 1e-6, W, b))
    return out
