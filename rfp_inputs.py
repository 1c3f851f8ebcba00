"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds only input recipes (random matrices with a prescribed
structure); none of the factorization, solve, inversion or packing
arithmetic lives here.  Every generator is a pure function of its arguments.

Recipes (the paper publishes no matrices; these are the workloads the
benchmark configurations describe):

* ``spd_bbt(n, seed)``: B with i.i.d. uniform[-1, 1] entries drawn from
  ``numpy.random.default_rng(seed)`` (PCG64), A = B B^T / n + I.  The
  condition number is O(1-10).  ``rhs(...)`` continues the same generator.
* ``spd_spectrum(n, seed, kappa)``: A = Q diag(lam) Q^T with Q Haar-random
  orthogonal (QR of a Gaussian matrix, signs fixed by diag(R) > 0), lam_1 = 1,
  lam_n = kappa and the others 10^U(0, log10 kappa): the 2-norm condition
  number is exactly kappa.  For n > 4096 the same recipe runs on a CUDA device
  with torch in FP64 (device RNG) when one is present.
* ``spd_butterfly(n, seed, kappa, device)``: A = Q diag(lam) Q^T with the
  same spectrum recipe and Q a random butterfly transform: log2(n) levels of
  Givens rotations with i.i.d. uniform angles pairing i and i + 2^l, so every
  eigenvector is spread over all coordinates (n must be a power of two).
  O(n^2 log n) work: the stand-in for a Haar Q at n = 32768, where the QR of
  a Gaussian matrix would cost ~1e14 FP64 flops.
* ``spd_reflectors(n, seed, kappa, device)``: A = Q diag(lam) Q^T with the
  same spectrum recipe and Q the product of 8 random Householder reflectors
  I - 2 v v^T (v uniform on the sphere): O(n^2) work per reflector, any n,
  every entry non-zero; the serving workload's generator (orders up to 8192
  for hundreds of matrices).
* ``spd_integer_factor(n, seed)``: A = L0 L0^T with L0 unit lower triangular
  with small integer entries; the exact Cholesky factor is L0.
* ``pascal(n)``: P_ij = C(i+j, i); its Cholesky factor is L_ij = C(i, j).
"""
from __future__ import annotations

from math import comb

import numpy as np


def spd_bbt(n: int, seed: int = 0, return_rng: bool = False):
    rng = np.random.default_rng(seed)
    B = rng.uniform(-1.0, 1.0, (n, n))
    A = B @ B.T / max(n, 1) + np.eye(n)
    A = 0.5 * (A + A.T)
    A = np.asfortranarray(A)
    return (A, rng) if return_rng else A


def rhs(n: int, nrhs: int, rng=None, seed: int | None = None):
    if rng is None:
        rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, (n, nrhs)))


def spectrum(n: int, kappa: float, rng) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    lam = 10.0 ** rng.uniform(0.0, np.log10(kappa), n)
    lam[0], lam[-1] = 1.0, float(kappa)
    return lam


def _preload_torch_linalg(torch):
    """torch loads its CUDA linear-algebra library lazily by file name; under
    a profiler's injection that lookup can fail, so load it by full path."""
    import ctypes
    import os
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def spd_spectrum(n: int, seed: int = 0, kappa: float = 1e4, device=None):
    """A = Q diag(lam) Q^T, Haar Q.  Returns numpy (CPU) unless ``device`` is a
    torch CUDA device, in which case a torch FP64 tensor on that device."""
    if device is not None:
        import torch
        _preload_torch_linalg(torch)
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        G = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
        Q, R = torch.linalg.qr(G)
        Q *= torch.sign(torch.diagonal(R)).unsqueeze(0)
        del G, R
        u = torch.rand(n, dtype=torch.float64, device=device, generator=g)
        lam = 10.0 ** (u * np.log10(kappa))
        lam[0], lam[-1] = 1.0, float(kappa)
        A = (Q * lam.unsqueeze(0)) @ Q.T
        del Q
        return 0.5 * (A + A.T)  # exactly symmetric: row- and column-major agree
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q *= np.sign(np.diag(R))[None, :]
    lam = spectrum(n, kappa, rng)
    A = (Q * lam[None, :]) @ Q.T
    return np.asfortranarray(0.5 * (A + A.T))


def spd_butterfly(n: int, seed: int = 0, kappa: float = 1e4, device=None):
    """A = Q diag(lam) Q^T, Q a random butterfly transform (torch FP64 on
    ``device``, returned as a torch tensor; symmetric, so row- and
    column-major storage agree)."""
    import torch
    if n & (n - 1):
        raise ValueError("the butterfly generator needs n a power of two")
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(n, dtype=torch.float64, device=device, generator=g)
    lam = 10.0 ** (u * np.log10(kappa))
    lam[0], lam[-1] = 1.0, float(kappa)
    A = torch.diag(lam)
    h = 1
    while h < n:
        theta = 2 * np.pi * torch.rand(n // 2, dtype=torch.float64, device=device, generator=g)
        c, s = torch.cos(theta), torch.sin(theta)
        # rotation on coordinate pairs (i, i + h) inside blocks of 2h: A <- G A G^T
        for dim in (0, 1):
            V = A.view(n // (2 * h), 2, h, n) if dim == 0 else A.view(n, n // (2 * h), 2, h)
            if dim == 0:
                x, y = V[:, 0].clone(), V[:, 1]
                cc, ss = c.view(n // (2 * h), h, 1), s.view(n // (2 * h), h, 1)
                V[:, 0] = cc * x - ss * y
                V[:, 1] = ss * x + cc * y
            else:
                x, y = V[:, :, 0].clone(), V[:, :, 1]
                cc, ss = c.view(1, n // (2 * h), h), s.view(1, n // (2 * h), h)
                V[:, :, 0] = cc * x - ss * y
                V[:, :, 1] = ss * x + cc * y
        h *= 2
    return 0.5 * (A + A.T)


def spd_reflectors(n: int, seed: int = 0, kappa: float = 1e4, device=None, reflectors: int = 8):
    """A = Q diag(lam) Q^T, Q = H_1 ... H_r with H_i = I - 2 v_i v_i^T (torch
    FP64 on ``device``, returned as a torch tensor)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = torch.rand(n, dtype=torch.float64, device=device, generator=g)
    lam = 10.0 ** (u * np.log10(kappa))
    lam[0] = 1.0
    if n > 1:
        lam[-1] = float(kappa)
    A = torch.diag(lam)
    for _ in range(reflectors):
        v = torch.randn(n, dtype=torch.float64, device=device, generator=g)
        v /= torch.linalg.vector_norm(v)
        # H A H with H = I - 2 v v^T:  A - 2 v w^T - 2 w v^T + 4 (v^T w) v v^T, w = A v
        w = A @ v
        A -= 2.0 * torch.outer(v, w) + 2.0 * torch.outer(w, v) - 4.0 * torch.dot(v, w) * torch.outer(v, v)
    return (A + A.T) * 0.5


def spd_integer_factor(n: int, seed: int = 0, lo: int = -2, hi: int = 2):
    """(A, L0) with A = L0 L0^T exactly in FP64 (small integers)."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.integers(lo, hi + 1, (n, n)).astype(np.float64), -1) + np.eye(n)
    A = L0 @ L0.T
    return np.asfortranarray(A), L0


def pascal(n: int):
    """(P, L) with P_ij = C(i+j, i) and L_ij = C(i, j) (0-based)."""
    P = np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    L = np.array([[comb(i, j) for j in range(n)] for i in range(n)], dtype=np.float64)
    return np.asfortranarray(P), L


def second_difference(n: int):
    """(K, K^{-1}) for the tridiagonal [-1, 2, -1] matrix; its inverse is
    min(i,j) (n+1-max(i,j)) / (n+1) with 1-based i, j."""
    K = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    i = np.arange(1, n + 1)
    Kinv = np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1)
    return np.asfortranarray(K), Kinv


LAYOUTS = [(t, u) for t in "NT" for u in "LU"]
