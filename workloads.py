"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input recipes only (no step of the SAP method).  Both the
CUDA library's tests/benchmark and the CPU oracle draw their inputs from here,
so the two sides see bit-identical data.  All randomness is NumPy PCG64 with an
explicit seed.

Workloads (sizes from the benchmark configurations; shapes follow the paper):

* ``moment_curve``   -- the trigonometric moment curve of Sec. V,
  phi(t) = (cos t, sin t, ..., cos m t, sin m t) in R^{2m}, t ~ U[0, 2 pi).
* ``blob_images``    -- 64 x 64 grey images of one isotropic Gaussian blob
  (sigma 4 px) whose centre is uniform on [16, 48]^2: a synthetic stand-in for
  the illumination-space images of Sec. VI-B (a two-parameter family).
* ``hyperspectral``  -- linear mixtures of 5 endmember spectra over 224 bands
  with Dirichlet(1) abundances and Gaussian noise: a synthetic stand-in for
  the Indian Pines cube of Sec. VI-C.
* ``random_basis``   -- the starting basis: Q factor (diag R > 0) of a seeded
  Gaussian n x k matrix.

Arrays follow the library's conventions: X is (N, n) C-contiguous, a basis is
a (k, n) C-contiguous FP64 array whose rows are the basis vectors (= an n x k
column-major matrix).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_bf16_exact(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even) and return them as
    FP32 (every value exactly representable in BF16)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).reshape(a.shape)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """The upper 16 bits of BF16-exact FP32 values, as uint16."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    return (a.view(np.uint32) >> 16).astype(np.uint16)


def moment_curve(N: int, m: int, seed: int, dtype=np.float32,
                 noise: float = 0.0, noise_seed: int | None = None):
    """N samples of the trigonometric moment curve in R^{2m} (Sec. V), with
    optional i.i.d. Gaussian noise of standard deviation ``noise`` per
    coordinate (Sec. VII).  Returns X (N, 2m) in ``dtype``."""
    t = rng(seed).random(N) * TWO_PI
    X = np.empty((N, 2 * m), dtype=np.float64)
    for q in range(1, m + 1):
        X[:, 2 * q - 2] = np.cos(q * t)
        X[:, 2 * q - 1] = np.sin(q * t)
    if noise > 0.0:
        X += rng(noise_seed if noise_seed is not None else seed + 7919).normal(
            0.0, noise, size=X.shape)
    return np.ascontiguousarray(X.astype(dtype))


def random_basis(n: int, k: int, seed: int) -> np.ndarray:
    """Orthonormal starting basis: Q of a seeded Gaussian n x k matrix with
    diag(R) > 0, returned as (k, n) FP64."""
    G = rng(seed).standard_normal((n, k))
    Q, R = np.linalg.qr(G)
    Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)
    return np.ascontiguousarray(Q.T)


def blob_images(N: int, seed: int, side: int = 64, sigma: float = 4.0,
                lo: float = 16.0, hi: float = 48.0) -> np.ndarray:
    """N images (side x side, flattened row-major) of one Gaussian blob with
    centre uniform on [lo, hi]^2; values in (0, 1], FP32."""
    c = rng(seed).uniform(lo, hi, size=(N, 2))
    u = np.arange(side, dtype=np.float64)
    gx = np.exp(-((u[None, :] - c[:, 0:1]) ** 2) / (2.0 * sigma * sigma))
    gy = np.exp(-((u[None, :] - c[:, 1:2]) ** 2) / (2.0 * sigma * sigma))
    img = gy[:, :, None] * gx[:, None, :]
    return np.ascontiguousarray(img.reshape(N, side * side).astype(np.float32))


def endmembers(seed: int, n_bands: int = 224, n_end: int = 5) -> np.ndarray:
    """n_end spectra, each a sum of 3 Gaussians over the band index with
    centre ~ U[0, n_bands), width ~ U[5, 30], amplitude ~ U[0.2, 1]."""
    g = rng(seed)
    b = np.arange(n_bands, dtype=np.float64)
    E = np.zeros((n_end, n_bands))
    for e in range(n_end):
        for _ in range(3):
            mu = g.uniform(0.0, n_bands)
            sd = g.uniform(5.0, 30.0)
            a = g.uniform(0.2, 1.0)
            E[e] += a * np.exp(-((b - mu) ** 2) / (2.0 * sd * sd))
    return E


def hyperspectral(N: int, seed: int, E: np.ndarray, noise: float = 0.01,
                  bf16: bool = True) -> np.ndarray:
    """N pixels: Dirichlet(1) mixtures of the endmembers E plus Gaussian
    noise; rounded to BF16 when ``bf16`` (returned as BF16-exact FP32)."""
    g = rng(seed)
    A = g.dirichlet(np.ones(E.shape[0]), size=N)
    X = A @ E + g.normal(0.0, noise, size=(N, E.shape[1]))
    X = X.astype(np.float32)
    return to_bf16_exact(X) if bf16 else np.ascontiguousarray(X)


def hyperspectral_batch(B: int, seed: int, n_min: int = 500,
                        n_max: int = 20000, n_bands: int = 224,
                        scale: float = 1.0):
    """B datasets with N log-uniform in [n_min, n_max] (scaled by ``scale`` for
    reduced test sizes).  Returns (list of X, list of N)."""
    g = rng(seed)
    E = endmembers(seed + 1, n_bands)
    Ns = [max(2, int(math.floor(math.exp(g.uniform(math.log(n_min),
                                                     math.log(n_max)))) * scale))
          for _ in range(B)]
    Xs = [hyperspectral(Nb, seed + 100 + b, E) for b, Nb in enumerate(Ns)]
    return Xs, Ns


def subsample_indices(N: int, R: int, m: int, seed: int) -> np.ndarray:
    """R subsets of m distinct row indices of range(N) (Sec. VI-C: repeated
    random subsamples of a large point set), as an (R, m) int64 array."""
    g = rng(seed)
    return np.stack([np.sort(g.permutation(N)[:m]) for _ in range(R)]).astype(np.int64)


# The benchmark configurations (sizes as stated for each workload).
CONFIGS = {
    "c1": dict(workload="moment_curve_fp64_N200_n10_k3", N=200, m=5, k=3,
               alpha=0.01, T=1000, dtype="f64", data_seed=1, basis_seed=2),
    "c2": dict(workload="moment_curve_fp32_N8192_n100_k5", N=8192, m=50, k=5,
               alpha=0.005, T=2000, dtype="f32", data_seed=1, basis_seed=2),
    "c3": dict(workload="blob_images_N4096_n4096_k1to20", N=4096, n=4096,
               kmax=20, T=500, alpha=0.01, threshold=0.1, dtype="f32",
               data_seed=3, basis_seed=4),
    "c4": dict(workload="hyperspectral_32x_N500to20000_n224_k10_eps0.05",
               B=32, n=224, k=10, eps=0.05, T=500, alpha=0.01, dtype="bf16",
               data_seed=5, basis_seed=6),
    "subsample": dict(workload="hyperspectral_N21025_n200_10x512_k1to10", N=21025, n=200, R=10,
                      m=512, kmax=10, T=100, alpha=0.01, threshold=0.1, dtype="f32", data_seed=7,
                      basis_seed=8, index_seed=9),
    "c5": dict(workload="moment_curve_softmin_N16384_n100_k5", N=16384, m=50,
               k=5, tau=0.01, steps=200, eta=0.005, dtype="f32", data_seed=1,
               basis_seed=2),
}
