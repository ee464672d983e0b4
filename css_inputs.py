"""Seeded synthetic inputs for greedy column subset selection.

This module is the only code shared by the CPU oracle side (tests, the CPU
baseline) and the CUDA side (tests, bench).  It draws random matrices and
formats them (bf16 rounding, column-major packing); it contains none of the
selection method's arithmetic.

Workloads (the paper's data sets are not available; these stand in for them
with the shapes of the paper's problems, Sec. 7):

* ``lowrank_uv``        A = U V + noise * N(0,1): U (m x rank), V (rank x n)
                        i.i.d. N(0,1).  Rank-r signal plus white noise.
* ``lowrank_decaying``  A = U diag(s) V^T + noise * N(0,1), U and V orthonormalised
                        Gaussians (QR), s_i = 1/i.
* ``gaussian_omega``    Omega (n x r) i.i.d. N(0, 1/r): the Gaussian random
                        projection of Sec. 5.1.
* ``lognormal_blocks``  c column-block widths ~ LogNormal(ln median, sigma), scaled
                        to sum to n with largest-remainder rounding, each >= min_w.
* ``batched_instances`` independent low-rank instances of uneven sizes.

All generators use ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lowrank_uv",
    "lowrank_decaying",
    "gaussian_omega",
    "lognormal_blocks",
    "batched_specs",
    "batched_instance",
    "round_bf16",
    "bf16_bits",
    "bits_to_f32",
    "CONFIGS",
]


def lowrank_uv(m, n, rank, noise, seed, dtype=np.float64):
    """A = U V + noise * N, U m x rank, V rank x n, N m x n, all i.i.d. N(0,1)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((rank, n))
    A = U @ V
    if noise:
        A += noise * rng.standard_normal((m, n))
    return A.astype(dtype, copy=False)


def lowrank_decaying(m, n, rank, noise, seed, dtype=np.float32, chunk=8192):
    """A = U diag(s) V^T + noise * N with s_i = 1/i, U (m x rank) and V (n x rank)
    orthonormalised Gaussians.  Built column-chunk by column-chunk so the
    float64 intermediate stays small at large n."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    s = 1.0 / np.arange(1, rank + 1, dtype=np.float64)
    US = U * s
    A = np.empty((m, n), dtype=dtype)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        blk = US @ V[c0:c1].T
        if noise:
            blk += noise * rng.standard_normal((m, c1 - c0))
        A[:, c0:c1] = blk
    return A


def gaussian_omega(n, r, seed, dtype=np.float32):
    """Omega (n x r), i.i.d. N(0, 1/r)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, r)) / np.sqrt(r)).astype(dtype)


def lognormal_blocks(n, c, median, sigma, seed, min_w=100):
    """Column block offsets (c+1 values) with log-normal widths summing to n."""
    rng = np.random.default_rng(seed)
    w = rng.lognormal(np.log(median), sigma, size=c)
    w = np.maximum(w, 1e-12)
    avail = n - min_w * c
    if avail < 0:
        raise ValueError("n too small for c blocks of min_w columns")
    share = w / w.sum() * avail
    base = np.floor(share).astype(np.int64)
    rem = int(avail - base.sum())
    order = np.argsort(-(share - base), kind="stable")
    base[order[:rem]] += 1
    widths = base + min_w
    return np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)


def batched_specs(count, seed, m_range=(64, 1024), n_range=(128, 4096),
                  k_range=(8, 64)):
    """Sizes (m, n, k) of ``count`` independent instances, each uniform on the
    inclusive integer ranges."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    ks = rng.integers(k_range[0], k_range[1] + 1, size=count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(ms, ns, ks)]


def batched_instance(m, n, k, seed, noise=1e-2, dtype=np.float32):
    """One batched instance: rank-k U V plus ``noise`` Gaussian noise."""
    return lowrank_uv(m, n, k, noise, seed, dtype=dtype)


def round_bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float32.  NaN/Inf are not expected in these workloads."""
    return bits_to_f32(bf16_bits(x))


def bf16_bits(x):
    """bfloat16 bit patterns (uint16) of float32 values, round-to-nearest-even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & np.uint32(1)
    r = (u + np.uint32(0x7FFF) + lsb) >> 16
    return r.astype(np.uint16)


def bits_to_f32(bits):
    """float32 values of bfloat16 bit patterns."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32)


# The workloads as named configurations (sizes, distributions and seeds).
CONFIGS = {
    # Centralized greedy, plain FP64: 500 x 1000, rank 50 + 0.01 noise, k = 50.
    "fp64_500x1000": dict(m=500, n=1000, rank=50, noise=0.01, seed=0, k=50),
    # Memory-efficient centralized greedy at scale: 4096 x 65536, rank 256,
    # s_i = 1/i, noise 1e-3, k = 256, streamed in FP32 and in BF16.
    "decay_4096x65536": dict(m=4096, n=65536, rank=256, noise=1e-3, seed=0, k=256),
    # Profiling case of the same model: half the columns, 16 iterations.
    "decay_4096x32768": dict(m=4096, n=32768, rank=256, noise=1e-3, seed=0, k=16),
    # Distributed-style GCSS: 2048 x 262144 BF16 rank 400, Omega 262144 x 400,
    # 64 log-normal blocks (median 3000, sigma 0.8), 100 per block, k = 100.
    "dist_2048x262144": dict(m=2048, n=262144, rank=400, noise=1e-3, seed=1,
                             r=400, omega_seed=2, blocks=64, block_median=3000,
                             block_sigma=0.8, block_seed=3, l_block=100, k=100),
    # Batched independent CSS: 1024 instances, FP32, rank k + 1e-2 noise.
    "batched_1024": dict(count=1024, seed=4, noise=1e-2),
    # The same model with 128 problems (the DRAM capture of the batched launch).
    "batched_128": dict(count=128, seed=4, noise=1e-2),
    # Adjoint of the reconstruction error: 4096 x 16384 FP32 rank 128 + 1e-3, k = 128.
    "adjoint_4096x16384": dict(m=4096, n=16384, rank=128, noise=1e-3, seed=5, k=128),
}
