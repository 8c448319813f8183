"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers: COO coordinates (uniform or Zipf
skewed per mode), nonzero values and dense factor matrices.  It holds none of
the MTTKRP / CP arithmetic, so the FP64 oracle and the CUDA path can both be
fed from it without sharing any of the method's code.

The paper measures on FROSTT and recommender-system tensors (Amazon,
Delicious, Music, Nell1, Twitch, Vast; Section 5.1.3, Table 3).  Those files
are not available here; the workloads below are synthetic stand-ins with the
shapes, nonzero counts and per-mode index skew of such tensors.

Recipe (all draws from ``torch.Generator`` seeded per call):
  * per mode k, an index is drawn either uniformly over [0, I_k) or from a
    Zipf(s) law over ranks 1..I_k by inverse CDF on the FP64 cumulative sum of
    r^-s; the rank is mapped through a seeded permutation of [0, I_k) so that
    the heavy indices are scattered over the index space;
  * coordinates are drawn in batches; repeats are dropped keeping the first
    draw, and drawing continues until ``nnz`` distinct coordinates exist; the
    first ``nnz`` distinct ones in draw order are kept;
  * values are FP32 U(0,1); factors are FP32 N(0,1) (times a scale).

Generation runs on the CPU for small cases and on a CUDA device (torch ops
only, for speed) for the large ones; a given (device, seed) is reproducible.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import torch

__all__ = ["TensorSpec", "WORKLOADS", "make_coo", "make_factors", "make_planted_targets",
           "workload"]


@dataclasses.dataclass(frozen=True)
class TensorSpec:
    name: str
    dims: tuple
    nnz: int
    skew: tuple          # per mode: 0.0 = uniform, s > 0 = Zipf(s)
    ranks: tuple         # ranks R the workload is run at
    seed: int            # tensor seed; factor k of rank R uses seed_f + 10*k


# The five workload families (sizes, skews and ranks of the paper-like tensors).
WORKLOADS = {
    "c1": TensorSpec("3-mode 200x150x100, 50k nnz uniform", (200, 150, 100), 50_000,
                     (0.0, 0.0, 0.0), (16,), 1001),
    "c2": TensorSpec("3-mode 120000x90000x2000000, 100M nnz, Zipf 1.1",
                     (120_000, 90_000, 2_000_000), 100_000_000, (1.1, 1.1, 1.1), (32,), 1002),
    "c3": TensorSpec("4-mode 1000000x20000x2000x500, 150M nnz, Zipf 1.2 on modes 0-1",
                     (1_000_000, 20_000, 2_000, 500), 150_000_000, (1.2, 1.2, 0.0, 0.0),
                     (32, 64), 1003),
    "c4a": TensorSpec("5-mode 500000x50000x5000x1000x200, 60M nnz, Zipf 1.1",
                      (500_000, 50_000, 5_000, 1_000, 200), 60_000_000, (1.1,) * 5,
                      (16, 32, 64), 1004),
    "c4b": TensorSpec("6-mode 200000x20000x2000x500x100x50, 40M nnz, Zipf 1.1",
                      (200_000, 20_000, 2_000, 500, 100, 50), 40_000_000, (1.1,) * 6,
                      (16, 32, 64), 1014),
    "c5": TensorSpec("3-mode CP completion 2000000x2000000x100000, 200M observed, Zipf 1.1",
                     (2_000_000, 2_000_000, 100_000), 200_000_000, (1.1, 1.1, 1.1), (64,), 1005),
    "c5fd": TensorSpec("3-mode CP completion 30x20x10, 500 observed (finite-difference copy)",
                       (30, 20, 10), 500, (1.1, 1.1, 1.1), (8,), 1015),
}


def workload(name: str) -> TensorSpec:
    return WORKLOADS[name]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _draw_mode(g, n: int, dim: int, s: float, perm: Optional[torch.Tensor], device) -> torch.Tensor:
    u = torch.rand(n, generator=g, dtype=torch.float64, device=device)
    if s == 0.0:
        idx = torch.clamp((u * dim).to(torch.int64), max=dim - 1)
        return idx
    r = torch.arange(1, dim + 1, dtype=torch.float64, device=device)
    w = torch.pow(r, -float(s))
    cdf = torch.cumsum(w, 0)
    cdf = cdf / cdf[-1]
    rank = torch.searchsorted(cdf, u, right=True)
    rank = torch.clamp(rank, max=dim - 1)
    return perm[rank]


def _keys(coo: torch.Tensor, dims: Sequence[int]) -> torch.Tensor:
    """64-bit key per coordinate: the linear index when it fits, else a hash.

    A hash collision between two distinct coordinates only drops one extra
    draw; equal coordinates always get equal keys, so the kept set is distinct.
    """
    total = 1
    for d in dims:
        total *= int(d)
    if total < 2 ** 62:
        key = torch.zeros(coo.shape[0], dtype=torch.int64, device=coo.device)
        for k, d in enumerate(dims):
            key = key * int(d) + coo[:, k]
        return key
    key = torch.full((coo.shape[0],), 0x1234567, dtype=torch.int64, device=coo.device)
    mult = 0x5DEECE66D  # odd multiplier; int64 products wrap modulo 2^64
    for k in range(coo.shape[1]):
        key = key * mult + coo[:, k] + 0x9E3779B1 * (k + 1)
        key = key ^ (key >> 29)
    return key


def make_coo(dims: Sequence[int], nnz: int, skew: Sequence[float], seed: int,
             device="cpu") -> tuple:
    """Distinct random coordinates and FP32 U(0,1) values.

    Returns ``(coo, vals)``: ``coo`` int64 [nnz, N] and ``vals`` float32 [nnz],
    on ``device``, in draw order (not sorted).
    """
    dims = [int(d) for d in dims]
    N = len(dims)
    g = _gen(seed, device)
    perms = []
    for k in range(N):
        if skew[k] > 0:
            perms.append(torch.randperm(dims[k], generator=g, device=device))
        else:
            perms.append(None)
    space = 1
    for d in dims:
        space *= d
    if nnz > space:
        raise ValueError("more nonzeros requested than coordinates exist")
    have = torch.empty((0, N), dtype=torch.int64, device=device)
    while have.shape[0] < nnz:
        need = nnz - have.shape[0]
        batch = int(need * 1.25) + 1024
        cols = [_draw_mode(g, batch, dims[k], float(skew[k]), perms[k], device) for k in range(N)]
        cand = torch.cat([have, torch.stack(cols, 1)], 0)
        key = _keys(cand, dims)
        _, inv = torch.unique(key, return_inverse=True)
        pos = torch.arange(cand.shape[0], device=device)
        first = torch.full((int(inv.max().item()) + 1,), cand.shape[0], dtype=torch.int64,
                           device=device)
        first.scatter_reduce_(0, inv, pos, reduce="amin", include_self=True)
        keep, _ = torch.sort(first)
        have = cand[keep]
        del cand, key, inv, pos, first, keep, cols
    coo = have[:nnz].contiguous()
    vals = torch.rand(nnz, generator=g, dtype=torch.float32, device=device)
    return coo, vals


def make_factors(dims: Sequence[int], rank: int, seed: int, device="cpu",
                 scale: float = 1.0, dtype=torch.float32) -> List[torch.Tensor]:
    """Dense factor matrices A_k (I_k x R, row-major), N(0,1) * scale, seed + 10*k."""
    out = []
    for k, d in enumerate(dims):
        g = _gen(seed + 10 * k, device)
        a = torch.randn(int(d), int(rank), generator=g, dtype=torch.float32, device=device)
        if scale != 1.0:
            a = a * scale
        out.append(a.to(dtype))
    return out


def make_planted_targets(coo: torch.Tensor, dims: Sequence[int], planted_rank: int,
                         noise_std: float, seed: int) -> torch.Tensor:
    """Observed entries of a planted low-rank model plus Gaussian noise.

    The planted factors are N(0,1) * planted_rank^(-1/(2N)) so that a model
    entry (a sum of planted_rank products of N factor entries) has unit
    variance; the noise is N(0, noise_std^2).  This builds the
    workload's target values only; the CP loss under test evaluates the model
    of different (fitted) factors.
    """
    N = len(dims)
    scale = float(planted_rank) ** (-1.0 / (2 * N))
    P = make_factors(dims, planted_rank, seed, device=coo.device, scale=scale)
    acc = torch.ones(coo.shape[0], planted_rank, dtype=torch.float64, device=coo.device)
    for k in range(N):
        acc = acc * P[k].to(torch.float64)[coo[:, k]]
    g = _gen(seed + 7, coo.device)
    noise = torch.randn(coo.shape[0], generator=g, dtype=torch.float64, device=coo.device)
    return (acc.sum(1) + noise_std * noise).to(torch.float32)


def factor_seed(config_index: int) -> int:
    """Factor seed base 2000 + 10*c for workload c (factor k adds 10*k)."""
    return 2000 + 10 * int(config_index)


def zipf_top_share(dim: int, s: float) -> float:
    """Probability mass of the most likely index of a Zipf(s) law over 1..dim."""
    h = sum(r ** (-s) for r in range(1, min(dim, 200000) + 1))
    if dim > 200000:  # tail by integral
        h += ((dim + 0.5) ** (1 - s) - (200000.5) ** (1 - s)) / (1 - s)
    return 1.0 / h if not math.isclose(h, 0.0) else 1.0
