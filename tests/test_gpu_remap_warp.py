"""GPU parity of form 3 of the fused kernel (warp blocks with one remap warp per
CTA: seven warps compute, the eighth stores the CTA's 960-nonzero write-order
tiles in destination order) against the FP64 oracle and against form 0.

Bit-exact: the remapped working copy after every mode (indices, values and the
remap ids of words 4..6), and the outputs against a form-0 plan with the same
blocks (the compute warps run form 0's arithmetic on the same blocks).  Numeric:
normwise relative error <= 1e-5 against the oracle (BF16 factors: against the
oracle on the BF16-rounded factors).  Outputs are pre-filled with NaN.  Sizes
cover fewer nonzeros than a tile, ragged last tiles, block counts that are not
a multiple of the CTA's seven compute warps, one CTA over the whole tensor, a
row split over every block, and graph replays.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def check_copy(p, c, v, m):
    """Indices, values and remap ids of the working copy, which is in mode-m order."""
    idx, val = p.elements()
    wi, wv = O.elements_in_order(c, v, m)
    assert np.array_equal(idx, wi), f"mode-{m} order: indices differ"
    assert np.array_equal(val.view(np.uint32), wv.view(np.uint32)), m
    raw = p.raw_elements()
    order = O.canonical_order(c, m)
    for k in range(3):
        pos = np.empty(c.shape[0], np.int64)
        pos[O.canonical_order(c, k)] = np.arange(c.shape[0])
        assert np.array_equal(raw[:, 4 + k] & 0x7fffffff, pos[order]), k


def run_pair(coo, vals, dims, R, dtype="f32", nblk=0, seed=3):
    """Form 3 and form 0 with the same blocks, mode by mode; returns both outputs."""
    c, v = coo.numpy(), vals.numpy()
    F = synth.make_factors(dims, R, seed=seed)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda() for f in F]
    p3 = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, checks=True, variant=3)
    p0 = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, checks=True, variant=0)
    assert p3.info()["variant"] == 3
    o3 = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    o0 = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    for n in range(3):
        p3.compute(n, Fd, o3[n])
        p0.compute(n, Fd, o0[n])
        check_copy(p3, c, v, (n + 1) % 3)
    torch.cuda.synchronize()
    got3 = [o.cpu().numpy() for o in o3]
    got0 = [o.cpu().numpy() for o in o0]
    Fh = [f.to(tdt).float().numpy() for f in F]
    p3.close()
    p0.close()
    return got3, got0, Fh


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_remap_warp_all_modes_match_oracle_and_form_0(R, dtype):
    dims = (600, 450, 3000)
    coo, vals = synth.make_coo(dims, 20_000, (1.1, 1.1, 1.1), seed=300 + R)
    got3, got0, Fh = run_pair(coo, vals, dims, R, dtype=dtype, nblk=37)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert np.all(np.isfinite(got3[n])), f"mode {n}: unwritten rows"
        assert np.array_equal(got3[n].view(np.uint32), got0[n].view(np.uint32)), n
        want = O.mttkrp(c, v, dims, Fh, n)
        assert O.relerr(got3[n].astype(np.float64), want) <= 1e-5, n


@pytest.mark.parametrize("nnz,nblk", [(100, 1), (959, 3), (960, 7), (961, 8), (7777, 1),
                                      (7777, 13), (7777, 2000), (50_000, 0), (123_457, 1217)])
def test_remap_warp_ragged_tiles_and_block_counts(nnz, nblk):
    dims = (500, 80, 6000)
    coo, vals = synth.make_coo(dims, nnz, (1.2, 1.1, 0.0), seed=nnz + 3 * nblk)
    got3, got0, Fh = run_pair(coo, vals, dims, 32, nblk=nblk)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert np.array_equal(got3[n].view(np.uint32), got0[n].view(np.uint32)), n
        assert O.relerr(got3[n].astype(np.float64), O.mttkrp(c, v, dims, Fh, n)) <= 1e-5, n


def test_remap_warp_heavy_row_split_over_every_block():
    n = 30_000
    g = torch.Generator().manual_seed(5)
    coo = torch.stack([torch.full((n,), 2, dtype=torch.int64),
                       torch.randperm(n, generator=g) % 300, torch.arange(n) // 300], 1)
    coo = torch.unique(coo, dim=0)
    coo = coo[torch.randperm(coo.shape[0], generator=g)]
    vals = torch.rand(coo.shape[0], generator=g)
    dims = (5, 300, 200)
    got3, got0, Fh = run_pair(coo, vals, dims, 32, nblk=64)
    c, v = coo.numpy(), vals.numpy()
    for m in range(3):
        assert np.array_equal(got3[m].view(np.uint32), got0[m].view(np.uint32)), m
        assert O.relerr(got3[m].astype(np.float64), O.mttkrp(c, v, dims, Fh, m)) <= 1e-5, m
    assert np.all(got3[0][[0, 1, 3, 4]] == 0.0)


def test_remap_warp_graph_sweeps_bit_identical_to_eager():
    dims = (700, 500, 9000)
    coo, vals = synth.make_coo(dims, 80_000, (1.1, 1.1, 1.1), seed=11)
    c, v = coo.numpy(), vals.numpy()
    F = [f.cuda() for f in synth.make_factors(dims, 32, seed=6)]
    p = Plan(c, v, dims, 32, variant=3, checks=True)
    o1 = [torch.empty(d, 32, device="cuda") for d in dims]
    o2 = [torch.empty(d, 32, device="cuda") for d in dims]
    p.sweep(F, o1)
    p.sweep(F, o2, graph=True)
    p.sweep(F, o2, graph=True)
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(o1[n], o2[n]), n
    check_copy(p, c, v, 0)
    p.close()
