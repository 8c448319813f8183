"""GPU parity of the tile form of the fused kernel (form 2: persistent CTAs,
960-nonzero tiles, remap stores in destination order) against the FP64 oracle.

Bit-exact: the remapped working copy after every mode (indices, values, the
remap ids in words 4..6 and the write orders in word 7).  Numeric: normwise
relative error <= 1e-5 (FP32 factors; BF16 factors against the oracle on the
BF16-rounded factors, and <= 1e-2 against the FP32 factors).  Outputs are
pre-filled with NaN.  Sizes cover ragged last tiles, blocks smaller than a
tile, one block spanning many tiles, several blocks per CTA, a row split over
every block and rows with no nonzero.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan

pytestmark = pytest.mark.gpu

TILE = 960


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def check_raw(p, coo, m):
    """Words 0..3, the remap ids (words 4..6) and the write orders (word 7) of the
    working copy, which is in mode-m order."""
    raw = p.raw_elements()
    order = O.canonical_order(coo, m)
    assert np.array_equal(raw[:, :3], coo[order].astype(np.int32))
    pos = [np.empty(coo.shape[0], np.int64) for _ in range(3)]
    for k in range(3):
        pos[k][O.canonical_order(coo, k)] = np.arange(coo.shape[0])
        assert np.array_equal(raw[:, 4 + k] & 0x7fffffff, pos[k][order]), k
    w = raw[:, 7].view(np.uint32)
    for k in range(3):
        want = O.tile_write_order(coo, k, TILE)[pos[k][order]]
        assert np.array_equal((w >> (10 * k)) & 1023, want), k
    # bit 31 of word 4 + k: i_k is one of the hot rows of factor k
    H = p.info()["hot_rows"]
    assert H > 0
    for k in range(3):
        hot = np.isin(coo[order, k], O.hot_rows(coo, k, H))
        assert np.array_equal(raw[:, 4 + k] < 0, hot), k


def run(coo, vals, dims, R, dtype="f32", nblk=0, seed=3, check_words=True):
    c, v = coo.numpy(), vals.numpy()
    F = synth.make_factors(dims, R, seed=seed)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda() for f in F]
    p = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, checks=True, variant=2)
    outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    if check_words:
        check_raw(p, c, 0)
    for n in range(3):
        p.compute(n, Fd, outs[n])
        idx, val = p.elements()
        wi, wv = O.elements_in_order(c, v, (n + 1) % 3)
        assert np.array_equal(idx, wi), f"mode {n}: remapped indices differ"
        assert np.array_equal(val.view(np.uint32), wv.view(np.uint32)), n
        if check_words:
            check_raw(p, c, (n + 1) % 3)
    torch.cuda.synchronize()
    got = [o.cpu().numpy().astype(np.float64) for o in outs]
    Fh = [f.to(tdt).float().numpy() for f in F]
    return p, got, F, Fh


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tile_form_all_modes_match_oracle(R, dtype):
    dims = (600, 450, 3000)
    coo, vals = synth.make_coo(dims, 20_000, (1.1, 1.1, 1.1), seed=200 + R)
    p, got, F, Fh = run(coo, vals, dims, R, dtype=dtype, nblk=37)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert np.all(np.isfinite(got[n])), f"mode {n}: unwritten rows"
        want = O.mttkrp(c, v, dims, Fh, n)
        assert O.relerr(got[n], want) <= 1e-5, (n, O.relerr(got[n], want))
        if dtype == "bf16":
            want32 = O.mttkrp(c, v, dims, [f.numpy() for f in F], n)
            assert O.relerr(got[n], want32) <= 1e-2
    p.close()


@pytest.mark.parametrize("nnz,nblk", [(TILE, 1), (TILE + 1, 1), (7777, 1), (7777, 3),
                                      (7777, 97), (7777, 2000), (50_000, 0), (50_000, 600),
                                      (123_457, 1217)])
def test_tile_form_ragged_tiles_and_block_counts(nnz, nblk):
    dims = (500, 80, 6000)
    coo, vals = synth.make_coo(dims, nnz, (1.2, 1.1, 0.0), seed=nnz + nblk)
    p, got, F, Fh = run(coo, vals, dims, 32, nblk=nblk, check_words=nnz < 60_000)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert np.all(np.isfinite(got[n])), n
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= 1e-5, n
    p.close()


def test_tile_form_heavy_row_split_over_every_block_and_empty_rows():
    n = 30_000
    g = torch.Generator().manual_seed(4)
    coo = torch.stack([torch.full((n,), 2, dtype=torch.int64),
                       torch.randperm(n, generator=g) % 300, torch.arange(n) // 300], 1)
    coo = torch.unique(coo, dim=0)
    coo = coo[torch.randperm(coo.shape[0], generator=g)]
    vals = torch.rand(coo.shape[0], generator=g)
    dims = (5, 300, 200)
    p, got, F, Fh = run(coo, vals, dims, 32, nblk=64)
    assert p.splits(0).tolist() == [[2, 0, 63]]
    c, v = coo.numpy(), vals.numpy()
    for m in range(3):
        assert O.relerr(got[m], O.mttkrp(c, v, dims, Fh, m)) <= 1e-5, m
    assert np.all(got[0][[0, 1, 3, 4]] == 0.0)
    p.close()


def test_tile_form_graph_sweeps_are_bit_identical_to_eager_and_form_0():
    dims = (700, 500, 9000)
    coo, vals = synth.make_coo(dims, 80_000, (1.1, 1.1, 1.1), seed=9)
    c, v = coo.numpy(), vals.numpy()
    F = [f.cuda() for f in synth.make_factors(dims, 32, seed=5)]
    p = Plan(c, v, dims, 32, variant=2)
    o1 = [torch.empty(d, 32, device="cuda") for d in dims]
    o2 = [torch.empty(d, 32, device="cuda") for d in dims]
    p.sweep(F, o1)
    p.sweep(F, o2, graph=True)
    p.sweep(F, o2, graph=True)
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(o1[n], o2[n]), n
    q = Plan(c, v, dims, 32, variant=0)
    o3 = [torch.empty(d, 32, device="cuda") for d in dims]
    q.sweep(F, o3)
    torch.cuda.synchronize()
    Fh = [f.cpu().numpy() for f in F]
    for n in range(3):
        want = O.mttkrp(c, v, dims, Fh, n)
        assert O.relerr(o1[n].cpu().numpy().astype(np.float64), want) <= 1e-5
        assert O.relerr(o3[n].cpu().numpy().astype(np.float64), want) <= 1e-5
    p.close()
    q.close()
