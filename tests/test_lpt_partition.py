"""Algorithm 1 partition (opts.partition = 1) against the oracle.

Host plans (CPU): every mode's working-copy order is (block of i_n, K_n) with the
oracle's LPT blocks, bit for bit: the mode-0 copy, next_pos of every mode, the
block bounds (block loads in block order), and no split rows.  GPU: every mode's
output against the FP64 oracle and the remapped copy after every pass against the
oracle's order, for both kernel forms, 16- and 32-byte nonzeros, 3 and 4 modes,
and a row heavier than any balanced block (never split by Algorithm 1).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, SpmError


def lpt_orders(c, kappa):
    """Per mode: rid (position of each input nonzero in the mode's order) and order."""
    out = []
    for n in range(c.shape[1]):
        rid = O.lpt_remap_ids(c, n, kappa)
        order = np.empty_like(rid)
        order[rid] = np.arange(rid.shape[0])
        out.append((rid, order))
    return out


CASES = [((60, 40, 30), 3000, (1.1, 1.1, 1.1), 7),
         ((40, 30, 20, 10), 2500, (1.2, 0.0, 1.1, 0.0), 13),
         ((300, 20, 10), 1500, (0.0, 0.0, 0.0), 64),
         ((25, 30), 400, (1.3, 0.0), 5)]


@pytest.mark.parametrize("dims,nnz,skew,kappa", CASES)
def test_host_plan_orders_match_oracle(dims, nnz, skew, kappa):
    coo, vals = synth.make_coo(dims, nnz, skew, seed=nnz + kappa)
    c, v = coo.numpy(), vals.numpy()
    p = Plan(c, v, dims, 8, nblk=kappa, host_only=True, partition=1)
    assert p.info()["partition"] == 1
    N = len(dims)
    ords = lpt_orders(c, kappa)
    idx, val = p.elements()
    assert np.array_equal(idx, c[ords[0][1]].astype(np.int32))
    assert np.array_equal(val.view(np.uint32), v[ords[0][1]].view(np.uint32))
    for n in range(N):
        want_np = ords[(n + 1) % N][0][ords[n][1]]
        assert np.array_equal(p.next_pos(n), want_np.astype(np.int32)), n
        deg = np.bincount(c[:, n], minlength=dims[n])
        _, load = O.lpt_partition(deg, kappa)
        assert np.array_equal(p.bounds(n), np.concatenate([[0], np.cumsum(load)])), n
        assert p.info(n)["nblk"] == kappa
        assert p.splits(n).shape[0] == 0
        # each row lives in exactly one block (no split) and blocks hold ascending rows
        rows = c[ords[n][1], n]
        b = p.bounds(n)
        seen = {}
        for j in range(kappa):
            seg = rows[b[j]:b[j + 1]]
            assert np.all(np.diff(seg) >= 0)
            for r in np.unique(seg):
                assert r not in seen
                seen[r] = j
    p.close()


def test_partition_option_errors():
    c = np.array([[0, 1, 2], [1, 1, 1], [2, 0, 0]], np.int64)
    v = np.ones(3, np.float32)
    with pytest.raises(SpmError) as ei:
        Plan(c, v, (3, 3, 3), 4, host_only=True, partition=2)
    assert ei.value.status == -1


@pytest.fixture(scope="module")
def gpu():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _all_modes(c, v, dims, R, kappa, dtype="f32", **kw):
    p = Plan(c, v, dims, R, dtype=dtype, nblk=kappa, checks=True, partition=1, **kw)
    F = synth.make_factors(dims, R, seed=41)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda() for f in F]
    Fh = [f.to(tdt).float().numpy() for f in F]
    ords = lpt_orders(c, kappa)
    N = len(dims)
    for rep in range(2):
        for n in range(N):
            out = torch.full((dims[n], R), float("nan"), device="cuda")
            p.compute(n, Fd, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got)), (rep, n, "unwritten rows")
            assert O.relerr(got, O.mttkrp(c, v, dims, Fh, n)) <= 1e-5, (rep, n)
            idx, _ = p.elements()
            assert np.array_equal(idx, c[ords[(n + 1) % N][1]].astype(np.int32)), (rep, n)
    return p, Fd


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nnz,skew,kappa", CASES[:3])
@pytest.mark.parametrize("variant,eb", [(0, 0), (0, 16), (1, 0)])
def test_gpu_all_modes_and_orders(gpu, dims, nnz, skew, kappa, variant, eb):
    if eb == 16 and len(dims) > 3:
        pytest.skip("16-byte nonzeros hold up to 3 modes")
    coo, vals = synth.make_coo(dims, nnz, skew, seed=nnz + kappa)
    p, _ = _all_modes(coo.numpy(), vals.numpy(), dims, 32, kappa, variant=variant,
                      element_bytes=eb)
    p.close()


@pytest.mark.gpu
def test_gpu_heavy_row_stays_in_one_block_bf16_and_sweeps(gpu):
    # row 3 of mode 0 holds half of the nonzeros: Algorithm 1 keeps it in one block
    n = 4000
    rng = np.random.default_rng(7)
    i0 = np.where(np.arange(n) % 2 == 0, 3, rng.integers(0, 50, n))
    c = np.stack([i0, np.arange(n) % 80, np.arange(n) // 80], 1).astype(np.int64)
    c = np.unique(c, axis=0)
    v = rng.random(c.shape[0]).astype(np.float32)
    dims = (50, 80, 50)
    p, Fd = _all_modes(c, v, dims, 16, 9, dtype="bf16")
    b = p.bounds(0)
    heavy = int(np.sum(c[:, 0] == 3))
    assert np.max(np.diff(b)) >= heavy
    # graph sweeps equal eager sweeps; the resident-copy option gives the same bits
    o1 = [torch.empty(d, 16, device="cuda") for d in dims]
    o2 = [torch.empty(d, 16, device="cuda") for d in dims]
    p.sweep(Fd, o1)
    p.sweep(Fd, o2, graph=True)
    p.sweep(Fd, o2, graph=True)
    pk = Plan(c, v, dims, 16, dtype="bf16", nblk=9, partition=1, keep_base=True)
    o3 = [torch.empty(d, 16, device="cuda") for d in dims]
    pk.sweep(Fd, o3)
    pk.sweep(Fd, o3, graph=True)
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(o1[k], o2[k]) and torch.equal(o1[k], o3[k])
    p.device_status()
    pk.close()
    p.close()


@pytest.mark.gpu
def test_gpu_autotune_keeps_the_blocks(gpu, tmp_path, monkeypatch):
    monkeypatch.setenv("SPMTTKRP_TUNE_CACHE", str(tmp_path / "tune.txt"))
    dims = (300, 200, 100)
    coo, vals = synth.make_coo(dims, 20000, (1.1, 1.1, 0.0), seed=3)
    c, v = coo.numpy(), vals.numpy()
    p = Plan(c, v, dims, 32, nblk=31, partition=1)
    F = [f.cuda() for f in synth.make_factors(dims, 32, seed=4)]
    scratch = [torch.empty(d, 32, device="cuda") for d in dims]
    p.autotune(F, scratch)
    assert p.info()["nblk"] == 31 and p.info()["partition"] == 1
    outs = [torch.full((d, 32), float("nan"), device="cuda") for d in dims]
    p.sweep(F, outs)
    torch.cuda.synchronize()
    Fh = [f.cpu().numpy() for f in F]
    for n in range(3):
        assert O.relerr(outs[n].cpu().numpy().astype(np.float64),
                        O.mttkrp(c, v, dims, Fh, n)) <= 1e-5
    p.close()
