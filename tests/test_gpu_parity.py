"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bit-exact: the remapped working copy after every mode, next_pos, block
boundaries and split tables.  Numeric: normwise relative error <= 1e-5 for
FP32 factors; BF16 factors <= 1e-5 against the oracle run on the BF16-rounded
factors and <= 1e-2 against the FP32 factors.  Outputs are pre-filled with
NaN so that a row the kernels fail to write shows up.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
BF16_Q_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_all_modes(coo, vals, dims, R, dtype="f32", nblk=0, tile=0, seed=3, graph=False,
                  check_order=True, scale=1.0, variant=0, element_bytes=0):
    c, v = coo.numpy(), vals.numpy()
    F = synth.make_factors(dims, R, seed=seed, scale=scale)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda() for f in F]
    p = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, tile=tile, checks=True, variant=variant,
             element_bytes=element_bytes)
    N = len(dims)
    outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    for n in range(N):
        p.compute(n, Fd, outs[n])
        if check_order:
            idx, val = p.elements()
            wi, wv = O.elements_in_order(c, v, (n + 1) % N)
            assert np.array_equal(idx, wi), f"mode {n}: remapped indices differ"
            assert np.array_equal(val.view(np.uint32), wv.view(np.uint32)), \
                f"mode {n}: remapped values differ"
    torch.cuda.synchronize()
    got = [o.cpu().numpy().astype(np.float64) for o in outs]
    Fh = [f.to(tdt).float().numpy() for f in F]
    return p, got, F, Fh


@pytest.mark.parametrize("N,R,dtype", [(3, 16, "f32"), (3, 32, "f32"), (3, 64, "f32"),
                                       (3, 128, "f32"), (3, 16, "bf16"), (3, 32, "bf16"),
                                       (3, 64, "bf16"), (4, 32, "f32"), (4, 64, "bf16"),
                                       (5, 16, "f32"), (6, 32, "f32"), (6, 32, "bf16")])
def test_all_modes_match_oracle(N, R, dtype):
    dims = [60, 45, 30, 20, 12, 9][:N]
    nnz = 6000 if N < 5 else 4000
    coo, vals = synth.make_coo(dims, nnz, (1.1,) * N, seed=100 + N)
    p, got, F, Fh = run_all_modes(coo, vals, dims, R, dtype=dtype, nblk=23, tile=256)
    c, v = coo.numpy(), vals.numpy()
    for n in range(N):
        assert np.all(np.isfinite(got[n])), f"mode {n}: unwritten rows"
        want_q = O.mttkrp(c, v, dims, Fh, n)
        assert O.relerr(got[n], want_q) <= F32_TOL, (n, O.relerr(got[n], want_q))
        if dtype == "bf16":
            want = O.mttkrp(c, v, dims, [f.numpy() for f in F], n)
            assert O.relerr(got[n], want) <= BF16_Q_TOL
    p.close()


def test_c1_workload_all_modes():
    spec = synth.workload("c1")
    coo, vals = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed)
    p, got, F, Fh = run_all_modes(coo, vals, spec.dims, 16, seed=synth.factor_seed(0))
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert O.relerr(got[n], O.mttkrp(c, v, spec.dims, Fh, n)) <= F32_TOL
        # device-side tables are the oracle's, bit for bit
        assert np.array_equal(p.next_pos(n), O.next_pos(c, n).astype(np.int32))
        rows = c[O.canonical_order(c, n), n]
        b = p.bounds(n)
        assert np.array_equal(b, O.contiguous_partition(rows, len(b) - 1))
        assert np.array_equal(p.splits(n), O.split_rows(rows, b))
    p.close()


@pytest.mark.parametrize("R", [1, 3, 4, 12, 17, 33, 100, 256])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("variant", [0, 1])
def test_odd_ranks_scalar_and_masked_paths(R, dtype, variant):
    dims = (40, 30, 20)
    coo, vals = synth.make_coo(dims, 2500, (1.1, 0.0, 1.1), seed=R)
    p, got, F, Fh = run_all_modes(coo, vals, dims, R, dtype=dtype, nblk=13, check_order=False,
                                  variant=variant)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert np.all(np.isfinite(got[n]))
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= F32_TOL
    p.close()


@pytest.mark.parametrize("N", [2, 7, 8, 9])
def test_generic_mode_counts(N):
    dims = [13, 11, 9, 7, 6, 5, 4, 4, 3][:N] if N > 2 else [300, 200]
    coo, vals = synth.make_coo(dims, 1500, (1.1,) + (0.0,) * (N - 1), seed=N)
    p, got, F, Fh = run_all_modes(coo, vals, dims, 16, nblk=11)
    c, v = coo.numpy(), vals.numpy()
    for n in range(N):
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= F32_TOL
    p.close()


@pytest.mark.parametrize("tile,nblk,variant", [(32, 1, 0), (64, 3, 0), (128, 7, 0), (256, 97, 0),
                                               (128, 0, 0), (128, 1, 1), (128, 5, 1),
                                               (128, 0, 1)])
def test_tiles_blocks_and_ragged_tails(tile, nblk, variant):
    # 7,777 nonzeros: not a multiple of any tile; blocks span several tiles
    dims = (500, 80, 60)
    coo, vals = synth.make_coo(dims, 7777, (1.2, 1.1, 0.0), seed=tile + nblk)
    p, got, F, Fh = run_all_modes(coo, vals, dims, 32, nblk=nblk, tile=tile, variant=variant)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= F32_TOL
    p.close()


def test_heavy_row_split_across_every_block():
    # every nonzero in output row 2 of mode 0: the row is split over all blocks
    n = 5000
    coo = torch.stack([torch.full((n,), 2, dtype=torch.int64), torch.arange(n) % 100,
                       torch.arange(n) // 100], 1)
    vals = torch.rand(n, generator=torch.Generator().manual_seed(0))
    dims = (5, 100, 50)
    p, got, F, Fh = run_all_modes(coo, vals, dims, 32, nblk=64, tile=256)
    assert p.splits(0).tolist() == [[2, 0, 63]]
    c, v = coo.numpy(), vals.numpy()
    for m in range(3):
        assert O.relerr(got[m], O.mttkrp(c, v, dims, Fh, m)) <= F32_TOL
    assert np.all(got[0][[0, 1, 3, 4]] == 0.0)
    p.close()


def test_empty_tensor_and_single_nonzero():
    dims = (7, 5, 3)
    p, got, _, _ = run_all_modes(torch.zeros((0, 3), dtype=torch.int64), torch.zeros(0),
                                 dims, 8, check_order=False)
    for n in range(3):
        assert np.all(got[n] == 0.0)
    p.close()
    coo = torch.tensor([[6, 0, 2]])
    vals = torch.tensor([0.5])
    p, got, F, Fh = run_all_modes(coo, vals, dims, 8, nblk=4)
    for n in range(3):
        assert O.relerr(got[n], O.mttkrp(coo.numpy(), vals.numpy(), dims, Fh, n)) <= F32_TOL
    p.close()


def test_sparse_rows_zero_filled():
    # huge dims with few nonzeros: most output rows are empty and must be zero
    dims = (5000, 3000, 20)
    coo, vals = synth.make_coo(dims, 800, (0.0, 0.0, 0.0), seed=77)
    p, got, F, Fh = run_all_modes(coo, vals, dims, 16, nblk=9)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        want = O.mttkrp(c, v, dims, Fh, n)
        assert np.all(got[n][np.all(want == 0, axis=1)] == 0.0)
        assert O.relerr(got[n], want) <= F32_TOL
    p.close()


def test_determinism_graph_and_remap():
    dims = (300, 200, 100)
    coo, vals = synth.make_coo(dims, 20000, (1.1, 1.1, 1.1), seed=5)
    F = [f.cuda() for f in synth.make_factors(dims, 32, seed=9)]
    p = Plan(coo.numpy(), vals.numpy(), dims, 32, nblk=40)
    o1 = [torch.empty(d, 32, device="cuda") for d in dims]
    o2 = [torch.empty(d, 32, device="cuda") for d in dims]
    o3 = [torch.empty(d, 32, device="cuda") for d in dims]
    p.sweep(F, o1)
    p.sweep(F, o2, graph=True)      # eager first run + capture
    p.sweep(F, o3, graph=True)      # graph replay (other buffer parity: N is odd)
    p.sweep(F, o3, graph=True)      # replay of the first parity
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(o1[n], o2[n]) and torch.equal(o1[n], o3[n])
    # remap-only passes land on the oracle's orders
    c = coo.numpy()
    for m in (2, 1, 0):
        p.remap(m)
        idx, _ = p.elements()
        assert np.array_equal(idx, O.elements_in_order(c, vals.numpy(), m)[0])
    # computing modes out of order remaps on demand
    out = torch.empty(dims[1], 32, device="cuda")
    p.compute(1, F, out)
    torch.cuda.synchronize()
    assert torch.equal(out, o1[1])
    p.device_status()
    p.close()


@pytest.mark.parametrize("eb", [0, 16, 32])
@pytest.mark.parametrize("variant,dtype,R", [(0, "f32", 32), (0, "bf16", 32), (1, "f32", 32),
                                             (0, "f32", 17), (0, "f32", 64), (0, "bf16", 16)])
def test_16_and_32_byte_elements(variant, dtype, R, eb):
    # 3-mode nonzeros unpadded (16 bytes) or in whole 32-byte sectors (the default):
    # same results, same remap order
    dims = (300, 200, 100)
    coo, vals = synth.make_coo(dims, 9000, (1.1, 1.1, 0.0), seed=R + variant)
    p, got, F, Fh = run_all_modes(coo, vals, dims, R, dtype=dtype, nblk=29, variant=variant,
                                  element_bytes=eb)
    assert p.info()["elem_bytes"] == (eb or 32)
    c, v = coo.numpy(), vals.numpy()
    for n in range(3):
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= F32_TOL
    for m in (2, 0):  # remap-only passes move whole sectors too
        p.remap(m)
        idx, _ = p.elements()
        assert np.array_equal(idx, O.elements_in_order(c, v, m)[0])
    p.close()


@pytest.mark.parametrize("keep_base", [False, True])
def test_compute_keep_order(keep_base):
    # a pass that writes no remap: same output, the copy stays in the mode's order
    dims = (300, 200, 100)
    coo, vals = synth.make_coo(dims, 20000, (1.1, 1.1, 0.0), seed=12)
    c, v = coo.numpy(), vals.numpy()
    F = [f.cuda() for f in synth.make_factors(dims, 32, seed=13)]
    p = Plan(c, v, dims, 32, nblk=40, checks=True, keep_base=keep_base)
    ref = [torch.empty(d, 32, device="cuda") for d in dims]
    p.sweep(F, ref)
    for n in (1, 2, 0, 2):
        out = torch.full((dims[n], 32), float("nan"), device="cuda")
        p.compute(n, F, out, keep_order=True)
        p.compute(n, F, out, keep_order=True)   # repeatable: still in mode-n order
        torch.cuda.synchronize()
        assert torch.equal(out, ref[n]), n
        assert p.info()["cur_mode"] == n
        assert np.array_equal(p.elements()[0], O.elements_in_order(c, v, n)[0]), n
    out = torch.empty(dims[2], 32, device="cuda")
    p.compute(2, F, out)                          # a plain pass remaps on to mode 0
    torch.cuda.synchronize()
    assert torch.equal(out, ref[2]) and p.info()["cur_mode"] == 0
    p.close()


def test_device_memory_cap_is_a_status():
    # fault injection through the allocation cap: plan creation fails cleanly with
    # SPM_ERR_OOM, and a plan within the cap works afterwards
    from paper_2405_08470_gb300 import SpmError
    dims = (300, 200, 100)
    coo, vals = synth.make_coo(dims, 50_000, (1.1, 1.1, 0.0), seed=6)
    c, v = coo.numpy(), vals.numpy()
    with pytest.raises(SpmError) as ei:
        Plan(c, v, dims, 16, max_bytes=1 << 20)   # the two 1.6 MB copies alone exceed it
    assert ei.value.status == -4
    p = Plan(c, v, dims, 16, max_bytes=1 << 30)
    assert 0 < p.info()["device_bytes"] <= 1 << 30
    F = [f.cuda() for f in synth.make_factors(dims, 16, seed=7)]
    out = torch.empty(dims[0], 16, device="cuda")
    p.compute(0, F, out)
    torch.cuda.synchronize()
    assert O.relerr(out.cpu().numpy().astype(np.float64),
                    O.mttkrp(c, v, dims, [f.cpu().numpy() for f in F], 0)) <= 1e-5
    p.close()


@pytest.mark.parametrize("dims,dtype,R", [((60, 45, 30, 20), "f32", 32),
                                          ((60, 45, 30, 20), "bf16", 32),
                                          ((30, 20, 12, 8, 6), "f32", 16),
                                          ((20, 15, 9, 7, 5, 4), "f32", 64),
                                          ((20, 15, 9, 7, 5, 4), "bf16", 16)])
def test_packed_16_byte_nonzeros_4_to_6_modes(dims, dtype, R):
    """Indices packed into bit fields (16-byte nonzeros, Section 3.5): the remapped
    working copy equals the oracle's order after every mode, outputs match the
    oracle, the device-built plan equals the host-built one byte for byte, and
    the device consistency check passes on the packed copy."""
    N = len(dims)
    coo, vals = synth.make_coo(dims, 5000, (1.1,) * N, seed=300 + N)
    c, v = coo.numpy(), vals.numpy()
    p, got, F, Fh = run_all_modes(coo, vals, dims, R, dtype=dtype, nblk=31, element_bytes=16)
    assert p.info()["elem_bytes"] == 16
    for n in range(N):
        assert np.all(np.isfinite(got[n])), n
        assert O.relerr(got[n], O.mttkrp(c, v, dims, Fh, n)) <= F32_TOL, n
    p.check()
    ph = Plan(c, v, dims, R, dtype=dtype, element_bytes=16, plan_on_host=True)
    pd = Plan(c, v, dims, R, dtype=dtype, element_bytes=16)
    assert np.array_equal(ph.raw_elements(), pd.raw_elements())
    order = O.canonical_order(c, 0)
    assert np.array_equal(pd.raw_elements().view(np.uint32), O.flycoo_pack(c[order], v[order], dims))
    for n in range(N):
        assert np.array_equal(pd.next_pos(n), O.next_pos(c, n).astype(np.int32))
    ph.close()
    pd.close()
    p.close()


def test_packed_nonzeros_cp_loss_and_als():
    """CP loss (plain forward + full backward) and CP-ALS on a packed 5-mode plan
    against the oracle."""
    from paper_2405_08470_gb300.cp import CPLoss
    dims, R = (30, 20, 12, 8, 6), 8
    coo, _ = synth.make_coo(dims, 4000, (1.1,) * 5, seed=17)
    x = synth.make_planted_targets(coo, dims, 4, 0.1, seed=18)
    c, xv = coo.numpy(), x.numpy()
    F = synth.make_factors(dims, R, seed=19, scale=0.3)
    p = Plan(c, xv, dims, R, element_bytes=16, nblk=13)
    Fd = [f.cuda().requires_grad_(True) for f in F]
    loss = CPLoss.apply(p, *Fd)
    loss.backward()
    F64 = [f.numpy().astype(np.float64) for f in F]
    want, _ = O.cp_loss(c, xv, F64)
    assert abs(loss.item() - want) <= 1e-5 * abs(want)
    G = O.cp_loss_grad(c, xv, dims, F64)
    for k in range(5):
        assert O.relerr(Fd[k].grad.cpu().numpy().astype(np.float64), G[k]) <= 1e-5, k
    Fa = [f.clone().cuda() for f in F]
    lam = torch.empty(R, device="cuda")
    Fo = F64
    for it in range(3):
        fit = p.als_iter(Fa, lam)
        Fo, lo, fo = O.cp_als_iter(c, xv, dims, Fo)
        assert abs(fit - fo) <= 1e-5, (it, fit, fo)
    p.close()
