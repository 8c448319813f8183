"""The allocation-free entry point (spmttkrp_compute_noalloc).

It serves callers that cannot call cudaMalloc (code in an allocator-free region
of a host framework, or a process whose device memory belongs to another pool):
they cannot create a plan, so they pass every buffer in and the call keeps its
scratch in a fixed static device array.  Checked here against the FP64 oracle
directly and against the existing plan-based entry point, on two calls in a row
(the static scratch keeps the previous call's contents).  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, lib

pytestmark = pytest.mark.gpu

P = ctypes.c_void_p


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = lib()
    L.spmttkrp_compute_noalloc.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                           ctypes.c_int, P, P, P, P, ctypes.c_int, P]
    L.spmttkrp_compute_noalloc.restype = ctypes.c_int


def device_elements(coo, vals, mode):
    """Nonzeros in mode-`mode` order in the engine's element layout, on the GPU."""
    N = coo.shape[1]
    words = (((4 * N + 4) + 15) // 16) * 4
    order = O.canonical_order(coo, mode)
    buf = np.zeros((coo.shape[0], words), dtype=np.int32)
    buf[:, :N] = coo[order]
    buf[:, N] = np.asarray(vals, np.float32)[order].view(np.int32)
    return torch.from_numpy(buf).cuda()


def call(elems, nnz, dims, mode, R, dtype, factors, out, elems_out=None, next_pos=None, nblk=0):
    fp = (ctypes.c_void_p * len(factors))(*[f.data_ptr() for f in factors])
    d = np.asarray(dims, dtype=np.int64)
    return lib().spmttkrp_compute_noalloc(
        elems.data_ptr() if nnz else None, nnz, len(dims), mode,
        d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), R, dtype, fp, out.data_ptr(),
        elems_out.data_ptr() if elems_out is not None else None,
        next_pos.data_ptr() if next_pos is not None else None, nblk,
        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dims,R,dtype,nblk", [((300, 200, 100), 32, "f32", 0),
                                               ((300, 200, 100), 32, "f32", 97),
                                               ((40, 30, 20, 10), 16, "bf16", 13)])
def test_noalloc_matches_plan_entry_point_twice(dims, R, dtype, nblk):
    N = len(dims)
    coo, vals = synth.make_coo(dims, 30_000 if N == 3 else 8_000, (1.1,) * N, seed=R + N)
    c, v = coo.numpy(), vals.numpy()
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    F = [f.to(tdt).cuda() for f in synth.make_factors(dims, R, seed=7)]
    Fo = [f.float().cpu().numpy().astype(np.float64) for f in F]   # as the GPU reads them
    plan = Plan(c, v, dims, R, dtype=dtype)
    for n in range(N):
        want = torch.empty(dims[n], R, device="cuda")
        plan.compute(n, F, want)                       # existing entry point
        elems = device_elements(c, v, n)
        npos = torch.from_numpy(O.next_pos(c, n).astype(np.int32)).cuda()
        nxt = device_elements(c, v, (n + 1) % N).cpu().numpy()
        exact = O.mttkrp(c, v, dims, Fo, n)             # Eq. 1 in FP64
        for rep in range(2):                           # two calls in a row
            out = torch.full((dims[n], R), float("nan"), device="cuda")
            eout = torch.zeros_like(elems)
            st = call(elems, c.shape[0], dims, n, R, 1 if dtype == "bf16" else 0, F, out,
                      eout, npos, nblk)
            assert st == 0, lib().spmttkrp_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got)), (n, rep)
            assert O.relerr(got, exact) <= 1e-5, (n, rep, O.relerr(got, exact))
            assert O.relerr(got, want.cpu().numpy()) <= 1e-5, (n, rep)
            assert np.array_equal(eout.cpu().numpy(), nxt), (n, rep)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dims, R = (10, 10, 10), 8
    coo, vals = synth.make_coo(dims, 100, (0.0,) * 3, seed=1)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=2)]
    elems = device_elements(coo.numpy(), vals.numpy(), 0)
    out = torch.empty(10, R, device="cuda")
    assert call(elems, 100, dims, 0, R, 0, F, out, nblk=4097) == -6
    big = [torch.empty(d, 257, device="cuda") for d in dims]
    assert call(elems, 100, dims, 0, 257, 0, big, torch.empty(10, 257, device="cuda")) == -6
    assert b"4096" in lib().spmttkrp_last_error() or b"256" in lib().spmttkrp_last_error()


def test_noalloc_head_row_over_every_block():
    """One row holding most nonzeros is split over all 4096 blocks; its partials
    are summed by the fix-up in fixed order, equal to the oracle and the same on
    two calls."""
    dims, R = (50, 3000, 2000), 32
    rng = np.random.default_rng(3)
    nnz = 200_000
    c = np.stack([np.where(rng.random(nnz) < 0.9, 7, rng.integers(0, 50, nnz)),
                  rng.integers(0, 3000, nnz), rng.integers(0, 2000, nnz)], 1)
    c = np.unique(c, axis=0)
    c = c[rng.permutation(c.shape[0])]
    v = rng.random(c.shape[0]).astype(np.float32)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=9)]
    Fo = [f.cpu().numpy().astype(np.float64) for f in F]
    elems = device_elements(c, v, 0)
    exact = O.mttkrp(c, v, dims, Fo, 0)
    outs = []
    for rep in range(2):
        out = torch.full((dims[0], R), float("nan"), device="cuda")
        st = call(elems, c.shape[0], dims, 0, R, 0, F, out, nblk=4096)
        assert st == 0, lib().spmttkrp_last_error()
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
        assert O.relerr(outs[-1].astype(np.float64), exact) <= 1e-5, rep
    assert np.array_equal(outs[0], outs[1])
