"""C-ABI library checks that need no GPU: exported symbols, host-side planning
(bit-exact against the oracle) and host-side error paths."""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, SpmError, binding, declared_functions, lib


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_library_exports_every_declared_symbol():
    L = lib()
    names = declared_functions()
    for must in ["spmttkrp_plan_create", "spmttkrp_plan_destroy", "spmttkrp_remap",
                 "spmttkrp_compute", "spmttkrp_sweep", "cp_als_iter", "cp_loss_fwd",
                 "cp_loss_bwd", "spmttkrp_autotune", "spmttkrp_plan_query",
                 "spmttkrp_last_error", "spmttkrp_opts_init", "spmttkrp_set_stream",
                 "spmttkrp_device_status", "spmttkrp_version", "spmttkrp_compute_ex",
                 "spmttkrp_compute_noalloc", "spmttkrp_check_elements",
                 "spmttkrp_plan_check"]:
        assert must in names
    for n in names:
        assert hasattr(L, n), n
    assert L.spmttkrp_version() >= 100


def _host_plan(coo, vals, dims, R=4, nblk=0):
    return Plan(coo, vals, dims, R, nblk=nblk, host_only=True)


@pytest.mark.parametrize("dims,nnz,skew,nblk", [
    ((200, 150, 100), 5000, (0.0, 0.0, 0.0), 0),
    ((50, 40, 30), 3000, (1.1, 1.1, 1.1), 17),
    ((30, 20, 10, 8), 2500, (1.2, 1.2, 0.0, 0.0), 9),
    ((12, 9, 7, 5, 4), 1500, (1.1,) * 5, 64),
    ((9, 3), 20, (0.0, 0.0), 40),                   # nblk > nnz
    ((6, 5, 4, 3, 3, 2, 2, 2, 2), 900, (0.0,) * 9, 5),  # 9 modes (runtime-N path)
])
def test_host_plan_matches_oracle_bit_exact(dims, nnz, skew, nblk):
    coo, vals = synth.make_coo(dims, nnz, skew, seed=sum(dims))
    c, v = coo.numpy(), vals.numpy()
    p = _host_plan(c, v, dims, nblk=nblk)
    N = len(dims)
    idx, val = p.elements()
    wi, wv = O.elements_in_order(c, v, 0)
    assert np.array_equal(idx, wi) and np.array_equal(val, wv)
    for n in range(N):
        assert np.array_equal(p.next_pos(n), O.next_pos(c, n).astype(np.int32))
        rows = c[O.canonical_order(c, n), n]
        nb = p.info(n)["nblk"]
        b = p.bounds(n)
        assert np.array_equal(b, O.contiguous_partition(rows, nb))
        assert np.array_equal(p.splits(n), O.split_rows(rows, b))
    assert p.info()["normx2"] == pytest.approx(float(np.sum(v.astype(np.float64) ** 2)),
                                               rel=1e-12)
    p.close()


def test_host_plan_heavy_single_row_split_everywhere():
    coo = np.stack([np.zeros(1000, np.int64), np.arange(1000) % 50, np.arange(1000) // 50], 1)
    vals = np.ones(1000, np.float32)
    p = _host_plan(coo, vals, (3, 50, 20), nblk=8)
    assert p.splits(0).tolist() == [[0, 0, 7]]
    rows = coo[O.canonical_order(coo, 0), 0]
    assert np.array_equal(p.bounds(0), O.contiguous_partition(rows, 8))


def test_host_plan_empty_tensor():
    p = _host_plan(np.zeros((0, 3), np.int64), np.zeros(0, np.float32), (4, 5, 6), nblk=3)
    assert p.info()["nnz"] == 0
    assert p.bounds(1).tolist() == [0, 0, 0, 0]


@pytest.mark.parametrize("case,status", [
    ("dup", -3), ("range", -2), ("neg", -2), ("nmodes", -1), ("rank0", -1), ("rank_big", -6),
    ("tile", -1), ("dims0", -1), ("partition", -1), ("dtype", -1), ("variant", -1),
])
def test_host_error_paths(case, status):
    coo = np.array([[0, 1, 2], [1, 1, 1], [2, 0, 0]], np.int64)
    vals = np.ones(3, np.float32)
    dims, R, kw = (3, 3, 3), 4, {}
    if case == "dup":
        coo[2] = coo[0]
    elif case == "range":
        coo[1, 2] = 3
    elif case == "neg":
        coo[1, 0] = -1
    elif case == "nmodes":
        coo, dims = coo[:, :1], (3,)
    elif case == "rank0":
        R = 0
    elif case == "rank_big":
        R = 257
    elif case == "tile":
        kw["tile"] = 300
    elif case == "dims0":
        dims = (3, 0, 3)
    elif case == "variant":
        kw["variant"] = 4  # forms 0..3
    if case in ("partition", "dtype"):
        L = lib()
        o = binding.Opts()
        L.spmttkrp_opts_init(ctypes.byref(o))
        o.host_only = 1
        if case == "partition":
            o.partition = 2  # 0 and 1 are the two partitions
        else:
            o.factor_dtype = 7
        h = ctypes.c_void_p()
        d = np.asarray(dims, np.int64)
        st = L.spmttkrp_plan_create(ctypes.byref(h), coo.ctypes.data, vals.ctypes.data, 3,
                                    d.ctypes.data_as(binding.I64P), 3, R, ctypes.byref(o))
        assert st == status
        assert L.spmttkrp_last_error()
        return
    with pytest.raises(SpmError) as ei:
        Plan(coo, vals, dims, R, host_only=True, **kw)
    assert ei.value.status == status


@pytest.mark.parametrize("N,eb,want", [(2, 0, 32), (3, 0, 32), (3, 16, 16), (3, 32, 32),
                                        (4, 0, 32), (7, 0, 32), (8, 0, 48), (4, 16, 16),
                                        (6, 16, 16), (3, 24, None), (8, 32, None)])
def test_element_stride_rules(N, eb, want):
    # default: one whole 32-byte sector per nonzero when N indices + value fit
    dims = (4,) * N
    coo = np.array([[i % 4] * N for i in range(3)], np.int64)
    coo[:, 0] = [0, 1, 2]
    vals = np.ones(3, np.float32)
    if want is None:
        with pytest.raises(SpmError) as ei:
            Plan(coo, vals, dims, 4, host_only=True, element_bytes=eb)
        assert ei.value.status == -1
        return
    p = Plan(coo, vals, dims, 4, host_only=True, element_bytes=eb)
    info = p.info()
    assert info["elem_bytes"] == want
    assert info["tile"] in (64, 128)  # 128, halved while two CTAs per SM would not fit
    assert info["stages"] == (3 if want == 16 else 2)
    p.close()


def test_null_pointer_and_state_errors():
    L = lib()
    assert L.spmttkrp_plan_create(None, None, None, 0, None, 3, 4, None) == -1
    h = ctypes.c_void_p()
    d = np.asarray((3, 3, 3), np.int64)
    assert L.spmttkrp_plan_create(ctypes.byref(h), None, None, 5, d.ctypes.data_as(binding.I64P),
                                  3, 4, None) == -1
    p = _host_plan(np.array([[0, 0, 0]]), np.ones(1, np.float32), (2, 2, 2))
    # compute on a host-only plan is a state error, not a crash
    assert L.spmttkrp_compute(p._h, 0, None, None) == -8
    assert L.spmttkrp_remap(p._h, 5) == -8
    p.close()


def test_als_and_loss_entry_points_reject_null_and_host_only_plans():
    """CP-ALS (one iteration and the loop), the CP loss and the autotuner return
    INVALID_ARG for a null plan and STATE for a host-only plan, before any
    argument or device is touched."""
    L = lib()
    fit = ctypes.c_double()
    fits = (ctypes.c_double * 4)()
    iters = ctypes.c_int()
    calls = {
        "cp_als_iter": lambda h: L.cp_als_iter(h, None, None, ctypes.byref(fit)),
        "cp_als_run": lambda h: L.cp_als_run(h, None, None, 4, 0.0, fits, ctypes.byref(iters)),
        "cp_loss_fwd": lambda h: L.cp_loss_fwd(h, None, None),
        "cp_loss_fwd_ex": lambda h: L.cp_loss_fwd_ex(h, None, None, 0),
        "cp_loss_bwd": lambda h: L.cp_loss_bwd(h, None, None, None),
        "spmttkrp_autotune": lambda h: L.spmttkrp_autotune(h, None, None, 0),
    }
    for name, call in calls.items():
        assert call(None) == -1, name
    p = _host_plan(np.array([[0, 0, 0], [1, 1, 1]]), np.ones(2, np.float32), (2, 2, 2))
    for name, call in calls.items():
        assert call(p._h) == -8, name
        assert L.spmttkrp_last_error()  # a message for the failed call
    p.close()


def test_check_argument_errors_need_no_device():
    """The consistency check rejects bad arguments before touching the device, and
    refuses host-only plans."""
    L = lib()
    dims_np = np.array([4, 4, 4], dtype=np.int64)
    dims = dims_np.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    cases = [(-1, 3, 32, 0), (8, 1, 32, 0), (8, 3, 24, 0), (8, 3, 12, 0), (8, 3, 32, 3),
             (8, 3, 32, 8)]
    buf = ctypes.c_void_p(1)  # never dereferenced: every case fails its argument checks
    for nnz, N, eb, aw in cases:
        assert L.spmttkrp_check_elements(buf, nnz, N, dims, eb, None, aw, None) == -1, \
            (nnz, N, eb, aw)
    coo, vals = synth.make_coo((20, 10, 5), 200, (0.0, 0.0, 0.0), seed=2)
    p = _host_plan(coo.numpy(), vals.numpy(), (20, 10, 5))
    with pytest.raises(SpmError) as ei:
        p.check()
    assert ei.value.status == -8
    p.close()


def test_binding_rejects_bad_tensors_before_the_c_abi():
    """The binding checks device, dtype, shape and layout of every tensor before a
    pointer reaches the C ABI (a host-only plan: nothing would run anyway)."""
    import torch
    coo, vals = synth.make_coo((20, 10, 5), 200, (0.0, 0.0, 0.0), seed=2)
    p = _host_plan(coo.numpy(), vals.numpy(), (20, 10, 5))
    F = [torch.zeros(d, 4) for d in (20, 10, 5)]
    with pytest.raises(ValueError, match="CUDA device"):
        p.compute(0, F, torch.zeros(20, 4))
    with pytest.raises(ValueError, match="expected 3 factors"):
        p.sweep(F[:2], F)
    p.close()


def test_packed_nonzeros_match_the_oracle_packing_and_order():
    """16-byte nonzeros with 4-6 modes hold the indices as bit fields of their
    exact widths (Section 3.5; oracle.flycoo_pack) and the value in word 3; the
    working copy, read back through the query, is the oracle's mode-0 order."""
    for dims in [(1000, 200, 50, 30), (500, 50, 5, 100, 20), (200, 20, 9, 5, 10, 5)]:
        N = len(dims)
        coo, vals = synth.make_coo(dims, 3000, (1.1,) * N, seed=N)
        c, v = coo.numpy(), vals.numpy()
        p = Plan(c, v, dims, 8, host_only=True, element_bytes=16)
        assert p.info()["elem_bytes"] == 16
        order = O.canonical_order(c, 0)
        want = O.flycoo_pack(c[order], v[order], dims)
        assert np.array_equal(p.raw_elements().view(np.uint32), want), dims
        idx, val = p.elements()
        wi, wv = O.elements_in_order(c, v, 0)
        assert np.array_equal(idx, wi) and np.array_equal(val.view(np.uint32), wv.view(np.uint32))
        p.close()


def test_packed_nonzeros_need_96_bits_at_most():
    dims = (2 ** 31 - 1,) * 4  # 4 x 31 bits do not fit
    coo = np.array([[0, 0, 0, 0], [1, 1, 1, 1]], np.int64)
    with pytest.raises(SpmError) as ei:
        Plan(coo, np.ones(2, np.float32), dims, 4, host_only=True, element_bytes=16)
    assert ei.value.status == -1
