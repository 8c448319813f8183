"""GPU: plans whose orders are built on the device equal host-built plans bit for bit.

The device build sorts every K_n order with the engine's radix sort, checks
duplicates, writes the mode-0 working copy and every mode's next_pos.  Every
K_n order is total (coordinates are distinct), so the working copy, next_pos,
block bounds and split tables must equal those of a plan built on the host, and
the host plans are checked against the oracle in the CPU tests.  Sizes cover
several radix tiles (4096 nonzeros) and scan chunks (8192) with ragged ends, keys
of 1 to 3 digit passes, and 2 to 9 modes.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, SpmError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def same_plans(c, v, dims, R=16, **kw):
    dev = Plan(c, v, dims, R, **kw)
    host = Plan(c, v, dims, R, plan_on_host=True, **kw)
    N = len(dims)
    a, b = dev.elements(), host.elements()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32),
                                                         b[1].view(np.uint32))
    for n in range(N):
        assert np.array_equal(dev.next_pos(n), host.next_pos(n)), n
        assert np.array_equal(dev.bounds(n), host.bounds(n)), n
        assert np.array_equal(dev.splits(n), host.splits(n)), n
    assert dev.info()["normx2"] == host.info()["normx2"]
    return dev, host


@pytest.mark.parametrize("dims,nnz,skew", [
    ((200, 150, 100), 50_000, (0.0, 0.0, 0.0)),
    ((3000, 2000, 70000), 123_457, (1.1, 1.1, 1.1)),          # 3 digit passes, ragged
    ((40, 30, 20, 10), 8_191, (1.2, 0.0, 1.1, 0.0)),
    ((12, 9, 7, 5, 4), 4_097, (1.1,) * 5),
    ((6, 5, 4, 3, 3, 2, 2, 2, 2), 900, (0.0,) * 9),
    ((300, 200), 1, (0.0, 0.0)),
    ((70000, 3), 5_000, (1.3, 0.0)),
])
def test_device_built_plan_equals_host_plan(dims, nnz, skew):
    coo, vals = synth.make_coo(dims, nnz, skew, seed=nnz % 997)
    c, v = coo.numpy(), vals.numpy()
    dev, host = same_plans(c, v, dims, nblk=37)
    # and the device-built plan computes every mode like the oracle
    R = 16
    F = synth.make_factors(dims, R, seed=5)
    Fd = [f.cuda() for f in F]
    Fh = [f.numpy() for f in F]
    for n in range(len(dims)):
        out = torch.full((dims[n], R), float("nan"), device="cuda")
        dev.compute(n, Fd, out)
        torch.cuda.synchronize()
        assert O.relerr(out.cpu().numpy().astype(np.float64),
                        O.mttkrp(c, v, dims, Fh, n)) <= 1e-5
    dev.close()
    host.close()


def test_device_build_with_options_and_one_million_nonzeros():
    dims = (120_000, 90_000, 200_000)
    coo, vals = synth.make_coo(dims, 1_000_003, (1.1, 1.1, 1.1), seed=9)
    c, v = coo.numpy(), vals.numpy()
    for kw in (dict(), dict(keep_base=True), dict(element_bytes=16), dict(dtype="bf16")):
        dev, host = same_plans(c, v, dims, **kw)
        assert dev.info()["nblk"] == host.info()["nblk"]
        dev.close()
        host.close()


def test_device_build_reports_duplicates():
    c = np.array([[0, 1, 2], [1, 1, 1], [0, 1, 2], [2, 0, 0]] * 3000, np.int64)
    c[4:, 0] = np.arange(4, c.shape[0]) % 50
    c[4:, 2] = np.arange(4, c.shape[0]) // 50
    v = np.ones(c.shape[0], np.float32)
    with pytest.raises(SpmError) as ei:
        Plan(c, v, (50, 3, 300), 8)
    assert ei.value.status == -3
