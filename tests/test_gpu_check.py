"""GPU: the device consistency check of a working copy (Section 3.5 invariants).

A correct working copy passes: indices inside dims, next_pos a permutation of
[0, nnz), remap ids carried in the nonzeros equal to next_pos.  Copies built
from the oracle and then damaged on the host (one index out of range, one remap
target duplicated, one carried id changed) must be reported with the right
status and the first damaged position, and the check itself must leave the
context usable.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, SpmError, check_elements

pytestmark = pytest.mark.gpu

INDEX_RANGE, STATE = -2, -8


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dims,kw", [((300, 200, 100), {}),
                                     ((300, 200, 100), {"element_bytes": 16}),
                                     ((300, 200, 100), {"keep_base": True}),
                                     ((50, 40, 30, 20), {}),
                                     ((400, 300), {"partition": 1})])
def test_plan_copy_passes_after_every_pass(dims, kw):
    R = 16
    coo, vals = synth.make_coo(dims, 7000, (1.1,) * len(dims), seed=3)
    p = Plan(coo.numpy(), vals.numpy(), dims, R, nblk=13, checks=True, **kw)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=4)]
    p.check()
    for _ in range(2):
        for n in range(len(dims)):
            out = torch.empty(dims[n], R, device="cuda")
            p.compute(n, F, out)
            p.check()
    p.close()


def oracle_copy(dims, n, eb, alpha):
    """Working copy of mode n built from the oracle only: records of eb bytes
    {int32 idx[N], float v, padding}; with alpha, word 4 + (n+1) % N holds next_pos."""
    N = len(dims)
    coo, vals = synth.make_coo(dims, 5000, (1.2,) * N, seed=9)
    c, v = coo.numpy(), vals.numpy()
    idx, val = O.elements_in_order(c, v, n)
    nxt = O.next_pos(c, n).astype(np.int32)
    rec = np.zeros((len(val), eb // 4), dtype=np.int32)
    rec[:, :N] = idx
    rec[:, N] = val.view(np.int32)
    if alpha:
        rec[:, 4 + (n + 1) % N] = nxt
    return rec, nxt


def run(rec, dims, nxt, aw):
    e = torch.from_numpy(rec.copy()).cuda()
    npos = None if nxt is None else torch.from_numpy(nxt.copy()).cuda()
    check_elements(e, rec.shape[0], dims, rec.shape[1] * 4, npos, aw)


@pytest.mark.parametrize("dims,n,eb,alpha", [((300, 200, 100), 0, 32, True),
                                             ((300, 200, 100), 2, 32, True),
                                             ((300, 200, 100), 1, 16, False),
                                             ((60, 50, 40, 30), 3, 32, False)])
def test_damaged_copies_are_reported(dims, n, eb, alpha):
    N = len(dims)
    aw = 4 + (n + 1) % N if alpha else 0
    rec, nxt = oracle_copy(dims, n, eb, alpha)
    run(rec, dims, nxt, aw)          # intact copy
    run(rec, dims, None, 0)          # indices only

    bad = rec.copy()
    bad[1234, n] = dims[n]           # one past the end of mode n
    with pytest.raises(SpmError) as ei:
        run(bad, dims, nxt, aw)
    assert ei.value.status == INDEX_RANGE and "first at 1234" in str(ei.value)
    bad[1234, n] = -1
    with pytest.raises(SpmError) as ei:
        run(bad, dims, None, 0)
    assert ei.value.status == INDEX_RANGE

    dup = nxt.copy()
    dup[700] = dup[701]              # one target hit twice, another never
    with pytest.raises(SpmError) as ei:
        run(rec, dims, dup, 0)
    assert ei.value.status == STATE and "not a permutation" in str(ei.value)
    out = nxt.copy()
    out[5] = len(nxt)                # outside [0, nnz)
    with pytest.raises(SpmError) as ei:
        run(rec, dims, out, 0)
    assert ei.value.status == STATE

    if alpha:
        wrong = rec.copy()
        wrong[42, aw] = (wrong[42, aw] + 1) % len(nxt)
        with pytest.raises(SpmError) as ei:
            run(wrong, dims, nxt, aw)
        assert ei.value.status == STATE and "differ from next_pos, first at 42" in str(ei.value)
    torch.cuda.synchronize()         # the context is still usable
    assert torch.ones(4, device="cuda").sum().item() == 4.0


def test_bad_arguments_are_rejected():
    e = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(SpmError):
        check_elements(e, 8, (4, 4, 4), 24)       # not a multiple of 16
    with pytest.raises(SpmError):
        check_elements(e, 8, (4, 4, 4), 32, None, 2)  # id word over the indices
    check_elements(e, 0, (4, 4, 4), 32)           # empty copy: nothing to check
