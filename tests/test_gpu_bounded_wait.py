"""Failure detection without a fault: the fused kernel's bounded waits.

Every wait of the fused kernel on its bulk-copy barriers has a time limit.  A
warp whose wait runs out records SPM_ERR_TIMEOUT in the plan's device error
word, waits (with the default limit) for its own copies still in flight, and
returns; nothing traps.  The test switch `inject_wait_stall` makes each warp's
first wait be on a barrier that nothing completes, so the give-up path runs
with a short `wait_limit_ns`; the host then reads the status, and the device
context stays usable for a plan without the switch.
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


def _tensor():
    dims, R = (60, 40, 30), 16
    coo, vals = synth.make_coo(dims, 4000, (1.1, 0.0, 1.1), seed=5)
    F = synth.make_factors(dims, R, seed=6)
    return dims, R, coo.numpy(), vals.numpy(), F


@pytest.mark.parametrize("variant", [0, 2, 3])
def test_wait_runs_out_reports_timeout_and_context_survives(variant):
    dims, R, c, v, F = _tensor()
    Fd = [f.cuda() for f in F]
    p = Plan(c, v, dims, R, variant=variant, wait_limit_ns=1_000_000, inject_wait_stall=True)
    out = torch.empty(dims[0], R, device="cuda")
    p.compute(0, Fd, out)                      # asynchronous: the error surfaces below
    with pytest.raises(SpmError) as ei:
        p.device_status()
    assert ei.value.status == -9
    p.device_status()                          # read and cleared: no error the second time
    p.close()
    # the same pass with the status read by the call itself (checks on)
    pc = Plan(c, v, dims, R, variant=variant, wait_limit_ns=1_000_000, inject_wait_stall=True,
              checks=True)
    with pytest.raises(SpmError) as ei:
        pc.compute(0, Fd, out)
    assert ei.value.status == -9
    pc.close()
    # the context is still usable: a plan with the default limit matches the oracle
    q = Plan(c, v, dims, R, variant=variant)
    outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    q.sweep(Fd, outs)
    q.device_status()
    Fo = [f.numpy().astype(np.float64) for f in F]
    for n in range(3):
        want = O.mttkrp(c, v, dims, Fo, n)
        assert O.relerr(outs[n].cpu().numpy().astype(np.float64), want) <= 1e-5, n
    q.close()
