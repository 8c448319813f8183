"""GPU: plans that keep the mode-0 copy resident (opts.keep_base).

The pass of mode N-1 then writes no remap and the next mode-0 pass reads the
resident copy.  Every result must equal, bit for bit, that of a plan that remaps
in every pass (same kernels, same order of arithmetic), and the working copy must
still be in the oracle's canonical order after every call.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan
from paper_2405_08470_gb300.cp import CPLoss

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def pair(dims, nnz, R, dtype="f32", nblk=17, seed=1, **kw):
    coo, vals = synth.make_coo(dims, nnz, (1.1,) * len(dims), seed=seed)
    c, v = coo.numpy(), vals.numpy()
    a = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, checks=True, **kw)
    b = Plan(c, v, dims, R, dtype=dtype, nblk=nblk, checks=True, keep_base=True, **kw)
    return c, v, a, b


@pytest.mark.parametrize("dims,variant,eb", [((300, 200, 100), 0, 0), ((300, 200, 100), 1, 0),
                                             ((300, 200, 100), 0, 32), ((50, 40, 30, 20), 0, 0),
                                             ((400, 300), 0, 0)])
def test_modes_and_orders_equal_plain_plan(dims, variant, eb):
    N, R = len(dims), 32
    c, v, a, b = pair(dims, 9000, R, variant=variant, element_bytes=eb)
    assert b.info()["keep_base"] == 1 and a.info()["keep_base"] == 0
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=5)]
    Fh = [f.numpy() for f in synth.make_factors(dims, R, seed=5)]
    for rep in range(2):  # the second cycle starts from the resident copy
        for n in range(N):
            oa = torch.full((dims[n], R), float("nan"), device="cuda")
            ob = torch.full((dims[n], R), float("nan"), device="cuda")
            a.compute(n, F, oa)
            b.compute(n, F, ob)
            torch.cuda.synchronize()
            assert torch.equal(oa, ob), (rep, n)
            assert O.relerr(ob.cpu().numpy().astype(np.float64), O.mttkrp(c, v, dims, Fh, n)) \
                <= 1e-5
            idx, val = b.elements()
            wi, wv = O.elements_in_order(c, v, (n + 1) % N)
            assert np.array_equal(idx, wi) and np.array_equal(val.view(np.uint32),
                                                              wv.view(np.uint32)), (rep, n)
    a.close()
    b.close()


def test_sweeps_graphs_remaps_and_out_of_order_calls():
    dims, R = (300, 200, 100), 16
    c, v, a, b = pair(dims, 20000, R, nblk=40, seed=7)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=9)]
    oa = [torch.empty(d, R, device="cuda") for d in dims]
    ob = [[torch.empty(d, R, device="cuda") for d in dims] for _ in range(4)]
    a.sweep(F, oa)
    b.sweep(F, ob[0])
    b.sweep(F, ob[1], graph=True)   # eager first run + capture
    b.sweep(F, ob[2], graph=True)   # replay
    b.sweep(F, ob[3], graph=True)   # replay again from the same state
    torch.cuda.synchronize()
    for o in ob:
        for n in range(3):
            assert torch.equal(oa[n], o[n])
    assert b.info()["cur_mode"] == 0
    # remap-only passes, including the free step from mode N-1 back to mode 0
    for m in (1, 2, 0, 2, 0):
        b.remap(m)
        assert np.array_equal(b.elements()[0], O.elements_in_order(c, v, m)[0]), m
    # a sweep from mode 1 (working buffer) and a single out-of-order mode
    b.remap(1)
    o1 = [torch.empty(d, R, device="cuda") for d in dims]
    b.sweep(F, o1, graph=True)
    b.sweep(F, o1, graph=True)
    out = torch.empty(dims[2], R, device="cuda")
    b.compute(2, F, out)
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(o1[n], oa[n])
    assert torch.equal(out, oa[2])
    assert np.array_equal(b.elements()[0], O.elements_in_order(c, v, 0)[0])
    b.device_status()
    a.close()
    b.close()


def test_als_iterations_equal_plain_plan():
    dims, R = (200, 150, 100), 16
    c, v, a, b = pair(dims, 40000, R, nblk=37, seed=11)
    Fa = [f.cuda() for f in synth.make_factors(dims, R, seed=2000)]
    Fb = [f.clone() for f in Fa]
    la, lb = torch.empty(R, device="cuda"), torch.empty(R, device="cuda")
    for it in range(4):  # eager, capture, replays
        fa = a.als_iter(Fa, la)
        fb = b.als_iter(Fb, lb)
        assert fa == fb, it
        assert torch.equal(la, lb)
        for k in range(3):
            assert torch.equal(Fa[k], Fb[k]), (it, k)
    a.close()
    b.close()


@pytest.mark.parametrize("start", [0, 1])
def test_cp_loss_and_gradients_equal_plain_plan(start):
    dims, R = (80, 60, 40), 16
    coo, _ = synth.make_coo(dims, 12000, (1.1, 1.1, 1.1), seed=21)
    x = synth.make_planted_targets(coo, dims, 8, 0.1, seed=22)
    c, xv = coo.numpy(), x.numpy()
    F = synth.make_factors(dims, R, seed=23, scale=0.3)
    grads, losses = [], []
    for keep in (False, True):
        p = Plan(c, xv, dims, R, nblk=19, keep_base=keep)
        p.remap(start)  # the residual sweep starts from the working copy's mode
        Fd = [f.cuda().requires_grad_(True) for f in F]
        loss = CPLoss.apply(p, *Fd)
        loss.backward()
        losses.append(loss.item())
        grads.append([f.grad.clone() for f in Fd])
        # the working copy is untouched by the residual sweep
        assert np.array_equal(p.elements()[0], O.elements_in_order(c, xv, start)[0])
        p.close()
    assert losses[0] == losses[1]
    for k in range(3):
        assert torch.equal(grads[0][k], grads[1][k]), k
    G = O.cp_loss_grad(c, xv, dims, [f.numpy().astype(np.float64) for f in F])
    for k in range(3):
        assert O.relerr(grads[1][k].cpu().numpy().astype(np.float64), G[k]) <= 1e-5
