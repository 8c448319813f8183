"""Parity at full size, in the launch configuration bench.py times (plan defaults).

The 3-mode 120000 x 90000 x 2000000 tensor with 100M Zipf(1.1) nonzeros, rank 32,
FP32 factors, default plan options (one warp per block, staged tiles).  The FP64
oracle cannot run the whole tensor here, so it checks sampled output rows one by one
(the heaviest row of every mode, rows split over many blocks, a light row, an empty
row when there is one, the first and the last row); the remapped working copy is
checked by properties that hold at any size (sorted by K_0 again after the sweep,
same multiset of nonzeros).  The 4-mode (150M nonzeros, FP32 and BF16 factors) and
6-mode (40M nonzeros) tensors are checked on sampled rows of at most 1M nonzeros.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = synth.workload("c2")
    coo, vals = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed, device="cuda")
    c, v = coo.cpu().numpy(), vals.cpu().numpy()
    del coo, vals
    torch.cuda.empty_cache()
    F = synth.make_factors(spec.dims, 32, seed=synth.factor_seed(1), device="cuda")
    return spec, c, v, F


def sample_rows(col, dim, plan_splits, rng):
    counts = np.bincount(col, minlength=dim)
    rows = {int(np.argmax(counts)), 0, dim - 1}
    nz = np.nonzero(counts)[0]
    rows.update(int(x) for x in rng.choice(nz, 4, replace=False))
    light = np.nonzero(counts == 1)[0]
    if light.size:
        rows.add(int(light[0]))
    empty = np.nonzero(counts == 0)[0]
    if empty.size:
        rows.add(int(empty[0]))
    if len(plan_splits):
        spans = plan_splits[:, 2] - plan_splits[:, 1]
        rows.add(int(plan_splits[np.argmax(spans), 0]))
        rows.add(int(plan_splits[0, 0]))
    return sorted(rows)


def test_full_size_sweep_sampled_rows_and_remap(c2):
    spec, c, v, F = c2
    plan = Plan(c, v, spec.dims, 32)
    outs = [torch.full((d, 32), float("nan"), device="cuda") for d in spec.dims]
    plan.sweep(F, outs)
    plan.device_status()
    torch.cuda.synchronize()
    Fh = [f.cpu().numpy() for f in F]
    rng = np.random.default_rng(0)
    for n in range(3):
        got = outs[n]
        assert not torch.isnan(got).any(), f"mode {n}: unwritten rows"
        rows = sample_rows(c[:, n], spec.dims[n], plan.splits(n), rng)
        want = O.mttkrp_rows(c, v, Fh, n, rows)
        g = got[rows].cpu().numpy().astype(np.float64)
        err = O.relerr(g, want)
        assert err <= 1e-5, (n, err)
        # each sampled row on its own as well (the heaviest row dominates the norm)
        for j, r in enumerate(rows):
            nrm = np.linalg.norm(want[j])
            if nrm > 0:
                assert np.linalg.norm(g[j] - want[j]) / nrm <= 1e-5, (n, r)
            else:
                assert np.all(g[j] == 0.0), (n, r)
    # after the sweep the working copy is back in mode-0 order: sorted by K_0 and
    # holding the same nonzeros
    idx, val = plan.elements()
    k0 = idx[:, 0].astype(np.int64)
    k2 = idx[:, 2].astype(np.int64)
    k1 = idx[:, 1].astype(np.int64)
    key = (k0 * spec.dims[2] + k2) * spec.dims[1] + k1   # K_0 = (i0, i2, i1) fits in int64
    assert np.all(np.diff(key) > 0)
    kin = (c[:, 0] * spec.dims[2] + c[:, 2]) * spec.dims[1] + c[:, 1]
    assert np.array_equal(key, np.sort(kin))
    assert float(np.sum(val.astype(np.float64))) == pytest.approx(
        float(np.sum(v.astype(np.float64))), rel=1e-12)
    # two sweeps are bit-identical (no atomics anywhere)
    outs2 = [torch.empty(d, 32, device="cuda") for d in spec.dims]
    plan.sweep(F, outs2, graph=True)
    torch.cuda.synchronize()
    for n in range(3):
        assert torch.equal(outs[n], outs2[n])
    plan.close()


def moderate_rows(col, dim, splits, rng, cap=1_000_000):
    """Rows of at most `cap` nonzeros (the oracle adds a row's nonzeros one by one): a
    split row spanning the most blocks among those, random nonempty rows, a light
    row, an empty row, and the first and last rows when they are small enough."""
    counts = np.bincount(col, minlength=dim)
    ok = lambda r: counts[r] <= cap  # noqa: E731
    rows = {r for r in (0, dim - 1) if ok(r)}
    nz = np.nonzero((counts > 0) & (counts <= cap))[0]
    rows.update(int(x) for x in rng.choice(nz, 4, replace=False))
    light = np.nonzero(counts == 1)[0]
    if light.size:
        rows.add(int(light[0]))
    empty = np.nonzero(counts == 0)[0]
    if empty.size:
        rows.add(int(empty[0]))
    if len(splits):
        small = [s for s in splits if ok(int(s[0]))]
        if small:
            rows.add(int(max(small, key=lambda s: s[2] - s[1])[0]))
    return sorted(rows)


@pytest.mark.parametrize("name,R,dtypes", [("c3", 32, ("f32", "bf16")), ("c4b", 32, ("f32",))])
def test_full_size_more_modes_sampled_rows(name, R, dtypes):
    # 4-mode 1M x 20k x 2k x 500 (150M nonzeros) and 6-mode (40M nonzeros) at full size
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spec = synth.workload(name)
    coo, vals = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed, device="cuda")
    c, v = coo.cpu().numpy(), vals.cpu().numpy()
    del coo, vals
    torch.cuda.empty_cache()
    N = len(spec.dims)
    F = synth.make_factors(spec.dims, R, seed=synth.factor_seed(3), device="cuda")
    rng = np.random.default_rng(1)
    for dt in dtypes:
        tdt = torch.bfloat16 if dt == "bf16" else torch.float32
        Fd = [f.to(tdt) for f in F]
        Fh = [f.float().cpu().numpy() for f in Fd]
        plan = Plan(c, v, spec.dims, R, dtype=dt)
        outs = [torch.full((d, R), float("nan"), device="cuda") for d in spec.dims]
        plan.sweep(Fd, outs)
        plan.device_status()
        torch.cuda.synchronize()
        for n in range(N):
            assert not torch.isnan(outs[n]).any(), (dt, n, "unwritten rows")
            rows = moderate_rows(c[:, n], spec.dims[n], plan.splits(n), rng)
            want = O.mttkrp_rows(c, v, Fh, n, rows)
            g = outs[n][rows].cpu().numpy().astype(np.float64)
            for j, r in enumerate(rows):
                nrm = np.linalg.norm(want[j])
                if nrm > 0:
                    assert np.linalg.norm(g[j] - want[j]) / nrm <= 1e-5, (dt, n, r)
                else:
                    assert np.all(g[j] == 0.0), (dt, n, r)
        plan.close()
