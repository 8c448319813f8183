"""GPU parity of CP-ALS, the CP loss / gradient and the autotuner against the oracle."""
import os

import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2405_08470_gb300 import Plan, SpmError
from paper_2405_08470_gb300.cp import CPLoss, cp_als

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dims,R,nnz", [((200, 150, 100), 16, 50_000),
                                        ((40, 30, 20, 10), 8, 6_000),
                                        ((30, 20, 12, 8, 6), 8, 4_000)])
def test_als_iterations_match_oracle(dims, R, nnz):
    """Five CP-ALS iterations (Section 2.1.4) on the GPU and in the FP64 oracle,
    both started from the same seeded factors.  Fit, lambda and every factor are
    held to the FP32 bar of 1e-5.  The condition number of each V = Hadamard of
    the other Grams is reported with any failure: A_n = M V^-1 amplifies the
    FP32 error of M by at most cond(V)."""
    N = len(dims)
    coo, vals = synth.make_coo(dims, nnz, (0.0,) * N, seed=nnz + N)
    c, v = coo.numpy(), vals.numpy()
    F0 = synth.make_factors(dims, R, seed=2000)
    Fd = [f.cuda() for f in F0]
    Fo = [f.numpy().astype(np.float64) for f in F0]
    p = Plan(c, v, dims, R, nblk=37)
    lam = torch.empty(R, device="cuda")
    for it in range(5):
        fit = p.als_iter(Fd, lam)           # first call eager, later calls graph replays
        conds = []
        A = [f.copy() for f in Fo]
        for n in range(N):                   # the oracle's sweep, mode by mode
            V = np.ones((R, R))
            for k in range(N):
                if k != n:
                    V = V * O.gram(A[k])
            conds.append(float(np.linalg.cond(V)))
            A, lo, _ = O.als_mode_update(c, v, dims, A, n)
        Fo, lo2, fo = O.cp_als_iter(c, v, dims, Fo)
        assert np.array_equal(lo, lo2)
        errs = [O.relerr(Fd[k].cpu().numpy(), Fo[k]) for k in range(N)]
        lerr = O.relerr(lam.cpu().numpy(), lo)
        info = dict(iteration=it, fit=(fit, fo), factor_err=errs, lambda_err=lerr,
                    cond_V=conds)
        assert abs(fit - fo) <= 1e-5, info
        assert lerr <= 1e-5, info
        assert max(errs) <= 1e-5, info
    p.close()


def test_als_fit_never_decreases_and_bf16_runs():
    dims, R = (120, 90, 60), 8
    coo, vals = synth.make_coo(dims, 20_000, (1.1, 1.1, 0.0), seed=3)
    p = Plan(coo.numpy(), vals.numpy(), dims, R)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=4)]
    _, fits = cp_als(p, F, 8)
    assert all(b >= a - 1e-6 for a, b in zip(fits, fits[1:])), fits
    p.close()
    pb = Plan(coo.numpy(), vals.numpy(), dims, R, dtype="bf16")
    Fb = [f.cuda().to(torch.bfloat16) for f in synth.make_factors(dims, R, seed=4)]
    _, fb = cp_als(pb, Fb, 8)
    assert abs(fb[-1] - fits[-1]) < 2e-2
    pb.close()


def test_als_not_spd_is_a_status_not_a_fault():
    dims, R = (20, 15, 10), 4
    coo, vals = synth.make_coo(dims, 500, (0.0,) * 3, seed=8)
    p = Plan(coo.numpy(), vals.numpy(), dims, R)
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=9)]
    F[1][:, 2] = 0.0           # zero column: V for mode 0 is singular
    lam = torch.empty(R, device="cuda")
    with pytest.raises(SpmError) as ei:
        p.als_iter(F, lam)
    assert ei.value.status == -7
    # the plan stays usable
    G = [f.cuda() for f in synth.make_factors(dims, R, seed=9)]
    fit = p.als_iter(G, lam)
    assert np.isfinite(fit)
    # the ALS loop graph reports the same status and stops at the failing iteration
    H = [f.cuda() for f in synth.make_factors(dims, R, seed=9)]
    H[1][:, 2] = 0.0
    with pytest.raises(SpmError) as ei:
        p.als_run(H, lam, 4, 0.0)
    assert ei.value.status == -7
    fits = p.als_run([f.cuda() for f in synth.make_factors(dims, R, seed=9)], lam, 3, 0.0)
    assert len(fits) == 3 and all(np.isfinite(fits))
    p.close()


@pytest.mark.parametrize("dtype,dims", [("f32", (80, 60, 40)), ("bf16", (80, 60, 40)),
                                        ("f32", (30, 20, 12, 8)), ("bf16", (30, 20, 12, 8)),
                                        ("f32", (12, 9, 7, 5, 4))])
def test_cp_loss_and_gradient_match_oracle(dtype, dims):
    R = 16
    nnz = 12_000 if len(dims) < 5 else 4_000
    coo, _ = synth.make_coo(dims, nnz, (1.1,) * len(dims), seed=21)
    x = synth.make_planted_targets(coo, dims, 8, 0.1, seed=22)
    c, xv = coo.numpy(), x.numpy()
    F = synth.make_factors(dims, R, seed=23, scale=0.3)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda().requires_grad_(True) for f in F]
    Fq = [f.to(tdt).float().numpy().astype(np.float64) for f in F]
    p = Plan(c, xv, dims, R, dtype=dtype, nblk=19)
    loss = CPLoss.apply(p, *Fd)
    loss.backward()
    want_loss, _ = O.cp_loss(c, xv, Fq)
    assert abs(loss.item() - want_loss) <= 1e-5 * abs(want_loss)
    G = O.cp_loss_grad(c, xv, dims, Fq)
    # the engine's FP32 gradients (before autograd casts them to the factor type)
    g32 = [torch.empty(d, R, device="cuda") for d in dims]
    lossb = torch.empty((), device="cuda")
    fs = [f.detach() for f in Fd]
    p.loss_fwd(fs, lossb)
    p.loss_bwd(fs, torch.ones((), device="cuda"), g32)
    torch.cuda.synchronize()
    for k in range(len(dims)):
        # accumulation error alone: FP64 oracle on the same (BF16-rounded) factors
        err = O.relerr(g32[k].cpu().numpy(), G[k])
        assert err <= 1e-5, (k, err)
        # the autograd gradient is that FP32 gradient in the factor's type
        assert torch.equal(Fd[k].grad, g32[k].to(tdt)), k
    if dtype == "bf16":  # quantisation error: FP64 oracle on the FP32 factors
        G32 = O.cp_loss_grad(c, xv, dims, [f.numpy().astype(np.float64) for f in F])
        for k in range(len(dims)):
            err = O.relerr(g32[k].cpu().numpy(), G32[k])
            assert err <= 1e-2, (k, err)
    p.close()


def test_cp_loss_backward_uses_its_own_forward():
    """Two forwards with different factors, then the first loss's backward: the
    gradient is the first forward's (its residuals are recomputed), and a second
    backward through a retained graph gives the same gradient again."""
    dims, R = (50, 40, 30), 8
    coo, _ = synth.make_coo(dims, 3_000, (1.1,) * 3, seed=41)
    x = synth.make_planted_targets(coo, dims, 4, 0.1, seed=42)
    c, xv = coo.numpy(), x.numpy()
    FA = synth.make_factors(dims, R, seed=43, scale=0.3)
    FB = synth.make_factors(dims, R, seed=44, scale=0.3)
    p = Plan(c, xv, dims, R)
    A = [f.cuda().requires_grad_(True) for f in FA]
    B = [f.cuda().requires_grad_(True) for f in FB]
    la = CPLoss.apply(p, *A)
    lb = CPLoss.apply(p, *B)
    la.backward(retain_graph=True)
    GA = O.cp_loss_grad(c, xv, dims, [f.numpy().astype(np.float64) for f in FA])
    first = [a.grad.clone() for a in A]
    for k in range(3):
        assert O.relerr(first[k].cpu().numpy(), GA[k]) <= 1e-5, k
    for a in A:
        a.grad = None
    la.backward()
    for k in range(3):
        assert torch.equal(A[k].grad, first[k]), k
    lb.backward()
    GB = O.cp_loss_grad(c, xv, dims, [f.numpy().astype(np.float64) for f in FB])
    for k in range(3):
        assert O.relerr(B[k].grad.cpu().numpy(), GB[k]) <= 1e-5, k
    p.close()


def test_cp_loss_gradient_finite_differences_small_copy():
    spec = synth.workload("c5fd")
    coo, _ = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed)
    x = synth.make_planted_targets(coo, spec.dims, 8, 0.1, spec.seed + 1)
    F = synth.make_factors(spec.dims, 8, seed=3000, scale=0.5)
    p = Plan(coo.numpy(), x.numpy(), spec.dims, 8)
    Fd = [f.cuda().requires_grad_(True) for f in F]
    loss = CPLoss.apply(p, *Fd)
    loss.backward()
    Fo = [f.numpy().astype(np.float64) for f in F]
    rng = np.random.default_rng(5)
    h = 1e-3
    for k in range(3):
        for _ in range(5):
            i, r = int(rng.integers(spec.dims[k])), int(rng.integers(8))
            Fp = [f.copy() for f in Fo]
            Fm = [f.copy() for f in Fo]
            Fp[k][i, r] += h
            Fm[k][i, r] -= h
            fd = (O.cp_loss(coo.numpy(), x.numpy(), Fp)[0] -
                  O.cp_loss(coo.numpy(), x.numpy(), Fm)[0]) / (2 * h)
            got = Fd[k].grad[i, r].item()
            assert abs(got - fd) <= 1e-4 * max(1.0, abs(fd)), (k, i, r, got, fd)
    p.close()


def test_autotune_keeps_results_and_caches(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SPMTTKRP_TUNE_CACHE", str(cache))
    dims, R = (3000, 2000, 1000), 32
    coo, vals = synth.make_coo(dims, 300_000, (1.1, 1.1, 1.1), seed=31, device="cuda")
    c, v = coo.cpu().numpy(), vals.cpu().numpy()
    F = [f.cuda() for f in synth.make_factors(dims, R, seed=32)]
    p = Plan(c, v, dims, R)
    scratch = [torch.empty(d, R, device="cuda") for d in dims]
    p.autotune(F, scratch)
    assert cache.exists() and cache.read_text().strip()
    key, nps, tile, variant, stages = cache.read_text().split()
    assert "_e32_" in key and int(variant) in (0, 1) and int(stages) in (2, 3)
    assert p.info()["tile"] == int(tile) or int(variant) == 1
    outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
    p.sweep(F, outs)
    torch.cuda.synchronize()
    Fh = [f.cpu().numpy() for f in F]
    for n in range(3):
        rows = np.unique(np.concatenate([c[:50, n], [0, dims[n] - 1]]))
        want = O.mttkrp_rows(c, v, Fh, n, rows)
        assert O.relerr(outs[n].cpu().numpy()[rows], want) <= 1e-5
    # a second plan of the same shape picks the cached configuration
    p2 = Plan(c, v, dims, R)
    p2.autotune(F, scratch)
    assert p2.info()["nblk"] == p.info()["nblk"]
    p.close()
    p2.close()


@pytest.mark.parametrize("eb", [0, 16])
@pytest.mark.parametrize("dtype,R", [("f32", 32), ("bf16", 32), ("f32", 64), ("bf16", 16)])
def test_fused_and_plain_forward_give_the_same_loss_and_gradients(dtype, R, eb):
    """The fused forward (residuals, the current mode's gradient and the residual
    copy in the next order, in one pass) against the plain forward followed by a
    full backward sweep: equal loss and gradients within FP32 summation order,
    both against the FP64 oracle, and the working copy untouched by either; for
    32-byte (default) and unpadded 16-byte nonzeros."""
    dims = (300, 200, 120)
    coo, _ = synth.make_coo(dims, 40_000, (1.1, 1.1, 1.1), seed=R + 5)
    x = synth.make_planted_targets(coo, dims, 8, 0.1, seed=6)
    c, xv = coo.numpy(), x.numpy()
    F = synth.make_factors(dims, R, seed=7, scale=0.3)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    Fd = [f.to(tdt).cuda() for f in F]
    Fq = [f.to(tdt).float().numpy().astype(np.float64) for f in F]
    p = Plan(c, xv, dims, R, dtype=dtype, nblk=57, element_bytes=eb)
    assert p.info()["elem_bytes"] == (eb or 32)
    want_loss, _ = O.cp_loss(c, xv, Fq)
    G = O.cp_loss_grad(c, xv, dims, Fq)
    idx0, _ = p.elements()
    for start in range(3):  # the fused pass runs in the working copy's current mode
        p.remap(start)
        got = {}
        for fo in (False, True):
            loss = torch.empty((), device="cuda")
            g = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
            p.loss_fwd(Fd, loss, forward_only=fo)
            p.loss_bwd(Fd, torch.full((), 2.0, device="cuda"), g)
            torch.cuda.synchronize()
            assert abs(loss.item() - want_loss) <= 1e-5 * abs(want_loss), (start, fo)
            for k in range(3):
                err = O.relerr(g[k].cpu().numpy().astype(np.float64), 2.0 * G[k])
                assert err <= 1e-5, (start, fo, k, err)
            got[fo] = g
        for k in range(3):
            assert O.relerr(got[False][k].cpu().numpy().astype(np.float64),
                            got[True][k].cpu().numpy().astype(np.float64)) <= 1e-5
    p.remap(0)
    idx1, _ = p.elements()
    assert np.array_equal(idx0, idx1)
    p.close()


@pytest.mark.parametrize("dims,R", [((200, 150, 100), 16), ((40, 30, 20, 10), 8),
                                    ((150, 120, 100), 72)])
def test_als_loop_graph_matches_single_iterations_and_stops_on_the_device(dims, R):
    """cp_als_run: max_iters iterations in one graph launch, with the column
    scales folded (no normalisation inside the loop, one after it), give the fits,
    factors and lambda of that many cp_als_iter calls and of the FP64 oracle's
    normalised iterations within 1e-5: the mode update followed by the
    normalisation does not depend on the other factors' column scales (the ALS
    update of Section 2.1.4, Kolda-Bader), so the two differ in rounding only.
    The returned factors have unit column norms; a loose tol stops after two
    iterations, decided on the device."""
    N = len(dims)
    coo, vals = synth.make_coo(dims, 30_000 if N == 3 else 6_000, (0.0,) * N, seed=77 + N)
    c, v = coo.numpy(), vals.numpy()
    F0 = synth.make_factors(dims, R, seed=78)
    pa = Plan(c, v, dims, R)
    pb = Plan(c, v, dims, R)
    Fa = [f.cuda() for f in F0]
    Fb = [f.cuda() for f in F0]
    la, lb = torch.empty(R, device="cuda"), torch.empty(R, device="cuda")
    fits = pa.als_run(Fa, la, 5, 0.0)
    ref = [pb.als_iter(Fb, lb) for _ in range(5)]
    assert len(fits) == 5
    assert max(abs(a - b) for a, b in zip(fits, ref)) <= 1e-6, (fits, ref)
    for k in range(N):
        assert O.relerr(Fa[k].cpu().numpy(), Fb[k].cpu().numpy()) <= 1e-5, k
        norms = torch.linalg.vector_norm(Fa[k].double(), dim=0)
        assert torch.allclose(norms, torch.ones_like(norms), rtol=0, atol=1e-6), k
    assert O.relerr(la.cpu().numpy(), lb.cpu().numpy()) <= 1e-5
    Fo = [f.numpy().astype(np.float64) for f in F0]
    for it in range(5):
        Fo, lo, fo = O.cp_als_iter(c, v, dims, Fo)
        assert abs(fits[it] - fo) <= 1e-5, (it, fits[it], fo)
    for k in range(N):
        assert O.relerr(Fa[k].cpu().numpy(), Fo[k]) <= 1e-5, k
    assert O.relerr(la.cpu().numpy(), lo) <= 1e-5
    # a second call replays the graph: five more iterations continue from there
    more = pa.als_run(Fa, la, 5, 0.0)
    assert len(more) == 5 and all(b >= a - 1e-6 for a, b in zip(more, more[1:]))
    # tol larger than any change: the device stops the loop after two iterations
    G = [f.cuda() for f in F0]
    two = pa.als_run(G, la, 10, 1.0)
    assert len(two) == 2
    for k in range(N):  # the normalisation after the loop ran after its early stop too
        norms = torch.linalg.vector_norm(G[k].double(), dim=0)
        assert torch.allclose(norms, torch.ones_like(norms), rtol=0, atol=1e-6), k
    # the working copy is still consistent after the loop
    outs = [torch.empty(d, R, device="cuda") for d in dims]
    pa.sweep(G, outs)
    torch.cuda.synchronize()
    Gh = [g.cpu().numpy().astype(np.float64) for g in G]
    for n in range(N):
        assert O.relerr(outs[n].cpu().numpy(), O.mttkrp(c, v, dims, Gh, n)) <= 1e-5, n
    pa.close()
    pb.close()


def test_als_loop_graph_bf16_factors():
    """cp_als_run on BF16 factors: the folded loop's fits track the FP32 loop's
    (BF16 bar 1e-2), lambda is positive, and the returned factors have unit column
    norms up to BF16 rounding."""
    dims, R = (120, 90, 60), 8
    coo, vals = synth.make_coo(dims, 20_000, (1.1, 1.1, 0.0), seed=3)
    c, v = coo.numpy(), vals.numpy()
    F0 = synth.make_factors(dims, R, seed=4)
    pf = Plan(c, v, dims, R)
    pb = Plan(c, v, dims, R, dtype="bf16")
    Ff = [f.cuda() for f in F0]
    Fb = [f.cuda().to(torch.bfloat16) for f in F0]
    lf, lb = torch.empty(R, device="cuda"), torch.empty(R, device="cuda")
    ff = pf.als_run(Ff, lf, 8, 0.0)
    fb = pb.als_run(Fb, lb, 8, 0.0)
    assert len(fb) == 8 and all(np.isfinite(fb))
    assert max(abs(a - b) for a, b in zip(ff, fb)) < 1e-2, (ff, fb)
    assert bool((lb > 0).all())
    for k in range(3):
        norms = torch.linalg.vector_norm(Fb[k].double(), dim=0)
        assert torch.allclose(norms, torch.ones_like(norms), rtol=0, atol=1e-2), k
    pf.close()
    pb.close()
