"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test checks an oracle function against the mathematics or the paper:
dense unfolding times an explicit Khatri-Rao product, closed forms, brute
force on tiny inputs, the worked partition example of Section 3.4, Graham's
list-scheduling bound, ALS monotonicity and central finite differences.
"""
import itertools
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_tensor(rng, N, maxdim=5, density=0.4):
    dims = [int(rng.integers(2, maxdim + 1)) for _ in range(N)]
    allc = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int64)
    keep = rng.random(allc.shape[0]) < density
    if not keep.any():
        keep[0] = True
    coo = allc[keep]
    coo = coo[rng.permutation(coo.shape[0])]
    vals = rng.standard_normal(coo.shape[0])
    return coo, vals, dims


# ---------------------------------------------------------------- spMTTKRP


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_mttkrp_matches_dense_unfolding_times_khatri_rao(N):
    rng = np.random.default_rng(10 + N)
    for _ in range(3):
        coo, vals, dims = tiny_tensor(rng, N, maxdim=4 if N >= 5 else 5)
        R = int(rng.integers(1, 6))
        F = [rng.standard_normal((d, R)) for d in dims]
        X = O.dense_from_coo(coo, vals, dims)
        for n in range(N):
            got = O.mttkrp(coo, vals, dims, F, n)
            want = O.mttkrp_dense(X, F, n)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12), (N, n)


def test_khatri_rao_and_unfold_definitions():
    # explicit index formulas of the Khatri-Rao product and the unfolding
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((3, 2)), rng.standard_normal((4, 2))
    K = O.khatri_rao([A, B])
    for i in range(3):
        for j in range(4):
            assert np.allclose(K[i * 4 + j], A[i] * B[j])
    X = rng.standard_normal((2, 3, 4))
    U = O.unfold(X, 1)
    for i0, i1, i2 in itertools.product(range(2), range(3), range(4)):
        assert U[i1, i0 + 2 * i2] == X[i0, i1, i2]


@pytest.mark.parametrize("N", [3, 4])
def test_mttkrp_rank1_closed_form(N):
    rng = np.random.default_rng(20 + N)
    dims = [3, 4, 2, 3][:N]
    u = [rng.standard_normal(d) for d in dims]
    coo = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int64)
    vals = np.ones(coo.shape[0])
    for k in range(N):
        vals = vals * u[k][coo[:, k]]
    R = 3
    F = [rng.standard_normal((d, R)) for d in dims]
    for n in range(N):
        want = np.outer(u[n], np.prod([u[k] @ F[k] for k in range(N) if k != n], axis=0))
        assert np.allclose(O.mttkrp(coo, vals, dims, F, n), want, rtol=1e-12, atol=1e-12)


def test_mttkrp_all_ones_factors_gives_row_sums():
    coo, vals = synth.make_coo((7, 5, 6), 60, (0.0, 1.1, 0.0), seed=5)
    coo, vals = coo.numpy(), vals.numpy().astype(np.float64)
    F = [np.ones((d, 4)) for d in (7, 5, 6)]
    for n in range(3):
        M = O.mttkrp(coo, vals, (7, 5, 6), F, n)
        sums = np.bincount(coo[:, n], weights=vals, minlength=(7, 5, 6)[n])
        assert np.allclose(M, sums[:, None] * np.ones((1, 4)), rtol=1e-14)


def test_mttkrp_rows_matches_full():
    coo, vals = synth.make_coo((40, 30, 20), 900, (1.1, 1.1, 0.0), seed=9)
    coo, vals = coo.numpy(), vals.numpy()
    F = [t.numpy() for t in synth.make_factors((40, 30, 20), 5, seed=7)]
    for n in range(3):
        M = O.mttkrp(coo, vals, (40, 30, 20), F, n)
        rows = [0, 3, int(coo[0, n]), (40, 30, 20)[n] - 1]
        assert np.allclose(O.mttkrp_rows(coo, vals, F, n, rows), M[rows], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- order / remap


@pytest.mark.parametrize("N", [2, 3, 4, 6])
def test_canonical_order_matches_python_sort_of_key_tuples(N):
    rng = np.random.default_rng(30 + N)
    coo, vals, dims = tiny_tensor(rng, N, maxdim=4)
    for n in range(N):
        assert np.array_equal(O.canonical_order(coo, n), O.brute_canonical_order(coo, n))


@pytest.mark.parametrize("N", [2, 3, 5])
def test_remap_chain_and_permutation(N):
    """Stable sort of the mode-n order by i_{n+1} is the mode-(n+1) order (Section 3.1)."""
    rng = np.random.default_rng(40 + N)
    coo, vals, dims = tiny_tensor(rng, N, maxdim=5)
    nnz = coo.shape[0]
    for n in range(N):
        on = O.canonical_order(coo, n)
        nxt = (n + 1) % N
        stable = on[np.argsort(coo[on, nxt], kind="stable")]
        assert np.array_equal(stable, O.canonical_order(coo, nxt))
        npos = O.next_pos(coo, n)
        assert np.array_equal(np.sort(npos), np.arange(nnz))       # Observation 1
        moved = np.empty_like(on)
        moved[npos] = on                                             # T_out[next_pos[p]] = x_p
        assert np.array_equal(moved, O.canonical_order(coo, nxt))
    # N remaps bring the copy back to mode-0 order (Algorithm 5's swap loop)
    cur = O.canonical_order(coo, 0)
    for n in range(N):
        out = np.empty_like(cur)
        out[O.next_pos(coo, n)] = cur
        cur = out
    assert np.array_equal(cur, O.canonical_order(coo, 0))


def test_duplicates_detected():
    coo = np.array([[0, 1, 2], [1, 1, 1], [0, 1, 2]])
    assert O.has_duplicates(coo)
    assert not O.has_duplicates(coo[:2])


def test_row_starts():
    rows = np.array([0, 0, 2, 2, 2, 5])
    assert list(O.row_starts(rows, 6)) == [0, 2, 2, 5, 5, 5, 6]


# ---------------------------------------------------------------- partition


def _check_partition(rows, nblk):
    nnz = rows.shape[0]
    b = O.contiguous_partition(rows, nblk)
    assert b[0] == 0 and b[-1] == nnz and np.all(np.diff(b) >= 0)
    T = -(-nnz // nblk) if nnz else 0
    uniq, starts = np.unique(rows, return_index=True)
    ends = np.append(starts[1:], nnz)
    deg = dict(zip(uniq.tolist(), (ends - starts).tolist()))
    start = dict(zip(uniq.tolist(), starts.tolist()))
    end = dict(zip(uniq.tolist(), ends.tolist()))
    for j in range(1, nblk):
        t = min(j * T, nnz)
        if t >= nnz:
            assert b[j] == nnz
            continue
        r = int(rows[t])
        if t == start[r]:
            assert b[j] == t
        elif deg[r] <= T:
            near = start[r] if t - start[r] <= end[r] - t else end[r]
            assert b[j] == near
        else:
            assert b[j] == t
    # block sizes stay within 2T (a snap moves a boundary by at most T/2)
    if nnz:
        assert np.all(np.diff(b) <= 2 * T)
    # split rows: exactly those with a boundary strictly inside them
    sr = O.split_rows(rows, b)
    want = [r for r in uniq if np.any((b[1:-1] > start[r]) & (b[1:-1] < end[r]))]
    assert sr[:, 0].tolist() == [int(r) for r in want]
    for r, fb, lb in sr:
        assert b[fb] <= start[r] < b[fb + 1]
        assert b[lb] <= end[r] - 1 < b[lb + 1]
        assert deg[r] > T                       # only heavy rows are split
    # every non-split row lies in exactly one block (Observation 2)
    for r in uniq:
        if r in set(sr[:, 0].tolist()):
            continue
        assert O.block_of(b, start[r]) == O.block_of(b, end[r] - 1)
    return b


def test_partition_rules_on_skewed_rows():
    rng = np.random.default_rng(50)
    for trial in range(40):
        nrows = int(rng.integers(1, 30))
        deg = rng.zipf(1.6, nrows)
        deg = np.minimum(deg, 200)
        rows = np.repeat(np.sort(rng.choice(1000, nrows, replace=False)), deg)
        for nblk in (1, 2, 3, 7, 16, 64):
            _check_partition(rows, nblk)


def test_partition_edge_cases():
    _check_partition(np.zeros(0, dtype=np.int64), 4)             # empty
    _check_partition(np.array([3]), 8)                           # single nonzero, nblk > nnz
    _check_partition(np.full(100, 5), 8)                         # one heavy row everywhere
    b = O.contiguous_partition(np.full(100, 5), 8)
    assert O.split_rows(np.full(100, 5), b).tolist() == [[5, 0, 7]]


def test_ownership_writes_every_row_once():
    rng = np.random.default_rng(60)
    for trial in range(30):
        dim = int(rng.integers(1, 60))
        nnz = int(rng.integers(0, 300))
        rows = np.sort(np.minimum(rng.zipf(1.3, nnz) - 1, dim - 1)) if nnz else np.zeros(0, int)
        for nblk in (1, 3, 8, 40):
            b = O.contiguous_partition(rows, nblk)
            assert np.all(O.ownership_writes(rows, b, dim) == 1)


def test_ownership_detects_a_wrong_split_table():
    # plant a mistake in the oracle's split detection: the rule must then fail
    rows = np.repeat(np.arange(4), [1, 30, 2, 1])
    b = O.contiguous_partition(rows, 4)
    good = O.ownership_writes(rows, b, 4)
    assert np.all(good == 1)
    orig = O.spmttkrp_oracle.split_rows
    try:
        O.spmttkrp_oracle.split_rows = lambda r, bb: np.zeros((0, 3), dtype=np.int64)
        bad = O.spmttkrp_oracle.ownership_writes(rows, b, 4)
    finally:
        O.spmttkrp_oracle.split_rows = orig
    assert not np.all(bad == 1)


# ---------------------------------------------------------------- Algorithm 1


def test_alg1_worked_example_of_section_3_4():
    g = json.load(open(os.path.join(GOLDEN, "alg1_worked_example.json")))
    assign, load = O.lpt_partition(g["mode0_degrees"], g["kappa"])
    assert assign.tolist() == g["expected_block_of_vertex"]
    assert load.tolist() == g["expected_loads"]


def test_alg1_graham_bound_against_brute_force_optimum():
    rng = np.random.default_rng(70)
    for trial in range(60):
        nv = int(rng.integers(1, 10))
        kappa = int(rng.integers(2, 4))
        deg = rng.integers(1, 20, nv)
        _, load = O.lpt_partition(deg, kappa)
        opt = O.all_partitions_opt(deg, kappa)
        assert load.sum() == deg.sum()
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3.0 * kappa)) * opt + 1e-9


def test_alg1_remap_ids_are_a_permutation_grouped_by_block():
    coo, vals = synth.make_coo((9, 7, 5), 120, (1.1, 0.0, 0.0), seed=3)
    coo = coo.numpy()
    rid = O.lpt_remap_ids(coo, 0, 3)
    assert np.array_equal(np.sort(rid), np.arange(coo.shape[0]))
    deg = np.bincount(coo[:, 0], minlength=9)
    assign, _ = O.lpt_partition(deg, 3)
    blk_in_order = assign[coo[np.argsort(rid), 0]]
    assert np.all(np.diff(blk_in_order) >= 0)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_alg1_remap_ids_within_block_order_is_canonical(N):
    """Section 3.4 orders the hyperedges by partition id; inside a block the
    reading is the canonical K_n order.  Pinned against Python ``sorted`` over
    explicit (block, K_n) tuples, and against the independently pinned
    canonical order filtered block by block: a reversed, rotated or shifted key
    inside a block fails both."""
    rng = np.random.default_rng(90 + N)
    for trial in range(4):
        coo, vals, dims = tiny_tensor(rng, N, maxdim=6)
        for n in range(N):
            for kappa in (2, 3, 4):
                rid = O.lpt_remap_ids(coo, n, kappa)
                deg = np.bincount(coo[:, n], minlength=int(coo[:, n].max()) + 1)
                assign, _ = O.lpt_partition(deg, kappa)
                blk = assign[coo[:, n]]
                rows = [tuple(int(x) for x in r) for r in coo]
                brute = sorted(range(len(rows)),
                               key=lambda e: (int(blk[e]),) +
                               tuple(rows[e][(n - j) % N] for j in range(N)))
                order = np.argsort(rid)
                assert np.array_equal(order, np.asarray(brute)), (N, n, kappa)
                canon = O.brute_canonical_order(coo, n)
                by_block = [e for b in range(kappa) for e in canon if blk[e] == b]
                assert np.array_equal(order, np.asarray(by_block)), (N, n, kappa)


@pytest.mark.parametrize("tile", [1, 3, 7, 960])
def test_tile_write_order_visits_destinations_in_increasing_order(tile):
    """Within every tile the write order is a permutation of the tile's local
    indices along which next_pos strictly increases; next_pos values are
    distinct, so these two properties fix it."""
    rng = np.random.default_rng(tile)
    for N in (2, 3, 4):
        coo, vals, dims = tiny_tensor(rng, N, maxdim=7, density=0.5)
        for n in range(N):
            w = O.tile_write_order(coo, n, tile)
            npos = O.next_pos(coo, n)
            for base in range(0, len(npos), tile):
                seg = [int(x) for x in npos[base:base + tile]]
                got = [int(x) for x in w[base:base + len(seg)]]
                assert sorted(got) == list(range(len(seg)))
                along = [seg[j] for j in got]
                assert all(x < y for x, y in zip(along, along[1:]))


def test_cp_loss_grad_rows_equal_full_gradient_rows():
    """The row-by-row CP-loss gradient equals the rows of the full gradient (itself
    checked against central differences), for every mode and for empty rows."""
    rng = np.random.default_rng(70)
    coo, vals, dims = tiny_tensor(rng, 3, maxdim=6, density=0.5)
    F = [rng.standard_normal((d, 4)) for d in dims]
    G = O.cp_loss_grad(coo, vals, dims, F)
    for n in range(3):
        rows = list(range(dims[n]))
        assert np.allclose(O.cp_loss_grad_rows(coo, vals, F, n, rows), G[n], rtol=1e-12,
                           atol=1e-12)


def test_hot_rows_are_the_most_frequent():
    """No row outside the hot set holds more nonzeros than one inside it, equal
    counts prefer the lower row id, and empty rows never count."""
    rng = np.random.default_rng(11)
    for trial in range(20):
        coo, vals, dims = tiny_tensor(rng, 3, maxdim=7, density=0.4)
        for k in range(3):
            for H in (1, 2, 3, 50):
                hot = set(O.hot_rows(coo, k, H).tolist())
                deg = np.bincount(coo[:, k], minlength=dims[k])
                nonempty = [r for r in range(dims[k]) if deg[r] > 0]
                assert len(hot) == min(H, len(nonempty))
                assert all(deg[r] > 0 for r in hot)
                for r in hot:
                    for s in nonempty:
                        if s not in hot:
                            assert deg[r] > deg[s] or (deg[r] == deg[s] and r < s)


def test_flycoo_pack_round_trip_and_widths():
    """Every index comes back from its bit field (shift and mask by hand), the
    widths are the ceil(log2 I) of the memory formula, and the value is word 3."""
    rng = np.random.default_rng(3)
    dims = (1000, 3, 1, 70000, 2)
    coo = np.stack([rng.integers(0, d, 50) for d in dims], 1)
    vals = rng.random(50).astype(np.float32)
    w = O.flycoo_pack(coo, vals, dims)
    assert [O.index_bits(d) for d in dims] == [10, 2, 1, 17, 1]
    for e in range(50):
        field = int(w[e, 0]) | (int(w[e, 1]) << 32) | (int(w[e, 2]) << 64)
        off = 0
        for k, d in enumerate(dims):
            b = O.index_bits(d)
            assert (field >> off) & ((1 << b) - 1) == coo[e, k]
            off += b
        assert field >> off == 0
        assert w[e, 3] == vals[e:e + 1].view(np.uint32)[0]


def test_flycoo_memory_formula():
    # Section 3.5.1: N log2|X| + sum log2 I_h + value bits
    assert O.flycoo_bits(2 ** 20, [2 ** 10] * 3) == pytest.approx(3 * 20 + 30 + 32)


# ---------------------------------------------------------------- CP-ALS


def test_als_residual_never_increases_per_mode():
    rng = np.random.default_rng(80)
    dims = (6, 5, 4)
    coo, vals, _ = tiny_tensor(rng, 3, maxdim=6, density=0.5)
    dims = tuple(int(coo[:, k].max()) + 1 for k in range(3))
    X = O.dense_from_coo(coo, vals, dims)
    R = 3
    A = [rng.standard_normal((d, R)) for d in dims]
    lam = np.ones(R)
    prev = np.linalg.norm(X - O.cp_full(A, lam))
    for it in range(6):
        for n in range(3):
            A, lam, _ = O.als_mode_update(coo, vals, dims, A, n)
            res = np.linalg.norm(X - O.cp_full(A, lam))
            assert res <= prev * (1 + 1e-10) + 1e-12
            prev = res


def test_als_fit_formula_matches_dense_residual():
    rng = np.random.default_rng(81)
    coo, vals, dims = tiny_tensor(rng, 4, maxdim=4, density=0.5)
    X = O.dense_from_coo(coo, vals, dims)
    A = [rng.standard_normal((d, 3)) for d in dims]
    A2, lam, fit = O.cp_als_iter(coo, vals, dims, A)
    want = 1 - np.linalg.norm(X - O.cp_full(A2, lam)) / np.linalg.norm(X)
    assert fit == pytest.approx(want, abs=1e-10)


def test_als_recovers_planted_exact_low_rank_tensor():
    rng = np.random.default_rng(82)
    dims, R = (6, 5, 7), 2
    P = [rng.standard_normal((d, R)) for d in dims]
    X = O.cp_full(P)
    coo = np.array(list(itertools.product(*[range(d) for d in dims])), dtype=np.int64)
    vals = X[tuple(coo.T)]
    A = [rng.standard_normal((d, R)) for d in dims]
    fit = 0
    for it in range(200):
        A, lam, fit = O.cp_als_iter(coo, vals, dims, A)
        if fit > 0.9999:
            break
    assert fit > 0.999


def test_als_update_ignores_the_other_factors_column_scales():
    """The mode update followed by the 2-norm normalisation (Section 2.1.4's ALS,
    Kolda-Bader) does not depend on positive column scales of the other factors;
    lambda absorbs them.  Then a sweep that never normalises inside the loop, and
    normalises once after it (lambda_r = prod_k |U_k[:, r]|), gives the factors and
    lambda of the normalised sweeps: the reading the folded ALS loop rests on."""
    rng = np.random.default_rng(83)
    coo, vals, dims = tiny_tensor(rng, 3, maxdim=6, density=0.6)
    R = 3
    A = [rng.standard_normal((d, R)) for d in dims]
    for n in range(3):
        c = [rng.uniform(0.2, 5.0, R) for _ in dims]
        B = [A[k] * c[k] if k != n else A[k] for k in range(3)]
        An, la, _ = O.als_mode_update(coo, vals, dims, A, n)
        Bn, lb, _ = O.als_mode_update(coo, vals, dims, B, n)
        assert np.allclose(An[n], Bn[n], rtol=0, atol=1e-10)
        scale = np.prod([c[k] for k in range(3) if k != n], axis=0)
        assert np.allclose(lb * scale, la, rtol=1e-10, atol=0)
    # three sweeps: normalised every mode against folded (never normalised inside)
    F, U = [a.copy() for a in A], [a.copy() for a in A]
    for it in range(3):
        F, lam, _ = O.cp_als_iter(coo, vals, dims, F)
        for n in range(3):
            M = O.mttkrp(coo, vals, dims, U, n)
            V = np.ones((R, R))
            for k in range(3):
                if k != n:
                    V = V * (U[k].T @ U[k])
            U[n] = np.linalg.solve(V, M.T).T
    norms = [np.linalg.norm(u, axis=0) for u in U]
    for k in range(3):
        assert np.allclose(U[k] / norms[k], F[k], rtol=0, atol=1e-8), k
    assert np.allclose(np.prod(norms, axis=0), lam, rtol=1e-8, atol=0)


def test_als_rejects_non_spd():
    coo = np.array([[0, 0, 0], [1, 1, 1]])
    vals = np.array([1.0, 2.0])
    A = [np.zeros((2, 2)) for _ in range(3)]
    with pytest.raises(np.linalg.LinAlgError):
        O.cp_als_iter(coo, vals, (2, 2, 2), A)


# ---------------------------------------------------------------- CP loss


def test_cp_loss_gradient_matches_central_differences():
    spec = synth.workload("c5fd")
    coo, _ = synth.make_coo(spec.dims, spec.nnz, spec.skew, spec.seed)
    x = synth.make_planted_targets(coo, spec.dims, 8, 0.1, spec.seed + 1).numpy()
    coo = coo.numpy()
    F = [t.numpy().astype(np.float64) for t in
         synth.make_factors(spec.dims, 8, seed=3000, scale=0.5)]
    G = O.cp_loss_grad(coo, x, spec.dims, F)
    rng = np.random.default_rng(90)
    h = 1e-6
    for k in range(3):
        for _ in range(8):
            i = int(rng.integers(0, spec.dims[k]))
            r = int(rng.integers(0, 8))
            Fp = [f.copy() for f in F]
            Fm = [f.copy() for f in F]
            Fp[k][i, r] += h
            Fm[k][i, r] -= h
            fd = (O.cp_loss(coo, x, Fp)[0] - O.cp_loss(coo, x, Fm)[0]) / (2 * h)
            assert fd == pytest.approx(G[k][i, r], rel=1e-6, abs=1e-7)
    # the loss itself against an explicit loop
    loss, _ = O.cp_loss(coo, x, F)
    want = 0.0
    for e in range(coo.shape[0]):
        m = sum(np.prod([F[k][coo[e, k], r] for k in range(3)]) for r in range(8))
        want += 0.5 * (m - x[e]) ** 2
    assert loss == pytest.approx(want, rel=1e-12)


def test_bf16_round_matches_torch():
    a = torch.randn(10000, generator=torch.Generator().manual_seed(1)) * 100
    want = a.to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(O.bf16_round(a.numpy()), want)


def test_planted_targets_have_unit_model_variance():
    coo, _ = synth.make_coo((50, 40, 30), 20000, (0.0, 0.0, 0.0), seed=4)
    x = synth.make_planted_targets(coo, (50, 40, 30), 8, 0.0, seed=5).numpy()
    assert 0.7 < np.var(x) < 1.3


def test_synth_coordinates_distinct_and_skewed():
    coo, vals = synth.make_coo((1000, 50, 40), 20000, (1.1, 0.0, 0.0), seed=6)
    c = coo.numpy()
    assert not O.has_duplicates(c)
    assert c.shape == (20000, 3)
    assert (vals.numpy() >= 0).all() and (vals.numpy() < 1).all()
    top = np.bincount(c[:, 0]).max() / c.shape[0]
    assert top > 0.05                       # the Zipf head is heavy
