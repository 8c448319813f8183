"""FP64 CPU oracle for all-mode sparse MTTKRP, its FLYCOO-style remap and CP-ALS.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU engine computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA path and imports
nothing from it.

Paper: Wijeratne, Kannan, Prasanna, "Sparse MTTKRP Acceleration for Tensor
Decomposition on GPU" (CF '24).  Each function cites the section, equation or
algorithm it follows.  Where the paper is silent the reading taken is stated
in the docstring.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (dense unfolding x explicit Khatri-Rao
product, closed forms, brute force on tiny inputs, the worked partition
example of Section 3.4, Graham's bound, ALS monotonicity, finite differences).
"""
from __future__ import annotations

import itertools
from typing import List, Sequence

import numpy as np

# --------------------------------------------------------------------------
# spMTTKRP (Eq. 1, Section 2.1.4; elementwise computation, Section 2.1.5)
# --------------------------------------------------------------------------


def mttkrp(coo, vals, dims, factors, n, chunk=1 << 20):
    """Mode-n spMTTKRP by its definition, in FP64.

    Eq. 1 / Section 2.1.5: for every nonzero x(i_0..i_{N-1}) = v, taken in
    input order, add v * (Hadamard product of rows A_k[i_k, :] for k != n) to
    output row M[i_n, :].  ``np.add.at`` accumulates unbuffered, in order.
    Chunking the nonzero list keeps the same order.
    """
    coo = np.asarray(coo)
    vals = np.asarray(vals, dtype=np.float64)
    N = coo.shape[1]
    R = np.asarray(factors[0]).shape[1]
    F = [np.asarray(f, dtype=np.float64) for f in factors]
    M = np.zeros((int(dims[n]), R), dtype=np.float64)
    for lo in range(0, coo.shape[0], chunk):
        hi = min(lo + chunk, coo.shape[0])
        ell = np.repeat(vals[lo:hi, None], R, axis=1)
        for k in range(N):
            if k == n:
                continue
            ell = ell * F[k][coo[lo:hi, k]]
        np.add.at(M, coo[lo:hi, n], ell)
    return M


def mttkrp_rows(coo, vals, factors, n, rows):
    """Selected output rows of mode-n spMTTKRP, each by its own definition.

    For every requested row i: sum over the nonzeros with i_n == i (in input
    order) of v * prod_{k != n} A_k[i_k, :].  Used to check single rows of
    workloads too large for the full oracle.
    """
    coo = np.asarray(coo)
    vals = np.asarray(vals, dtype=np.float64)
    N = coo.shape[1]
    R = np.asarray(factors[0]).shape[1]
    out = np.zeros((len(rows), R), dtype=np.float64)
    col = coo[:, n]
    for j, i in enumerate(rows):
        sel = np.nonzero(col == i)[0]
        ell = np.repeat(vals[sel, None], R, axis=1)
        for k in range(N):
            if k == n:
                continue
            ell = ell * np.asarray(factors[k], dtype=np.float64)[coo[sel, k]]
        acc = np.zeros(R, dtype=np.float64)
        for t in range(ell.shape[0]):
            acc += ell[t]
        out[j] = acc
    return out


def dense_from_coo(coo, vals, dims):
    X = np.zeros(tuple(int(d) for d in dims), dtype=np.float64)
    X[tuple(np.asarray(coo).T)] = np.asarray(vals, dtype=np.float64)
    return X


def unfold(X, n):
    """Mode-n matricization X_(n) (Section 2.1.3; Kolda-Bader column order).

    Column j of X_(n) = sum_{k != n} i_k * prod_{m < k, m != n} I_m, i.e. the
    lowest remaining mode varies fastest.
    """
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1, order="F")


def khatri_rao(mats):
    """Column-wise Kronecker product; the first matrix's row index varies slowest."""
    out = np.asarray(mats[0], dtype=np.float64)
    for m in mats[1:]:
        m = np.asarray(m, dtype=np.float64)
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, out.shape[1])
    return out


def mttkrp_dense(X, factors, n):
    """Brute-force M_n = X_(n) (A_{N-1} (.) ... (.) A_{n+1} (.) A_{n-1} (.) ... (.) A_0).

    Eq. 1 writes the Khatri-Rao operands in cyclic order; any consistent pair
    of unfolding and Khatri-Rao order gives the same M_n.  This uses Kolda's.
    """
    N = X.ndim
    mats = [factors[k] for k in reversed(range(N)) if k != n]
    return unfold(X, n) @ khatri_rao(mats)


# --------------------------------------------------------------------------
# Canonical per-mode order, remap ids (Section 3.1, 3.4, 3.5; Algorithm 3)
# --------------------------------------------------------------------------


def canonical_order(coo, n):
    """Mode-n order: nonzeros sorted lexicographically by K_n.

    Reading (the paper leaves the order inside a partition open, Section 3.4):
    K_n = (i_n, i_{n-1}, ..., i_0, i_{N-1}, ..., i_{n+1}), most significant
    first.  With distinct coordinates this order is total.  ``np.lexsort``
    takes the primary key last.
    """
    coo = np.asarray(coo)
    N = coo.shape[1]
    keys = [coo[:, (n + 1 + j) % N] for j in range(N)]
    return np.lexsort(keys)


def next_pos(coo, n):
    """Remap ids for the dynamic remap of mode n (Section 3.1; Algorithm 3).

    next_pos[p] = position, in the mode-(n+1 mod N) order, of the nonzero at
    position p of the mode-n order.  Writing element p to T_out[next_pos[p]]
    turns a mode-n-ordered copy into the mode-(n+1)-ordered copy.
    """
    coo = np.asarray(coo)
    N = coo.shape[1]
    on = canonical_order(coo, n)
    onext = canonical_order(coo, (n + 1) % N)
    inv = np.empty_like(onext)
    inv[onext] = np.arange(onext.shape[0])
    return inv[on].astype(np.int64)


def has_duplicates(coo):
    """Duplicate coordinates, found by comparing neighbours after the K_0 sort.

    Reading: the paper is silent on duplicates (FROSTT tensors have none); the
    engine rejects them.
    """
    coo = np.asarray(coo)
    if coo.shape[0] < 2:
        return False
    s = coo[canonical_order(coo, 0)]
    return bool(np.any(np.all(s[1:] == s[:-1], axis=1)))


def row_starts(sorted_rows, dim):
    """S[i] = first position of row i in a row-sorted list; S[dim] = nnz."""
    sorted_rows = np.asarray(sorted_rows)
    return np.searchsorted(sorted_rows, np.arange(int(dim) + 1), side="left").astype(np.int64)


# --------------------------------------------------------------------------
# Atomic-free contiguous block split (in the spirit of Section 3.4 and
# Observation 2; heavy-row splitting is this engine's reading)
# --------------------------------------------------------------------------


def contiguous_partition(sorted_rows, nblk):
    """Block boundaries over a row-sorted nonzero list.

    Reading (Section 3.4 gives no rule for rows heavier than a block): with
    T = ceil(nnz / nblk), for j = 1..nblk-1 take t = min(j*T, nnz) and the row
    r that holds position t.  If t is r's start, the boundary is t.  Else if
    r's degree is <= T, the boundary snaps to r's start or end, whichever is
    nearer (ties to the start).  Else r is heavy, the boundary stays at t and
    r becomes a split row.  bounds[0] = 0, bounds[nblk] = nnz.
    """
    rows = np.asarray(sorted_rows)
    nnz = rows.shape[0]
    nblk = int(nblk)
    bounds = np.zeros(nblk + 1, dtype=np.int64)
    bounds[nblk] = nnz
    if nnz == 0:
        return bounds
    T = -(-nnz // nblk)
    for j in range(1, nblk):
        t = min(j * T, nnz)
        if t >= nnz:
            bounds[j] = nnz
            continue
        r = rows[t]
        s = int(np.searchsorted(rows, r, side="left"))
        e = int(np.searchsorted(rows, r, side="right"))
        if t == s:
            bounds[j] = t
        elif e - s <= T:
            bounds[j] = s if (t - s) <= (e - t) else e
        else:
            bounds[j] = t
    return bounds


def block_of(bounds, p):
    """The block b with bounds[b] <= p < bounds[b+1] (empty blocks hold nothing)."""
    return int(np.searchsorted(bounds, p, side="right") - 1)


def split_rows(sorted_rows, bounds):
    """Rows with a block boundary strictly inside them, as (row, first_blk, last_blk).

    first_blk holds the row's first nonzero, last_blk its last; the partial
    sums of blocks first_blk..last_blk are added in ascending block order.
    """
    rows = np.asarray(sorted_rows)
    nnz = rows.shape[0]
    out = []
    if nnz == 0:
        return np.zeros((0, 3), dtype=np.int64)
    uniq, starts = np.unique(rows, return_index=True)
    ends = np.append(starts[1:], nnz)
    inner = bounds[1:-1]
    for r, s, e in zip(uniq, starts, ends):
        if np.any((inner > s) & (inner < e)):
            out.append((int(r), block_of(bounds, s), block_of(bounds, e - 1)))
    return np.asarray(out, dtype=np.int64).reshape(-1, 3)


def ownership_writes(sorted_rows, bounds, dim):
    """Simulated count of writes per output row under the engine's ownership rule.

    Rule (this engine's reading of Observation 2 plus zero rows): every row
    that holds nonzeros is written by the one block that holds all of it, or,
    if it is split, by the fix-up alone.  Whoever writes row r also writes the
    empty rows strictly between the previous nonempty row and r; whoever
    writes the last nonempty row also writes the empty rows after it.  With no
    nonzeros at all, one zero fill writes every row.
    """
    rows = np.asarray(sorted_rows)
    bounds = np.asarray(bounds)
    cnt = np.zeros(int(dim), dtype=np.int64)
    nnz = rows.shape[0]
    if nnz == 0:
        cnt += 1
        return cnt
    last_row = int(rows[-1])

    def write(r, prev):
        cnt[prev + 1:r] += 1          # empty rows between the previous row and r
        cnt[r] += 1
        if r == last_row:
            cnt[r + 1:] += 1          # empty rows after the last nonempty row

    nblk = bounds.shape[0] - 1
    for b in range(nblk):
        lo, hi = int(bounds[b]), int(bounds[b + 1])
        p = lo
        while p < hi:
            r = int(rows[p])
            q = p
            while q < hi and rows[q] == r:
                q += 1
            starts_before = p > 0 and rows[p - 1] == r
            ends_after = q < nnz and rows[q] == r
            if not (starts_before or ends_after):
                write(r, int(rows[p - 1]) if p > 0 else -1)
            p = q
    for r, fb, lb in split_rows(rows, bounds):
        s = int(np.searchsorted(rows, r, side="left"))
        write(int(r), int(rows[s - 1]) if s > 0 else -1)
    return cnt


# --------------------------------------------------------------------------
# Tensor partitioning scheme (Algorithm 1, Section 3.4)
# --------------------------------------------------------------------------


def lpt_partition(degrees, kappa):
    """Algorithm 1: vertices in descending degree, each to the least-filled block.

    Readings (Algorithm 1 says "least filled", the prose says "cyclic"; the
    worked example of Section 3.4 is only reproduced by the greedy form):
    fill is the number of hyperedges already in the block; equal degrees are
    taken in ascending vertex index; ties between blocks go to the lowest
    block id; the loop runs over the |I_d| vertices (j < |I_d|).
    Returns ``assign`` (block per vertex) and the per-block loads.
    """
    deg = np.asarray(degrees, dtype=np.int64)
    order = sorted(range(deg.shape[0]), key=lambda v: (-int(deg[v]), v))
    load = [0] * int(kappa)
    assign = np.zeros(deg.shape[0], dtype=np.int64)
    for v in order:
        b = min(range(int(kappa)), key=lambda w: (load[w], w))
        assign[v] = b
        load[b] += int(deg[v])
    return assign, np.asarray(load, dtype=np.int64)


def lpt_remap_ids(coo, n, kappa):
    """Remap id b_n of each nonzero: its position after ordering by (block, K_n).

    Section 3.4: hyperedges follow their mode-n vertex into its block; they are
    ordered by block id and numbered.  Inside a block the K_n order is used
    (reading).  Returns the remap id per nonzero (input order).
    """
    coo = np.asarray(coo)
    deg = np.bincount(coo[:, n], minlength=int(coo[:, n].max()) + 1)
    assign, _ = lpt_partition(deg, kappa)
    blk = assign[coo[:, n]]
    N = coo.shape[1]
    keys = [coo[:, (n + 1 + j) % N] for j in range(N)] + [blk]
    order = np.lexsort(keys)
    rid = np.empty(coo.shape[0], dtype=np.int64)
    rid[order] = np.arange(coo.shape[0])
    return rid


def tile_write_order(coo, n, tile):
    """Write order of one mode pass cut into tiles of `tile` consecutive
    positions of the mode-n order: for each tile, its tile-local indices sorted
    by destination in the mode-(n+1) order (next_pos, Section 3.1).  Storing a
    tile's nonzeros in this order visits their destinations in increasing
    order; the remap itself (where each nonzero goes) is unchanged.
    Returns int64 [nnz]: entry base + j is the local index written j-th."""
    npos = next_pos(coo, n)
    out = np.empty_like(npos)
    for base in range(0, npos.shape[0], int(tile)):
        seg = npos[base:base + int(tile)]
        out[base:base + seg.shape[0]] = np.argsort(seg, kind="stable")
    return out


def hot_rows(coo, k, H):
    """The H rows of mode k holding the most nonzeros (ties to the lower row id;
    rows without nonzeros never count).  These factor rows are the ones gathered
    most often in the other modes' passes.  Returns a sorted int64 array."""
    col = np.asarray(coo)[:, k]
    if col.size == 0:
        return np.zeros(0, dtype=np.int64)
    deg = np.bincount(col)
    rows = np.nonzero(deg)[0]
    order = sorted(rows.tolist(), key=lambda r: (-int(deg[r]), r))
    return np.sort(np.asarray(order[:int(H)], dtype=np.int64))


def index_bits(dim):
    """Bits of a mode-k index: ceil(log2 I_k), at least 1 (Section 3.5.1)."""
    b = 1
    while (1 << b) < int(dim):
        b += 1
    return b


def flycoo_pack(coo, vals, dims):
    """Nonzeros (in the given order) packed into 16 bytes each: the N indices as
    bit fields of index_bits(I_k) bits, index k starting at the sum of the widths
    before it, in a 96-bit little-endian field (words 0..2), and the FP32 value
    in word 3.  Section 3.5 stores a nonzero's indices with log2 I_h bits each.
    Returns uint32 [nnz, 4]."""
    coo = np.asarray(coo)
    widths = [index_bits(d) for d in dims]
    if sum(widths) > 96:
        raise ValueError("indices need more than 96 bits")
    out = np.zeros((coo.shape[0], 4), dtype=np.uint32)
    vbits = np.asarray(vals, dtype=np.float32).view(np.uint32)
    for e in range(coo.shape[0]):
        field, off = 0, 0
        for k, b in enumerate(widths):
            field |= int(coo[e, k]) << off
            off += b
        out[e, 0] = field & 0xFFFFFFFF
        out[e, 1] = (field >> 32) & 0xFFFFFFFF
        out[e, 2] = (field >> 64) & 0xFFFFFFFF
        out[e, 3] = vbits[e]
    return out


def flycoo_bits(nnz, dims, value_bits=32):
    """Bits per nonzero of the FLYCOO element (Section 3.5.1).

    N * log2|X| bits of remap ids + sum_h log2 I_h bits of indices + the value.
    """
    N = len(dims)
    return N * np.log2(nnz) + sum(np.log2(d) for d in dims) + value_bits


# --------------------------------------------------------------------------
# CP-ALS (Section 2.1.4; the update is Kolda-Bader's, which the paper cites)
# --------------------------------------------------------------------------


def gram(A):
    A = np.asarray(A, dtype=np.float64)
    return A.T @ A


def als_mode_update(coo, vals, dims, factors, n):
    """One ALS mode update: returns (factors with A_n replaced, lambda, M_n).

    M = mttkrp(n); V = Hadamard over k != n of A_k^T A_k; A_n = M V^-1 via the
    Cholesky factor of V; lambda = column 2-norms; A_n <- A_n / lambda.
    """
    N = len(dims)
    A = [np.asarray(f, dtype=np.float64) for f in factors]
    R = A[0].shape[1]
    M = mttkrp(coo, vals, dims, A, n)
    V = np.ones((R, R))
    for k in range(N):
        if k != n:
            V = V * gram(A[k])
    L = np.linalg.cholesky(V)
    # A_n = M V^-1  <=>  V A_n^T = M^T
    Y = np.linalg.solve(L, M.T)
    An = np.linalg.solve(L.T, Y).T
    lam = np.sqrt((An * An).sum(0))
    A = list(A)
    A[n] = An / lam
    return A, lam, M


def cp_als_iter(coo, vals, dims, factors):
    """One CP-ALS sweep over modes 0..N-1 in FP64.

    Per mode n: M = mttkrp(n); V = Hadamard of the Gram matrices of the other
    factors; A_n = M V^-1 (Cholesky); lambda = column 2-norms of A_n;
    A_n <- A_n / lambda.  Fit after the sweep:
    1 - sqrt(|X|^2 + |Y|^2 - 2<X,Y>) / |X| with |Y|^2 = lambda^T (Hadamard of
    all Grams) lambda and <X,Y> = sum_r lambda_r sum_i M_{N-1}[i,r] A_{N-1}[i,r].
    Readings: 2-norm normalisation every iteration, no regularisation.
    Raises ``np.linalg.LinAlgError`` when V is not positive definite.
    """
    N = len(dims)
    A = [np.asarray(f, dtype=np.float64).copy() for f in factors]
    R = A[0].shape[1]
    lam = np.ones(R)
    M = None
    for n in range(N):
        A, lam, M = als_mode_update(coo, vals, dims, A, n)
    normx2 = float(np.sum(np.asarray(vals, dtype=np.float64) ** 2))
    H = np.ones((R, R))
    for k in range(N):
        H = H * gram(A[k])
    normy2 = float(lam @ H @ lam)
    inner = float(np.sum(lam * np.sum(M * A[N - 1], axis=0)))
    resid2 = max(normx2 + normy2 - 2.0 * inner, 0.0)
    fit = 1.0 - np.sqrt(resid2) / np.sqrt(normx2)
    return A, lam, fit


def cp_full(factors, lam=None):
    """Dense reconstruction sum_r lambda_r a^0_r o ... o a^{N-1}_r (tiny tensors only)."""
    N = len(factors)
    R = np.asarray(factors[0]).shape[1]
    lam = np.ones(R) if lam is None else np.asarray(lam, dtype=np.float64)
    shape = tuple(np.asarray(f).shape[0] for f in factors)
    X = np.zeros(shape)
    for r in range(R):
        t = np.array(lam[r])
        for k in range(N):
            t = np.multiply.outer(t, np.asarray(factors[k], dtype=np.float64)[:, r])
        X += t
    return X


# --------------------------------------------------------------------------
# CP loss on observed entries and its gradient (completion form)
# --------------------------------------------------------------------------


def cp_model_at(coo, factors):
    """m_e = sum_r prod_k A_k[i_k(e), r] for each observed coordinate."""
    coo = np.asarray(coo)
    R = np.asarray(factors[0]).shape[1]
    acc = np.ones((coo.shape[0], R))
    for k in range(coo.shape[1]):
        acc = acc * np.asarray(factors[k], dtype=np.float64)[coo[:, k]]
    return acc.sum(1)


def cp_loss(coo, vals, factors):
    """L = 1/2 sum_{e observed} (m_e - x_e)^2 (sum reduction, no regulariser)."""
    e = cp_model_at(coo, factors) - np.asarray(vals, dtype=np.float64)
    return 0.5 * float(np.sum(e * e)), e


def cp_loss_grad(coo, vals, dims, factors):
    """dL/dA_n = mode-n spMTTKRP of the residual tensor (values m_e - x_e)."""
    _, e = cp_loss(coo, vals, factors)
    return [mttkrp(coo, e, dims, factors, n) for n in range(len(dims))]


def cp_loss_grad_rows(coo, vals, factors, n, rows):
    """Selected rows of dL/dA_n for workloads too large for ``cp_loss_grad``.

    For every requested row i: the observed entries with i_n == i (input
    order), their residuals m_e - x_e, and the mode-n spMTTKRP row of those
    residuals (``mttkrp_rows``)."""
    coo = np.asarray(coo)
    vals = np.asarray(vals, dtype=np.float64)
    R = np.asarray(factors[0]).shape[1]
    out = np.zeros((len(rows), R), dtype=np.float64)
    col = coo[:, n]
    for j, i in enumerate(rows):
        sel = np.nonzero(col == i)[0]
        if sel.size == 0:
            continue
        r = cp_model_at(coo[sel], factors) - vals[sel]
        out[j] = mttkrp_rows(coo[sel], r, factors, n, [i])[0]
    return out


# --------------------------------------------------------------------------
# Small helpers used by tests
# --------------------------------------------------------------------------


def brute_canonical_order(coo, n):
    """Python ``sorted`` on explicit K_n tuples (pin for ``canonical_order``)."""
    coo = [tuple(int(x) for x in row) for row in np.asarray(coo)]
    N = len(coo[0]) if coo else 0
    return np.asarray(sorted(range(len(coo)),
                             key=lambda e: tuple(coo[e][(n - j) % N] for j in range(N))),
                      dtype=np.int64)


def all_partitions_opt(degrees, kappa):
    """Optimal makespan over all assignments of indivisible vertices (brute force)."""
    deg = list(int(d) for d in degrees)
    best = None
    for assign in itertools.product(range(int(kappa)), repeat=len(deg)):
        load = [0] * int(kappa)
        for v, b in enumerate(assign):
            load[b] += deg[v]
        m = max(load)
        best = m if best is None or m < best else best
    return best


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def elements_in_order(coo, vals, n):
    """Expected working copy in mode-n order: (int32 indices [nnz, N], float32 values)."""
    o = canonical_order(coo, n)
    return np.asarray(coo)[o].astype(np.int32), np.asarray(vals, dtype=np.float32)[o]


def bf16_round(a):
    """Round FP32 to the nearest BF16 (ties to even), returned as FP32."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


__all__ = [n for n in dir() if not n.startswith("_")]
