"""The multi-threaded C FP64 oracle (timing) against the pinned NumPy oracle and the dense
definition.

Built without floating-point contraction and summing each output entry in input order,
it must equal ``oracle.mttkrp`` bit for bit, on one thread and on all; on tiny tensors it
must also match the dense unfolding times the explicit Khatri-Rao product.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import ref_c


@pytest.mark.parametrize("dims,nnz,R,skew", [((7, 5, 4), 60, 3, (0.0, 0.0, 0.0)),
                                             ((6, 5), 20, 4, (0.0, 0.0)),
                                             ((4, 3, 3, 2), 40, 2, (0.0,) * 4)])
def test_c_oracle_matches_dense_definition(dims, nnz, R, skew):
    coo, vals = synth.make_coo(dims, nnz, skew, seed=nnz)
    c, v = coo.numpy(), vals.numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    F = [rng.standard_normal((d, R)) for d in dims]
    X = O.dense_from_coo(c, v, dims)
    for n in range(len(dims)):
        got = ref_c.mttkrp(c, v, dims, F, n)
        want = O.mttkrp_dense(X, F, n)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12), n


@pytest.mark.parametrize("dims,nnz,R,skew", [((200, 150, 100), 20_000, 16, (1.1, 1.1, 0.0)),
                                             ((40, 30, 20, 10), 6_000, 8, (1.2, 0.0, 1.1, 0.0)),
                                             ((12, 9, 7, 5, 4), 3_000, 5, (1.1,) * 5),
                                             ((500, 20), 3_000, 33, (1.3, 0.0))])
def test_c_oracle_equals_numpy_oracle_bitwise(dims, nnz, R, skew):
    coo, vals = synth.make_coo(dims, nnz, skew, seed=R)
    c, v = coo.numpy(), vals.numpy()
    F = [f.numpy().astype(np.float64) for f in synth.make_factors(dims, R, seed=4)]
    for n in range(len(dims)):
        want = O.mttkrp(c, v, dims, F, n)
        for t in (1, 0):
            got = ref_c.mttkrp(c, v, dims, F, n, nthreads=t)
            assert np.array_equal(got, want), (n, t)


def test_c_oracle_empty_and_errors():
    dims = (5, 4, 3)
    F = [np.ones((d, 2)) for d in dims]
    out = ref_c.mttkrp(np.zeros((0, 3), np.int64), np.zeros(0), dims, F, 1)
    assert out.shape == (4, 2) and np.all(out == 0.0)
    with pytest.raises(ValueError):
        ref_c.mttkrp(np.zeros((1, 3), np.int64), np.ones(1), dims, F, 3)
    assert ref_c.threads() >= 1
