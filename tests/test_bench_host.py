"""Host-side logic of bench.py that needs no GPU: the committed DRAM traffic is
reported only for the configuration it was captured on, and the algorithmic byte
count follows its definition (elements read, remap ids, remapped write, each
touched factor row once, output once)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def captured():
    d = json.load(open(os.path.join(ROOT, "profiles", "mttkrp_remap_traffic.json")))
    return d, d["entries"]["c2_R32_f32"]


def test_traffic_only_for_the_captured_configuration():
    """Committed traffic is scaled per nonzero from the small capture, and only for
    the captured kernel sources and launch configuration."""
    d, e = captured()
    cfg = dict(e["config"])
    nnz = 100_000_000
    if d["kernel_digest"] != bench.kernel_digest():
        assert bench.ncu_traffic("c2", 32, "f32", nnz, cfg) is None
        return
    per = e["dram_bytes_per_nonzero_per_launch"]
    assert bench.ncu_traffic("c2", 32, "f32", nnz, cfg) == per * nnz
    assert bench.ncu_traffic("c2", 32, "f32", nnz // 5, cfg) == per * (nnz // 5)
    for k in cfg:
        other = dict(cfg, **{k: cfg[k] + 1})
        assert bench.ncu_traffic("c2", 32, "f32", nnz, other) is None, k
    # each factor type reads its own entry; a rank without an entry has none
    eb = d["entries"].get("c2_R32_bf16")
    want_bf16 = None if eb is None else eb["dram_bytes_per_nonzero_per_launch"] * nnz
    assert bench.ncu_traffic("c2", 32, "bf16", nnz, cfg) == want_bf16
    assert bench.ncu_traffic("c2", 64, "f32", nnz, cfg) is None


def test_compulsory_bytes_by_hand():
    # 3 modes, 10 nonzeros, R = 2, FP32: E = 16 bytes per nonzero unpadded
    dims, nnz, R, s, N = (4, 3, 5), 10, 2, 4, 3
    touched = [4, 2, 5]
    got = bench.compulsory_bytes(dims, nnz, R, s, touched, N)
    want = []
    for n in range(N):
        stream = nnz * (16 + 4 + 16)
        rows = sum(touched[k] for k in range(N) if k != n) * R * s
        want.append(stream + rows + dims[n] * R * 4)
    assert list(got) == want
    # the resident mode-0 copy: the last pass reads no remap ids and writes no copy
    kb = bench.compulsory_bytes(dims, nnz, R, s, touched, N, keep_base=True)
    assert list(kb[:-1]) == want[:-1]
    assert kb[-1] == want[-1] - nnz * (4 + 16)
