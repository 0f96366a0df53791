"""The skewed configuration at its full size, against the oracle on full state
(needs a B300): N = 2^24 records of 64 B (8 B key + 56 B value) under a 2 GB
HBM budget (alpha = 0.2), built from device-resident inputs, then 2^20
Zipf(0.99) accesses, 70% GET / 30% PUT, through bolt_access_device_batches
with the trace recorder off -- the launch configuration the benchmark times.
The op stream is cut into four runs of batch widths 1, 64, 4096 and 65536
(the oracle uses the same partition).  Every value and status byte, every
page ciphertext, the bin loads, the position-map rows and the live HBM-store
and stash counts must equal the oracle's, after the width-1 run and at the
end."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")

N, VB, BUDGET = 1 << 24, 56, 2 * 10**9
N_OPS = 1 << 20
SEED_DATA, SEED_OPS, SEED_MAP = 0x5EED0002, 0x5EED0102, 0x5EED0202
# (first op, end op, batch width): 4096 single-op batches (Alg. 1 one command
# at a time), then 1024 batches of 64, 64 of 4096, and 65536-op batches with a
# ragged last one
RUNS = [(0, 4096, 1), (4096, 69632, 64), (69632, 331776, 4096), (331776, N_OPS, 65536)]


def _state_equal(o, g, what):
    assert np.array_equal(o.loads(), g.loads()), f"bin loads differ {what}"
    assert np.array_equal(o.rowcounts().astype(np.uint8), g.rowcounts()), f"pm rows differ {what}"
    so, sg = o.stats(), g.stats()
    for f in ("n_hbm", "n_stash", "max_load", "max_row", "peak_hbm", "peak_stash", "peak_load"):
        assert so[f] == sg[f], f"{f} differs {what}: oracle {so[f]}, gpu {sg[f]}"
    M = o.info()["M"]
    op = o.pages()
    step = 1 << 18  # compare the 1.6 GB page store in slices
    for lo in range(0, M, step):
        cnt = min(step, M - lo)
        assert np.array_equal(op[lo:lo + cnt], g.pages(lo, cnt)), \
            f"page ciphertexts differ in pages [{lo}, {lo + cnt}) {what}"
    assert sg["trace_len"] == 0


def test_skewed_config_full_size_matches_oracle():
    import torch
    o = O.OracleMap(N, VB, hbm_budget=BUDGET, trace=False)
    g = B.BoltMap(N, VB, hbm_budget=BUDGET)
    info = g.info()
    assert o.info() == info and info["alpha"] == 0.2
    keys, vals = W.records(N, VB, SEED_DATA)
    assert o.init(keys, vals, SEED_MAP) == 0
    d_keys = torch.from_numpy(keys.view(np.int64)).cuda()
    d_vals = torch.from_numpy(vals).cuda()
    assert g.init_device(d_keys, d_vals, SEED_MAP) == 0
    del d_keys, d_vals
    ops, k, vin = W.op_stream(N, N_OPS, VB, SEED_OPS, get_frac=0.7, zipf_theta=0.99)
    t_ops = torch.from_numpy(ops).cuda()
    t_k = torch.from_numpy(k.view(np.int64)).cuda()
    t_vin = torch.from_numpy(vin).cuda()
    t_out = torch.zeros((N_OPS, VB), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(N_OPS, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    vo = np.zeros((N_OPS, VB), np.uint8)
    so = np.zeros(N_OPS, np.uint8)
    for lo, hi, w in RUNS:
        s = slice(lo, hi)
        assert g.access_device_batches(t_ops[s], t_k[s], t_vin[s], t_out[s], t_st[s], w,
                                       stream=stream) == 0
        o.set_param(O.PARAM_BATCH, w)
        rc, vo[s], so[s] = o.access(ops[s], k[s], vin[s])
        assert rc == 0
        if w == 1:
            assert g.sync() == 0
            _state_equal(o, g, "after the width-1 run")
    assert g.sync() == 0
    assert np.array_equal(so, t_st.cpu().numpy()), "status differs"
    assert np.array_equal(vo, t_out.cpu().numpy()), "values differ"
    _state_equal(o, g, "at the end")
    assert g.stats()["batches"] == sum((hi - lo + w - 1) // w for lo, hi, w in RUNS)
    o.close()
    g.close()
