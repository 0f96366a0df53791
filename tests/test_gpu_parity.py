"""CUDA path vs the CPU oracle, element by element (needs a B300).

Every comparison is exact: the map's outputs are bytes and integers, so the
bar is bit-exact equality of values, status flags, page ciphertexts, page
versions, bin loads, position-map row counts and the host-access trace.
Inputs are seeded and synthetic (paper_2509_01742_b300.workload).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W
from tests.dict_model import DictModel

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _pair(N, vb, batch=None, alpha=None, c=None, budget=2**64 - 1, trace=True):
    """An oracle map and a GPU map of the same sizing.  trace=False leaves the
    GPU map's trace recorder off, as the benchmark and the server run it (the
    batch's kernel chain is then shorter); the oracle records nothing either."""
    o = O.OracleMap(N, vb, hbm_budget=budget, alpha=alpha, c=c, batch=batch, trace=trace)
    g = B.BoltMap(N, vb, hbm_budget=budget, alpha=alpha, c=c, trace=trace, batch=batch)
    assert o.info() == g.info()
    return o, g


def _assert_state_equal(o, g, what="", trace=True):
    """Full map state: page ciphertexts (every record's page, value and
    version), bin loads, position-map row counts, live HBM-store and stash
    items, and (trace on) the host-access trace."""
    assert np.array_equal(o.pages(), g.pages()), f"page ciphertexts differ {what}"
    assert np.array_equal(o.loads(), g.loads()), f"bin loads differ {what}"
    assert np.array_equal(o.rowcounts().astype(np.uint8), g.rowcounts()), f"pm rows differ {what}"
    so, sg = o.stats(), g.stats()
    for f in ("n_hbm", "n_stash", "max_load", "max_row", "peak_hbm", "peak_stash", "peak_load"):
        assert so[f] == sg[f], f"{f} differs {what}: oracle {so[f]}, gpu {sg[f]}"
    if trace:
        assert np.array_equal(o.trace(), g.trace()), f"host trace differs {what}"
    else:
        assert g.stats()["trace_len"] == 0, f"trace recorded with the recorder off {what}"


def _run_batch(o, g, ops, keys, vin, what=""):
    rc_o, vo, so = o.access(ops, keys, vin)
    rc_g, vg, sg = g.access(ops, keys, vin)
    assert rc_o == rc_g == 0, (rc_o, rc_g)
    assert np.array_equal(so, sg), f"status differs {what}"
    assert np.array_equal(vo, vg), f"values differ {what}"
    return vg, sg


@pytest.mark.parametrize("N,prf", [(1 << 16, 0), (1 << 16, 1), (1 << 16, 2), (1 << 20, 1)])
def test_build_parity_small_config(N, prf):
    """Records of 16 B (8 B key + 8 B value): the build's pages, loads and
    position-map rows equal the oracle's, with the records' PRF computed
    where the build picks (prf = 0), inside the persistent P2C rounds (1;
    on these maps the automatic choice is a pass) or in a pass before them
    (2), and with every access afterwards too."""
    o, g = _pair(N, 8)
    g.set_param(B.BOLT_PARAM_ROUNDS_PRF, prf)
    keys, vals = W.records(N, 8, 0x5EED0001)
    assert o.init(keys, vals, 42) == 0
    assert g.init(keys, vals, 42) == 0
    _assert_state_equal(o, g, "after build")
    ops, k, vin = W.op_stream(N, 2048, 8, 0x5EED0002, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.1)
    _run_batch(o, g, ops, k, vin, "after the build")
    _assert_state_equal(o, g, "after a batch")
    o.close(); g.close()


def test_access_parity_small_config():
    """N=2^16, then 4096 accesses (50% GET / 50% PUT, 10% absent keys,
    uniform) in one batch, then more batches with deletes and duplicates."""
    N = 1 << 16
    o, g = _pair(N, 8)
    keys, vals = W.records(N, 8, 0x5EED0001)
    assert o.init(keys, vals, 42) == 0 and g.init(keys, vals, 42) == 0
    model = DictModel(keys, vals)
    ops, k, vin = W.op_stream(N, 4096, 8, 0x5EED0101, get_frac=0.5, absent_frac=0.1)
    vg, sg = _run_batch(o, g, ops, k, vin, "batch 0")
    ev, es = model.apply(ops, k, vin, 8)
    assert np.array_equal(vg, ev) and np.array_equal(sg, es)
    _assert_state_equal(o, g, "after batch 0")
    for rep in range(3):
        ops, k, vin = W.op_stream(N, 3000, 8, 0x5EED0200 + rep, get_frac=0.4, del_frac=0.2,
                                  absent_frac=0.2)
        k[::7] = k[1]  # a hot key repeated inside the batch
        vg, sg = _run_batch(o, g, ops, k, vin, f"batch {rep + 1}")
        ev, es = model.apply(ops, k, vin, 8)
        assert np.array_equal(vg, ev) and np.array_equal(sg, es)
        _assert_state_equal(o, g, f"after batch {rep + 1}")
    o.close(); g.close()


@pytest.mark.parametrize("batch,fused", [(1, 1), (7, 1), (32, 1), (1, 0), (7, 0), (333, 1)])
def test_access_parity_batch_widths(batch, fused):
    """Small batches (one op per batch is Alg. 1) on a 2^12 map, 24 B values,
    through bolt_access.  Batches of at most 32 ops run as one fused launch
    (fused = 1) or through the multi-kernel chain (fused = 0)."""
    N = 1 << 12
    o, g = _pair(N, 24, batch=batch)
    g.set_param(B.BOLT_PARAM_FUSED, fused)
    keys, vals = W.records(3500, 24, 7)
    assert o.init(keys, vals, 9) == 0 and g.init(keys, vals, 9) == 0
    _assert_state_equal(o, g, "after build")
    for rep in range(2):
        ops, k, vin = W.op_stream(3500, 700, 24, 40 + rep, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.2)
        _run_batch(o, g, ops, k, vin, f"rep {rep}")
        _assert_state_equal(o, g, f"rep {rep}")
    o.close(); g.close()


@pytest.mark.parametrize("N,batch", [(1 << 12, 2), (1 << 14, 8), (1 << 16, 32)])
def test_one_round_fused_batches_match_oracle(N, batch):
    """Fused batches that fit one P2C round (batch <= W_r): the launch decides
    on bin, row and reverse-index counts read while its pages are in flight,
    less what find_remove takes out, and places beside the eviction.  Keys
    from a small pool (duplicates, deletes and re-inserts inside a batch)
    and absent keys (new rows) on maps small enough that a removal's bin or
    a deleted key's row often meets another op's choices."""
    o, g = _pair(N, 8, batch=batch)
    assert g.info()["round_width"] >= batch
    g.set_param(B.BOLT_PARAM_FUSED, 1)
    keys, vals = W.records(N * 3 // 4, 8, 0x0E0D)
    assert o.init(keys, vals, 17) == 0 and g.init(keys, vals, 17) == 0
    for rep, (pool, dfrac, afrac) in enumerate([(64, 0.2, 0.2), (N * 3 // 4, 0.1, 0.3),
                                                (16, 0.3, 0.1)]):
        ops, k, vin = W.op_stream(pool, 1500, 8, 0x0E10 + rep, get_frac=0.3, del_frac=dfrac,
                                  absent_frac=afrac)
        _run_batch(o, g, ops, k, vin, f"rep {rep}")
        _assert_state_equal(o, g, f"rep {rep}")
    o.close(); g.close()


@pytest.mark.parametrize("trace", [True, False])
def test_fused_and_chain_batches_interleaved_match_oracle(trace):
    """Calls whose batches run as single fused launches (widths 1, 5, 32)
    between calls that run the multi-kernel chain (widths 33, 300), through
    bolt_access_device_batches and bolt_access_device without a host sync in
    between: a fused batch right after a chain batch whose host write-back is
    still in flight, and a chain batch right after fused ones.  Keys repeat
    (1500 keys on a 2^12 map), deletes, misses.  Everything equals the oracle
    with the same batch partition."""
    import torch
    N, vb = 1 << 12, 16
    o, g = _pair(N, vb, trace=trace)
    keys, vals = W.records(1500, vb, 81)
    assert o.init(keys, vals, 4) == 0 and g.init(keys, vals, 4) == 0
    plan = [(64, 1), (300, 300), (40, 5), (330, 33), (96, 32), (1, 1), (600, 300), (7, 1)]
    total = sum(n for n, _ in plan)
    ops, k, vin = W.op_stream(1500, total, vb, 82, get_frac=0.4, del_frac=0.15,
                              absent_frac=0.2)
    t_ops = torch.from_numpy(ops).cuda()
    t_k = torch.from_numpy(k.view(np.int64)).cuda()
    t_vin = torch.from_numpy(vin).cuda()
    t_out = torch.zeros((total, vb), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(total, dtype=torch.uint8, device="cuda")
    lo = 0
    vo_all, so_all = [], []
    for n, w in plan:
        s = slice(lo, lo + n)
        if n == w:
            assert g.access_device(t_ops[s], t_k[s], t_vin[s], t_out[s], t_st[s]) == 0
        else:
            assert g.access_device_batches(t_ops[s], t_k[s], t_vin[s], t_out[s], t_st[s], w) == 0
        for b in range(lo, lo + n, w):
            e = min(lo + n, b + w)
            rc, vo, so = o.access(ops[b:e], k[b:e], vin[b:e])
            assert rc == 0
            vo_all.append(vo)
            so_all.append(so)
        lo += n
    assert g.sync() == 0
    assert np.array_equal(np.concatenate(so_all), t_st.cpu().numpy())
    assert np.array_equal(np.concatenate(vo_all), t_out.cpu().numpy())
    _assert_state_equal(o, g, "fused and chain batches", trace=trace)
    o.close(); g.close()


@pytest.mark.parametrize("key_bytes,trace", [(8, True), (8, False), (4, False)])
def test_small_host_calls_match_oracle(key_bytes, trace):
    """bolt_access calls of 1..32 operations, each one batch: a single fused
    launch reads the call's inputs from the pinned staging and writes its
    results back there (no copies).  Interleaved with calls of 33..200 ops in
    batches of 64 (the chain, copies through the staging).  Values, status
    and state equal the oracle's with the same batch partition."""
    N, vb = 1 << 13, 24
    o = O.OracleMap(N, vb, batch=64, trace=trace)
    g = B.BoltMap(N, vb, trace=trace, batch=64, key_bytes=key_bytes)
    rng = np.random.default_rng(101)
    if key_bytes == 4:
        keys = rng.choice(2**32, size=6001, replace=False).astype(np.uint64)
    else:
        keys = W.key_of(np.arange(6001, dtype=np.uint64))
    _, vals = W.records(6000, vb, 102)
    assert o.init(keys[:6000], vals, 7) == 0
    assert g.init(keys[:6000].astype(np.uint32) if key_bytes == 4 else keys[:6000], vals, 7) == 0
    for call in range(300):
        n = int(rng.integers(1, 33)) if call % 10 else int(rng.integers(33, 201))
        idx = rng.integers(0, 6001, n)  # index 6000 is an absent key
        ops = rng.integers(0, 3, n).astype(np.uint8)
        vin = rng.integers(0, 256, (n, vb), dtype=np.uint8)
        k = keys[idx]
        rc_o, vo, so = o.access(ops, k, vin)
        rc_g, vg, sg = g.access(ops, k.astype(np.uint32) if key_bytes == 4 else k, vin)
        assert rc_o == rc_g == 0
        assert np.array_equal(so, sg) and np.array_equal(vo, vg), f"call {call}"
    _assert_state_equal(o, g, "small host calls", trace=trace)
    o.close(); g.close()


@pytest.mark.parametrize("batch", [1, 4096])
def test_extreme_keys_match_oracle(batch):
    """Keys at the ends of the key space -- 0, 1, 2^63, 2^64 - 2 and 2^64 - 1
    (the value the page build's and the eviction's warp sort give an empty
    lane) -- among random keys: the build places them, Gets return their
    values, Puts and Deletes change them, in single-op fused launches and in a
    4096-op chain batch; pages and state equal the oracle's."""
    N, vb = 1 << 12, 8
    o, g = _pair(N, vb, batch=batch)
    keys, vals = W.records(3000, vb, 91)
    special = np.array([0, 1, 1 << 63, (1 << 64) - 2, (1 << 64) - 1], dtype=np.uint64)
    keys[[5, 700, 1400, 2100, 2999]] = special
    assert o.init(keys, vals, 6) == 0 and g.init(keys, vals, 6) == 0
    _assert_state_equal(o, g, "after build")
    model = DictModel(keys, vals)
    rng = np.random.default_rng(92)
    for rep in range(3):
        idx = rng.integers(0, 3000, 200)
        kk = keys[idx]
        kk[::4] = special[rng.integers(0, 5, len(kk[::4]))]
        ops = rng.integers(0, 3, len(kk)).astype(np.uint8)
        vin = rng.integers(0, 256, (len(kk), vb), dtype=np.uint8)
        vg, sg = _run_batch(o, g, ops, kk, vin, f"rep {rep}")
        ev, es = model.apply(ops, kk, vin, vb)
        assert np.array_equal(vg, ev) and np.array_equal(sg, es)
        _assert_state_equal(o, g, f"rep {rep}")
    o.close(); g.close()


def test_access_parity_multi_tile_batch_zipf():
    """A 20000-op batch (multi-tile grouping sort) with Zipf(0.99) keys, 56 B
    values, 70% GET / 30% PUT -- the skewed configuration's shape."""
    N = 1 << 15
    o, g = _pair(N, 56)
    keys, vals = W.records(N, 56, 11)
    assert o.init(keys, vals, 3) == 0 and g.init(keys, vals, 3) == 0
    ops, k, vin = W.op_stream(N, 20000, 56, 12, get_frac=0.7, zipf_theta=0.99)
    assert len(np.unique(k)) < 15000  # heavy duplication
    _run_batch(o, g, ops, k, vin, "zipf")
    _assert_state_equal(o, g, "zipf")
    o.close(); g.close()


def test_access_parity_max_batch_zipf():
    """One full 65536-op batch (Zipf 0.99, 70/30) on a 2^20 map."""
    N = 1 << 20
    o, g = _pair(N, 56)
    keys, vals = W.records(N, 56, 14)
    assert o.init(keys, vals, 3) == 0 and g.init(keys, vals, 3) == 0
    ops, k, vin = W.op_stream(N, 65536, 56, 13, get_frac=0.7, zipf_theta=0.99)
    _run_batch(o, g, ops, k, vin, "zipf 65536")
    _assert_state_equal(o, g, "zipf 65536")
    o.close(); g.close()


def test_batch_wider_than_map():
    """A 65536-op batch on a 2^15 map (the batch remaps a quarter of all keys
    at once; the value store's batch headroom absorbs it)."""
    N = 1 << 15
    o, g = _pair(N, 56)
    keys, vals = W.records(N, 56, 11)
    assert o.init(keys, vals, 3) == 0 and g.init(keys, vals, 3) == 0
    ops, k, vin = W.op_stream(N, 65536, 56, 13, get_frac=0.7, zipf_theta=0.99)
    _run_batch(o, g, ops, k, vin, "65536 on 2^15")
    _assert_state_equal(o, g, "65536 on 2^15")
    o.close(); g.close()


def test_alpha_zero_and_large_alpha():
    """Edge settings: no HBM bins (alpha = 0) and alpha = 0.5."""
    for alpha in (0.0, 0.5):
        N = 1 << 12
        o, g = _pair(N, 8, alpha=alpha)
        keys, vals = W.records(N, 8, 5)
        assert o.init(keys, vals, 1) == 0 and g.init(keys, vals, 1) == 0
        _assert_state_equal(o, g, f"alpha {alpha} build")
        ops, k, vin = W.op_stream(N, 2048, 8, 6, del_frac=0.1, absent_frac=0.1)
        _run_batch(o, g, ops, k, vin, f"alpha {alpha}")
        _assert_state_equal(o, g, f"alpha {alpha}")
        o.close(); g.close()


def test_empty_and_partial_init():
    """n = 0 records (every page a dummy page) and n < N."""
    N = 1 << 12
    for n in (0, 1000):
        o, g = _pair(N, 8)
        keys, vals = W.records(n, 8, 2)
        assert o.init(keys, vals, 5) == 0 and g.init(keys, vals, 5) == 0
        _assert_state_equal(o, g, f"n={n}")
        ops, k, vin = W.op_stream(max(n, 1), 500, 8, 3, get_frac=0.3, absent_frac=0.5)
        _run_batch(o, g, ops, k, vin, f"n={n}")
        _assert_state_equal(o, g, f"n={n} access")
        o.close(); g.close()


@pytest.mark.parametrize("case", ["far_apart", "salt_key", "distinct_with_salt_key"])
def test_duplicate_keys_detected_at_scale(case):
    """The build's key-uniqueness check (a hashed table on the side stream)
    on 2^17 keys: a duplicate pair far apart, the key that the table encodes
    as its empty value given twice, and that key given once among distinct
    keys (no false alarm)."""
    N = 1 << 17
    keys, vals = W.records(N, 8, 71)
    salt = np.uint64(0x9E3779B97F4A7C15)
    if case == "far_apart":
        keys[N - 1] = keys[3]
    elif case == "salt_key":
        keys[10] = salt
        keys[N - 5] = salt
    else:
        keys[10] = salt
    g = B.BoltMap(N, 8)
    rc = g.init(keys, vals, 3)
    assert rc == (0 if case == "distinct_with_salt_key" else B.BOLT_E_DUPKEY)
    g.close()


def test_overflow_and_dupkey_match_oracle():
    o, g = _pair(64, 8)
    k = np.array([5, 6, 5], dtype=np.uint64)
    v = np.zeros((3, 8), np.uint8)
    assert o.init(k, v, 1) == O.E_DUPKEY and g.init(k, v, 1) == B.BOLT_E_DUPKEY
    keys, vals = W.records(60, 8, 1)
    assert o.init(keys, vals, 1) == 0 and g.init(keys, vals, 1) == 0
    newk = W.key_of(np.arange(1000, 1400))
    for lo in range(0, 400, 50):
        ops = np.ones(50, np.uint8)
        vin = np.ones((50, 8), np.uint8)
        rc_o, _, _ = o.access(ops, newk[lo:lo + 50], vin)
        rc_g, _, _ = g.access(ops, newk[lo:lo + 50], vin)
        assert rc_o == rc_g
        if rc_o:
            break
    assert rc_g == B.BOLT_E_OVERFLOW
    rc, _, _ = g.access(np.zeros(1, np.uint8), keys[:1], np.zeros((1, 8), np.uint8))
    assert rc == B.BOLT_E_STATE
    assert g.init(keys, vals, 2) == 0
    o.close(); g.close()


def test_build_barrier_wait_gives_up_and_map_recovers():
    """The build's P2C rounds run in one cooperative kernel whose blocks meet at
    a software grid barrier between the decide and apply phases of each round;
    every wait there is bounded.  With the bound set to zero iterations a
    block that finds the barrier still closed gives up at once (N = 2^22: 8
    blocks, 4096 barriers): bolt_init returns BOLT_E_TIMEOUT, the map refuses
    accesses (BOLT_E_STATE) but the CUDA context is unharmed, and with the
    bound restored the next bolt_init builds the map the oracle builds."""
    N, vb = 1 << 22, 8
    o, g = _pair(N, vb, trace=False)
    keys, vals = W.records(N, vb, 33)
    g.set_param(B.BOLT_PARAM_SPIN_LIMIT, 0)
    assert g.init(keys, vals, 3) == B.BOLT_E_TIMEOUT
    rc, _, _ = g.access(np.zeros(1, np.uint8), keys[:1], np.zeros((1, vb), np.uint8))
    assert rc == B.BOLT_E_STATE
    g.set_param(B.BOLT_PARAM_SPIN_LIMIT, 1 << 22)
    assert o.init(keys, vals, 3) == 0 and g.init(keys, vals, 3) == 0
    _assert_state_equal(o, g, "after the re-init", trace=False)
    ops, k, vin = W.op_stream(N, 4096, vb, 34, del_frac=0.1, absent_frac=0.1)
    _run_batch(o, g, ops, k, vin, "after the re-init")
    _assert_state_equal(o, g, "after a batch", trace=False)
    o.close(); g.close()


def test_device_pointer_path_matches_host_path():
    """bolt_init_device / bolt_access_device on torch tensors give the same
    outputs and pages as the host-pointer calls."""
    import torch
    N = 1 << 14
    keys, vals = W.records(N, 24, 21)
    ops, k, vin = W.op_stream(N, 4096, 24, 22, del_frac=0.1, absent_frac=0.1)
    h = B.BoltMap(N, 24)
    assert h.init(keys, vals, 77) == 0
    rc, vh, sh = h.access(ops, k, vin)
    assert rc == 0
    d = B.BoltMap(N, 24)
    tk = torch.from_numpy(keys.view(np.int64)).cuda()
    tv = torch.from_numpy(vals).cuda()
    assert d.init_device(tk, tv, 77) == 0
    t_ops = torch.from_numpy(ops).cuda()
    t_k = torch.from_numpy(k.view(np.int64)).cuda()
    t_vin = torch.from_numpy(vin).cuda()
    t_out = torch.zeros((4096, 24), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert d.access_device(t_ops, t_k, t_vin, t_out, t_st) == 0
    assert d.sync() == 0
    assert np.array_equal(t_out.cpu().numpy(), vh)
    assert np.array_equal(t_st.cpu().numpy(), sh)
    assert np.array_equal(h.pages(), d.pages())
    h.close(); d.close()


@pytest.mark.parametrize("trace", [True, False])
def test_device_batches_back_to_back_match_oracle(trace):
    """Twenty device-path batches enqueued without a host sync in between on
    a 2^12 map: consecutive batches often touch the same pages while the
    previous batch's write-back is still in flight.  Outputs, pages, loads
    and (recorder on) the trace equal the oracle's with the same batch
    partition; with the recorder off the kernel chain is the benchmark's."""
    import torch
    N, vb, bw = 1 << 12, 8, 300
    o, g = _pair(N, vb, trace=trace)
    keys, vals = W.records(3000, vb, 31)
    assert o.init(keys, vals, 8) == 0 and g.init(keys, vals, 8) == 0
    ops, k, vin = W.op_stream(3000, 20 * bw, vb, 32, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.2)
    t_ops = torch.from_numpy(ops).cuda()
    t_k = torch.from_numpy(k.view(np.int64)).cuda()
    t_vin = torch.from_numpy(vin).cuda()
    t_out = torch.zeros((len(ops), vb), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(len(ops), dtype=torch.uint8, device="cuda")
    for lo in range(0, len(ops), bw):
        sl = slice(lo, lo + bw)
        assert g.access_device(t_ops[sl], t_k[sl], t_vin[sl], t_out[sl], t_st[sl]) == 0
    assert g.sync() == 0
    vo_all, so_all = [], []
    for lo in range(0, len(ops), bw):
        rc, vo, so = o.access(ops[lo:lo + bw], k[lo:lo + bw], vin[lo:lo + bw])
        assert rc == 0
        vo_all.append(vo)
        so_all.append(so)
    assert np.array_equal(np.concatenate(vo_all), t_out.cpu().numpy())
    assert np.array_equal(np.concatenate(so_all), t_st.cpu().numpy())
    _assert_state_equal(o, g, "back-to-back device batches", trace=trace)
    o.close(); g.close()


@pytest.mark.parametrize("lookahead,defer,trace", [
    (0, 0, True), (0, 1, True), (0, 2, True), (0.3, 1, True), (1, 1, True),
    # the benchmark's configuration (recorder off, no lookahead, no deferral)
    # and the other pipelines with the shorter chain
    (0, 0, False), (0, 1, False), (0.3, 1, False)])
def test_device_batches_call_matches_oracle(lookahead, defer, trace):
    """bolt_access_device_batches (the next batch's preparation, and with
    lookahead its position-map search and page reads, run ahead on an
    internal stream; without lookahead each batch's host write-back either
    follows its eviction or waits for the next batch's page reads) over 21
    batches of width 300 with a ragged tail of 123,
    then one plain device batch, then batches of width 1000 on a caller
    stream: outputs and state equal the oracle's with the same batch
    partition.  Keys repeat across consecutive batches (3000 keys), so
    predicted bins, re-checked hits and pages rewritten by the previous batch
    are all exercised."""
    import torch
    N, vb = 1 << 12, 8
    o, g = _pair(N, vb, trace=trace)
    g.set_param(B.BOLT_PARAM_LOOKAHEAD, lookahead)
    g.set_param(B.BOLT_PARAM_DEFER_FLUSH, defer)
    keys, vals = W.records(3000, vb, 41)
    assert o.init(keys, vals, 9) == 0 and g.init(keys, vals, 9) == 0
    n1, n2, n3 = 20 * 300 + 123, 257, 3500
    ops, k, vin = W.op_stream(3000, n1 + n2 + n3, vb, 42, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.2)
    t_ops = torch.from_numpy(ops).cuda()
    t_k = torch.from_numpy(k.view(np.int64)).cuda()
    t_vin = torch.from_numpy(vin).cuda()
    t_out = torch.zeros((len(ops), vb), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(len(ops), dtype=torch.uint8, device="cuda")
    a, b, c = slice(0, n1), slice(n1, n1 + n2), slice(n1 + n2, n1 + n2 + n3)
    assert g.access_device_batches(t_ops[a], t_k[a], t_vin[a], t_out[a], t_st[a], 300) == 0
    assert g.access_device(t_ops[b], t_k[b], t_vin[b], t_out[b], t_st[b]) == 0
    side = torch.cuda.Stream()
    assert g.access_device_batches(t_ops[c], t_k[c], t_vin[c], t_out[c], t_st[c], 1000,
                                   stream=side) == 0
    assert g.sync() == 0
    parts = [(lo, min(n1, lo + 300)) for lo in range(0, n1, 300)] + [(n1, n1 + n2)]
    parts += [(lo, min(n1 + n2 + n3, lo + 1000)) for lo in range(n1 + n2, n1 + n2 + n3, 1000)]
    vo_all, so_all = [], []
    for lo, hi in parts:
        rc, vo, so = o.access(ops[lo:hi], k[lo:hi], vin[lo:hi])
        assert rc == 0
        vo_all.append(vo)
        so_all.append(so)
    assert np.array_equal(np.concatenate(so_all), t_st.cpu().numpy())
    assert np.array_equal(np.concatenate(vo_all), t_out.cpu().numpy())
    _assert_state_equal(o, g, "pipelined device batches", trace=trace)
    assert g.stats()["batches"] == len(parts)
    o.close(); g.close()


@pytest.mark.parametrize("pinned,cap,bw,with_status,trace", [
    (False, 1000, 300, True, True),   # pageable: every chunk packed through staging
    (True, 1000, 300, True, True),    # pinned but small chunks: packed as well
    (True, 4000, 1300, True, True),   # pinned 3900-op chunk copied directly, ragged 1100 packed
    (True, 4000, 1300, False, True),  # the same without a status array
    (False, 4000, 1300, True, True),  # pageable large chunks
    (False, 1000, 300, True, False),  # recorder off (the end-to-end benchmark's calls)
    (True, 4000, 1300, True, False),
])
def test_host_call_over_many_chunks_matches_oracle(pinned, cap, bw, with_status, trace):
    """bolt_access over 5000 ops with a batch capacity below the call:
    chunks of whole batches alternate between two device I/O sets, each
    chunk a pipelined run of batches.  Pageable or small chunks cross the
    link packed (one copy per direction through pinned staging), large
    pinned ones are copied directly from and to the caller's arrays.
    Outputs and state equal the oracle's with the same batch width."""
    import ctypes
    import torch
    N, vb = 1 << 14, 16
    o = O.OracleMap(N, vb, batch=bw, trace=trace)
    g = B.BoltMap(N, vb, trace=trace)
    g.set_param(B.BOLT_PARAM_BATCH_CAP, cap)
    g.set_param(B.BOLT_PARAM_BATCH, bw)
    keys, vals = W.records(12000, vb, 51)
    assert o.init(keys, vals, 5) == 0 and g.init(keys, vals, 5) == 0
    ops, k, vin = W.op_stream(12000, 5000, vb, 52, get_frac=0.5, del_frac=0.1, absent_frac=0.1)
    rc_o, vo, so = o.access(ops, k, vin)
    assert rc_o == 0
    if pinned:
        t = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
             for a in (ops, k.view(np.int64), vin)]
        out = torch.zeros((len(ops), vb), dtype=torch.uint8).pin_memory()
        st = torch.zeros(len(ops), dtype=torch.uint8).pin_memory()
        ptrs = [ctypes.c_void_p(x.data_ptr()) for x in (*t, out)]
        ptrs.append(ctypes.c_void_p(st.data_ptr() if with_status else 0))
        rc = B.bolt_access(g.handle, *ptrs, len(ops))
        vg, sg = out.numpy(), st.numpy()
    else:
        rc, vg, sg = g.access(ops, k, vin)
    assert rc == 0
    if with_status:
        assert np.array_equal(so, sg)
    else:
        assert not sg.any()
    assert np.array_equal(vo, vg)
    _assert_state_equal(o, g, "chunked host call", trace=trace)
    assert g.stats()["batches"] == (5000 + bw - 1) // bw
    o.close(); g.close()


def test_four_byte_keys_match_the_oracle_on_widened_keys():
    """A map created with 4-byte keys takes uint32 keys at its host-pointer
    calls and holds them zero-extended: build, a single-chunk call and a
    chunked call (batch capacity 1000, width 300) give the same values,
    status, pages, loads, rows and trace as the oracle on the same keys as
    uint64."""
    N, vb = 1 << 14, 8
    o = O.OracleMap(N, vb, batch=300)
    g = B.BoltMap(N, vb, trace=True, key_bytes=4)
    assert g.info()["key_bytes"] == 4
    rng = np.random.default_rng(71)
    k32 = rng.choice(2**32, size=13000, replace=False).astype(np.uint32)
    keys32 = k32[:12000]
    _, vals = W.records(12000, vb, 72)
    assert o.init(keys32.astype(np.uint64), vals, 73) == 0
    assert g.init(keys32, vals, 73) == 0
    _assert_state_equal(o, g, "after init")
    g.set_param(B.BOLT_PARAM_BATCH, 300)
    for n, cap in [(300, None), (5000, 1000)]:
        if cap:
            g.set_param(B.BOLT_PARAM_BATCH_CAP, cap)
            g.set_param(B.BOLT_PARAM_BATCH, 300)
            g.set_param(B.BOLT_PARAM_TRACE, 1)
            assert g.init(keys32, vals, 73) == 0
            o.close()
            o = O.OracleMap(N, vb, batch=300)
            assert o.init(keys32.astype(np.uint64), vals, 73) == 0
        idx = rng.integers(0, 13000, n)  # indices >= 12000 are absent keys
        ops = rng.integers(0, 3, n).astype(np.uint8)
        vin = rng.integers(0, 256, (n, vb), dtype=np.uint8)
        rc_o, vo, so = o.access(ops, k32[idx].astype(np.uint64), vin)
        rc_g, vg, sg = g.access(ops, k32[idx], vin)
        assert rc_o == rc_g == 0
        assert np.array_equal(so, sg) and np.array_equal(vo, vg)
        _assert_state_equal(o, g, f"after {n} ops")
    with pytest.raises(ValueError):
        g.access(ops[:1], np.array([1 << 40], dtype=np.uint64), vin[:1])
    o.close(); g.close()


def test_autotune_keeps_results():
    """bolt_autotune picks a tile and a batch width by measurement; the map's
    contents are unchanged (its tuning Gets only remap keys) and later builds
    with the picked tile still match the oracle."""
    N, vb = 1 << 16, 8
    keys, vals = W.records(N, vb, 41)
    g = B.BoltMap(N, vb)
    assert g.init(keys, vals, 5) == 0
    t = g.autotune(sample_keys=keys[:20000], max_batch_us=0)
    assert t["sort_log_tile"] in (12, 13) and t["batch_width"] in (64, 256, 1024, 4096, 16384, 65536)
    assert all(x > 0 for x in t["sort_ms"])
    model = DictModel(keys, vals)
    ops, k, vin = W.op_stream(N, 5000, vb, 42, del_frac=0.1, absent_frac=0.1)
    rc, vout, st = g.access(ops, k, vin)
    ev, es = model.apply(ops, k, vin, vb)
    assert rc == 0 and np.array_equal(vout, ev) and np.array_equal(st, es)
    o = O.OracleMap(N, vb)
    assert o.init(keys, vals, 6) == 0 and g.init(keys, vals, 6) == 0  # tuned tile
    assert np.array_equal(o.pages(), g.pages())
    o.close(); g.close()


def test_large_config_scaled_replica():
    """The 2^30-record, 64 B, 16 GB-budget configuration (alpha = 0.1 under
    that budget) on a scaled replica the oracle can run: N = 2^22, alpha 0.1,
    Zipf(0.99) keys, 90% GET / 10% PUT, batches of 4096."""
    N, vb = 1 << 22, 56
    o, g = _pair(N, vb, alpha=0.1)
    keys, vals = W.records(N, vb, 0x5EED0004)
    assert o.init(keys, vals, 99) == 0 and g.init(keys, vals, 99) == 0
    assert np.array_equal(o.pages(), g.pages())
    for rep in range(4):
        ops, k, vin = W.op_stream(N, 4096, vb, 0x5EED0104 + rep, get_frac=0.9,
                                  zipf_theta=0.99)
        _run_batch(o, g, ops, k, vin, f"replica batch {rep}")
    _assert_state_equal(o, g, "scaled replica")
    o.close(); g.close()


def test_link_probe_leaves_pages_unchanged():
    """bolt_probe_link reads random pages of the map's own store and writes
    earlier-read pages back: rates are positive and every page ciphertext is
    unchanged, so the map still matches the oracle afterwards."""
    N, vb = 1 << 14, 8
    o, g = _pair(N, vb)
    keys, vals = W.records(N, vb, 61)
    assert o.init(keys, vals, 3) == 0 and g.init(keys, vals, 3) == 0
    before = g.pages().copy()
    r = g.probe_link(512, launches=5)
    assert r["read_pages_per_s"] > 0 and r["pipelined_pages_per_s"] > 0
    assert np.array_equal(before, g.pages())
    ops, k, vin = W.op_stream(N, 2048, vb, 62, get_frac=0.5)
    _run_batch(o, g, ops, k, vin, "after the probe")
    _assert_state_equal(o, g, "after the probe")
    o.close(); g.close()


@pytest.mark.parametrize("vb", [248, 504])
@pytest.mark.parametrize("batch,sealed", [(None, False), (16, False), (None, True), (16, True)])
def test_largest_values_match_oracle(vb, batch, sealed):
    """Values up to the ABI's limit (504 B; pages of several 512-byte chunks,
    ~3.3 and ~6.7 KB here) through the multi-kernel chain (batches of 700)
    and the fused single-CTA launch (batches of 16, fewer eviction warps fit
    its shared memory), plain and sealed: values, status, page bytes, loads,
    rows and trace equal the oracle's."""
    N = 1 << 12
    o = O.OracleMap(N, vb, batch=batch, integrity=sealed)
    g = B.BoltMap(N, vb, trace=True, batch=batch, integrity=sealed)
    assert o.info() == g.info()
    assert g.info()["page_bytes"] > 3000
    keys, vals = W.records(3000, vb, 0x1AD0 + vb)
    assert o.init(keys, vals, 12) == 0 and g.init(keys, vals, 12) == 0
    _assert_state_equal(o, g, "after build")
    for rep in range(2):
        ops, k, vin = W.op_stream(3000, 700, vb, 0x1AD8 + rep, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.2)
        _run_batch(o, g, ops, k, vin, f"rep {rep}")
        _assert_state_equal(o, g, f"after rep {rep}")
    o.close(); g.close()


def test_fused_batches_after_kernels_that_write_their_inputs():
    """Each call's inputs are written by torch kernels on the same stream
    right before it (keys XOR-ed into place, values and ops copied from
    device scratch), then run as batches of one op (fused launches chained by
    programmatic dependent launch, from the second batch on reading their
    inputs before their wait).  Repeated over many calls; results and state
    equal the oracle's."""
    import torch
    N, vb = 1 << 12, 16
    o, g = _pair(N, vb, trace=False)
    keys, vals = W.records(2000, vb, 91)
    assert o.init(keys, vals, 5) == 0 and g.init(keys, vals, 5) == 0
    stream = torch.cuda.Stream()
    mask = np.uint64(0x9E3779B97F4A7C15)
    n, calls = 24, 12
    t_out = torch.zeros((n, vb), dtype=torch.uint8, device="cuda")
    t_st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    for c in range(calls):
        ops, k, vin = W.op_stream(2000, n, vb, 920 + c, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.2)
        # the keys reach the device masked; a kernel on the call's stream
        # unmasks them in place just before the call
        src_k = torch.from_numpy((k ^ mask).view(np.int64)).cuda()
        src_v = torch.from_numpy(vin).cuda()
        src_o = torch.from_numpy(ops).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            t_k = torch.bitwise_xor(src_k, torch.tensor(np.int64(mask.view(np.int64)),
                                                        device="cuda"))
            t_vin = src_v.clone()
            t_ops = src_o.clone()
        assert g.access_device_batches(t_ops, t_k, t_vin, t_out, t_st, 1, stream=stream) == 0
        stream.synchronize()
        for b in range(n):
            rc, vo, so = o.access(ops[b:b + 1], k[b:b + 1], vin[b:b + 1])
            assert rc == 0
            assert np.array_equal(vo[0], t_out[b].cpu().numpy()), f"call {c} op {b}"
            assert so[0] == t_st[b].item(), f"call {c} op {b}"
    assert g.sync() == 0
    _assert_state_equal(o, g, "after the calls", trace=False)
    o.close(); g.close()
