"""The continuous-batching server: admission by HBM budget, results that do
not depend on how requests were batched or interleaved, and an oracle replay
of each map's logged batch partition that reproduces its page ciphertexts."""
import threading

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W
from tests.dict_model import DictModel

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _requests(n_records, count, vb, seed, max_n):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        ops, k, vin = W.op_stream(n_records, max(1, n), vb, seed * 1000 + r, get_frac=0.6,
                                  del_frac=0.1, absent_frac=0.15,
                                  zipf_theta=0.99 if r % 2 else None)
        out.append((ops, k, vin))
    return out


def test_mixed_results_equal_alone_and_oracle_replay():
    vb = 24
    sizes = [1 << 12, 1 << 13, 1 << 15, 1 << 16]
    srv = B.BoltServer(hbm_budget=8 << 30, max_batch=1024)
    maps, data, reqs = [], [], []
    for j, N in enumerate(sizes):
        keys, vals = W.records(N * 3 // 4, vb, 500 + j)
        maps.append(srv.add_map(N, vb, keys, vals, 77 + j))
        data.append((N, keys, vals))
        reqs.append(_requests(N * 3 // 4, 40, vb, 600 + j, 700))
    # submit interleaved from two client threads while batches run
    order = [(j, r) for r in range(40) for j in range(len(sizes))]
    ids = {}
    lock = threading.Lock()

    def client(part):
        for j, r in part:
            ops, k, vin = reqs[j][r]
            rid = srv.submit(maps[j], ops, k, vin)
            with lock:
                ids[(j, r)] = rid
    # one thread per map keeps each map's arrival order
    threads = [threading.Thread(target=client, args=([x for x in order if x[0] == j],))
               for j in range(len(sizes))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = {}
    for (j, r), rid in ids.items():
        rc, vout, st, info = srv.wait(rid, len(reqs[j][r][0]), maps[j], timeout_ms=120000)
        assert rc == 0, rc
        assert info.done_us >= info.start_us >= info.submit_us
        got[(j, r)] = (vout, st)
    for j, (N, keys, vals) in enumerate(data):
        # alone: the same requests through a plain dict, one after another
        model = DictModel(keys, vals)
        for r in range(40):
            ops, k, vin = reqs[j][r]
            ev, es = model.apply(ops, k, vin, vb)
            assert np.array_equal(got[(j, r)][0], ev) and np.array_equal(got[(j, r)][1], es)
        # oracle replay of the logged batch partition reproduces the pages
        sizes_log = srv.batches(maps[j])
        allops = np.concatenate([reqs[j][r][0] for r in range(40)])
        allk = np.concatenate([reqs[j][r][1] for r in range(40)])
        allv = np.concatenate([reqs[j][r][2] for r in range(40)])
        assert sizes_log.sum() == len(allops)
        o = O.OracleMap(N, vb)
        assert o.init(keys, vals, 77 + j) == 0
        lo = 0
        for s in sizes_log:
            rc, _, _ = o.access(allops[lo:lo + s], allk[lo:lo + s], allv[lo:lo + s])
            assert rc == 0
            lo += s
        assert np.array_equal(o.pages(), srv.map_pages(maps[j]))
        o.close()
    st = srv.stats()
    assert st["maps_ready"] == len(sizes) and st["queued"] == 0
    srv.close()


def test_sixteen_maps_full_batches_match_oracle():
    """Sixteen maps of N log-uniform in [2^12, 2^20] (32 B records) behind one
    server with 4096-op batches; requests of log-uniform size 1..4096 (half
    Zipf(0.99)) arrive from four client threads at once, so batches of
    different maps overlap on the device and a map's queued requests share
    batches.  Each request's values and status equal a plain dict applying
    that map's requests alone, in order; the oracle replaying each map's
    logged batch partition reproduces its page ciphertexts, bin loads,
    position-map rows and stash and HBM-store counts."""
    vb, n_maps, n_req, max_batch = 24, 16, 24, 4096
    rng = np.random.default_rng(0x5EED0015)
    sizes = [int(2 ** x) for x in rng.uniform(12, 20, n_maps)]
    srv = B.BoltServer(hbm_budget=64 << 30, max_batch=max_batch)
    maps, data, reqs = [], [], []
    for j, N in enumerate(sizes):
        keys, vals = W.records(N, vb, 900 + j)
        maps.append(srv.add_map(N, vb, keys, vals, 1000 + j))
        data.append((N, keys, vals))
        reqs.append(_requests(N, n_req, vb, 1100 + j, max_batch))
    ids = {}
    lock = threading.Lock()

    def client(part):
        for j in part:
            for r in range(n_req):
                ops, k, vin = reqs[j][r]
                rid = srv.submit(maps[j], ops, k, vin)
                with lock:
                    ids[(j, r)] = rid
    # four threads, four maps each: a map's requests keep their order
    threads = [threading.Thread(target=client, args=(list(range(t, n_maps, 4)),))
               for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = {}
    for (j, r), rid in ids.items():
        rc, vout, st, info = srv.wait(rid, len(reqs[j][r][0]), maps[j], timeout_ms=300000)
        assert rc == 0, rc
        got[(j, r)] = (vout, st)
    shared = 0
    for j, (N, keys, vals) in enumerate(data):
        model = DictModel(keys, vals)
        for r in range(n_req):
            ops, k, vin = reqs[j][r]
            ev, es = model.apply(ops, k, vin, vb)
            assert np.array_equal(got[(j, r)][0], ev) and np.array_equal(got[(j, r)][1], es), \
                f"map {j} request {r}"
        log = srv.batches(maps[j])
        assert log.sum() == sum(len(reqs[j][r][0]) for r in range(n_req))
        assert log.max() <= max_batch
        shared += n_req - len(log)
        allops = np.concatenate([reqs[j][r][0] for r in range(n_req)])
        allk = np.concatenate([reqs[j][r][1] for r in range(n_req)])
        allv = np.concatenate([reqs[j][r][2] for r in range(n_req)])
        o = O.OracleMap(N, vb, trace=False)
        assert o.init(keys, vals, 1000 + j) == 0
        lo = 0
        for s in log:
            rc, _, _ = o.access(allops[lo:lo + s], allk[lo:lo + s], allv[lo:lo + s])
            assert rc == 0
            lo += s
        assert np.array_equal(o.pages(), srv.map_pages(maps[j])), f"pages of map {j}"
        st = srv.map_stats(maps[j])
        so = o.stats()
        for f in ("n_hbm", "n_stash", "max_load", "max_row", "peak_hbm", "peak_stash",
                  "peak_load"):
            assert so[f] == st[f], f"map {j}: {f} oracle {so[f]} server {st[f]}"
        assert np.array_equal(o.loads(), srv.map_loads(maps[j])), f"loads of map {j}"
        o.close()
    assert shared > 0, "no two requests of a map ever shared a batch"
    srv.close()


def test_submit_many_matches_dict_and_rejects_all_or_nothing():
    """Requests of four maps queued by one bolt_server_submit_many call
    (interleaved, in array order per map) give each request the values and
    status of a plain dict applying that map's requests alone, in order.  A
    call with one bad op code queues nothing (BOLT_E_ARG)."""
    vb, n_req = 24, 20
    sizes = [1 << 12, 1 << 14, 1 << 15, 1 << 17]
    srv = B.BoltServer(hbm_budget=32 << 30, max_batch=4096)
    maps, data, reqs = [], [], []
    for j, N in enumerate(sizes):
        keys, vals = W.records(N, vb, 1300 + j)
        maps.append(srv.add_map(N, vb, keys, vals, 1400 + j))
        data.append((keys, vals))
        reqs.append(_requests(N, n_req, vb, 1500 + j, 4096))
    batch = [(maps[j], *reqs[j][r]) for r in range(n_req) for j in range(len(sizes))]
    bad = [list(x) for x in batch[:3]]
    bad[2][1] = bad[2][1].copy()
    bad[2][1][0] = 7
    with pytest.raises(B.BoltError) as e:
        srv.submit_many([tuple(x) for x in bad])
    assert e.value.rc == B.BOLT_E_ARG
    ids = srv.submit_many(batch)
    assert len(set(ids)) == len(batch)
    for j, (keys, vals) in enumerate(data):
        model = DictModel(keys, vals)
        for r in range(n_req):
            ops, k, vin = reqs[j][r]
            rid = ids[r * len(sizes) + j]
            rc, vout, st, info = srv.wait(rid, len(ops), maps[j], timeout_ms=300000)
            assert rc == 0
            ev, es = model.apply(ops, k, vin, vb)
            assert np.array_equal(vout, ev) and np.array_equal(st, es), f"map {j} request {r}"
        # the rejected call queued nothing: the map ran exactly these ops
        assert srv.batches(maps[j]).sum() == sum(len(reqs[j][r][0]) for r in range(n_req))
    srv.close()


def test_admission_by_budget():
    import time
    vb, N = 24, 1 << 16
    keys, vals = W.records(N // 2, vb, 5)
    # a server map's planned resident footprint, as the server accounts it
    probe = B.BoltServer(hbm_budget=1 << 40, max_batch=512)
    pid = probe.add_map(N, vb, keys, vals, 1)
    t0 = time.time()
    while probe.map_state(pid) == 0 and time.time() - t0 < 60:
        time.sleep(0.01)
    fixed = B.BOLT_NOALLOC_SCRATCH_BYTES  # counted once by every server
    res = probe.stats()["used"] - fixed
    probe.close()
    _, build = B.plan_bytes(N, vb, batch_cap=512, n_init=N // 2)
    # room for two maps (plus one build) but not three
    srv = B.BoltServer(hbm_budget=fixed + 2 * res + build + (res // 2), max_batch=512)
    ids = [srv.add_map(N, vb, keys, vals, 10 + j) for j in range(3)]
    ops, k, vin = W.op_stream(N // 2, 100, vb, 6)
    r0 = srv.submit(ids[0], ops, k, vin)
    assert srv.wait(r0, 100, ids[0], timeout_ms=60000)[0] == 0
    t0 = time.time()
    while srv.map_state(ids[1]) == 0 and time.time() - t0 < 60:
        time.sleep(0.01)
    assert srv.map_state(ids[0]) == 1 and srv.map_state(ids[1]) == 1
    time.sleep(0.2)
    assert srv.map_state(ids[2]) == 0  # pending: does not fit
    assert srv.stats()["maps_pending"] == 1
    r2 = srv.submit(ids[2], ops, k, vin)  # queued until admitted
    srv.remove_map(ids[0])
    rc, vout, st, info = srv.wait(r2, 100, ids[2], timeout_ms=60000)
    assert rc == 0 and srv.map_state(ids[2]) == 1 and srv.map_state(ids[0]) == 2
    with pytest.raises(B.BoltError):
        srv.submit(ids[0], ops, k, vin)  # removed
    srv.close()


def test_footprint_estimate_matches_allocation():
    for N, vb in [(1 << 14, 8), (1 << 16, 24)]:
        m = B.BoltMap(N, vb)
        res, _ = m.footprint()
        est, _ = B.plan_bytes(N, vb)
        assert res == est, (N, vb, res, est)
        m.close()
