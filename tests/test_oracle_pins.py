"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test ties the oracle to something other than itself: an independent
ChaCha20 implementation, the numbers the paper prints (slack table, HBM-usage
example, validation-experiment maxima), a plain dict, brute-force recounts of
the data-structure invariants, and exact predictions of the host trace from
the PRF definition.  None of them needs a GPU.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W
from tests.dict_model import DictModel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DOM_INIT, DOM_PM, DOM_REMAP, DOM_DUMMY = 1, 2, 3, 4


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def decode_page(plain, info):
    """Page format: u64 bitmap, u64 zero, lmax slots of (u64 key, value)."""
    vb, rec = info["val_bytes"], info["rec_bytes"]
    bitmap = int(np.frombuffer(plain[:8].tobytes(), dtype=np.uint64)[0])
    header2 = int(np.frombuffer(plain[8:16].tobytes(), dtype=np.uint64)[0])
    cnt = 0
    while cnt < 64 and (bitmap >> cnt) & 1:
        cnt += 1
    assert bitmap == (1 << cnt) - 1, "occupied slots must be a prefix"
    assert header2 == 0
    assert cnt <= info["lmax"]
    keys, vals = [], []
    for s in range(cnt):
        off = 16 + s * rec
        keys.append(int(np.frombuffer(plain[off:off + 8].tobytes(), dtype=np.uint64)[0]))
        vals.append(plain[off + 8:off + 8 + vb].tobytes())
    assert keys == sorted(keys), "reals are stored in ascending key order"
    assert not plain[16 + cnt * rec:].any(), "dummy slots and padding are zero"
    return keys, vals


def check_invariants(m: O.OracleMap, model: DictModel):
    """Every live key is in exactly one place with its current value; loads
    equal recounted occupancies (Sec. 3.1 bins; Sec. 4.2 storage)."""
    info, st = m.info(), m.stats()
    loads = m.loads().astype(np.int64)
    K, M = info["K"], info["M"]
    page_keys = {}
    host_total = 0
    stash_by_page = 0
    for q in range(M):
        keys, vals = decode_page(m.decrypt_page(q), info)
        host_total += len(keys)
        assert loads[K + q] >= len(keys)
        stash_by_page += loads[K + q] - len(keys)
        for k, v in zip(keys, vals):
            assert k not in page_keys
            page_keys[k] = v
            assert model.d[k] == v
    assert host_total == st["n_host"]
    assert stash_by_page == st["n_stash"]
    assert loads[:K].sum() == st["n_hbm"]
    assert loads.sum() == len(model.d)
    assert st["n_hbm"] + st["n_stash"] + st["n_host"] == len(model.d)
    assert loads.max() <= info["lmax"]


# --------------------------------------------------------------------------
# ChaCha20 against an independent implementation


def test_chacha20_matches_cryptography():
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    rng = np.random.default_rng(1)
    for _ in range(20):
        key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
        nonce = rng.integers(0, 256, 12, dtype=np.uint8).tobytes()
        counter = int(rng.integers(0, 2**31))
        length = int(rng.integers(1, 300))
        enc = Cipher(algorithms.ChaCha20(key, counter.to_bytes(4, "little") + nonce),
                     mode=None).encryptor()
        expect = enc.update(bytes(length))
        got = O.chacha20_xor(np.frombuffer(key, dtype=np.uint32), counter,
                             np.frombuffer(nonce, dtype=np.uint32), bytes(length))
        assert got == expect


def test_chacha20_block_is_keystream():
    key = np.arange(8, dtype=np.uint32) * 0x01010101
    nonce = np.array([9, 0x4a, 0], dtype=np.uint32)
    blk = O.chacha20_block(key, 1, nonce)
    ks = O.chacha20_xor(key, 1, nonce, bytes(64))
    assert np.frombuffer(ks, dtype=np.uint32).tolist() == blk.tolist()


# --------------------------------------------------------------------------
# Sizing against the paper's printed numbers


def test_lmax_pins_slack_table():
    # Fig. 5 table: bin-load slack 2 at rel .143 (c=8) and .091 (c=16) => the
    # analytical bin-load bounds at N=2^20 are 14 and 22.
    for row in _golden("slack_table.txt"):
        if row[0] != "binload":
            continue
        c, abs_slack, rel = int(row[1]), int(row[3]), float(row[4])
        lmax = O.sizing(1 << 20, c, float(row[2]), 8)["lmax"]
        assert round(abs_slack / lmax, 3) == rel


def test_bound_pins_slack_table():
    # Claim 3.3 (HBM sum) and Claim 3.4 (stash) bounds at N=2^20 reproduce the
    # printed relative slacks slack/bound.
    for row in _golden("slack_table.txt"):
        metric, c, alpha, abs_slack, rel = row[0], int(row[1]), float(row[2]), \
            int(row[3]), float(row[4])
        if metric == "binload":
            continue
        s = O.sizing(1 << 20, c, alpha, 8)
        bound = s["beta1"] if metric == "hbm" else s["beta2"]
        digits = len(row[4].split(".")[1])
        tol = 0.5 * 10 ** -digits + 1e-9 if metric == "hbm" else 0.0075
        assert abs(abs_slack / bound - rel) <= tol, (row, bound, abs_slack / bound)


def test_hbm_usage_example_claim_5_2():
    # Claim 5.2 applied to the paper's example: 1e9 records, 32-bit keys, c=8,
    # position map of N/16 rows with d=4, no HBM store (alpha = 0).
    N = 10**9
    for row in _golden("hbm_usage.txt"):
        vbytes, percent = int(row[0]), float(row[1])
        s = O.sizing(N, 8, 0.0, 8)
        vs_bits = vbytes * 8
        ks = 32
        rows = N / 16
        pm_bits = (2 * math.log2(N) + ks) * (N + rows * math.log2(math.log2(N)) / math.log2(4))
        total_bits = (s["beta1"] + s["beta2"]) * vs_bits + pm_bits
        raw_bits = N * (ks + vs_bits)
        assert abs(100.0 * total_bits / raw_bits - percent) <= 1.0, (vbytes, total_bits / raw_bits)


def test_alpha_policy_and_derived_sizes():
    # config sizes (N, val_bytes, budget) -> alpha on the grid {.2,.1,.05,.01,0}
    m = O.OracleMap(1 << 16, 8)
    i = m.info()
    assert (i["B"], i["K"], i["M"], i["lmax"], i["R"], i["page_bytes"]) == \
        (8192, 1638, 6554, 13, 18, 256)
    assert i["alpha"] == 0.2 and i["round_width"] == 32
    m.close()
    s = O.sizing(1 << 28, 8, 0.2, 24)
    assert (s["lmax"], s["R"], s["page_bytes"], s["B"]) == (14, 19, 512, 1 << 25)
    # a budget that only fits alpha = 0.01
    need = {a: O.sizing(1 << 16, 8, a, 8)["vs_cap"] * 16 for a in (0.2, 0.1, 0.05, 0.01)}
    m = O.OracleMap(1 << 16, 8, hbm_budget=need[0.01])
    assert m.info()["alpha"] == 0.01
    m.close()
    with pytest.raises(O.OracleError):
        O.OracleMap(1 << 16, 8, hbm_budget=1000)


# --------------------------------------------------------------------------
# The paper's validation experiment (Sec. 3.3 "Dimensions in practice")


@pytest.mark.parametrize("alpha", [0.01, 0.2])
def test_dimensional_validation(alpha):
    """N=2^20, c=8, one operation per batch (Alg. 1), uniform random accesses:
    peak bin load, HBM load and stash land on the paper's empirical maxima
    (analytical bound minus printed slack), measured here over 10^6 accesses
    instead of 10^9."""
    N = 1 << 20
    m = O.OracleMap(N, 8, alpha=alpha, nocrypt=True, trace=False, batch=1)
    keys, vals = W.records(N, 8, 1)
    assert m.init(keys, vals, 7) == 0
    info = m.info()
    stash = []
    for rep in range(4):
        ops, k, vin = W.op_stream(N, 250000, 8, 100 + rep)
        rc, _, _ = m.access(ops, k, vin)
        assert rc == 0
        stash.append(m.stats()["n_stash"])
    st = m.stats()
    table = {(r[0], float(r[2])): int(r[3]) for r in _golden("slack_table.txt") if r[1] == "8"}
    emp_hbm = info["beta1"] - table[("hbm", alpha)]
    emp_stash = info["beta2"] - table[("stash", alpha)]
    emp_load = info["lmax"] - table[("binload", alpha)]
    assert st["peak_load"] == emp_load
    assert abs(st["peak_hbm"] / emp_hbm - 1) < 0.03, (st, emp_hbm)
    assert -0.03 < st["peak_stash"] / emp_stash - 1 < 0.01, (st, emp_stash)
    if alpha == 0.01:
        # drift equilibrium x* = (1+alpha) M / 2 (proof of Claim 3.4)
        xstar = (1 + alpha) * info["M"] / 2
        assert abs(np.mean(stash[1:]) / xstar - 1) < 0.02
    m.close()


# --------------------------------------------------------------------------
# Results against the plain dictionary, invariants by brute force


@pytest.mark.parametrize("batch", [1, 7, 4096])
def test_results_match_dict(batch):
    N = 1 << 12
    n0 = 3000
    keys, vals = W.records(n0, 8, 3)
    m = O.OracleMap(N, 8, batch=batch)
    assert m.init(keys, vals, 11) == 0
    model = DictModel(keys, vals)
    for rep in range(3):
        ops, k, vin = W.op_stream(n0, 2000, 8, 50 + rep, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.15)
        # heavy duplicates inside a batch
        k[::5] = k[0]
        rc, vout, status = m.access(ops, k, vin)
        assert rc == 0
        evout, estatus = model.apply(ops, k, vin, 8)
        assert np.array_equal(status, estatus)
        assert np.array_equal(vout, evout)
        check_invariants(m, model)
    m.close()


def test_brute_force_tiny_every_op():
    N = 64
    keys, vals = W.records(40, 16, 5)
    m = O.OracleMap(N, 16, batch=1, alpha=0.25)
    assert m.init(keys, vals, 3) == 0
    model = DictModel(keys, vals)
    check_invariants(m, model)
    rng = np.random.default_rng(9)
    for step in range(300):
        ops, k, vin = W.op_stream(40, 1, 16, 1000 + step, get_frac=0.4, del_frac=0.2,
                                  absent_frac=0.3)
        rc, vout, status = m.access(ops, k, vin)
        if rc == O.E_OVERFLOW:  # tiny maps may legitimately overflow
            break
        assert rc == 0
        evout, estatus = model.apply(ops, k, vin, 16)
        assert np.array_equal(vout, evout) and np.array_equal(status, estatus)
        check_invariants(m, model)
    assert step > 50
    m.close()


def test_init_layout_brute_force():
    """After init every record sits in the bin P2C gives it (round-synchronous
    rounds of W_r records on round-start loads, first choice on ties)."""
    N = 1 << 12
    keys, vals = W.records(N, 8, 21)
    m = O.OracleMap(N, 8)
    assert m.init(keys, vals, 5) == 0
    info = m.info()
    kprf, _ = m.keys()
    B, K, Wr = info["B"], info["K"], info["round_width"]
    load = np.zeros(B, dtype=np.int64)
    dest = np.zeros(N, dtype=np.int64)
    for lo in range(0, N, Wr):
        idx = range(lo, min(N, lo + Wr))
        pairs = [O.pair(kprf, DOM_INIT, i, B) for i in idx]
        d = [a if load[a] <= load[b] else b for a, b in pairs]
        for i, b in zip(idx, d):
            dest[i] = b
        for b in d:
            load[b] += 1
    assert np.array_equal(load, m.loads().astype(np.int64))
    for q in range(info["M"]):
        pk, pv = decode_page(m.decrypt_page(q), info)
        expect = sorted(int(keys[i]) for i in np.nonzero(dest == K + q)[0])
        assert pk == expect
    m.close()


# --------------------------------------------------------------------------
# Host-access trace (obliviousness invariants)


def _host_bins(pairs, K):
    out = []
    for a, b in pairs:
        for p in (a, b):
            if p >= K:
                out.append(p - K)
    return out


def _expected_trace(reads):
    seen, writes = set(), []
    for q in reads:
        if q not in seen:
            seen.add(q)
            writes.append(q | 0x80000000)
    return np.array(reads + writes, dtype=np.uint32)


def test_trace_predicted_from_prf():
    """First batch after init: leaders of distinct existing keys read the
    bins of their init pair, misses and duplicates the DUMMY pair of their
    global sequence number; each distinct page is then written once in
    first-read order (Alg. 1 lines 5-10, simulator of Sec. 3.2)."""
    N = 1 << 12
    keys, vals = W.records(N, 8, 4)
    m = O.OracleMap(N, 8)
    assert m.init(keys, vals, 77) == 0
    info = m.info()
    kprf, _ = m.keys()
    B, K = info["B"], info["K"]
    rng = np.random.default_rng(0)
    idx = rng.choice(N, 300, replace=False)
    k = keys[idx].copy()
    k[10:20] = W.key_of(np.arange(N + 5, N + 15))  # absent
    k[30] = k[29]  # duplicate
    ops = np.zeros(300, dtype=np.uint8)
    vin = np.zeros((300, 8), dtype=np.uint8)
    m.trace()
    rc, _, _ = m.access(ops, k, vin)
    assert rc == 0
    pairs = []
    for i in range(300):
        if 10 <= i < 20 or i == 30:
            pairs.append(O.pair(kprf, DOM_DUMMY, i, B))
        else:
            pairs.append(O.pair(kprf, DOM_INIT, int(idx[i]), B))
    assert np.array_equal(m.trace(), _expected_trace(_host_bins(pairs, K)))
    # second batch: the same keys were remapped with REMAP pairs at t = their index
    rc, _, _ = m.access(ops[:5], k[:5], vin[:5])
    pairs2 = [O.pair(kprf, DOM_REMAP, i, B) for i in range(5)]
    assert np.array_equal(m.trace(), _expected_trace(_host_bins(pairs2, K)))
    m.close()


def test_trace_independent_of_ops_and_payloads():
    """O4: at a fixed state, opcodes and payloads leave no trace footprint."""
    N = 1 << 12
    keys, vals = W.records(N, 8, 4)
    traces = []
    for variant in range(3):
        m = O.OracleMap(N, 8)
        assert m.init(keys, vals, 5) == 0
        ops, k, vin = W.op_stream(N, 1000, 8, 8, absent_frac=0.2)
        if variant == 1:
            ops = (ops + 1) % 3
        if variant == 2:
            vin = 255 - vin
        m.trace()
        rc, _, _ = m.access(ops, k, vin)
        assert rc == 0
        traces.append(m.trace())
        m.close()
    assert np.array_equal(traces[0], traces[1]) and np.array_equal(traces[0], traces[2])


def test_pair_uniformity_chi2():
    """The pair map is uniform over ordered pairs of distinct bins (Sec. 3.2)."""
    from scipy.stats import chisquare
    kprf = np.arange(8, dtype=np.uint32) + 17
    B = 7
    counts = np.zeros((B, B), dtype=np.int64)
    for x in range(42 * 400):
        a, b = O.pair(kprf, DOM_REMAP, x, B)
        assert a != b and a < B and b < B
        counts[a, b] += 1
    obs = counts[~np.eye(B, dtype=bool)]
    assert chisquare(obs).pvalue > 1e-3


def test_repeated_key_trace_uniform():
    """O3: hammering one key gives a stream of fresh uniform pairs; with
    alpha = 0 every bin is a host page so the trace shows whole pairs."""
    from scipy.stats import chisquare
    m = O.OracleMap(64, 8, alpha=0.0, batch=1)
    keys, vals = W.records(40, 8, 2)
    assert m.init(keys, vals, 1) == 0
    B = m.info()["B"]
    n = 56 * 150
    ops = np.zeros(n, dtype=np.uint8)
    k = np.full(n, keys[3], dtype=np.uint64)
    rc, _, _ = m.access(ops, k, np.zeros((n, 8), dtype=np.uint8))
    assert rc == 0
    tr = m.trace()
    reads = tr[(tr >> 31) == 0].reshape(-1, 2)
    assert len(reads) == n
    counts = np.zeros((B, B), dtype=np.int64)
    for a, b in reads:
        counts[a, b] += 1
    assert chisquare(counts[~np.eye(B, dtype=bool)]).pvalue > 1e-3
    m.close()


# --------------------------------------------------------------------------
# Error paths


def test_dupkey_and_overflow_poison():
    m = O.OracleMap(64, 8)
    k = np.array([5, 6, 5], dtype=np.uint64)
    assert m.init(k, np.zeros((3, 8), np.uint8), 1) == O.E_DUPKEY
    keys, vals = W.records(60, 8, 1)
    assert m.init(keys, vals, 1) == 0
    # insert far more keys than the capacity: some bin or row must overflow
    newk = W.key_of(np.arange(1000, 1400))
    rc = 0
    for lo in range(0, 400, 50):
        rc, _, _ = m.access(np.ones(50, np.uint8), newk[lo:lo + 50], np.ones((50, 8), np.uint8))
        if rc:
            break
    assert rc == O.E_OVERFLOW
    rc2, _, _ = m.access(np.zeros(1, np.uint8), keys[:1], np.zeros((1, 8), np.uint8))
    assert rc2 == O.E_STATE
    assert m.init(keys, vals, 2) == 0  # re-init clears the poison
    m.close()


def test_standalone_kdf_and_page_codec_match_a_built_map():
    """oracle.kdf / oracle.page_decrypt (used to check sampled pages of maps
    too large for the oracle to build) agree with an oracle map's own keys and
    page decryption."""
    N, vb, seed = 1 << 10, 8, 0x1234567
    keys, vals = W.records(N, vb, 3)
    o = O.OracleMap(N, vb)
    assert o.init(keys, vals, seed) == 0
    kprf, kenc = O.kdf(seed)
    k2 = o.keys()
    assert np.array_equal(kprf, k2[0]) and np.array_equal(kenc, k2[1])
    pages = o.pages()
    for q in (0, 1, o.info()["M"] - 1):
        assert np.array_equal(O.page_decrypt(kenc, q, 0, pages[q]), o.decrypt_page(q))
    o.close()


def _chacha_ref(key_words, nonce_words, length, counter=0):
    """Keystream of the `cryptography` package's ChaCha20 (RFC 7539 block
    layout: 32-bit little-endian counter followed by a 96-bit nonce)."""
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    key = np.asarray(key_words, dtype="<u4").tobytes()
    nonce = np.asarray(nonce_words, dtype="<u4").tobytes()
    enc = Cipher(algorithms.ChaCha20(key, counter.to_bytes(4, "little") + nonce),
                 mode=None).encryptor()
    return np.frombuffer(enc.update(bytes(length)), dtype=np.uint8)


def test_keys_and_page_cipher_match_cryptography():
    """The working keys and every page ciphertext, rebuilt with a third-party
    ChaCha20 from their definitions: K_prf || K_enc is the first key-stream
    block under the 64-bit seed (little-endian, zero-extended to 256 bits)
    and the nonce "BOLT"; page q at version v is its plaintext XOR the key
    stream under K_enc and the nonce (q, v) from block 0 (Sec. 4.1 step 3
    encryption; Sec. 4.2 page contents).  The plaintext decoded this way
    holds exactly the init records that P2C put in the page, and after one
    batch every page it wrote decrypts under its bumped version."""
    N, vb, seed = 1 << 11, 8, 0x0123456789ABCDEF
    keys, vals = W.records(N, vb, 8)
    m = O.OracleMap(N, vb)
    assert m.init(keys, vals, seed) == 0
    info = m.info()
    kprf, kenc = m.keys()
    blk = _chacha_ref([seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0],
                      [int.from_bytes(b"BOLT", "little"), 0, 0], 64).view("<u4")
    assert np.array_equal(kprf, blk[:8]) and np.array_equal(kenc, blk[8:])

    M, P = info["M"], info["page_bytes"]
    val_of = {int(k): vals[i].tobytes() for i, k in enumerate(keys)}

    def decrypt(q, v):
        ks = _chacha_ref(kenc, [q, v & 0xFFFFFFFF, v >> 32], P)
        return m.pages()[q] ^ ks

    seen = 0
    for q in range(M):
        pk, pv = decode_page(decrypt(q, 0), info)
        assert [val_of[k] for k in pk] == pv
        seen += len(pk)
    assert seen == m.stats()["n_host"]

    rng = np.random.default_rng(3)
    idx = rng.choice(N, 64, replace=False)
    ops = np.full(64, 1, dtype=np.uint8)  # PUT
    vin = rng.integers(0, 256, (64, vb), dtype=np.uint8)
    m.trace()
    assert m.access(ops, keys[idx], vin)[0] == 0
    written = [int(e) & 0x7FFFFFFF for e in m.trace() if int(e) & 0x80000000]
    ver = m.versions()
    assert written and all(ver[q] == 1 for q in written)
    assert sum(int(v) for v in ver) == len(written)
    for q in written:
        decode_page(decrypt(q, 1), info)
    m.close()


def test_init_position_map_rows_brute_force():
    """Position-map placement at init (Sec. 4.2, d = 4 choices): a key's
    candidate rows are four 64-bit words of PRF(K_prf, PM, key), each scaled
    to [0, rows) by its high product, recomputed here with a third-party
    ChaCha20; every key goes to its least-occupied candidate on the counts
    at the start of its P2C round (W_r records, Sec. 3.3), the first of equal
    candidates on ties.  The recount equals the oracle's row occupancies and
    no row exceeds R."""
    N = 1 << 16
    keys, vals = W.records(N, 8, 13)
    m = O.OracleMap(N, 8)
    assert m.init(keys, vals, 99) == 0
    info = m.info()
    kprf, _ = m.keys()
    rows, Wr = info["rows"], info["round_width"]
    assert Wr > 1
    cand = np.empty((N, 4), dtype=np.int64)
    for i, k in enumerate(keys):
        k = int(k)
        w = _chacha_ref(kprf, [DOM_PM, k & 0xFFFFFFFF, k >> 32], 64).view("<u4")
        for j in range(4):
            r = int(w[2 * j]) | (int(w[2 * j + 1]) << 32)
            cand[i, j] = (r * rows) >> 64
    cnt = np.zeros(rows, dtype=np.int64)
    for lo in range(0, N, Wr):
        c = cand[lo:lo + Wr]
        pick = c[np.arange(len(c)), np.argmin(cnt[c], axis=1)]  # argmin: first of ties
        np.add.at(cnt, pick, 1)
    assert np.array_equal(cnt, m.rowcounts().astype(np.int64))
    assert cnt.max() <= info["R"]
    m.close()


def test_pair_from_independent_prf():
    """The bin pair of (domain, x): PRF block under K_prf with the nonce
    (domain, x); the first bin scales its first 64-bit word to [0, B), the
    second scales the next word to [0, B - 1) and skips the first (Sec. 3.2,
    two distinct uniformly random bins), recomputed with a third-party
    ChaCha20 for all four domains, B = 2 and large B."""
    rng = np.random.default_rng(17)
    kprf, _ = O.kdf(0xC0FFEE)
    for B in (2, 3, 8192, (1 << 25) + 7):
        for dom in (DOM_INIT, DOM_PM, DOM_REMAP, DOM_DUMMY):
            for x in [0, 1, (1 << 64) - 1] + [int(v) for v in rng.integers(0, 2**63, 5)]:
                w = _chacha_ref(kprf, [dom, x & 0xFFFFFFFF, x >> 32], 64).view("<u4")
                r0 = int(w[0]) | (int(w[1]) << 32)
                r1 = int(w[2]) | (int(w[3]) << 32)
                first = (r0 * B) >> 64
                second = (r1 * (B - 1)) >> 64
                second += second >= first
                assert O.pair(kprf, dom, x, B) == (first, second)
                assert first != second and 0 <= first < B and 0 <= second < B


@pytest.mark.parametrize("N", [1 << 12, 1 << 16])
def test_per_access_block_counts(N):
    """The fixed block set of one access (Sec. 4.3 overhead claim: constant
    rounds and O(1) + O(log2 log2 N) bandwidth per access; Alg. 1):
    with one operation per batch every access reads at most two host pages
    (the host bins of its pair, in pair order) and writes back exactly the
    distinct pages it read; every page is page_bytes long with
    lmax = c + ceil(log2 log2 N) + 1 slots, and a key's position-map search
    covers d = 4 rows of R = 16 + ceil(log2 log2 N / log2 d) slots -- the O(1)
    + O(log log N) bound.  Over 3000 accesses of a Zipf-skewed mix with
    deletes and misses the mean number of page reads per access is 2(1 - alpha)
    within sampling error."""
    m = O.OracleMap(N, 8, batch=1)
    keys, vals = W.records(N // 2, 8, 21)
    assert m.init(keys, vals, 6) == 0
    info = m.info()
    llg = math.ceil(math.log2(math.log2(N)))
    assert info["lmax"] == info["c"] + llg + 1
    assert info["R"] == 16 + math.ceil(math.log2(math.log2(N)) / 2)
    assert info["page_bytes"] == (16 + info["lmax"] * info["rec_bytes"] + 63) // 64 * 64
    ops, k, vin = W.op_stream(N // 2, 3000, 8, 22, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.1, zipf_theta=0.99)
    m.trace()
    assert m.access(ops, k, vin)[0] == 0
    tr = [int(e) for e in m.trace()]
    reads_per_access, i = [], 0
    while i < len(tr):
        reads = []
        while i < len(tr) and not tr[i] & 0x80000000:
            reads.append(tr[i])
            i += 1
        writes = []
        while i < len(tr) and tr[i] & 0x80000000:
            writes.append(tr[i] & 0x7FFFFFFF)
            i += 1
        assert 1 <= len(reads) <= 2
        assert writes == list(dict.fromkeys(reads))
        assert all(q < info["M"] for q in reads)
        reads_per_access.append(len(reads))
    # accesses whose two bins are both HBM bins leave no trace entry
    n_host = len(reads_per_access)
    assert n_host <= 3000
    mean = sum(reads_per_access) / 3000
    alpha = info["K"] / info["B"]
    expect = 2 * (1 - alpha)
    assert abs(mean - expect) < 5 * math.sqrt(2 * alpha * (1 - alpha) / 3000) + 0.01
    m.close()


@pytest.mark.parametrize("batch", [1, 64])
def test_host_residents_sit_in_a_bin_of_their_current_pair(batch):
    """After a run of batches every record found in host page q has bin K + q
    in its current pair: the INIT pair of its input index if no batch touched
    it, else the REMAP pair drawn at the global sequence number of the first
    operation on it in the last batch that touched it (Alg. 1 remap; Sec. 3.2
    pairs; batch leaders).  Pairs come from the PRF definition recomputed here
    with a third-party ChaCha20, pages from the oracle's ciphertexts decrypted
    the same way."""
    N = 1 << 12
    keys, vals = W.records(N // 2, 8, 31)
    m = O.OracleMap(N, 8, batch=batch)
    assert m.init(keys, vals, 12) == 0
    info = m.info()
    kprf, kenc = m.keys()
    K, B, P = info["K"], info["B"], info["page_bytes"]
    n_ops = 2048
    ops, k, vin = W.op_stream(N // 2, n_ops, 8, 32, get_frac=0.6, zipf_theta=0.9)
    assert m.access(ops, k, vin)[0] == 0

    def pair(dom, x):
        w = _chacha_ref(kprf, [dom, x & 0xFFFFFFFF, x >> 32], 64).view("<u4")
        first = ((int(w[0]) | (int(w[1]) << 32)) * B) >> 64
        second = ((int(w[2]) | (int(w[3]) << 32)) * (B - 1)) >> 64
        return first, second + (second >= first)

    index = {int(x): i for i, x in enumerate(keys)}
    leader_t = {}
    for lo in range(0, n_ops, batch):
        seen = set()
        for t in range(lo, min(n_ops, lo + batch)):
            kk = int(k[t])
            if kk not in seen:
                seen.add(kk)
                leader_t[kk] = t
    ver = m.versions()
    checked = 0
    for q in range(info["M"]):
        v = int(ver[q])
        plain = m.pages()[q] ^ _chacha_ref(kenc, [q, v & 0xFFFFFFFF, v >> 32], P)
        pk, _ = decode_page(plain, info)
        for kk in pk:
            cur = pair(DOM_REMAP, leader_t[kk]) if kk in leader_t else pair(DOM_INIT, index[kk])
            assert K + q in cur, (q, kk)
            checked += 1
    assert checked > N // 4
    m.close()


def test_remap_p2c_choice_one_op_at_a_time():
    """P2C at access time, checked op by op on the bin loads (Alg. 1 remap;
    Sec. 3.1 P2C with ties to the first bin): an op on a present key removes
    it from one bin of its current pair; if the key is present afterwards it
    goes to the less loaded bin of the REMAP pair drawn at the op's sequence
    number, on the loads after that removal, the first bin on ties.  A Get or
    Delete of an absent key changes no load.  Pairs are recomputed with a
    third-party ChaCha20; presence follows a plain dict."""
    N = 1 << 12
    keys, vals = W.records(N // 2, 8, 41)
    m = O.OracleMap(N, 8, batch=1)
    assert m.init(keys, vals, 14) == 0
    info = m.info()
    kprf, _ = m.keys()
    B = info["B"]

    def pair(dom, x):
        w = _chacha_ref(kprf, [dom, x & 0xFFFFFFFF, x >> 32], 64).view("<u4")
        first = ((int(w[0]) | (int(w[1]) << 32)) * B) >> 64
        second = ((int(w[2]) | (int(w[3]) << 32)) * (B - 1)) >> 64
        return first, second + (second >= first)

    cur = {int(x): pair(DOM_INIT, i) for i, x in enumerate(keys)}
    ops, k, vin = W.op_stream(N // 2, 600, 8, 42, get_frac=0.4, del_frac=0.2,
                              absent_frac=0.2)
    before = m.loads().astype(np.int64)
    for t in range(len(ops)):
        assert m.access(ops[t:t + 1], k[t:t + 1], vin[t:t + 1])[0] == 0
        after = m.loads().astype(np.int64)
        kk, op = int(k[t]), int(ops[t])
        present_after = op == W.PUT or (op == W.GET and kk in cur)
        olds = cur[kk] if kk in cur else (None,)
        ok = False
        for old in olds:
            mid = before.copy()
            if old is not None:
                mid[old] -= 1
            expect = mid.copy()
            if present_after:
                r1, r2 = pair(DOM_REMAP, t)
                expect[r1 if mid[r1] <= mid[r2] else r2] += 1
            ok |= np.array_equal(expect, after)
        assert ok, (t, op, kk in cur)
        if present_after:
            cur[kk] = pair(DOM_REMAP, t)
        else:
            cur.pop(kk, None)
        before = after
    m.close()


def test_written_pages_hold_exactly_their_bin():
    """Trace, eviction and write-back checked op by op (Alg. 1: read both pages,
    remove the key, evict the stash items bound for the pages, write them
    back; the remapped key then waits in the stash or the HBM store): after
    each single-op batch, every page the trace shows written holds exactly
    the present keys whose bin is that page, except the op's own key if it
    was just remapped there, each with its current value; the trace itself is
    the host bins of the key's stored pair (a DUMMY pair at the op's sequence
    number for an absent key), then each page once as a write.  Bins are tracked
    from the INIT P2C rounds and the REMAP rule, pairs recomputed with a
    third-party ChaCha20, values from a plain dict."""
    N = 1 << 12
    keys, vals = W.records(N // 2, 8, 51)
    m = O.OracleMap(N, 8, batch=1)
    assert m.init(keys, vals, 15) == 0
    info = m.info()
    kprf, kenc = m.keys()
    B, K, Wr, P = info["B"], info["K"], info["round_width"], info["page_bytes"]

    def pair(dom, x):
        w = _chacha_ref(kprf, [dom, x & 0xFFFFFFFF, x >> 32], 64).view("<u4")
        first = ((int(w[0]) | (int(w[1]) << 32)) * B) >> 64
        second = ((int(w[2]) | (int(w[3]) << 32)) * (B - 1)) >> 64
        return first, second + (second >= first)

    # bins after init: round-synchronous P2C on round-start loads
    load = np.zeros(B, dtype=np.int64)
    bin_of, pair_of = {}, {}
    for lo in range(0, len(keys), Wr):
        chosen = []
        for i in range(lo, min(len(keys), lo + Wr)):
            a, b = pair(DOM_INIT, i)
            pair_of[int(keys[i])] = (a, b)
            chosen.append((int(keys[i]), a if load[a] <= load[b] else b))
        for kk, d in chosen:
            bin_of[kk] = d
            load[d] += 1
    assert np.array_equal(load, m.loads().astype(np.int64))
    value = {int(x): vals[i].tobytes() for i, x in enumerate(keys)}
    ops, k, vin = W.op_stream(N // 2, 400, 8, 52, get_frac=0.4, del_frac=0.2,
                              absent_frac=0.2)
    m.trace()
    for t in range(len(ops)):
        assert m.access(ops[t:t + 1], k[t:t + 1], vin[t:t + 1])[0] == 0
        kk, op = int(k[t]), int(ops[t])
        # the trace: the host bins of the stored pair (a DUMMY pair for an
        # absent key), then each page once as a write
        read_pair = pair_of[kk] if kk in bin_of else pair(DOM_DUMMY, t)
        reads = [p - K for p in read_pair if p >= K]
        trace = m.trace()
        assert [int(e) for e in trace] == reads + [q | 0x80000000 for q in dict.fromkeys(reads)]
        if kk in bin_of:
            load[bin_of.pop(kk)] -= 1
        if op == W.PUT:
            value[kk] = vin[t].tobytes()
        elif op == W.DEL:
            value.pop(kk, None)
        if kk in value:
            r1, r2 = pair(DOM_REMAP, t)
            pair_of[kk] = (r1, r2)
            bin_of[kk] = r1 if load[r1] <= load[r2] else r2
            load[bin_of[kk]] += 1
        assert np.array_equal(load, m.loads().astype(np.int64)), t
        ver = m.versions()
        for e in trace:
            if not int(e) & 0x80000000:
                continue
            q = int(e) & 0x7FFFFFFF
            v = int(ver[q])
            plain = m.pages()[q] ^ _chacha_ref(kenc, [q, v & 0xFFFFFFFF, v >> 32], P)
            pk, pv = decode_page(plain, info)
            expect = sorted(x for x, d in bin_of.items() if d == K + q and x != kk)
            assert pk == expect, (t, q)
            assert pv == [value[x] for x in pk]
    m.close()


@pytest.mark.parametrize("width", [37, 64, 4096])
def test_batches_follow_the_stated_semantics(width):
    """Batches of several ops against an independent model of the batch
    reading of Alg. 1 (grouping by key; the first op on a present key reads
    its stored pair, misses and repeats read a DUMMY pair at their sequence
    number; every read page is written once, in first-read order, holding
    the keys of its bin after the batch's removals; keys present afterwards
    are remapped by P2C in rounds of W_r op slots decided on round-start
    loads, ties to the first bin).  Checked per batch: the trace, the bin
    loads and every written page (keys and values), at N = 2^16 where a
    round holds 32 op slots (batches of 4096 make keys of one round compete
    for bins, so deciding a round's keys one after another fails).  Pairs
    come from a third-party ChaCha20."""
    N = 1 << 16
    keys, vals = W.records(N // 2, 8, 61)
    m = O.OracleMap(N, 8, batch=width)
    assert m.init(keys, vals, 16) == 0
    info = m.info()
    kprf, kenc = m.keys()
    B, K, Wr, P = info["B"], info["K"], info["round_width"], info["page_bytes"]
    assert Wr == 32

    def pair(dom, x):
        w = _chacha_ref(kprf, [dom, x & 0xFFFFFFFF, x >> 32], 64).view("<u4")
        first = ((int(w[0]) | (int(w[1]) << 32)) * B) >> 64
        second = ((int(w[2]) | (int(w[3]) << 32)) * (B - 1)) >> 64
        return first, second + (second >= first)

    load = np.zeros(B, dtype=np.int64)
    bin_of, pair_of = {}, {}
    for lo in range(0, len(keys), Wr):
        chosen = []
        for i in range(lo, min(len(keys), lo + Wr)):
            p = pair(DOM_INIT, i)
            pair_of[int(keys[i])] = p
            chosen.append((int(keys[i]), p[0] if load[p[0]] <= load[p[1]] else p[1]))
        for kk, d in chosen:
            bin_of[kk] = d
            load[d] += 1
    value = {int(x): vals[i].tobytes() for i, x in enumerate(keys)}
    n_ops = min(8 * width, 3 * 4096)
    ops, k, vin = W.op_stream(N // 2, n_ops, 8, 62, get_frac=0.4, del_frac=0.2,
                              absent_frac=0.15, zipf_theta=1.1)
    m.trace()
    for t0 in range(0, n_ops, width):
        n = min(width, n_ops - t0)
        assert m.access(ops[t0:t0 + n], k[t0:t0 + n], vin[t0:t0 + n])[0] == 0
        bk = [int(x) for x in k[t0:t0 + n]]
        first = {}
        for i, kk in enumerate(bk):
            first.setdefault(kk, i)
        reads = []
        for i, kk in enumerate(bk):
            p = pair_of[kk] if first[kk] == i and kk in bin_of else pair(DOM_DUMMY, t0 + i)
            reads += [b - K for b in p if b >= K]
        written = list(dict.fromkeys(reads))
        trace = [int(e) for e in m.trace()]
        assert trace == reads + [q | 0x80000000 for q in written]
        for kk in first:
            if kk in bin_of:
                load[bin_of.pop(kk)] -= 1
        for i, kk in enumerate(bk):
            if ops[t0 + i] == W.PUT:
                value[kk] = vin[t0 + i].tobytes()
            elif ops[t0 + i] == W.DEL:
                value.pop(kk, None)
        ver = m.versions()
        pages = m.pages()
        by_page = {}
        for x, d in bin_of.items():
            if d >= K:
                by_page.setdefault(d - K, []).append(x)
        for q in written:
            v = int(ver[q])
            plain = pages[q] ^ _chacha_ref(kenc, [q, v & 0xFFFFFFFF, v >> 32], P)
            pk, pv = decode_page(plain, info)
            assert pk == sorted(by_page.get(q, [])), (t0, q)
            assert pv == [value[x] for x in pk]
        for lo in range(0, n, Wr):
            chosen = []
            for i in range(lo, min(n, lo + Wr)):
                kk = bk[i]
                if first[kk] == i and kk in value:
                    p = pair(DOM_REMAP, t0 + i)
                    chosen.append((kk, p, p[0] if load[p[0]] <= load[p[1]] else p[1]))
            for kk, p, d in chosen:
                pair_of[kk], bin_of[kk] = p, d
                load[d] += 1
        assert np.array_equal(load, m.loads().astype(np.int64)), t0
    m.close()


def test_position_map_rows_one_op_at_a_time():
    """Position-map occupancy op by op (Sec. 4.2 d-choice at insertion; a
    delete frees the key's slot): with one op per batch a Put of an absent
    key adds one to the least-occupied of its four candidate rows (the
    first of equal ones), a Delete of a present key frees its row's slot,
    and every other op leaves the rows unchanged.  Candidate rows come from
    the PRF recomputed with a third-party ChaCha20; rows of the init keys
    from the init placement rule."""
    N = 1 << 12
    keys, vals = W.records(N // 2, 8, 81)
    m = O.OracleMap(N, 8, batch=1)
    assert m.init(keys, vals, 18) == 0
    info = m.info()
    kprf, _ = m.keys()
    rows, Wr = info["rows"], info["round_width"]

    def cand(kk):
        w = _chacha_ref(kprf, [DOM_PM, kk & 0xFFFFFFFF, kk >> 32], 64).view("<u4")
        return [((int(w[2 * j]) | (int(w[2 * j + 1]) << 32)) * rows) >> 64 for j in range(4)]

    cnt = np.zeros(rows, dtype=np.int64)
    row_of = {}
    for lo in range(0, len(keys), Wr):
        chosen = []
        for i in range(lo, min(len(keys), lo + Wr)):
            c = cand(int(keys[i]))
            chosen.append((int(keys[i]), c[int(np.argmin(cnt[c]))]))
        for kk, r in chosen:
            row_of[kk] = r
            cnt[r] += 1
    assert np.array_equal(cnt, m.rowcounts().astype(np.int64))
    ops, k, vin = W.op_stream(N // 2, 800, 8, 82, get_frac=0.3, del_frac=0.3,
                              absent_frac=0.3)
    for t in range(len(ops)):
        assert m.access(ops[t:t + 1], k[t:t + 1], vin[t:t + 1])[0] == 0
        kk, op = int(k[t]), int(ops[t])
        if op == W.PUT and kk not in row_of:
            c = cand(kk)
            row_of[kk] = c[int(np.argmin(cnt[c]))]
            cnt[row_of[kk]] += 1
        elif op == W.DEL and kk in row_of:
            cnt[row_of.pop(kk)] -= 1
        assert np.array_equal(cnt, m.rowcounts().astype(np.int64)), t
    m.close()


@pytest.mark.parametrize("batch", [1, 64, 4096])
def test_openmp_build_is_byte_identical(batch):
    """The multi-core CPU baseline is the oracle's own source built with
    OpenMP (its independent loops -- PRF draws, per-round decisions, page
    decryption and encryption -- on several threads).  On the same seeded
    inputs it gives the same pages, trace, loads, rows, statistics, values
    and status as the single-threaded build, at any thread count."""
    N, vb = 1 << 14, 24
    keys, vals = W.records(12000, vb, 61)
    ops, k, vin = W.op_stream(12000, 6000, vb, 62, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.1, zipf_theta=0.99)
    one = O.OracleMap(N, vb, batch=batch)
    assert one.init(keys, vals, 9) == 0
    r1 = one.access(ops, k, vin)
    for nthreads in (2, 7):
        assert O.threads(nthreads) == nthreads
        many = O.OracleMap(N, vb, batch=batch, omp=True)
        assert many.init(keys, vals, 9) == 0
        r2 = many.access(ops, k, vin)
        assert r1[0] == r2[0] == 0
        assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
        assert np.array_equal(one.pages(), many.pages())
        assert np.array_equal(one.loads(), many.loads())
        assert np.array_equal(one.rowcounts(), many.rowcounts())
        assert one.stats() == many.stats()
        assert np.array_equal(one.trace(clear=False), many.trace(clear=False))
        many.close()
    one.close()


def test_owner_image_matches_the_built_map():
    """The data owner's image (Sec. 4.2 "Fast data initialization"): records
    in bin-major order (HBM bins first, then host pages; ascending record
    index within a bin), each with the pair PRF(INIT, i), the bin it sits in,
    and a position-map row among its d = 4 candidate rows.  Checked against
    the map the same call builds: per-bin counts equal the bin loads, the rows
    recount to the position-map row counts, every host page decrypts to
    exactly its bin's run of the image."""
    N, vb = 1 << 14, 16
    keys, vals = W.records(12000, vb, 41)
    m = O.OracleMap(N, vb)
    rc, img = m.prepare(keys, vals, 5)
    assert rc == 0
    info = m.info()
    K, B_ = info["K"], info["B"]
    assert np.array_equal(img["counts"], m.loads())
    assert int(img["counts"].sum()) == len(keys)
    idx_of = {int(k): i for i, k in enumerate(keys)}
    src = np.array([idx_of[int(k)] for k in img["keys"]])
    assert sorted(src.tolist()) == list(range(len(keys)))  # a permutation
    assert np.array_equal(img["vals"], vals[src])
    b1 = (img["pairs"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    b2 = (img["pairs"] >> np.uint64(32)).astype(np.int64)
    in_b2 = (img["rows"] >> np.uint32(31)).astype(bool)
    rows = (img["rows"] & np.uint32(0x7FFFFFFF)).astype(np.int64)
    bins = np.where(in_b2, b2, b1)
    assert np.all(np.diff(bins) >= 0), "bin-major order"
    same = np.diff(bins) == 0
    assert np.all(np.diff(src)[same] > 0), "ascending record index within a bin"
    assert np.array_equal(np.bincount(bins, minlength=B_), img["counts"].astype(np.int64))
    kprf, _ = m.keys()
    for j in range(0, len(keys), 97):
        assert O.pair(kprf, 1, int(src[j]), B_) == (b1[j], b2[j])
        # the row is one of the key's d = 4 candidates PRF(PM, key) (Sec. 4.2)
        k = int(img["keys"][j])
        w = O.chacha20_block(kprf, 0, [2, k & 0xFFFFFFFF, k >> 32]).astype(np.uint64)
        cand = [((int(w[2 * t]) | (int(w[2 * t + 1]) << 32)) * info["rows"]) >> 64 for t in range(4)]
        assert rows[j] in cand
    assert np.array_equal(np.bincount(rows, minlength=info["rows"]), m.rowcounts())
    starts = np.concatenate([[0], np.cumsum(img["counts"].astype(np.int64))])
    rec = 8 + vb
    for q in range(0, info["M"], 37):
        plain = m.decrypt_page(q)
        cnt = int(img["counts"][K + q])
        lo = starts[K + q]
        slots = plain[16:16 + cnt * rec].reshape(cnt, rec)
        got = slots[:, :8].copy().view(np.uint64)[:, 0]
        assert np.array_equal(got, np.sort(img["keys"][lo:lo + cnt]))
    m.close()


# --------------------------------------------------------------------------
# Page integrity (NEXT-4): pages sealed by ChaCha20-Poly1305, bound to (page, version)


def test_poly1305_matches_the_cryptography_package():
    """The oracle's Poly1305 (RFC 8439 Sec. 2.5, three 64-bit limbs) against
    an independent implementation, on random keys and messages of every
    length class (empty, short, exact blocks, ragged tails), and on keys
    whose r and s sit at the edges of their ranges."""
    from cryptography.hazmat.primitives.poly1305 import Poly1305
    rng = np.random.default_rng(301)
    keys = [rng.bytes(32) for _ in range(40)]
    keys += [b"\xff" * 32, b"\x00" * 16 + b"\xff" * 16, b"\xff" * 16 + b"\x00" * 16]
    for j, key in enumerate(keys):
        for n in (0, 1, 15, 16, 17, 31, 32, 33, 64, 100, 511, 512, 1000):
            msg = rng.bytes(n) if j % 3 else b"\xff" * n
            assert O.poly1305(key, msg) == Poly1305.generate_tag(key, msg), (j, n)


def test_sealed_pages_are_the_chacha20_poly1305_aead():
    """With integrity on, every page of a built map, and every page an access
    batch rewrote (under its bumped version), is the RFC 8439 AEAD
    encryption of its plaintext under K_enc with nonce page || version and
    no additional data -- checked by decrypting with the `cryptography`
    package, which verifies the tag -- and the oracle's own decryption gives
    the same plaintext.  The page size leaves room for the 16-byte tag."""
    from cryptography.hazmat.primitives.ciphers.aead import ChaCha20Poly1305
    N, vb = 1 << 12, 24
    m = O.OracleMap(N, vb, integrity=True)
    info = m.info()
    assert info["page_bytes"] == (16 + info["lmax"] * (8 + vb) + 16 + 63) // 64 * 64
    keys, vals = W.records(3000, vb, 302)
    assert m.init(keys, vals, 7) == 0
    _, kenc = m.keys()
    aead = ChaCha20Poly1305(kenc.astype("<u4").tobytes())

    def check_all():
        pages = m.pages()
        vers = m.versions()
        for q in range(info["M"]):
            nonce = int(q).to_bytes(4, "little") + int(vers[q]).to_bytes(8, "little")
            plain = aead.decrypt(nonce, pages[q].tobytes(), None)
            assert plain == m.decrypt_page(q)[:info["page_bytes"] - 16].tobytes()
        return vers

    v0 = check_all()
    assert not v0.any()
    ops, k, vin = W.op_stream(3000, 500, vb, 303, del_frac=0.1, absent_frac=0.1)
    rc, vout, st = m.access(ops, k, vin)
    assert rc == 0
    model = DictModel(keys, vals)
    ev, es = model.apply(ops, k, vin, vb)
    assert np.array_equal(vout, ev) and np.array_equal(st, es)
    assert check_all().any()
    m.close()


@pytest.mark.parametrize("attack", ["flip", "replay", "swap"])
def test_sealed_pages_detect_host_changes(attack):
    """A host that changes a page (one bit), replays an older version of it,
    or puts another page's sealed bytes in its place is caught when the page
    is next read: the access returns ORC_E_INTEGRITY (the version lives in
    HBM, so an old ciphertext no longer matches its nonce).  Untouched pages
    read fine."""
    N, vb = 1 << 12, 8
    m = O.OracleMap(N, vb, integrity=True, batch=1)
    keys, vals = W.records(3000, vb, 304)
    assert m.init(keys, vals, 9) == 0
    store = m.host_pages()
    old = store.copy()
    # one access rewrites the pages of key 0's two bins (and the versions)
    rc, _, _ = m.access(np.zeros(1, np.uint8), keys[:1], np.zeros((1, vb), np.uint8))
    assert rc == 0
    tr = m.trace()
    written = sorted({int(e) & 0x7FFFFFFF for e in tr if e & 0x80000000})
    q = written[0]
    if attack == "flip":
        store[q, 37] ^= 0x10
    elif attack == "replay":
        store[q] = old[q]
    else:
        other = (q + 1) % m.info()["M"]
        store[q] = store[other]
    # a Get whose DUMMY or stored pair reads page q: run single-op Gets on
    # keys until one reads q (the trace says which pages each op read)
    rc = 0
    for i in range(1, 3000):
        rc, _, _ = m.access(np.zeros(1, np.uint8), keys[i:i + 1], np.zeros((1, vb), np.uint8))
        reads = {int(e) for e in m.trace() if not e & 0x80000000}
        if rc != 0 or q in reads:
            break
    assert rc == O.E_INTEGRITY
    m.close()
