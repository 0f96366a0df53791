"""The headline map at full size (N = 2^28 records of 32 B), checked on
samples the oracle computes one by one and on properties that hold at any
size (needs a B300; ~14 GB of pinned host memory).

The oracle cannot rebuild a 2^28-record map in test time, so this test
checks what it can compute per record and per page: a record's two INIT bins
from the PRF, a page's plaintext from its ciphertext, and Get/Put results,
in the launch configuration the benchmark times (device-resident inputs,
batches of 4096 through bolt_access_device_batches)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _parse(plain: np.ndarray, lmax: int, vb: int):
    bitmap = int(plain[:8].view(np.uint64)[0])
    rec = 8 + vb
    slots = plain[16:16 + lmax * rec].reshape(lmax, rec)
    keys = slots[:, :8].copy().view(np.uint64)[:, 0]
    return bitmap, keys, slots[:, 8:]


def test_full_size_headline_map_sampled():
    import torch
    N, vb, seed, batch = 1 << 28, 24, 0x5EED0203, 4096
    torch.cuda.set_device(0)
    d_keys = W.key_of_torch(torch.arange(N, device="cuda", dtype=torch.int64))
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    d_vals = torch.randint(0, 256, (N, vb), dtype=torch.uint8, device="cuda", generator=g)
    m = B.BoltMap(N, vb)
    assert m.init_device(d_keys, d_vals, seed) == 0
    assert m.sync() == 0
    info = m.info()
    K, Bn, lmax, pb = info["K"], info["B"], info["lmax"], info["page_bytes"]
    kprf, kenc = O.kdf(seed)

    # bin loads: every record counted once, none above lmax (Claim 3.2)
    loads = m.loads()
    assert int(loads.max()) <= lmax
    assert int(loads.sum(dtype=np.int64)) == N

    rng = np.random.default_rng(12)
    idx = rng.choice(N, size=2000, replace=False).astype(np.uint64)
    keys = W.key_of(idx)
    vals = d_vals[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
    seen_pages = {}
    both_host = 0
    for j, i in enumerate(idx):
        b1, b2 = O.pair(kprf, 1, int(i), Bn)  # INIT pair of record i
        assert b1 != b2 and b1 < Bn and b2 < Bn
        found = 0
        for b in (b1, b2):
            if b < K:
                continue
            q = b - K
            if q not in seen_pages:
                plain = O.page_decrypt(kenc, q, 0, m.pages(q, 1)[0])
                bitmap, pk, pv = _parse(plain, lmax, vb)
                cnt = bin(bitmap).count("1")
                # page invariants: reals in the first slots, ascending keys,
                # count = the bin's load, zero dummies
                assert bitmap == (1 << cnt) - 1 and cnt == int(loads[b])
                assert np.all(pk[1:cnt] > pk[:cnt - 1])
                assert not plain[16 + cnt * (8 + vb):].any()
                seen_pages[q] = (pk[:cnt], pv[:cnt])
            pk, pv = seen_pages[q]
            hit = np.flatnonzero(pk == keys[j])
            if len(hit):
                found += 1
                assert np.array_equal(pv[hit[0]], vals[j])
        if b1 >= K and b2 >= K:
            both_host += 1
            assert found == 1, f"record {i} must sit in exactly one of its two pages"
        else:
            assert found <= 1
    assert both_host > 1000  # alpha = 0.2: ~64% of records have two host bins

    # Get / Put in the benchmark's launch configuration
    n = 2 * batch
    gidx = rng.choice(N, size=batch, replace=False).astype(np.uint64)
    gvals = d_vals[torch.from_numpy(gidx.astype(np.int64)).cuda()].cpu().numpy()
    pidx = rng.choice(N, size=batch, replace=False).astype(np.uint64)
    newv = rng.integers(0, 256, size=(batch, vb), dtype=np.uint8)
    ops = np.concatenate([np.zeros(batch, np.uint8), np.ones(batch, np.uint8)])
    akeys = np.concatenate([W.key_of(gidx), W.key_of(pidx)])
    avin = np.concatenate([np.zeros((batch, vb), np.uint8), newv])
    t = [torch.from_numpy(x).cuda() for x in (ops, akeys.view(np.int64), avin)]
    out = torch.zeros((n, vb), dtype=torch.uint8, device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    assert m.access_device_batches(t[0], t[1], t[2], out, st, batch) == 0
    assert m.sync() == 0
    assert st.cpu().numpy().all()
    assert np.array_equal(out[:batch].cpu().numpy(), gvals)
    assert not out[batch:].cpu().numpy().any()  # PUT responses are zero
    # the new values are read back
    ops2 = np.zeros(batch, np.uint8)
    t2 = [torch.from_numpy(x).cuda() for x in (ops2, W.key_of(pidx).view(np.int64),
                                               np.zeros((batch, vb), np.uint8))]
    out2 = torch.zeros((batch, vb), dtype=torch.uint8, device="cuda")
    st2 = torch.zeros(batch, dtype=torch.uint8, device="cuda")
    assert m.access_device_batches(t2[0], t2[1], t2[2], out2, st2, batch) == 0
    assert m.sync() == 0
    assert st2.cpu().numpy().all()
    assert np.array_equal(out2.cpu().numpy(), newv)
    m.close()
