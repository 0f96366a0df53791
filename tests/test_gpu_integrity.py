"""Sealed pages (BOLT_PARAM_INTEGRITY) on the GPU against the oracle (needs a B300).

With integrity on, every host page is the ChaCha20-Poly1305 AEAD (RFC 8439
Sec. 2.8) of its plaintext under nonce (page, version): the device seals
pages in the build and in every write-back and checks each page's tag when
a batch reads it.  The bar is the same as for plain pages -- page bytes
(ciphertext and tag), values, status, loads, rows and trace equal the
oracle's -- plus the same verdict as the oracle on pages the host altered.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _pair(N, vb, batch=None):
    o = O.OracleMap(N, vb, integrity=True, batch=batch)
    g = B.BoltMap(N, vb, trace=True, batch=batch, integrity=True)
    assert o.info() == g.info()
    return o, g


def _state_equal(o, g, what):
    assert np.array_equal(o.pages(), g.pages()), f"sealed pages differ {what}"
    assert np.array_equal(o.loads(), g.loads()), f"bin loads differ {what}"
    assert np.array_equal(o.rowcounts().astype(np.uint8), g.rowcounts()), f"pm rows differ {what}"
    assert np.array_equal(o.trace(), g.trace()), f"host trace differs {what}"


# 8-, 56- and 120-byte values: sealed pages of 256, 896 and 1728 bytes, so the
# tag spans one, two and four 512-byte chunks of the warp's Poly1305
@pytest.mark.parametrize("vb", [8, 56, 120])
def test_sealed_build_and_batches_match_oracle(vb):
    """Build, then batches through the multi-kernel chain: every sealed page
    byte equals the oracle's, and so do the results."""
    N = 1 << 12
    o, g = _pair(N, vb)
    i = g.info()
    assert i["page_bytes"] == (16 + i["lmax"] * (8 + vb) + 16 + 63) // 64 * 64
    keys, vals = W.records(3500, vb, 0x1A7E + vb)
    assert o.init(keys, vals, 5) == 0 and g.init(keys, vals, 5) == 0
    _state_equal(o, g, "after build")
    for rep in range(3):
        ops, k, vin = W.op_stream(3500, 900, vb, 0x1A80 + rep, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.2)
        rc_o, vo, so = o.access(ops, k, vin)
        rc_g, vg, sg = g.access(ops, k, vin)
        assert rc_o == rc_g == 0, (rc_o, rc_g)
        assert np.array_equal(so, sg) and np.array_equal(vo, vg), f"results differ, rep {rep}"
        _state_equal(o, g, f"after batch {rep}")
    o.close(); g.close()


@pytest.mark.parametrize("batch,fused", [(1, 1), (32, 1), (7, 0)])
def test_sealed_small_batches_match_oracle(batch, fused):
    """Batches of 1..32 ops as one fused launch (the page read, tag check and
    sealed write-back inside one CTA) or through the chain."""
    N, vb = 1 << 12, 24
    o, g = _pair(N, vb, batch=batch)
    g.set_param(B.BOLT_PARAM_FUSED, fused)
    keys, vals = W.records(3000, vb, 0x1A90)
    assert o.init(keys, vals, 6) == 0 and g.init(keys, vals, 6) == 0
    ops, k, vin = W.op_stream(3000, 300, vb, 0x1A91, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.2)
    rc_o, vo, so = o.access(ops, k, vin)
    rc_g, vg, sg = g.access(ops, k, vin)
    assert rc_o == rc_g == 0
    assert np.array_equal(so, sg) and np.array_equal(vo, vg)
    _state_equal(o, g, "after the batches")
    o.close(); g.close()


@pytest.mark.parametrize("attack", ["flip", "replay", "swap"])
@pytest.mark.parametrize("fused", [1, 0])
def test_altered_page_fails_like_the_oracle(attack, fused):
    """The host changes one bit of a page, puts back the page's previous
    sealed version, or copies another page over it: the first batch that
    reads the page returns BOLT_E_INTEGRITY on the GPU at the same operation
    as ORC_E_INTEGRITY on the oracle, every earlier batch succeeds with the
    oracle's results, and the map is poisoned afterwards on both."""
    N, vb = 1 << 12, 8
    o, g = _pair(N, vb, batch=1)
    g.set_param(B.BOLT_PARAM_FUSED, fused)
    keys, vals = W.records(3000, vb, 0x1AA0)
    assert o.init(keys, vals, 8) == 0 and g.init(keys, vals, 8) == 0
    old = g.pages()
    z = np.zeros((1, vb), np.uint8)
    get = np.zeros(1, np.uint8)
    # the first Get that reads (and so rewrites) a host page: its pair may
    # also fall on two HBM bins, which the host never sees
    written, j = [], 0
    while not written:
        assert o.access(get, keys[j:j + 1], z)[0] == 0 and g.access(get, keys[j:j + 1], z)[0] == 0
        tr = g.trace()
        assert np.array_equal(tr, o.trace())
        written = sorted({int(e) & 0x7FFFFFFF for e in tr if e & 0x80000000})
        j += 1
    q = written[0]
    now = g.pages()
    page = now[q].copy()
    if attack == "flip":
        page[37] ^= 0x10
    elif attack == "replay":
        page = old[q].copy()
        assert not np.array_equal(page, now[q])
    else:
        page = now[(q + 1) % now.shape[0]].copy()
    g.write_pages(q, page[None, :])
    o.host_pages()[q] = page
    assert np.array_equal(o.pages(), g.pages())
    hit = None
    for i in range(j, 3000):
        rc_o, vo, so = o.access(get, keys[i:i + 1], z)
        rc_g, vg, sg = g.access(get, keys[i:i + 1], z)
        assert rc_o == rc_g, (i, rc_o, rc_g)
        if rc_g:
            assert rc_g == B.BOLT_E_INTEGRITY and rc_o == O.E_INTEGRITY
            hit = i
            break
        assert np.array_equal(vo, vg) and np.array_equal(so, sg)
        tr = g.trace()
        assert np.array_equal(tr, o.trace())
        assert q not in {int(e) for e in tr if not e & 0x80000000}
    assert hit is not None, "no operation read the altered page"
    assert o.access(get, keys[:1], z)[0] == O.E_STATE
    assert g.access(get, keys[:1], z)[0] == B.BOLT_E_STATE
    # a rebuild clears the poison
    assert g.init(keys, vals, 8) == 0
    assert g.access(get, keys[:1], z)[0] == 0
    o.close(); g.close()


def test_integrity_excludes_lookahead():
    """Pages read ahead are not checked, so the two settings exclude each
    other (BOLT_E_ARG either way round)."""
    g = B.BoltMap(1 << 12, 8, integrity=True)
    with pytest.raises(B.BoltError) as e:
        g.set_param(B.BOLT_PARAM_LOOKAHEAD, 0.5)
    assert e.value.rc == B.BOLT_E_ARG
    g.set_param(B.BOLT_PARAM_INTEGRITY, 0)
    g.set_param(B.BOLT_PARAM_LOOKAHEAD, 0.5)
    with pytest.raises(B.BoltError) as e:
        g.set_param(B.BOLT_PARAM_INTEGRITY, 1)
    assert e.value.rc == B.BOLT_E_ARG
    g.close()


def test_sealed_prepared_load_matches_oracle():
    """A data owner's image (Sec. 4.2) loaded into a sealed map gives the
    oracle's sealed pages, and accesses afterwards the oracle's results."""
    import torch
    from tests.test_gpu_owner_build import _to_device
    N, vb = 1 << 14, 24
    keys, vals = W.records(12000, vb, 0x1AB0)
    seed = 0x5EED0031
    o = O.OracleMap(N, vb, integrity=True)
    rc, img = o.prepare(keys, vals, seed)
    assert rc == 0
    g = B.BoltMap(N, vb, trace=True, integrity=True)
    assert g.info() == o.info()
    assert g.init_prepared(_to_device(img), len(keys), seed) == 0
    assert np.array_equal(o.pages(), g.pages()), "sealed pages differ after the prepared load"
    ops, k, vin = W.op_stream(12000, 2000, vb, 0x1AB1, get_frac=0.5, del_frac=0.1,
                              absent_frac=0.1)
    rc_o, vo, so = o.access(ops, k, vin)
    rc_g, vg, sg = g.access(ops, k, vin)
    assert rc_o == rc_g == 0
    assert np.array_equal(so, sg) and np.array_equal(vo, vg)
    _state_equal(o, g, "after a batch")
    o.close(); g.close()


def test_sealed_allocation_free_build_matches_oracle():
    """bolt_init_device_noalloc (pages stored straight to the host from the
    SMs) seals them as the oracle does."""
    import ctypes
    import torch
    N, vb = 1 << 14, 8
    keys, vals = W.records(N, vb, 0x1AC0)
    seed = 0x5EED0032
    o = O.OracleMap(N, vb, integrity=True)
    assert o.init(keys, vals, seed) == 0
    g = B.BoltMap(N, vb, integrity=True)
    tk = torch.from_numpy(keys.view(np.int64)).cuda()
    tv = torch.from_numpy(vals.copy()).cuda()
    assert B.bolt_init_device_noalloc(g.handle, ctypes.c_void_p(tk.data_ptr()),
                                      ctypes.c_void_p(tv.data_ptr()), N, seed,
                                      ctypes.c_void_p(0)) == 0
    assert np.array_equal(o.pages(), g.pages()), "sealed pages differ after the build"
    assert np.array_equal(o.loads(), g.loads())
    o.close(); g.close()
