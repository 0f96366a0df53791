"""bolt_init_device_noalloc: the build for callers that cannot allocate.

Some callers cannot allocate device memory at the moment they (re)build a map:
a serving loop that re-keys maps in place must not stall its other streams on
cudaMalloc/cudaFree, and some processes hand all device memory to another
allocator.  For them the library has one entry point whose scratch lives in a
fixed array compiled into the library.  This test calls it through the C ABI
twice in a row (the second call on different data, so stale contents of the
shared array would show) and checks that the map it builds is the map
bolt_init_device builds: same page ciphertexts, bin loads and position-map
rows, and the same results for a batch of accesses afterwards.  The file sorts
last so a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2509_01742_b300 import workload as W

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _noalloc_init(m, tk, tv, seed):
    return B.bolt_init_device_noalloc(m.handle, ctypes.c_void_p(tk.data_ptr()),
                                      ctypes.c_void_p(tv.data_ptr()), tk.numel(), seed,
                                      ctypes.c_void_p(0))


def test_noalloc_build_matches_device_build_twice():
    import torch
    N, vb = 1 << 16, 8
    ref = B.BoltMap(N, vb)
    nal = B.BoltMap(N, vb)
    for call, (n, seed) in enumerate([(N, 0x5EED0001), (40000, 0x5EED0002)]):
        keys, vals = W.records(n, vb, 100 + call)
        tk = torch.from_numpy(keys.view(np.int64)).cuda()
        tv = torch.from_numpy(vals.copy()).cuda()
        assert ref.init_device(tk, tv, seed) == 0
        assert _noalloc_init(nal, tk, tv, seed) == 0
        # nothing was allocated for the build: this handle never ran
        # bolt_init or bolt_init_device, so it holds no build scratch
        assert nal.footprint()[1] == 0
        assert np.array_equal(ref.pages(), nal.pages()), f"pages differ on call {call}"
        assert np.array_equal(ref.loads(), nal.loads()), f"loads differ on call {call}"
        assert np.array_equal(ref.rowcounts(), nal.rowcounts()), f"rows differ on call {call}"
        ops, k, vin = W.op_stream(n, 4096, vb, 7 + call, del_frac=0.1, absent_frac=0.1)
        rc1, v1, s1 = ref.access(ops, k, vin)
        rc2, v2, s2 = nal.access(ops, k, vin)
        assert rc1 == rc2 == 0
        assert np.array_equal(v1, v2) and np.array_equal(s1, s2)
        assert np.array_equal(ref.pages(), nal.pages())
        assert nal.footprint()[1] == 0
    ref.close()
    nal.close()


@pytest.mark.parametrize("case", ["far_apart", "max_key_twice", "max_key_once"])
def test_noalloc_key_check(case):
    """The allocation-free build checks key uniqueness (Sec. 2.1) by sorting a
    copy of the keys, padded with all-ones words, and comparing neighbours:
    a duplicate pair far apart is found, the all-ones key given twice is
    found, and given once among distinct keys (equal to the padding) it is
    not mistaken for a duplicate.  2^17 keys, within the array's limit."""
    import torch
    n = 1 << 17
    keys, vals = W.records(n, 8, 91)
    top = np.uint64(0xFFFFFFFFFFFFFFFF)
    if case == "far_apart":
        keys[n - 1] = keys[2]
    elif case == "max_key_twice":
        keys[7] = top
        keys[n - 3] = top
    else:
        keys[n // 2] = top
    m = B.BoltMap(n, 8)
    tk = torch.from_numpy(keys.view(np.int64)).cuda()
    tv = torch.from_numpy(vals.copy()).cuda()
    rc = _noalloc_init(m, tk, tv, 4)
    assert rc == (0 if case == "max_key_once" else B.BOLT_E_DUPKEY)
    assert m.footprint()[1] == 0
    if rc == 0:
        # the map built beside the padding value serves its keys
        ops = np.zeros(64, np.uint8)
        idx = np.arange(n // 2 - 32, n // 2 + 32)
        rc2, vout, st = m.access(ops, keys[idx], np.zeros((64, 8), np.uint8))
        assert rc2 == 0 and st.all() and np.array_equal(vout, vals[idx])
    m.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    big = B.BoltMap(1 << 22, 8)  # 2^22 / 8 bins -> more than 2^18 host pages
    tk = torch.zeros(16, dtype=torch.int64, device="cuda")
    tv = torch.zeros((16, 8), dtype=torch.uint8, device="cuda")
    assert _noalloc_init(big, tk, tv, 1) == B.BOLT_E_ARG
    big.close()
    small = B.BoltMap(1 << 20, 8)  # 2^17 bins: fits; 2^18 + 1 records do not
    n = (1 << 18) + 1
    tk = torch.arange(n, dtype=torch.int64, device="cuda")
    tv = torch.zeros((n, 8), dtype=torch.uint8, device="cuda")
    assert _noalloc_init(small, tk, tv, 1) == B.BOLT_E_ARG
    small.close()
