"""The owner-side build (Sec. 4.2 "Fast data initialization") against the
oracle (needs a B300).  The paper's data owner pre-organizes the records --
random pairs, power-of-two-choices bins, position-map rows -- and the device
loads that layout with sequential reads and writes.  Checked here:
  - the image bolt_prepare_device exports equals the oracle's image of the
    same records and seed, array by array;
  - bolt_init_prepared, given the oracle's image, builds the oracle's map:
    page ciphertexts, bin loads, position-map rows, HBM-store and stash
    counts; and access batches afterwards give the oracle's values, status,
    pages and trace;
  - an image that does not fit the map (a count above lmax, a row out of
    range, counts that do not add up) is refused with BOLT_E_OVERFLOW and the
    handle builds again afterwards."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_01742_b300 import workload as W
from tests.test_gpu_parity import _assert_state_equal, _run_batch

pytestmark = pytest.mark.gpu

B = pytest.importorskip("paper_2509_01742_b300.bolt")


def _to_device(img):
    import torch
    return {"keys": torch.from_numpy(img["keys"].view(np.int64)).cuda(),
            "vals": torch.from_numpy(img["vals"]).cuda(),
            "pairs": torch.from_numpy(img["pairs"].view(np.int64)).cuda(),
            "rows": torch.from_numpy(img["rows"].view(np.int32)).cuda(),
            "counts": torch.from_numpy(img["counts"]).cuda()}


@pytest.mark.parametrize("N,n,vb,alpha", [(1 << 16, 1 << 16, 16, None), (1 << 20, 900000, 24, 0.01),
                                          (1 << 12, 0, 8, None)])
def test_owner_image_and_prepared_load_match_oracle(N, n, vb, alpha):
    import torch
    keys, vals = W.records(n, vb, 61)
    seed = 0x5EED0011
    o = O.OracleMap(N, vb, alpha=alpha)
    rc, img_o = o.prepare(keys, vals, seed)
    assert rc == 0
    # the exported image
    g = B.BoltMap(N, vb, alpha=alpha)
    assert g.info() == o.info()
    tk = torch.from_numpy(keys.view(np.int64)).cuda()
    tv = torch.from_numpy(vals.copy()).cuda()
    rc, img_g = g.prepare_device(tk, tv, seed)
    assert rc == 0
    assert np.array_equal(img_g["counts"].cpu().numpy(), img_o["counts"])
    for k in ("keys", "pairs"):
        assert np.array_equal(img_g[k].cpu().numpy().view(np.uint64), img_o[k]), k
    assert np.array_equal(img_g["rows"].cpu().numpy().view(np.uint32), img_o["rows"])
    assert np.array_equal(img_g["vals"].cpu().numpy(), img_o["vals"])
    # the prepared load of the oracle's image
    p = B.BoltMap(N, vb, alpha=alpha, trace=True)
    assert p.init_prepared(_to_device(img_o), n, seed) == 0
    _assert_state_equal(o, p, "after the prepared load")
    assert np.array_equal(p.pages(), g.pages())
    for rep in range(3):
        ops, k, vin = W.op_stream(max(n, 1), 3000, vb, 70 + rep, get_frac=0.5, del_frac=0.1,
                                  absent_frac=0.1)
        _run_batch(o, p, ops, k, vin, f"batch {rep}")
        _assert_state_equal(o, p, f"after batch {rep}")
    o.close(); g.close(); p.close()


def test_prepared_load_refuses_images_that_do_not_fit():
    import torch
    N, vb = 1 << 14, 8
    keys, vals = W.records(N, vb, 62)
    o = O.OracleMap(N, vb)
    rc, img = o.prepare(keys, vals, 3)
    assert rc == 0
    g = B.BoltMap(N, vb)
    lmax = g.info()["lmax"]
    bad = {k: v.copy() for k, v in img.items()}
    bad["counts"][5] = lmax + 1           # a bin above lmax (and a wrong total)
    assert g.init_prepared(_to_device(bad), N, 3) == B.BOLT_E_OVERFLOW
    bad = {k: v.copy() for k, v in img.items()}
    bad["rows"][100] = np.uint32(0x7FFFFFF)  # a row out of range
    assert g.init_prepared(_to_device(bad), N, 3) == B.BOLT_E_OVERFLOW
    assert g.init_prepared(_to_device(img), N - 1, 3) == B.BOLT_E_OVERFLOW  # counts != n
    rc, _, _ = g.access(np.zeros(1, np.uint8), keys[:1], np.zeros((1, vb), np.uint8))
    assert rc == B.BOLT_E_STATE
    assert g.init_prepared(_to_device(img), N, 3) == 0
    assert np.array_equal(g.pages(), o.pages())
    o.close(); g.close()
