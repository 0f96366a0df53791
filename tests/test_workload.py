"""The seeded input generators (harness code, no method arithmetic)."""
import numpy as np

from paper_2509_01742_b300 import workload as W


def test_device_key_generator_matches_host():
    """key_of_torch gives the same 64-bit keys as key_of (it generates the
    inputs of the largest configuration on the device)."""
    import torch
    idx = np.concatenate([np.arange(5000, dtype=np.uint64),
                          np.array([2**30 - 1, 2**31 + 7, 2**40 + 3], dtype=np.uint64)])
    host = W.key_of(idx).view(np.int64)
    dev = W.key_of_torch(torch.from_numpy(idx.view(np.int64))).numpy()
    assert np.array_equal(host, dev)


def test_keys_distinct_and_op_indices_consistent():
    keys = W.key_of(np.arange(1 << 16, dtype=np.uint64))
    assert len(np.unique(keys)) == len(keys)
    ops, k, vin, idx = W.op_stream(1 << 16, 4096, 8, 7, get_frac=0.9, zipf_theta=0.99,
                                   return_index=True)
    assert np.array_equal(W.key_of(idx), k)
    assert (idx < (1 << 16)).all()
    ops2, k2, vin2 = W.op_stream(1 << 16, 4096, 8, 7, get_frac=0.9, zipf_theta=0.99)
    assert np.array_equal(ops, ops2) and np.array_equal(k, k2) and np.array_equal(vin, vin2)
