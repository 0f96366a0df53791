"""Seeded synthetic workloads for the oblivious map (harness code).

Holds none of the method's arithmetic: it only draws keys, values and
operation streams.  Both the tests (for the CPU oracle and the CUDA path) and
the benchmark draw their inputs from here, so the two sides see identical
bytes.  Shapes follow the paper's evaluation workload (Sec. 5.3: uniform
random GET/PUT over an initial key set, "YCSB-like"), plus Zipf-skewed key
popularity for the skewed configurations.
"""
from __future__ import annotations

import numpy as np

GET, PUT, DEL = 0, 1, 2
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_KEY_SALT = np.uint64(0x5DEECE66D2B7E151)


def mix64(x: np.ndarray) -> np.ndarray:
    """A bijective 64-bit mixer (xor-shift / odd-multiply rounds)."""
    x = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(30)
        x *= _M1
        x ^= x >> np.uint64(27)
        x *= _M2
        x ^= x >> np.uint64(31)
    return x


def key_of(index: np.ndarray) -> np.ndarray:
    """Distinct 64-bit keys: record i has key mix64(i ^ salt); indices >= N give
    keys that are absent from an N-record map."""
    return mix64(np.asarray(index, dtype=np.uint64) ^ _KEY_SALT)


def _s64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def key_of_torch(index):
    """key_of for an integer torch tensor on any device: the same 64 bits, as
    int64 (right shifts are made logical by masking the sign-extended bits)."""
    import torch
    x = index.to(torch.int64) ^ _s64(int(_KEY_SALT))
    x = x ^ ((x >> 30) & ((1 << 34) - 1))
    x = x * _s64(int(_M1))
    x = x ^ ((x >> 27) & ((1 << 37) - 1))
    x = x * _s64(int(_M2))
    x = x ^ ((x >> 31) & ((1 << 33) - 1))
    return x


def records(n: int, val_bytes: int, seed: int):
    """n distinct keys (uint64) and n random values (uint8[n, val_bytes])."""
    rng = np.random.default_rng(seed)
    keys = key_of(np.arange(n, dtype=np.uint64))
    vals = rng.integers(0, 256, size=(n, val_bytes), dtype=np.uint8)
    return keys, vals


class Zipf:
    """Zipf(theta) ranks over [0, n) by the Gray et al. (SIGMOD '94) closed-form
    sampler; rank 0 is the most popular.  zeta(n, theta) is summed once."""

    def __init__(self, n: int, theta: float):
        self.n, self.theta = n, theta
        zeta = 0.0
        step = 1 << 24
        for lo in range(1, n + 1, step):
            i = np.arange(lo, min(n, lo + step - 1) + 1, dtype=np.float64)
            zeta += float(np.sum(i ** -theta))
        self.zetan = zeta
        self.zeta2 = 1.0 + 0.5 ** theta
        self.alpha = 1.0 / (1.0 - theta)
        self.eta = (1.0 - (2.0 / n) ** (1.0 - theta)) / (1.0 - self.zeta2 / self.zetan)

    def sample(self, rng: np.random.Generator, size: int) -> np.ndarray:
        u = rng.random(size)
        uz = u * self.zetan
        r = np.floor(self.n * (self.eta * u - self.eta + 1.0) ** self.alpha)
        r = np.where(uz < 1.0 + 0.5 ** self.theta, 1.0, r)
        r = np.where(uz < 1.0, 0.0, r)
        return np.minimum(r, self.n - 1).astype(np.uint64)


def op_stream(n_records: int, n_ops: int, val_bytes: int, seed: int, get_frac=0.5,
              del_frac=0.0, absent_frac=0.0, zipf_theta=None, return_index=False):
    """An operation stream over an n_records map.

    Returns (ops uint8[n], keys uint64[n], vals_in uint8[n, val_bytes]).
    Keys are existing records drawn uniformly or Zipf-skewed (popular ranks are
    scattered over the key space by the mixer), with `absent_frac` of them
    replaced by keys that were never inserted; ops are GET with probability
    `get_frac`, DEL with `del_frac`, else PUT.  With return_index, the record
    index of each op's key (key = key_of(index)) is returned fourth.
    """
    rng = np.random.default_rng(seed)
    if zipf_theta is None:
        idx = rng.integers(0, n_records, size=n_ops, dtype=np.uint64)
    else:
        ranks = Zipf(n_records, zipf_theta).sample(rng, n_ops)
        idx = mix64(ranks) % np.uint64(n_records)
    absent = rng.random(n_ops) < absent_frac
    idx = np.where(absent, np.uint64(n_records) + rng.integers(0, 1 << 40, size=n_ops,
                                                                dtype=np.uint64), idx)
    keys = key_of(idx)
    u = rng.random(n_ops)
    ops = np.where(u < get_frac, GET, np.where(u < get_frac + del_frac, DEL, PUT))
    ops = ops.astype(np.uint8)
    vals = rng.integers(0, 256, size=(n_ops, val_bytes), dtype=np.uint8)
    if return_index:
        return ops, keys, vals, idx
    return ops, keys, vals
