"""ctypes binding of the CPU oracle (oracle/bolt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the
CPU-baseline leg of bench.py -- never by the product package.  The oracle is a
plain single-threaded C implementation of the BOLT oblivious map (Alg. 1,
Sec. 3.1; architecture Sec. 4.1-4.2) that shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
OMP_LIB_PATH = os.path.join(HERE, "liboracle_omp.so")
SRC_PATH = os.path.join(HERE, "bolt_oracle.c")

PARAM_ALPHA, PARAM_C, PARAM_NOCRYPT, PARAM_TRACE, PARAM_BATCH = 1, 2, 3, 4, 5
PARAM_INTEGRITY = 6
OK, E_ARG, E_NOMEM, E_OVERFLOW, E_STATE, E_DUPKEY = 0, -1, -2, -3, -4, -5
E_INTEGRITY = -8
GET, PUT, DEL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler: oracle/liboracle.so
    (single-threaded, the oracle proper) and oracle/liboracle_omp.so (the
    same source with OpenMP on: its independent loops run on all host cores,
    the multi-core CPU baseline)."""
    hdr = os.path.join(HERE, "bolt_oracle.h")
    for path, extra in ((LIB_PATH, ["-Wno-unknown-pragmas"]), (OMP_LIB_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < max(
                os.path.getmtime(SRC_PATH), os.path.getmtime(hdr)):
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", *extra, "-shared", "-fPIC",
                                   "-o", path, SRC_PATH, "-lm"])
    return LIB_PATH


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint64), ("B", ctypes.c_uint64), ("K", ctypes.c_uint64),
                ("M", ctypes.c_uint64), ("rows", ctypes.c_uint64),
                ("key_bytes", ctypes.c_uint32), ("val_bytes", ctypes.c_uint32),
                ("c", ctypes.c_uint32), ("d", ctypes.c_uint32), ("lmax", ctypes.c_uint32),
                ("R", ctypes.c_uint32), ("page_bytes", ctypes.c_uint32),
                ("rec_bytes", ctypes.c_uint32), ("round_width", ctypes.c_uint64),
                ("vs_cap", ctypes.c_uint64), ("alpha", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_uint64), ("n_hbm", ctypes.c_uint64),
                ("n_stash", ctypes.c_uint64), ("n_host", ctypes.c_uint64),
                ("peak_stash", ctypes.c_uint64), ("peak_hbm", ctypes.c_uint64),
                ("max_load", ctypes.c_uint32), ("peak_load", ctypes.c_uint32),
                ("max_row", ctypes.c_uint32), ("pad", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


_lib = None
_omp_lib = None


def omp_lib():
    """The OpenMP build (multi-core CPU baseline): same entry points."""
    global _omp_lib
    if _omp_lib is None:
        lib()
        _omp_lib = _bind_all(ctypes.CDLL(OMP_LIB_PATH))
    return _omp_lib


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _bind_all(ctypes.CDLL(LIB_PATH))
    return _lib


def _bind_all(L):
    """ctypes signatures of the oracle's entry points."""
    if L is not None:
        P, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.oracle_create.argtypes = [u64, u32, u32, u64, ctypes.POINTER(P)]
        L.oracle_set_param.argtypes = [P, i32, ctypes.c_double]
        L.oracle_init.argtypes = [P, P, P, u64, u64]
        L.oracle_access.argtypes = [P, P, P, P, P, P, u64]
        L.oracle_destroy.argtypes = [P]
        L.oracle_destroy.restype = None
        L.oracle_info.argtypes = [P, ctypes.POINTER(Info)]
        L.oracle_stats.argtypes = [P, ctypes.POINTER(Stats)]
        L.oracle_pages.argtypes = [P]
        L.oracle_pages.restype = P
        L.oracle_loads.argtypes = [P, P]
        L.oracle_versions.argtypes = [P, P]
        L.oracle_rowcounts.argtypes = [P, P]
        L.oracle_trace_len.argtypes = [P]
        L.oracle_trace_len.restype = u64
        L.oracle_trace_copy.argtypes = [P, P, u64]
        L.oracle_trace_copy.restype = u64
        L.oracle_trace_clear.argtypes = [P]
        L.oracle_trace_clear.restype = None
        L.oracle_decrypt_page.argtypes = [P, u64, P]
        L.oracle_keys.argtypes = [P, P, P]
        L.oracle_chacha20_block.argtypes = [P, u32, P, P]
        L.oracle_chacha20_block.restype = None
        L.oracle_chacha20_xor.argtypes = [P, u32, P, P, u64]
        L.oracle_chacha20_xor.restype = None
        L.oracle_sizing.argtypes = [u64, u32, ctypes.c_double, u32, ctypes.POINTER(Info)]
        L.oracle_pair.argtypes = [P, u32, u64, u64, ctypes.POINTER(u32), ctypes.POINTER(u32)]
        L.oracle_kdf.argtypes = [u64, P, P]
        L.oracle_kdf.restype = None
        L.oracle_page_decrypt.argtypes = [P, u64, u64, P, P, u64]
        L.oracle_page_decrypt.restype = None
        L.oracle_threads.argtypes = [i32]
        L.oracle_prepare.argtypes = [P, P, P, u64, u64, P, P, P, P, P]
        L.oracle_poly1305.argtypes = [P, P, u64, P]
        L.oracle_poly1305.restype = None
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def chacha20_block(key_words, counter, nonce_words) -> np.ndarray:
    k = np.ascontiguousarray(key_words, dtype=np.uint32)
    nn = np.ascontiguousarray(nonce_words, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    lib().oracle_chacha20_block(_ptr(k), counter, _ptr(nn), _ptr(out))
    return out


def chacha20_xor(key_words, counter, nonce_words, data: bytes) -> bytes:
    k = np.ascontiguousarray(key_words, dtype=np.uint32)
    nn = np.ascontiguousarray(nonce_words, dtype=np.uint32)
    buf = np.frombuffer(bytearray(data), dtype=np.uint8).copy()
    lib().oracle_chacha20_xor(_ptr(k), counter, _ptr(nn), _ptr(buf), len(buf))
    return buf.tobytes()


def poly1305(key: bytes, msg: bytes) -> bytes:
    """The oracle's Poly1305 tag of msg under a 32-byte one-time key."""
    k = np.frombuffer(bytes(key), dtype=np.uint8).copy()
    mm = np.frombuffer(bytes(msg) + b"\0", dtype=np.uint8).copy()
    tag = np.zeros(16, dtype=np.uint8)
    lib().oracle_poly1305(_ptr(k), _ptr(mm), len(msg), _ptr(tag))
    return tag.tobytes()


def sizing(N: int, c: int, alpha: float, val_bytes: int) -> dict:
    o = Info()
    rc = lib().oracle_sizing(N, c, alpha, val_bytes, ctypes.byref(o))
    if rc:
        raise ValueError(f"oracle_sizing rc={rc}")
    return o.as_dict()


def kdf(seed: int):
    """(K_prf, K_enc) derived from a map seed, 8 uint32 words each."""
    kprf = np.zeros(8, dtype=np.uint32)
    kenc = np.zeros(8, dtype=np.uint32)
    lib().oracle_kdf(seed, _ptr(kprf), _ptr(kenc))
    return kprf, kenc


def page_decrypt(kenc_words, q: int, version: int, ciphertext: np.ndarray) -> np.ndarray:
    """Plaintext of page q's ciphertext at `version` under K_enc."""
    k = np.ascontiguousarray(kenc_words, dtype=np.uint32)
    c = np.ascontiguousarray(ciphertext, dtype=np.uint8)
    out = np.empty_like(c)
    lib().oracle_page_decrypt(_ptr(k), q, version, _ptr(c), _ptr(out), c.size)
    return out


def pair(kprf_words, dom: int, x: int, B: int):
    k = np.ascontiguousarray(kprf_words, dtype=np.uint32)
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib().oracle_pair(_ptr(k), dom, x, B, ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise ValueError(rc)
    return a.value, b.value


def threads(n: int = 0) -> int:
    """Threads the OpenMP build uses (n > 0 sets them)."""
    return omp_lib().oracle_threads(n)


class OracleError(RuntimeError):
    def __init__(self, rc, what):
        super().__init__(f"{what} failed rc={rc}")
        self.rc = rc


class OracleMap:
    """One oracle map instance (same call shapes as the product C ABI)."""

    def __init__(self, N, val_bytes, hbm_budget=2**64 - 1, key_bytes=8, alpha=None,
                 c=None, nocrypt=False, trace=True, batch=None, omp=False, integrity=False):
        """omp=True runs the same oracle from its OpenMP build (independent
        loops on all host cores; results identical to the plain build)."""
        self._L = omp_lib() if omp else lib()
        self._h = ctypes.c_void_p()
        rc = self._L.oracle_create(N, key_bytes, val_bytes, hbm_budget, ctypes.byref(self._h))
        if rc:
            raise OracleError(rc, "oracle_create")
        if c is not None:
            self.set_param(PARAM_C, c)
        if alpha is not None:
            self.set_param(PARAM_ALPHA, alpha)
        if integrity:
            self.set_param(PARAM_INTEGRITY, 1)
        if nocrypt:
            self.set_param(PARAM_NOCRYPT, 1)
        if not trace:
            self.set_param(PARAM_TRACE, 0)
        if batch is not None:
            self.set_param(PARAM_BATCH, batch)
        self.vb = val_bytes

    def set_param(self, which, v):
        rc = self._L.oracle_set_param(self._h, which, float(v))
        if rc:
            raise OracleError(rc, "oracle_set_param")

    def close(self):
        if self._h:
            self._L.oracle_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, keys: np.ndarray, vals: np.ndarray, seed: int) -> int:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        return self._L.oracle_init(self._h, _ptr(keys), _ptr(vals), len(keys), seed)

    def prepare(self, keys: np.ndarray, vals: np.ndarray, seed: int):
        """The data owner's bin-major image of this map's placement (and the
        map built as by init): (rc, dict of keys, vals, pairs, rows, counts)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        n = len(keys)
        img = {"keys": np.zeros(n, np.uint64), "vals": np.zeros((n, self.vb), np.uint8),
               "pairs": np.zeros(n, np.uint64), "rows": np.zeros(n, np.uint32),
               "counts": np.zeros(self.info()["B"], np.uint8)}
        rc = self._L.oracle_prepare(self._h, _ptr(keys), _ptr(vals), n, seed, _ptr(img["keys"]),
                                    _ptr(img["vals"]), _ptr(img["pairs"]), _ptr(img["rows"]),
                                    _ptr(img["counts"]))
        return rc, img

    def access(self, ops, keys, vals_in):
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vin = np.ascontiguousarray(vals_in, dtype=np.uint8)
        n = len(ops)
        vout = np.zeros((n, self.vb), dtype=np.uint8)
        status = np.zeros(n, dtype=np.uint8)
        rc = self._L.oracle_access(self._h, _ptr(ops), _ptr(keys), _ptr(vin), _ptr(vout),
                                 _ptr(status), n)
        return rc, vout, status

    def info(self) -> dict:
        o = Info()
        self._L.oracle_info(self._h, ctypes.byref(o))
        return o.as_dict()

    def stats(self) -> dict:
        s = Stats()
        self._L.oracle_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def pages(self) -> np.ndarray:
        i = self.info()
        size = i["M"] * i["page_bytes"]
        addr = self._L.oracle_pages(self._h)
        buf = (ctypes.c_uint8 * size).from_address(addr)
        return np.frombuffer(buf, dtype=np.uint8).copy().reshape(i["M"], i["page_bytes"])

    def loads(self) -> np.ndarray:
        out = np.zeros(self.info()["B"], dtype=np.uint8)
        self._L.oracle_loads(self._h, _ptr(out))
        return out

    def versions(self) -> np.ndarray:
        out = np.zeros(self.info()["M"], dtype=np.uint64)
        self._L.oracle_versions(self._h, _ptr(out))
        return out

    def rowcounts(self) -> np.ndarray:
        out = np.zeros(self.info()["rows"], dtype=np.uint32)
        self._L.oracle_rowcounts(self._h, _ptr(out))
        return out

    def trace(self, clear=True) -> np.ndarray:
        n = self._L.oracle_trace_len(self._h)
        out = np.zeros(n, dtype=np.uint32)
        self._L.oracle_trace_copy(self._h, _ptr(out), n)
        if clear:
            self._L.oracle_trace_clear(self._h)
        return out

    def host_pages(self):
        """The host page store itself (writable: a test standing in for a
        host that alters or replays pages)."""
        i = self.info()
        size = i["M"] * i["page_bytes"]
        addr = self._L.oracle_pages(self._h)
        buf = (ctypes.c_uint8 * size).from_address(addr)
        return np.frombuffer(buf, dtype=np.uint8).reshape(i["M"], i["page_bytes"])

    def decrypt_page(self, q) -> np.ndarray:
        out = np.zeros(self.info()["page_bytes"], dtype=np.uint8)
        rc = self._L.oracle_decrypt_page(self._h, q, _ptr(out))
        if rc:
            raise OracleError(rc, "oracle_decrypt_page")
        return out

    def keys(self):
        a = np.zeros(8, dtype=np.uint32)
        b = np.zeros(8, dtype=np.uint32)
        rc = self._L.oracle_keys(self._h, _ptr(a), _ptr(b))
        if rc:
            raise OracleError(rc, "oracle_keys")
        return a, b
