"""ctypes binding of libbolt.so (the C ABI declared in include/bolt.h).

Argument marshalling only: every step of the build and of the access path runs
in the library's CUDA kernels.  Host-pointer calls take numpy arrays;
device-pointer calls take torch CUDA tensors (PyTorch is used for device
memory and streams only).  Importing this module loads the in-tree library and
raises if it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbolt.so")

BOLT_OK, BOLT_E_ARG, BOLT_E_NOMEM, BOLT_E_OVERFLOW = 0, -1, -2, -3
BOLT_E_STATE, BOLT_E_DUPKEY, BOLT_E_CUDA, BOLT_E_TIMEOUT, BOLT_E_INTERNAL = -4, -5, -6, -7, -9
BOLT_E_INTEGRITY = -8
BOLT_GET, BOLT_PUT, BOLT_DEL = 0, 1, 2
BOLT_MAX_BATCH = 65536
BOLT_NOALLOC_SCRATCH_BYTES = 7340800
BOLT_PARAM_ALPHA, BOLT_PARAM_C, BOLT_PARAM_TRACE, BOLT_PARAM_BATCH = 1, 2, 4, 5
BOLT_PARAM_TRACE_CAP, BOLT_PARAM_CHECK_KEYS, BOLT_PARAM_PROFILE = 6, 7, 8
BOLT_PARAM_BATCH_CAP, BOLT_PARAM_LOOKAHEAD, BOLT_PARAM_DEFER_FLUSH = 9, 10, 11
BOLT_PARAM_SPIN_LIMIT, BOLT_PARAM_FUSED, BOLT_PARAM_INTEGRITY = 12, 13, 14
BOLT_PARAM_ROUNDS_PRF = 15
BOLT_PROF_CLASSES = 19
PROF_NAMES = ("sort_global", "sort_tile", "page_build", "p2c_rounds", "key_check",
              "access_batch", "gather", "evict", "build", "group", "ksort_global",
              "ksort_tile", "flush", "ahead", "page_group", "pages", "find_exec", "remap",
              "stage")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2509_01742_b300.build_ext` (no CPU fallback exists)")
_lib = ctypes.CDLL(LIB_PATH)


class bolt_info_t(ctypes.Structure):
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


class bolt_stats_t(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_uint64), ("n_hbm", ctypes.c_uint64),
                ("n_stash", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("trace_len", ctypes.c_uint64), ("max_load", ctypes.c_uint32),
                ("max_row", ctypes.c_uint32), ("peak_hbm", ctypes.c_uint64),
                ("peak_stash", ctypes.c_uint64), ("peak_load", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class bolt_profile_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("spans", ctypes.c_uint64 * BOLT_PROF_CLASSES),
                ("ms", ctypes.c_double * BOLT_PROF_CLASSES)]


class bolt_tune_t(ctypes.Structure):
    _fields_ = [("sort_log_tile", ctypes.c_uint32), ("batch_width", ctypes.c_uint32),
                ("sort_ms", ctypes.c_double * 2), ("widths", ctypes.c_uint32 * 6),
                ("width_us", ctypes.c_double * 6)]


class bolt_image_t(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("pairs", ctypes.c_void_p),
                ("rows", ctypes.c_void_p), ("counts", ctypes.c_void_p)]


class bolt_req_info_t(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("map", ctypes.c_uint32), ("n", ctypes.c_uint32),
                ("rc", ctypes.c_int), ("submit_us", ctypes.c_double),
                ("start_us", ctypes.c_double), ("done_us", ctypes.c_double)]


class bolt_server_stats_t(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_uint64), ("used", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("ops", ctypes.c_uint64),
                ("maps_pending", ctypes.c_uint32), ("maps_ready", ctypes.c_uint32),
                ("queued", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P, _u64, _u32, _i = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_SIGS = {
    "bolt_create": ([_u64, _u32, _u32, _u64, ctypes.POINTER(_P)], _i),
    "bolt_plan": ([_u64, _u32, _u32, _u64, ctypes.c_double, _u32, ctypes.POINTER(bolt_info_t)], _i),
    "bolt_set_param": ([_P, _i, ctypes.c_double], _i),
    "bolt_init": ([_P, _P, _P, _u64, _u64], _i),
    "bolt_init_device": ([_P, _P, _P, _u64, _u64, _P], _i),
    "bolt_init_device_noalloc": ([_P, _P, _P, _u64, _u64, _P], _i),
    "bolt_prepare_device": ([_P, _P, _P, _u64, _u64, ctypes.POINTER(bolt_image_t), _P], _i),
    "bolt_init_prepared": ([_P, ctypes.POINTER(bolt_image_t), _u64, _u64, _P], _i),
    "bolt_access": ([_P, _P, _P, _P, _P, _P, _u64], _i),
    "bolt_access_device": ([_P, _P, _P, _P, _P, _P, _u64, _P], _i),
    "bolt_access_device_batches": ([_P, _P, _P, _P, _P, _P, _u64, ctypes.c_uint32, _P], _i),
    "bolt_sync": ([_P], _i),
    "bolt_probe_link": ([_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double)], _i),
    "bolt_destroy": ([_P], _i),
    "bolt_get_info": ([_P, ctypes.POINTER(bolt_info_t)], _i),
    "bolt_get_stats": ([_P, ctypes.POINTER(bolt_stats_t)], _i),
    "bolt_read_pages": ([_P, _u64, _u64, _P], _i),
    "bolt_write_pages": ([_P, _u64, _u64, _P], _i),
    "bolt_read_trace": ([_P, _P, _u64, ctypes.POINTER(_u64)], _i),
    "bolt_read_loads": ([_P, _P], _i),
    "bolt_read_rowcounts": ([_P, _P], _i),
    "bolt_read_profile": ([_P, ctypes.POINTER(bolt_profile_t), _i], _i),
    "bolt_trim": ([_P], _i),
    "bolt_autotune": ([_P, _P, _u64, ctypes.c_double, ctypes.POINTER(bolt_tune_t)], _i),
    "bolt_footprint": ([_P, ctypes.POINTER(_u64), ctypes.POINTER(_u64)], _i),
    "bolt_plan_bytes": ([_u64, _u32, _u64, _u32, _u64, ctypes.POINTER(_u64),
                         ctypes.POINTER(_u64)], _i),
    "bolt_server_create": ([_u64, _u32, ctypes.POINTER(_P)], _i),
    "bolt_server_add_map": ([_P, _u64, _u32, _P, _P, _u64, _u64, ctypes.POINTER(_u32)], _i),
    "bolt_server_map_state": ([_P, _u32], _i),
    "bolt_server_remove_map": ([_P, _u32], _i),
    "bolt_server_submit": ([_P, _u32, _P, _P, _P, _u32, ctypes.POINTER(_u64)], _i),
    "bolt_server_submit_many": ([_P, _u32, _P, _P, _P, _P, _P, _P], _i),
    "bolt_server_wait": ([_P, _u64, _P, _P, ctypes.POINTER(bolt_req_info_t), _i], _i),
    "bolt_server_map_batches": ([_P, _u32, _P, _u64, ctypes.POINTER(_u64)], _i),
    "bolt_server_map_handle": ([_P, _u32, ctypes.POINTER(_P)], _i),
    "bolt_server_stats": ([_P, ctypes.POINTER(bolt_server_stats_t)], _i),
    "bolt_server_destroy": ([_P], _i),
    "bolt_strerror": ([_i], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class BoltError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"{what}: {bolt_strerror(rc).decode()} ({rc})")
        self.rc = rc


def _check(rc: int, what: str) -> int:
    if rc != BOLT_OK:
        raise BoltError(rc, what)
    return rc


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def plan(N: int, val_bytes: int, hbm_budget: int = 2**64 - 1, alpha: float = -1.0,
         c: int = 8, key_bytes: int = 8) -> dict:
    o = bolt_info_t()
    _check(bolt_plan(N, key_bytes, val_bytes, hbm_budget, alpha, c, ctypes.byref(o)),
           "bolt_plan")
    return o.as_dict()


class BoltMap:
    """One oblivious map handle (owns its device state and pinned pages)."""

    def __init__(self, N: int, val_bytes: int, hbm_budget: int = 2**64 - 1, alpha=None,
                 c=None, trace: bool = False, batch=None, check_keys=None, key_bytes: int = 8,
                 integrity: bool = False):
        self._h = ctypes.c_void_p()
        _check(bolt_create(N, key_bytes, val_bytes, hbm_budget, ctypes.byref(self._h)),
               "bolt_create")
        self.vb = val_bytes
        # host-pointer calls take keys of this width (device calls take uint64)
        self._kdt = np.uint32 if key_bytes == 4 else np.uint64
        if c is not None:
            self.set_param(BOLT_PARAM_C, c)
        if integrity:
            self.set_param(BOLT_PARAM_INTEGRITY, 1)
        if alpha is not None:
            self.set_param(BOLT_PARAM_ALPHA, alpha)
        if trace:
            self.set_param(BOLT_PARAM_TRACE, 1)
        if batch is not None:
            self.set_param(BOLT_PARAM_BATCH, batch)
        if check_keys is not None:
            self.set_param(BOLT_PARAM_CHECK_KEYS, int(check_keys))

    def _keys(self, keys):
        keys = np.asarray(keys)
        if self._kdt is np.uint32 and keys.dtype.itemsize > 4 and keys.size and \
                int(keys.max()) > 0xFFFFFFFF:
            raise ValueError("a map of 4-byte keys takes keys below 2^32")
        return np.ascontiguousarray(keys, dtype=self._kdt)

    def set_param(self, which: int, value: float):
        _check(bolt_set_param(self._h, which, float(value)), "bolt_set_param")

    def close(self):
        if self._h:
            bolt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        o = bolt_info_t()
        _check(bolt_get_info(self._h, ctypes.byref(o)), "bolt_get_info")
        return o.as_dict()

    def stats(self) -> dict:
        s = bolt_stats_t()
        _check(bolt_get_stats(self._h, ctypes.byref(s)), "bolt_get_stats")
        return s.as_dict()

    # --- host-pointer calls ------------------------------------------------
    def init(self, keys: np.ndarray, vals: np.ndarray, seed: int) -> int:
        keys = self._keys(keys)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        if vals.size != len(keys) * self.vb:
            raise ValueError(f"{len(keys)} keys need {len(keys) * self.vb} value bytes")
        return bolt_init(self._h, _np_ptr(keys), _np_ptr(vals), len(keys), seed)

    def access(self, ops, keys, vals_in):
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = self._keys(keys)
        vin = np.ascontiguousarray(vals_in, dtype=np.uint8)
        n = len(ops)
        if len(keys) != n or vin.size != n * self.vb:
            raise ValueError(f"array sizes do not match {n} ops of {self.vb}-byte values")
        vout = np.zeros((n, self.vb), dtype=np.uint8)
        status = np.zeros(n, dtype=np.uint8)
        rc = bolt_access(self._h, _np_ptr(ops), _np_ptr(keys), _np_ptr(vin), _np_ptr(vout),
                         _np_ptr(status), n)
        return rc, vout, status

    # --- device-pointer calls (torch CUDA tensors) --------------------------
    def init_device(self, keys, vals, seed: int, stream=None) -> int:
        if keys.element_size() != 8 or vals.element_size() != 1 or \
                vals.numel() != keys.numel() * self.vb:
            raise ValueError("keys must be 8-byte, values uint8 of n * val_bytes")
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        return bolt_init_device(self._h, ctypes.c_void_p(keys.data_ptr()),
                                ctypes.c_void_p(vals.data_ptr()), keys.numel(), seed, s)

    def _image(self, img: dict):
        return bolt_image_t(*(ctypes.c_void_p(img[k].data_ptr())
                              for k in ("keys", "vals", "pairs", "rows", "counts")))

    def prepare_device(self, keys, vals, seed: int, stream=None):
        """bolt_prepare_device: build the map from device tensors and return
        (rc, image) with the image's arrays as device tensors (keys, vals,
        pairs, rows, counts)."""
        import torch
        n = keys.numel()
        img = {"keys": torch.empty(n, dtype=torch.int64, device=keys.device),
               "vals": torch.empty((n, self.vb), dtype=torch.uint8, device=keys.device),
               "pairs": torch.empty(n, dtype=torch.int64, device=keys.device),
               "rows": torch.empty(n, dtype=torch.int32, device=keys.device),
               "counts": torch.empty(self.info()["B"], dtype=torch.uint8, device=keys.device)}
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        rc = bolt_prepare_device(self._h, ctypes.c_void_p(keys.data_ptr()),
                                 ctypes.c_void_p(vals.data_ptr()), n, seed,
                                 ctypes.byref(self._image(img)), s)
        return rc, img

    def init_prepared(self, img: dict, n: int, seed: int, stream=None) -> int:
        """bolt_init_prepared from an image of device tensors."""
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        return bolt_init_prepared(self._h, ctypes.byref(self._image(img)), n, seed, s)

    def _check_io(self, ops, keys, vals_in, vals_out, status):
        n = ops.numel()
        vb = self.vb
        if keys.numel() != n or vals_in.numel() != n * vb or vals_out.numel() != n * vb or \
                (status is not None and status.numel() != n):
            raise ValueError(f"array sizes do not match {n} ops of {vb}-byte values")
        if ops.element_size() != 1 or keys.element_size() != 8 or \
                vals_in.element_size() != 1 or vals_out.element_size() != 1 or \
                (status is not None and status.element_size() != 1):
            raise ValueError("ops, values and status are bytes; keys are 8-byte integers")
        for t in (ops, keys, vals_in, vals_out) + ((status,) if status is not None else ()):
            if not t.is_contiguous():
                raise ValueError("arrays must be contiguous")

    def access_device(self, ops, keys, vals_in, vals_out, status=None, stream=None) -> int:
        self._check_io(ops, keys, vals_in, vals_out, status)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        st = ctypes.c_void_p(status.data_ptr()) if status is not None else ctypes.c_void_p(0)
        return bolt_access_device(self._h, ctypes.c_void_p(ops.data_ptr()),
                                  ctypes.c_void_p(keys.data_ptr()),
                                  ctypes.c_void_p(vals_in.data_ptr()),
                                  ctypes.c_void_p(vals_out.data_ptr()), st, ops.numel(), s)

    def access_device_batches(self, ops, keys, vals_in, vals_out, status, width: int = 0,
                              stream=None) -> int:
        """Consecutive batches of `width` ops over device tensors (one call)."""
        self._check_io(ops, keys, vals_in, vals_out, status)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        return bolt_access_device_batches(self._h, ctypes.c_void_p(ops.data_ptr()),
                                          ctypes.c_void_p(keys.data_ptr()),
                                          ctypes.c_void_p(vals_in.data_ptr()),
                                          ctypes.c_void_p(vals_out.data_ptr()),
                                          ctypes.c_void_p(status.data_ptr()), ops.numel(),
                                          width, s)

    def sync(self) -> int:
        return bolt_sync(self._h)

    def probe_link(self, pages: int, launches: int = 50) -> dict:
        """Random-page zero-copy read rate, and the read + previous-set write-back
        rate, over this map's own pinned pages."""
        r, w = ctypes.c_double(), ctypes.c_double()
        _check(bolt_probe_link(self._h, pages, launches, ctypes.byref(r), ctypes.byref(w)),
               "bolt_probe_link")
        return {"read_pages_per_s": r.value, "pipelined_pages_per_s": w.value}

    # --- inspection ----------------------------------------------------------
    def pages(self, first: int = 0, count=None) -> np.ndarray:
        i = self.info()
        count = i["M"] - first if count is None else count
        out = np.zeros((count, i["page_bytes"]), dtype=np.uint8)
        _check(bolt_read_pages(self._h, first, count, _np_ptr(out)), "bolt_read_pages")
        return out

    def write_pages(self, first: int, pages: np.ndarray):
        """Overwrite host pages (the untrusted host's own move)."""
        pages = np.ascontiguousarray(pages, dtype=np.uint8)
        i = self.info()
        if pages.ndim != 2 or pages.shape[1] != i["page_bytes"]:
            raise ValueError("pages must be (count, page_bytes) bytes")
        _check(bolt_write_pages(self._h, first, pages.shape[0], _np_ptr(pages)),
               "bolt_write_pages")

    def trace(self, cap: int = 1 << 24) -> np.ndarray:
        out = np.zeros(cap, dtype=np.uint32)
        n = ctypes.c_uint64()
        _check(bolt_read_trace(self._h, _np_ptr(out), cap, ctypes.byref(n)), "bolt_read_trace")
        if n.value > cap:
            raise BoltError(BOLT_E_ARG, f"trace overflow ({n.value} > {cap})")
        return out[:n.value].copy()

    def profile(self, reset: bool = True) -> dict:
        p = bolt_profile_t()
        _check(bolt_read_profile(self._h, ctypes.byref(p), int(reset)), "bolt_read_profile")
        out = {"launches": int(p.launches)}
        for c, name in enumerate(PROF_NAMES):
            out[name] = {"spans": int(p.spans[c]), "ms": float(p.ms[c])}
        return out

    def autotune(self, sample_keys=None, max_batch_us: float = 0.0) -> dict:
        t = bolt_tune_t()
        if sample_keys is not None:
            sk = self._keys(sample_keys)
            rc = bolt_autotune(self._h, _np_ptr(sk), len(sk), max_batch_us, ctypes.byref(t))
        else:
            rc = bolt_autotune(self._h, None, 0, max_batch_us, ctypes.byref(t))
        _check(rc, "bolt_autotune")
        return {"sort_log_tile": t.sort_log_tile, "batch_width": t.batch_width,
                "sort_ms": list(t.sort_ms), "widths": list(t.widths),
                "width_us": list(t.width_us)}

    def footprint(self):
        r, s = ctypes.c_uint64(), ctypes.c_uint64()
        _check(bolt_footprint(self._h, ctypes.byref(r), ctypes.byref(s)), "bolt_footprint")
        return r.value, s.value

    def loads(self) -> np.ndarray:
        out = np.zeros(self.info()["B"], dtype=np.uint8)
        _check(bolt_read_loads(self._h, _np_ptr(out)), "bolt_read_loads")
        return out

    def rowcounts(self) -> np.ndarray:
        out = np.zeros(self.info()["rows"], dtype=np.uint8)
        _check(bolt_read_rowcounts(self._h, _np_ptr(out)), "bolt_read_rowcounts")
        return out


def plan_bytes(N: int, val_bytes: int, batch_cap: int = BOLT_MAX_BATCH, n_init: int = 0,
               hbm_budget: int = 2**64 - 1):
    r, s = ctypes.c_uint64(), ctypes.c_uint64()
    _check(bolt_plan_bytes(N, val_bytes, hbm_budget, batch_cap, n_init, ctypes.byref(r),
                           ctypes.byref(s)), "bolt_plan_bytes")
    return r.value, s.value


class BoltServer:
    """Continuous-batching server over many maps (bolt_server_* calls)."""

    def __init__(self, hbm_budget: int, max_batch: int = 4096):
        self._s = ctypes.c_void_p()
        _check(bolt_server_create(hbm_budget, max_batch, ctypes.byref(self._s)),
               "bolt_server_create")
        self.max_batch = max_batch
        self.vb = {}

    def close(self):
        if self._s:
            bolt_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_map(self, N: int, val_bytes: int, keys, vals, seed: int) -> int:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vals = np.ascontiguousarray(vals, dtype=np.uint8)
        mid = ctypes.c_uint32()
        _check(bolt_server_add_map(self._s, N, val_bytes, _np_ptr(keys), _np_ptr(vals),
                                   len(keys), seed, ctypes.byref(mid)), "bolt_server_add_map")
        self.vb[mid.value] = val_bytes
        return mid.value

    def map_state(self, mid: int) -> int:
        return bolt_server_map_state(self._s, mid)

    def remove_map(self, mid: int):
        _check(bolt_server_remove_map(self._s, mid), "bolt_server_remove_map")

    def submit(self, mid: int, ops, keys, vals_in) -> int:
        ops = np.ascontiguousarray(ops, dtype=np.uint8)
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        vin = np.ascontiguousarray(vals_in, dtype=np.uint8)
        rid = ctypes.c_uint64()
        _check(bolt_server_submit(self._s, mid, _np_ptr(ops), _np_ptr(keys), _np_ptr(vin),
                                  len(ops), ctypes.byref(rid)), "bolt_server_submit")
        return rid.value

    def submit_many(self, reqs) -> list:
        """Queue several requests in one call: reqs = [(map id, ops, keys,
        vals_in), ...]; returns their ids."""
        arrs = []
        for mid, ops, keys, vin in reqs:
            arrs.append((mid, np.ascontiguousarray(ops, dtype=np.uint8),
                         np.ascontiguousarray(keys, dtype=np.uint64),
                         np.ascontiguousarray(vin, dtype=np.uint8)))
        c = len(arrs)
        mids = np.array([a[0] for a in arrs], dtype=np.uint32)
        ns = np.array([len(a[1]) for a in arrs], dtype=np.uint32)
        P = ctypes.c_void_p * max(c, 1)
        po = P(*[a[1].ctypes.data for a in arrs])
        pk = P(*[a[2].ctypes.data for a in arrs])
        pv = P(*[a[3].ctypes.data for a in arrs])
        ids = np.zeros(max(c, 1), dtype=np.uint64)
        _check(bolt_server_submit_many(self._s, c, _np_ptr(mids), po, pk, pv, _np_ptr(ns),
                                       _np_ptr(ids)), "bolt_server_submit_many")
        return [int(x) for x in ids[:c]]

    def wait(self, rid: int, n: int, mid: int, timeout_ms: int = -1):
        vout = np.zeros((n, self.vb[mid]), dtype=np.uint8)
        status = np.zeros(n, dtype=np.uint8)
        info = bolt_req_info_t()
        rc = bolt_server_wait(self._s, rid, _np_ptr(vout), _np_ptr(status), ctypes.byref(info),
                              timeout_ms)
        return rc, vout, status, info

    def batches(self, mid: int) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(bolt_server_map_batches(self._s, mid, None, 0, ctypes.byref(cnt)), "batches")
        out = np.zeros(max(1, cnt.value), dtype=np.uint32)
        _check(bolt_server_map_batches(self._s, mid, _np_ptr(out), cnt.value, ctypes.byref(cnt)),
               "batches")
        return out[:cnt.value]

    def map_pages(self, mid: int) -> np.ndarray:
        h = ctypes.c_void_p()
        _check(bolt_server_map_handle(self._s, mid, ctypes.byref(h)), "bolt_server_map_handle")
        o = bolt_info_t()
        _check(bolt_get_info(h, ctypes.byref(o)), "bolt_get_info")
        out = np.zeros((o.M, o.page_bytes), dtype=np.uint8)
        _check(bolt_read_pages(h, 0, o.M, _np_ptr(out)), "bolt_read_pages")
        return out

    def _map_handle(self, mid: int):
        h = ctypes.c_void_p()
        _check(bolt_server_map_handle(self._s, mid, ctypes.byref(h)), "bolt_server_map_handle")
        return h

    def map_stats(self, mid: int) -> dict:
        """bolt_get_stats of a ready map (the server must be quiescent)."""
        s = bolt_stats_t()
        _check(bolt_get_stats(self._map_handle(mid), ctypes.byref(s)), "bolt_get_stats")
        return s.as_dict()

    def map_loads(self, mid: int) -> np.ndarray:
        h = self._map_handle(mid)
        o = bolt_info_t()
        _check(bolt_get_info(h, ctypes.byref(o)), "bolt_get_info")
        out = np.zeros(o.B, dtype=np.uint8)
        _check(bolt_read_loads(h, _np_ptr(out)), "bolt_read_loads")
        return out

    def stats(self) -> dict:
        s = bolt_server_stats_t()
        _check(bolt_server_stats(self._s, ctypes.byref(s)), "bolt_server_stats")
        return s.as_dict()
