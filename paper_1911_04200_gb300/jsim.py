"""Thin ctypes binding of the jsim C-ABI (include/jsim.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (its caching allocator, through the
library's allocator hooks) and the CUDA stream.  There is no CPU fallback:
if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_native

JSIM_OK = 0
ERRORS = {1: "JSIM_ERR_ARG", 2: "JSIM_ERR_UNSORTED", 3: "JSIM_ERR_OVERFLOW", 4: "JSIM_ERR_ID_RANGE",
          5: "JSIM_ERR_OOM", 6: "JSIM_ERR_CUDA", 7: "JSIM_ERR_TIMEOUT", 8: "JSIM_ERR_CANCELLED",
          9: "JSIM_ERR_UNSUPPORTED", 10: "JSIM_ERR_INCOMPLETE", 11: "JSIM_ERR_CHECKPOINT"}
MEM_HOST, MEM_DEVICE = 0, 1
VARIANTS = {"auto": 0, "popc": 1, "b1": 2, "i8": 3, "f8": 4, "tc": 5, "tc2": 6, "sparse": 7}
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}

_u64p = ctypes.POINTER(ctypes.c_uint64)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class JsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


class Sets(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("offsets", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("mem", ctypes.c_int)]


def partition_batches(minid: int, maxid: int, batch_rows: int, parts: int):
    """The row batches [begin, end) (batch index = value // batch_rows) of each
    part of jsim_all_pairs_part, by the library's own rule
    (jsim_partition_batches; batch_rows 0: the automatic size)."""
    lib = load()
    out = []
    for p in range(parts):
        b0, b1, mt = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib.jsim_partition_batches(minid, maxid, batch_rows, p, parts, ctypes.byref(b0), ctypes.byref(b1),
                                        ctypes.byref(mt))
        if rc:
            raise JsimError(rc, "jsim_partition_batches")
        out.append((b0.value, b1.value))
    return out


def check_tc_schedule(jobs, grid: int, tile_n: int = 256, stage_bits: int = 256):
    """Host-side check of the job-table tensor-core product's schedule for
    jobs [(n, W, stride, rows), ...] over `grid` CTAs, with stages of
    `stage_bits` bit-rows: (code, message), code 0 when every check passes
    (jsim_check_tc_schedule)."""
    lib = load()
    k = len(jobs)
    arr = [(ctypes.c_uint64 * k)(*[int(j[f]) for j in jobs]) for f in range(4)]
    buf = ctypes.create_string_buffer(256)
    rc = lib.jsim_check_tc_schedule(k, arr[0], arr[1], arr[2], arr[3], grid, tile_n, stage_bits, buf, 256)
    return rc, buf.value.decode()


class Checkpoint(ctypes.Structure):
    _fields_ = [("path", ctypes.c_char_p), ("every", ctypes.c_uint32), ("max_supers", ctypes.c_uint32),
                ("resume", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("batch_rows", ctypes.c_uint64), ("word_bits", ctypes.c_int), ("variant", ctypes.c_int),
                ("count_bits", ctypes.c_int), ("id_bits", ctypes.c_int), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", ctypes.c_void_p), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("timeout_ms", ctypes.c_int), ("profile", ctypes.c_int),
                ("filter_min", ctypes.c_int), ("distance", ctypes.c_int), ("count_useful", ctypes.c_int),
                ("tile_n", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("rows_nonzero", ctypes.c_uint64), ("words", ctypes.c_uint64),
                ("batch_rows", ctypes.c_uint64), ("variant", ctypes.c_int), ("product_launches", ctypes.c_int),
                ("launches", ctypes.c_int), ("ms_total", ctypes.c_double), ("ms_h2d", ctypes.c_double),
                ("ms_validate", ctypes.c_double), ("ms_filter", ctypes.c_double), ("ms_scan", ctypes.c_double),
                ("ms_pack", ctypes.c_double), ("ms_product", ctypes.c_double), ("ms_epilogue", ctypes.c_double),
                ("ms_d2h", ctypes.c_double), ("bitops_dense", ctypes.c_double),
                ("bitops_useful", ctypes.c_double), ("bitops_done", ctypes.c_double), ("tile_n", ctypes.c_uint64),
                ("pack_bytes", ctypes.c_uint64),
                ("h2d_copies", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64),
                ("h2d_pieces", ctypes.c_uint64),
                ("windows", ctypes.c_uint64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["variant"] = VARIANT_NAMES.get(d["variant"], d["variant"])
        return d


class ServeOptions(ctypes.Structure):
    _fields_ = [("max_batch_samples", ctypes.c_uint64), ("max_batch_values", ctypes.c_uint64),
                ("slots", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    _fields_ = [("requests_submitted", ctypes.c_uint64), ("requests_done", ctypes.c_uint64),
                ("samples_done", ctypes.c_uint64), ("values_done", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("rows_read", ctypes.c_uint64),
                ("ms_device", ctypes.c_double), ("ms_product", ctypes.c_double),
                ("index_bytes_read", ctypes.c_double),
                ("bitops_dense", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every C-ABI entry point declared in include/jsim.h, with its ctypes signature.
SIGNATURES = {
    "jsim_partition_batches": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "jsim_check_tc_schedule": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_char_p, ctypes.c_size_t]),
    "jsim_default_options": (None, [ctypes.POINTER(Options)]),
    "jsim_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Options)]),
    "jsim_destroy": (None, [ctypes.c_void_p]),
    "jsim_all_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int]),
    "jsim_all_pairs_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_uint64,
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                              ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "jsim_all_pairs_streamed": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64]),
    "jsim_all_pairs_streamed_ckpt": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                                    ctypes.POINTER(Checkpoint)]),
    "jsim_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, _u64p, ctypes.c_void_p,
                                 ctypes.c_int]),
    "jsim_product": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]),
    "jsim_product_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]),
    "jsim_serve_default_options": (None, [ctypes.POINTER(ServeOptions)]),
    "jsim_index_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.POINTER(ServeOptions),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "jsim_index_destroy": (None, [ctypes.c_void_p]),
    "jsim_index_info": (ctypes.c_int, [ctypes.c_void_p, _u64p, _u64p, ctypes.c_void_p]),
    "jsim_index_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServeStats)]),
    "jsim_query_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.POINTER(ctypes.c_void_p)]),
    "jsim_request_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int]),
    "jsim_request_latency": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "jsim_request_free": (None, [ctypes.c_void_p]),
    "jsim_topk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int]),
    "jsim_all_pairs_part": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Sets), ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "jsim_finish": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "jsim_threshold": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _u64p,
                                      ctypes.c_int]),
    "jsim_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "jsim_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "jsim_last_cuda_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "jsim_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return build_native.LIB


def load(build: bool = True):
    """Load libjsim.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_native.build() if build else build_native.LIB
            if not os.path.exists(path):
                raise RuntimeError("libjsim.so is not built: %s" % path)
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, ctx_ptr=None):
    if rc != JSIM_OK:
        lib = load()
        msg = lib.jsim_strerror(rc).decode()
        if rc == 6 and ctx_ptr:
            msg += ": " + lib.jsim_last_cuda_error(ctx_ptr).decode()
        raise JsimError(rc, msg)


def _torch():
    import torch
    return torch


class Context:
    """A jsim context on one CUDA device.

    Device memory comes from PyTorch's caching allocator and work runs on the
    given torch stream (default: the device's current stream).
    """

    def __init__(self, device: int = 0, variant: str | int = "auto", batch_rows: int = 0, word_bits: int = 64,
                 count_bits: int = 32, id_bits: int = 64, profile: bool = False, stream=None,
                 use_torch_allocator: bool = True, timeout_ms: int = 2000, filter_min: int = 1,
                 distance: bool = False, count_useful: bool = False, allocator=None, tile_n: int = 0):
        """``allocator`` (optional) replaces PyTorch's caching allocator as the
        library's device allocator: an object with ``alloc(nbytes, stream) ->
        int`` (a device pointer, or 0 when it cannot serve the request: the
        library then returns JSIM_ERR_OOM) and ``free(ptr, nbytes, stream)``."""
        torch = _torch()
        self._lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.Stream(device)
        self.stream = stream
        o = Options()
        self._lib.jsim_default_options(ctypes.byref(o))
        o.batch_rows = batch_rows
        o.word_bits = word_bits
        o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o.count_bits = count_bits
        o.id_bits = id_bits
        o.device = device
        o.profile = 1 if profile else 0
        o.timeout_ms = timeout_ms
        o.filter_min = filter_min
        o.distance = 1 if distance else 0
        o.count_useful = 1 if count_useful else 0
        o.tile_n = tile_n
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        self._keep = []
        if allocator is not None:
            def _alloc_user(nbytes, st, user):
                try:
                    return int(allocator.alloc(int(nbytes), int(st or 0))) or None
                except Exception:
                    return None

            def _free_user(ptr, nbytes, st, user):
                if ptr:
                    allocator.free(int(ptr), int(nbytes), int(st or 0))

            a, f = ALLOC_FN(_alloc_user), FREE_FN(_free_user)
            self._keep += [a, f]
            o.alloc, o.free = a, f
        elif use_torch_allocator:
            dev = device

            def _alloc(nbytes, st, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(st or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, st, user):
                if ptr:
                    torch.cuda.caching_allocator_delete(int(ptr))

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f]
            o.alloc, o.free = a, f
        self.count_bits = count_bits
        self._opts = o
        h = ctypes.c_void_p()
        _check(self._lib.jsim_create(ctypes.byref(h), ctypes.byref(o)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.jsim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers -----------------------------------------------------------------
    @staticmethod
    def _ptr(x):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            return x.ctypes.data
        return x.data_ptr()

    def _sets(self, offsets, ids):
        torch = _torch()
        is_dev = isinstance(offsets, torch.Tensor) and offsets.is_cuda
        if is_dev:
            assert offsets.dtype == torch.uint64 or offsets.dtype == torch.int64
            assert offsets.is_contiguous() and ids.is_contiguous()
            n = offsets.numel() - 1
        else:
            offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
            ids = np.ascontiguousarray(ids, dtype=np.uint64)
            n = offsets.size - 1
        s = Sets()
        s.n = n
        s.offsets = self._ptr(offsets)
        s.ids = self._ptr(ids) if (ids is not None and (ids.numel() if is_dev else ids.size)) else None
        s.mem = MEM_DEVICE if is_dev else MEM_HOST
        return s, (offsets, ids), is_dev

    def _order(self):
        """The library's stream waits for work already queued on torch's current stream."""
        torch = _torch()
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def stats(self) -> dict:
        st = Stats()
        _check(self._lib.jsim_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    # -- entry points --------------------------------------------------------------
    def all_pairs(self, offsets, ids, want_C=True, want_J=True, want_sizes=True, out_device=None, out=None):
        """C (n x n), sizes (n), J (n x n) of one collection.

        Host inputs (numpy) give numpy outputs unless out_device=True; CUDA
        tensors give CUDA tensor outputs.  ``out`` may pass preallocated
        (C, sizes, J) buffers of the right kind.
        """
        s, keep, is_dev = self._sets(offsets, ids)
        dev_out = is_dev if out_device is None else out_device
        C, sizes, J = out if out is not None else self._outputs(s.n, dev_out, want_C, want_sizes, want_J)
        self._order()
        rc = self._lib.jsim_all_pairs(self._h, ctypes.byref(s), self._ptr(C), self._ptr(sizes), self._ptr(J),
                                      MEM_DEVICE if dev_out else MEM_HOST)
        _check(rc, self._h)
        return C, sizes, J

    def all_pairs_part(self, offsets, ids, part: int, parts: int, out_device=None):
        """(C, sizes): the counts of part `part` of `parts` of the collection's
        row batches (see jsim_all_pairs_part); sum C over the parts and call
        finish()."""
        s, keep, is_dev = self._sets(offsets, ids)
        dev_out = is_dev if out_device is None else out_device
        C, sizes, _ = self._outputs(s.n, dev_out, True, True, False)
        self._order()
        rc = self._lib.jsim_all_pairs_part(self._h, ctypes.byref(s), int(part), int(parts), self._ptr(C),
                                           self._ptr(sizes), MEM_DEVICE if dev_out else MEM_HOST)
        _check(rc, self._h)
        return C, sizes

    def finish(self, C, sizes, want_C=True, want_J=True):
        """(C, J) from summed part counts and the sizes (jsim_finish); device
        tensors in, device tensors out."""
        torch = _torch()
        is_dev = isinstance(C, torch.Tensor) and C.is_cuda
        n = int(C.shape[0])
        if not is_dev:
            cdt = np.uint64 if self.count_bits == 64 else np.uint32
            C = np.ascontiguousarray(C, dtype=cdt)
            sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
        Co, _, J = self._outputs(n, is_dev, want_C, False, want_J)
        self._order()
        rc = self._lib.jsim_finish(self._h, n, self._ptr(C), self._ptr(sizes), self._ptr(Co), self._ptr(J),
                                   MEM_DEVICE if is_dev else MEM_HOST)
        _check(rc, self._h)
        return Co, J

    def _outputs(self, n, dev_out, want_C, want_sizes, want_J):
        torch = _torch()
        if dev_out:
            d = torch.device("cuda", self.device)
            cdt = torch.uint64 if self.count_bits == 64 else torch.uint32
            return (torch.empty((n, n), dtype=cdt, device=d) if want_C else None,
                    torch.empty(n, dtype=torch.uint64, device=d) if want_sizes else None,
                    torch.empty((n, n), dtype=torch.float64, device=d) if want_J else None)
        cdt = np.uint64 if self.count_bits == 64 else np.uint32
        return (np.empty((n, n), dtype=cdt) if want_C else None,
                np.empty(n, dtype=np.uint64) if want_sizes else None,
                np.empty((n, n), dtype=np.float64) if want_J else None)

    def all_pairs_streamed(self, offsets, ids, staging_bytes: int = 1 << 30, want_C=True, want_J=True,
                           want_sizes=True, out_device=False, out=None, checkpoint: dict | None = None):
        """As all_pairs for a collection in host memory, streamed through two
        pinned staging buffers of ``staging_bytes`` each (host->device copies
        overlap the device's work).  ``checkpoint`` = {"path": ..., "every": k,
        "max_supers": m, "resume": bool} keeps progress in a file (see
        jsim_all_pairs_streamed_ckpt); a stop after m super-batches raises
        JsimError JSIM_ERR_INCOMPLETE."""
        s, keep, is_dev = self._sets(offsets, ids)
        if is_dev:
            raise ValueError("all_pairs_streamed reads its input from host memory")
        C, sizes, J = out if out is not None else self._outputs(s.n, out_device, want_C, want_sizes, want_J)
        self._order()
        mem = MEM_DEVICE if out_device else MEM_HOST
        if checkpoint is None:
            rc = self._lib.jsim_all_pairs_streamed(self._h, ctypes.byref(s), self._ptr(C), self._ptr(sizes),
                                                   self._ptr(J), mem, int(staging_bytes))
        else:
            ck = Checkpoint()
            path = checkpoint.get("path")
            ck.path = os.fsencode(path) if path else None
            ck.every = int(checkpoint.get("every", 0))
            ck.max_supers = int(checkpoint.get("max_supers", 0))
            ck.resume = 1 if checkpoint.get("resume", False) else 0
            rc = self._lib.jsim_all_pairs_streamed_ckpt(self._h, ctypes.byref(s), self._ptr(C), self._ptr(sizes),
                                                        self._ptr(J), mem, int(staging_bytes), ctypes.byref(ck))
        _check(rc, self._h)
        return C, sizes, J

    def all_pairs_batched(self, collections, out_device=None, want_C=True, want_J=True, want_sizes=True):
        """Independent collections [(offsets, ids), ...] in one call -> [(C, sizes, J), ...]."""
        torch = _torch()
        k = len(collections)
        sets = (Sets * max(k, 1))()
        keep = []
        dev_in = None
        for c, (off, ids) in enumerate(collections):
            s, kp, is_dev = self._sets(off, ids)
            sets[c] = s
            keep.append(kp)
            dev_in = is_dev if dev_in is None else dev_in
        dev_out = bool(dev_in) if out_device is None else out_device
        cdt_np = np.uint64 if self.count_bits == 64 else np.uint32
        cdt_t = torch.uint64 if self.count_bits == 64 else torch.uint32
        outs = []
        for c in range(k):
            n = sets[c].n
            if dev_out:
                d = torch.device("cuda", self.device)
                outs.append((torch.empty((n, n), dtype=cdt_t, device=d) if want_C else None,
                             torch.empty(n, dtype=torch.uint64, device=d) if want_sizes else None,
                             torch.empty((n, n), dtype=torch.float64, device=d) if want_J else None))
            else:
                outs.append((np.empty((n, n), dtype=cdt_np) if want_C else None,
                             np.empty(n, dtype=np.uint64) if want_sizes else None,
                             np.empty((n, n), dtype=np.float64) if want_J else None))
        arr = lambda q: (ctypes.c_void_p * max(k, 1))(*[self._ptr(o[q]) for o in outs])
        Cp, Sp, Jp = arr(0), arr(1), arr(2)
        self._order()
        rc = self._lib.jsim_all_pairs_batched(self._h, sets, k, Cp if want_C else None, Sp if want_sizes else None,
                                              Jp if want_J else None, MEM_DEVICE if dev_out else MEM_HOST)
        _check(rc, self._h)
        return outs

    def pack(self, offsets, ids, lo: int, width: int, want_filter=True, want_words=True, want_sizes=True,
             stride: int | None = None):
        """One row batch: (filter words, packed words [n, stride], R, per-batch sizes) on the host."""
        s, keep, is_dev = self._sets(offsets, ids)
        n = s.n
        R = ctypes.c_uint64(0)
        # ask for R first
        self._order()
        rc = self._lib.jsim_pack(self._h, ctypes.byref(s), lo, width, None, None, 0, ctypes.byref(R), None,
                                 MEM_HOST)
        _check(rc, self._h)
        W = (R.value + 63) // 64
        if stride is None:
            stride = max(W, 1)
        filt = np.empty(width // 64, dtype=np.uint64) if want_filter else None
        words = np.empty((n, stride), dtype=np.uint64) if want_words else None
        sz = np.empty(n, dtype=np.uint64) if want_sizes else None
        rc = self._lib.jsim_pack(self._h, ctypes.byref(s), lo, width, self._ptr(filt), self._ptr(words), stride,
                                 ctypes.byref(R), self._ptr(sz), MEM_HOST)
        _check(rc, self._h)
        return filt, words, R.value, sz

    def topk(self, J, k: int, want_val: bool = True):
        """(idx n x k uint64, val n x k binary64 or None): the k samples with the
        largest J of every sample (itself excluded), ties to the smaller index."""
        torch = _torch()
        is_dev = isinstance(J, torch.Tensor) and J.is_cuda
        n = J.shape[0]
        if is_dev:
            idx = torch.empty((n, k), dtype=torch.uint64, device=J.device)
            val = torch.empty((n, k), dtype=torch.float64, device=J.device) if want_val else None
        else:
            J = np.ascontiguousarray(J, dtype=np.float64)
            idx = np.empty((n, k), dtype=np.uint64)
            val = np.empty((n, k), dtype=np.float64) if want_val else None
        self._order()
        _check(self._lib.jsim_topk(self._h, self._ptr(J), n, k, self._ptr(idx), self._ptr(val),
                                   MEM_DEVICE if is_dev else MEM_HOST), self._h)
        return idx, val

    def threshold(self, J, tau: float, below: bool = False, cap: int | None = None, want_val: bool = True):
        """Pairs i < j with J >= tau (below: J <= tau, for distances), row-major:
        (pi uint64, pj uint64, val binary64 or None, count).  cap (default: every
        pair that passes, found by a counting call first) bounds the pairs
        written; count is the total that pass."""
        torch = _torch()
        is_dev = isinstance(J, torch.Tensor) and J.is_cuda
        n = J.shape[0]
        if not is_dev:
            J = np.ascontiguousarray(J, dtype=np.float64)
        mem = MEM_DEVICE if is_dev else MEM_HOST
        cnt = ctypes.c_uint64(0)
        self._order()
        if cap is None:
            _check(self._lib.jsim_threshold(self._h, self._ptr(J), n, float(tau), int(bool(below)), 0, None, None,
                                            None, ctypes.byref(cnt), mem), self._h)
            cap = cnt.value
        if is_dev:
            pi = torch.empty(cap, dtype=torch.uint64, device=J.device)
            pj = torch.empty(cap, dtype=torch.uint64, device=J.device)
            val = torch.empty(cap, dtype=torch.float64, device=J.device) if want_val else None
        else:
            pi = np.empty(cap, dtype=np.uint64)
            pj = np.empty(cap, dtype=np.uint64)
            val = np.empty(cap, dtype=np.float64) if want_val else None
        _check(self._lib.jsim_threshold(self._h, self._ptr(J), n, float(tau), int(bool(below)), cap,
                                        self._ptr(pi) if cap else None, self._ptr(pj) if cap else None,
                                        self._ptr(val) if cap else None, ctypes.byref(cnt), mem), self._h)
        w = min(cap, cnt.value)
        return pi[:w], pj[:w], (val[:w] if val is not None else None), cnt.value

    def product(self, words, n: int, W: int, stride: int, C=None, variant: str | int = "auto"):
        """C = X X^T over (AND, popcount, +) of device-resident packed words."""
        torch = _torch()
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        if C is None:
            C = torch.empty((n, n), dtype=torch.uint64 if self.count_bits == 64 else torch.uint32,
                            device=torch.device("cuda", self.device))
        self._order()
        rc = self._lib.jsim_product(self._h, self._ptr(words), n, W, stride, self._ptr(C), v)
        _check(rc, self._h)
        return C


    def product_noalloc(self, words, n: int, W: int, stride: int, C, variant: str | int = "auto"):
        """jsim_product without device allocation (see include/jsim.h): C must
        be preallocated by the caller; scratch is the library's fixed array."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        self._order()
        rc = self._lib.jsim_product_noalloc(self._h, self._ptr(words), n, W, stride, self._ptr(C), v)
        _check(rc, self._h)
        return C


class Index:
    """A resident reference index with its query server (jsim_index_build).

    ``submit`` queues query samples (host arrays) and returns a Request; the
    arrays are kept referenced by the Request until it is freed, because the
    server reads them until the request is done.
    """

    def __init__(self, ctx: Context, offsets, ids, max_batch_samples: int = 64, max_batch_values: int = 1 << 27,
                 slots: int = 3):
        self._lib = ctx._lib
        self.ctx = ctx
        self.count_bits = ctx.count_bits
        s, self._ref_keep, _ = ctx._sets(offsets, ids)
        opt = ServeOptions(max_batch_samples, max_batch_values, slots)
        h = ctypes.c_void_p()
        ctx._order()
        _check(self._lib.jsim_index_build(ctx._h, ctypes.byref(s), ctypes.byref(opt), ctypes.byref(h)), ctx._h)
        self._h = h
        self._ref_keep = None  # the index holds its own copy
        n_ref, rows = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.jsim_index_info(self._h, ctypes.byref(n_ref), ctypes.byref(rows), None))
        self.n_ref, self.rows = n_ref.value, rows.value

    def ref_sizes(self):
        out = np.empty(self.n_ref, dtype=np.uint64)
        _check(self._lib.jsim_index_info(self._h, None, None, out.ctypes.data))
        return out

    def submit(self, offsets, ids) -> "Request":
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        s = Sets()
        s.n = offsets.size - 1
        s.offsets = offsets.ctypes.data
        s.ids = ids.ctypes.data if ids.size else None
        s.mem = MEM_HOST
        h = ctypes.c_void_p()
        _check(self._lib.jsim_query_submit(self._h, ctypes.byref(s), ctypes.byref(h)))
        return Request(self, h, s.n, (offsets, ids))

    def stats(self) -> dict:
        st = ServeStats()
        _check(self._lib.jsim_index_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self._h is not None:
            self._lib.jsim_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Request:
    """One submitted query request (jsim_query_submit)."""

    def __init__(self, index: Index, h, q: int, keep):
        self._lib = index._lib
        self._index = index  # the index outlives its requests
        self._h = h
        self.q = q
        self.n_ref = index.n_ref
        self.count_bits = index.count_bits
        self._keep = keep

    def wait(self, timeout_ms: int = -1):
        """(C q x n_ref, sizes q, J q x n_ref) as numpy arrays."""
        C = np.empty((self.q, self.n_ref), dtype=np.uint64 if self.count_bits == 64 else np.uint32)
        sizes = np.empty(self.q, dtype=np.uint64)
        J = np.empty((self.q, self.n_ref), dtype=np.float64)
        _check(self._lib.jsim_request_wait(self._h, C.ctypes.data, sizes.ctypes.data, J.ctypes.data,
                                           int(timeout_ms)))
        return C, sizes, J

    def latency(self):
        """(submit -> admitted, submit -> done) in ms, host clock."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.jsim_request_latency(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def free(self):
        if self._h is not None:
            self._lib.jsim_request_free(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def version() -> str:
    return load().jsim_version().decode()
