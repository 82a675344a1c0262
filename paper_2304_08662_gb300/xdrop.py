"""Thin ctypes binding of the C ABI in include/xdrop.h (argument marshalling only).

Every function of the header is exposed under the same name.  There is no CPU path: if
libxd.so cannot be built or loaded, importing the binding raises.  Arrays are numpy
arrays (host) or objects exposing ``data_ptr()`` (device tensors, for xd_run_device).
"""
import ctypes
import os

import numpy as np

from . import build as _build

XD_OK, XD_PENDING, XD_EINVAL, XD_ENOMEM, XD_ETIMEDOUT, XD_EDEVICE, XD_ENOTFOUND = 0, 1, -1, -2, -3, -4, -5
XD_DNA2, XD_PROT5 = 0, 1
STATUS_NAMES = {0: "XD_OK", 1: "XD_PENDING", -1: "XD_EINVAL", -2: "XD_ENOMEM", -3: "XD_ETIMEDOUT",
                -4: "XD_EDEVICE", -5: "XD_ENOTFOUND"}

SIDE_DTYPE = np.dtype([("score", np.int32), ("h_ext", np.uint32), ("v_ext", np.uint32),
                       ("flags", np.uint32), ("cells", np.uint64)])
RESULT_DTYPE = np.dtype([("left", SIDE_DTYPE), ("right", SIDE_DTYPE), ("total", np.int64)])
PAIR_DTYPE = np.dtype([("h_id", np.uint32), ("v_id", np.uint32), ("h_seed", np.uint32),
                       ("v_seed", np.uint32), ("seed_len", np.uint32)])


class xd_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("store_bytes_cap", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int32), ("tune_table", ctypes.c_char_p),
                ("batching", ctypes.c_int32), ("max_batch_pairs", ctypes.c_uint32)]


class xd_scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap", ctypes.c_int32),
                ("matrix20x20", ctypes.c_void_p)]


class xd_batch(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int), ("n_seqs", ctypes.c_uint32), ("n_codes", ctypes.c_uint64),
                ("seq_codes", ctypes.c_void_p), ("seq_offsets", ctypes.c_void_p),
                ("seq_lengths", ctypes.c_void_p), ("n_pairs", ctypes.c_uint32),
                ("pairs", ctypes.c_void_p), ("scoring", xd_scoring), ("X", ctypes.c_int32),
                ("delta_b", ctypes.c_uint32), ("z_drop", ctypes.c_int32)]


class xd_pairs_batch(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int), ("n_pairs", ctypes.c_uint32), ("pairs", ctypes.c_void_p),
                ("scoring", xd_scoring), ("X", ctypes.c_int32), ("delta_b", ctypes.c_uint32),
                ("z_drop", ctypes.c_int32)]


class xd_stats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("pairs", ctypes.c_uint64), ("cells", ctypes.c_uint64),
                ("units_tier", ctypes.c_uint64 * 3), ("escalations", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("host_launches", ctypes.c_uint64),
                ("host_requests", ctypes.c_uint64), ("graph_captures", ctypes.c_uint64),
                ("graph_replays", ctypes.c_uint64), ("mixed_launches", ctypes.c_uint64)]


class xd_timing(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64),
                ("pack_ms", ctypes.c_float), ("units_ms", ctypes.c_float), ("order_ms", ctypes.c_float),
                ("tier_ms", ctypes.c_float * 3), ("totals_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("tier_units", ctypes.c_uint64 * 3), ("tier_cells", ctypes.c_uint64 * 3),
                ("escalations", ctypes.c_uint64), ("discarded_cells", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("window_shifts", ctypes.c_uint64),
                ("register_band_cells", ctypes.c_uint64), ("register_slot_cells", ctypes.c_uint64)]


assert ctypes.sizeof(xd_batch) == 96 and RESULT_DTYPE.itemsize == 56 and ctypes.sizeof(xd_config) == 40

_LIB = None


def lib():
    """Load libxd.so, building it with nvcc first if it is missing or stale."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P, V = ctypes.c_void_p, ctypes.c_void_p
        L.xd_create.argtypes = [ctypes.POINTER(xd_config), ctypes.POINTER(P)]
        L.xd_submit_batch.argtypes = [P, ctypes.POINTER(xd_batch), ctypes.POINTER(ctypes.c_uint64)]
        L.xd_poll.argtypes = [P, ctypes.c_uint64, V, ctypes.c_int32]
        L.xd_run_device.argtypes = [P, ctypes.POINTER(xd_batch), V, V]
        L.xd_reserve.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        L.xd_device_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
        L.xd_get_stats.argtypes = [P, ctypes.POINTER(xd_stats)]
        L.xd_set_timing.argtypes = [P, ctypes.c_int32]
        L.xd_get_timing.argtypes = [P, ctypes.POINTER(xd_timing)]
        L.xd_probe.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.xd_set_trace.argtypes = [P, ctypes.c_int32]
        L.xd_run_device_many.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(xd_batch), V, V]
        L.xd_get_trace.argtypes = [P, V, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.xd_run_device_noalloc.argtypes = [ctypes.POINTER(xd_batch), ctypes.c_uint32, V, V]
        L.xd_autotune.argtypes = [P, ctypes.POINTER(xd_batch), ctypes.c_char_p, ctypes.POINTER(ctypes.c_float)]
        L.xd_store_add.argtypes = [P, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, V, V, V, V]
        L.xd_store_info.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        L.xd_submit_pairs.argtypes = [P, ctypes.POINTER(xd_pairs_batch), ctypes.POINTER(ctypes.c_uint64)]
        L.xd_destroy.argtypes = [P]
        L.xd_last_error.argtypes = [P]
        L.xd_last_error.restype = ctypes.c_char_p
        L.xd_version.restype = ctypes.c_char_p
        for name in ("xd_create", "xd_submit_batch", "xd_poll", "xd_run_device", "xd_reserve",
                     "xd_device_status", "xd_get_stats", "xd_destroy", "xd_set_timing", "xd_get_timing", "xd_probe", "xd_run_device_noalloc", "xd_autotune",
                     "xd_set_trace", "xd_get_trace", "xd_run_device_many",
                     "xd_store_add", "xd_store_info", "xd_submit_pairs"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


class XdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- C names

def xd_version():
    return lib().xd_version().decode()


def xd_last_error(ctx=None):
    return lib().xd_last_error(ctx).decode()


def xd_create(device=0, store_bytes_cap=0, max_inflight=0, tune_table=None, batching=0,
              max_batch_pairs=0):
    cfg = xd_config(device, store_bytes_cap, max_inflight,
                    None if tune_table is None else tune_table.encode(), batching, max_batch_pairs)
    out = ctypes.c_void_p()
    rc = lib().xd_create(ctypes.byref(cfg), ctypes.byref(out))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(None))
    return out


def xd_destroy(ctx):
    return lib().xd_destroy(ctx)


class BatchArgs:
    """Keeps the arrays of one xd_batch alive while the C call reads them."""

    def __init__(self, alphabet, codes, offsets, lengths, pairs, match, mismatch, gap, matrix, X, delta, zdrop=0):
        self.keep = [codes, offsets, lengths, pairs, matrix]
        self.matrix = None if matrix is None else np.ascontiguousarray(matrix, dtype=np.int8)
        sc = xd_scoring(int(match), int(mismatch), int(gap), None if self.matrix is None else _ptr(self.matrix))
        n_codes = int(codes.numel() if hasattr(codes, "numel") else codes.size)
        n_seqs = int(lengths.numel() if hasattr(lengths, "numel") else lengths.size)
        n_pairs = int(pairs.shape[0])
        self.c = xd_batch(XD_DNA2 if alphabet == "dna" else XD_PROT5, n_seqs, n_codes, _ptr(codes),
                          _ptr(offsets), _ptr(lengths), n_pairs, _ptr(pairs), sc, int(X), int(delta), int(zdrop))

    @classmethod
    def from_host(cls, b):
        """From a synth.Batch-like object holding numpy arrays."""
        pairs = np.ascontiguousarray(b.pairs, dtype=np.uint32).reshape(-1, 5)
        return cls(b.alphabet, np.ascontiguousarray(b.codes, dtype=np.uint8),
                   np.ascontiguousarray(b.offsets, dtype=np.uint64),
                   np.ascontiguousarray(b.lengths, dtype=np.uint32), pairs,
                   b.match, b.mismatch, b.gap, b.matrix, b.X, b.delta, getattr(b, "zdrop", 0))


def xd_submit_batch(ctx, args):
    t = ctypes.c_uint64()
    rc = lib().xd_submit_batch(ctx, ctypes.byref(args.c), ctypes.byref(t))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return t.value


def xd_poll(ctx, ticket, out, wait_ms=-1):
    """Returns the status; raises only for errors other than XD_PENDING / XD_ETIMEDOUT."""
    rc = lib().xd_poll(ctx, ticket, _ptr(out), int(wait_ms))
    if rc not in (XD_OK, XD_PENDING, XD_ETIMEDOUT):
        raise XdError(rc, xd_last_error(ctx))
    return rc


def xd_run_device(ctx, args, d_out, stream=None):
    rc = lib().xd_run_device(ctx, ctypes.byref(args.c), _ptr(d_out), stream)
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))


def xd_run_device_many(ctx, args_list, d_out, stream=None):
    """Several device batches (BatchArgs) in one pass; d_out holds their results in order."""
    arr = (xd_batch * len(args_list))(*[a.c for a in args_list])
    rc = lib().xd_run_device_many(ctx, len(args_list), arr, _ptr(d_out), stream)
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))


def xd_run_device_noalloc(args, max_side_len, d_out, stream=None):
    """Allocation-free run on device inputs (see include/xdrop.h); returns the status."""
    return lib().xd_run_device_noalloc(ctypes.byref(args.c), int(max_side_len), _ptr(d_out), stream)


def xd_reserve(ctx, n_codes, n_seqs, n_pairs, max_seq_len):
    rc = lib().xd_reserve(ctx, int(n_codes), int(n_seqs), int(n_pairs), int(max_seq_len))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))


def xd_device_status(ctx):
    f = ctypes.c_uint32()
    rc = lib().xd_device_status(ctx, ctypes.byref(f))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return f.value


def xd_get_stats(ctx):
    s = xd_stats()
    rc = lib().xd_get_stats(ctx, ctypes.byref(s))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return {"batches": s.batches, "pairs": s.pairs, "cells": s.cells,
            "units_tier": list(s.units_tier), "escalations": s.escalations,
            "kernel_launches": s.kernel_launches, "host_launches": s.host_launches,
            "host_requests": s.host_requests, "graph_captures": s.graph_captures,
            "graph_replays": s.graph_replays, "mixed_launches": s.mixed_launches}


def xd_set_timing(ctx, enable=True):
    rc = lib().xd_set_timing(ctx, 1 if enable else 0)
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))


def xd_get_timing(ctx):
    t = xd_timing()
    rc = lib().xd_get_timing(ctx, ctypes.byref(t))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return {"batches": t.batches, "pack_ms": t.pack_ms, "units_ms": t.units_ms, "order_ms": t.order_ms,
            "tier_ms": list(t.tier_ms), "totals_ms": t.totals_ms, "total_ms": t.total_ms,
            "tier_units": list(t.tier_units), "tier_cells": list(t.tier_cells),
            "escalations": t.escalations, "discarded_cells": t.discarded_cells,
            "launches": t.launches, "window_shifts": t.window_shifts,
            "register_band_cells": t.register_band_cells, "register_slot_cells": t.register_slot_cells}


PROBE_OPS = {"add": 0, "max": 1, "dpx_addmax": 2, "dpx_max3": 3, "lop3": 4, "imad": 5,
             "cmp_sel": 6, "prmt": 7, "dpx_addmax_16x2": 8, "dpx_max3_16x2": 9, "max_16x2": 10,
             "cell_dna": 100, "cell_prot": 101, "cell_dna16": 102, "cell_prot16": 103}


TRACE_DTYPE = np.dtype([("start_ns", np.uint64), ("dur_ns", np.uint32), ("diags", np.uint32),
                        ("window", np.uint16), ("smid", np.uint16), ("lanes", np.uint8), ("level", np.uint8),
                        ("outcome", np.uint16)])
assert TRACE_DTYPE.itemsize == 24
TRACE_VISITS = 8


def xd_set_trace(ctx, enable):
    rc = lib().xd_set_trace(ctx, 1 if enable else 0)
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))


def xd_get_trace(ctx):
    """Records of the last traced xd_run_device batch: array [n_units, 8] of TRACE_DTYPE."""
    n = ctypes.c_uint64()
    rc = lib().xd_get_trace(ctx, None, 0, ctypes.byref(n))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    out = np.zeros((n.value, TRACE_VISITS), dtype=TRACE_DTYPE)
    rc = lib().xd_get_trace(ctx, out.ctypes.data_as(ctypes.c_void_p), out.nbytes, ctypes.byref(n))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return out


def xd_probe(ctx, op):
    r = ctypes.c_double()
    rc = lib().xd_probe(ctx, PROBE_OPS.get(op, op) if isinstance(op, str) else int(op), ctypes.byref(r))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return r.value


def xd_autotune(ctx, args, path=None):
    """Tune on a host sample (BatchArgs); returns the winner's milliseconds."""
    ms = ctypes.c_float()
    rc = lib().xd_autotune(ctx, ctypes.byref(args.c), None if path is None else str(path).encode(),
                           ctypes.byref(ms))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return ms.value


def xd_store_add(ctx, alphabet, codes, offsets, lengths):
    """Add sequences to the resident store; returns one uint32 handle per sequence."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    handles = np.zeros(lengths.size, dtype=np.uint32)
    rc = lib().xd_store_add(ctx, XD_DNA2 if alphabet == "dna" else XD_PROT5, lengths.size, codes.size,
                            _ptr(codes), _ptr(offsets), _ptr(lengths), _ptr(handles))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return handles


def xd_store_info(ctx, alphabet):
    n, b = ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().xd_store_info(ctx, XD_DNA2 if alphabet == "dna" else XD_PROT5, ctypes.byref(n), ctypes.byref(b))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return n.value, b.value


def xd_submit_pairs(ctx, alphabet, pairs, match=1, mismatch=-1, gap=-1, matrix=None, X=20, delta=0, zdrop=0):
    """Submit seed tuples whose h_id / v_id are resident-store handles; returns a ticket."""
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 5)
    mat = None if matrix is None else np.ascontiguousarray(matrix, dtype=np.int8)
    sc = xd_scoring(int(match), int(mismatch), int(gap), None if mat is None else _ptr(mat))
    pb = xd_pairs_batch(XD_DNA2 if alphabet == "dna" else XD_PROT5, pairs.shape[0], _ptr(pairs), sc, int(X),
                        int(delta), int(zdrop))
    t = ctypes.c_uint64()
    rc = lib().xd_submit_pairs(ctx, ctypes.byref(pb), ctypes.byref(t))
    if rc != XD_OK:
        raise XdError(rc, xd_last_error(ctx))
    return t.value


# ----------------------------------------------------------------------------- helpers

def extend_host(ctx, batch, wait_ms=-1):
    """Submit a host batch and wait for its results (numpy RESULT_DTYPE array)."""
    args = BatchArgs.from_host(batch)
    ticket = xd_submit_batch(ctx, args)
    out = np.zeros(batch.n_pairs, dtype=RESULT_DTYPE)
    rc = xd_poll(ctx, ticket, out, wait_ms)
    if rc != XD_OK:
        raise XdError(rc, "batch did not finish")
    return out


def header_symbols():
    """Function names declared in include/xdrop.h."""
    import re
    here = os.path.dirname(os.path.abspath(__file__))
    text = open(os.path.join(os.path.dirname(here), "include", "xdrop.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(xd_\w+)\s*\(", text, re.M)))
