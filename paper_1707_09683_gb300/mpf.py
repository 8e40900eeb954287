"""ctypes binding of libmpf.so (argument marshalling only).

Every scan step runs in the CUDA kernels of ``csrc/``; this module converts
torch tensors and numpy arrays to pointers and status codes to exceptions.
There is no CPU fallback: if ``libmpf.so`` is missing, importing the
functions raises ``MpfLibraryMissing``.

The C entry points are declared in ``include/mpf.h``; the names here match.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpf.so")
# The same library with the kernels' debug index checks (build(debug=True)).
DEBUG_LIB_PATH = os.path.join(_HERE, "libmpf_debug.so")

MPF_OK, MPF_EINVAL, MPF_ENOMEM, MPF_ECUDA, MPF_ETIMEOUT, MPF_EUNSUPPORTED, MPF_EDEVICE = range(7)
MSV, SSV = 0, 1
MSV_SSV = 2   # batches and plans: both filters; outputs hold the MSV block, then the SSV block
ARITH_AUTO, ARITH_I16, ARITH_F16 = 0, 1, 2
TABLE_AUTO, TABLE_SHARED, TABLE_TENSOR = 0, 1, 2


class MpfLibraryMissing(RuntimeError):
    pass


class MpfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libmpf.so (built by ``paper_1707_09683_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise MpfLibraryMissing(
            f"{path} not found: build it with `python -m paper_1707_09683_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, u8p, f32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_void_p
    i32, u32, u64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "mpf_max_model_length": (i32, []),
        "mpf_max_striped_length": (i32, []),
        "mpf_strerror": (ctypes.c_char_p, [i32]),
        "mpf_ctx_create": (i32, [i32, vp, ctypes.POINTER(vp)]),
        "mpf_ctx_destroy": (None, [vp]),
        "mpf_ctx_stream": (vp, [vp]),
        "mpf_sync": (i32, [vp]),
        "mpf_profile_create": (i32, [vp, i32, i32, vp, ctypes.c_uint8, ctypes.c_uint8,
                                     ctypes.c_uint8, ctypes.c_uint8, vp, u32, ctypes.c_float,
                                     ctypes.c_uint8, ctypes.POINTER(vp)]),
        "mpf_profile_destroy": (None, [vp]),
        "mpf_profile_set_config": (i32, [vp, i32, i32, i32]),
        "mpf_profile_get_config": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "mpf_profile_set_arith": (i32, [vp, i32, i32]),
        "mpf_db_upload": (i32, [vp, vp, u64, vp, vp, u64, ctypes.POINTER(vp)]),
        "mpf_db_destroy": (None, [vp]),
        "mpf_db_n_seqs": (u64, [vp]),
        "mpf_db_n_residues": (u64, [vp]),
        "mpf_msv_scan": (i32, [vp, vp, vp, vp, vp, vp]),
        "mpf_ssv_scan": (i32, [vp, vp, vp, vp, vp, vp]),
        "mpf_scan_batch": (i32, [vp, i32, vp, i32, vp, vp, vp, vp]),
        "mpf_plan_create": (i32, [vp, i32, vp, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "mpf_plan_launch": (i32, [vp]),
        "mpf_plan_capture_graph": (i32, [vp]),
        "mpf_plan_kernel_launches": (i32, [vp]),
        "mpf_plan_group_count": (i32, [vp]),
        "mpf_plan_pack_sets": (i32, [i32, vp, i32, i32, vp]),
        "mpf_plan_group_info": (i32, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "mpf_plan_destroy": (None, [vp]),
        "mpf_scan_noalloc": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "mpf_profile_footprint": (i32, [vp, i32, vp, vp]),
        "mpf_profile_set_table_memory": (i32, [vp, i32, i32]),
        "mpf_profile_set_shard_factor": (i32, [vp, i32, i32]),
        "mpf_profile_get_shard_factor": (i32, [vp, i32, vp]),
        "mpf_profile_get_table_memory": (i32, [vp, i32, vp]),
        "mpf_pipeline_scan": (i32, [vp, vp, i32, vp, ctypes.c_float, vp, vp, vp, vp, vp, vp, vp]),
        "mpf_pvalues": (i32, [vp, vp, u64, ctypes.c_float, ctypes.c_float, vp]),
        "mpf_debug_check_selftest": (i32, [vp]),
        "mpf_vit_profile_create": (i32, [vp, i32, i32, vp, vp, vp, i32, ctypes.c_float,
                                         ctypes.POINTER(vp)]),
        "mpf_vit_profile_destroy": (None, [vp]),
        "mpf_viterbi_scan": (i32, [vp, vp, i32, vp, vp, vp, vp]),
        "mpf_viterbi_rescore": (i32, [vp, vp, i32, vp, vp, vp, ctypes.c_float, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return load().mpf_strerror(int(status)).decode()
    except MpfLibraryMissing:
        return f"status {status}"


def _check(status: int, where: str):
    if status != MPF_OK:
        raise MpfError(status, where)


def _ptr(a) -> Optional[int]:
    """Address of a torch tensor or numpy array (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def max_model_length() -> int:
    return int(load().mpf_max_model_length())


def max_striped_length() -> int:
    return int(load().mpf_max_striped_length())


# Handles a context owns, destroyed in this order before the context itself.
_CHILD_ORDER = ("mpf_plan_destroy", "mpf_vit_profile_destroy", "mpf_profile_destroy",
                "mpf_db_destroy")


class Context:
    """``mpf_ctx``: a device and the stream the library launches on.

    Without an explicit ``stream`` the context launches on a new
    ``torch.cuda.Stream`` that this object keeps alive, so torch (its events,
    its pinned-memory bookkeeping) never sees a stream the library destroyed.

    The context records the handles created in it (profiles, databases,
    plans); closing it destroys the ones still live first, so the C rule
    "destroy children before their context" holds whatever order Python
    finalises objects in (reference cycles, interpreter exit).
    """

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        self._live = {}
        self._torch_stream = None
        if stream is None:
            import torch
            self._torch_stream = torch.cuda.Stream(device=torch.device("cuda", int(device)))
            handle = self._torch_stream.cuda_stream
        elif hasattr(stream, "cuda_stream"):
            self._torch_stream = stream
            handle = stream.cuda_stream
        else:
            handle = int(stream)
        h = ctypes.c_void_p()
        _check(lib.mpf_ctx_create(int(device), handle or None, ctypes.byref(h)), "mpf_ctx_create")
        self.handle = h
        self.device = int(device)

    @property
    def stream(self) -> int:
        return int(load().mpf_ctx_stream(self.handle) or 0)

    def torch_stream(self):
        if self._torch_stream is not None:
            return self._torch_stream
        import torch
        return torch.cuda.ExternalStream(self.stream, device=torch.device("cuda", self.device))

    def sync(self):
        _check(load().mpf_sync(self.handle), "mpf_sync")

    def _own(self, handle, destroy: str):
        self._live[int(handle.value)] = destroy

    def _release(self, handle) -> bool:
        """True if ``handle`` was still live (the caller destroys it now)."""
        return self._live.pop(int(handle.value), None) is not None

    def close(self):
        if getattr(self, "handle", None):
            lib = load()
            live = getattr(self, "_live", {})
            for fn in _CHILD_ORDER:
                for h in [h for h, d in live.items() if d == fn]:
                    del live[h]
                    getattr(lib, fn)(ctypes.c_void_p(h))
            lib.mpf_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Profile:
    """``mpf_profile`` built from a profile record (``synth.Profile`` or any
    object with ``M, K, cost, bias, tbm, tec, tjb_fixed, tjb_by_len, scale,
    base``)."""

    def __init__(self, ctx: Context, prof):
        lib = load()
        cost = np.ascontiguousarray(prof.cost, dtype=np.uint8)
        K, M = cost.shape
        lut = getattr(prof, "tjb_by_len", None)
        lut = None if lut is None else np.ascontiguousarray(lut, dtype=np.uint8)
        h = ctypes.c_void_p()
        _check(lib.mpf_profile_create(
            ctx.handle, int(M), int(K), cost.ctypes.data, int(prof.bias), int(prof.tbm),
            int(prof.tec), int(prof.tjb_fixed), None if lut is None else lut.ctypes.data,
            0 if lut is None else int(lut.size), float(prof.scale), int(prof.base),
            ctypes.byref(h)), "mpf_profile_create")
        self.handle = h
        self.ctx = ctx
        self.M = int(M)
        ctx._own(h, "mpf_profile_destroy")

    def set_config(self, filter: int, lanes: int, words: int):
        _check(load().mpf_profile_set_config(self.handle, int(filter), int(lanes), int(words)),
               "mpf_profile_set_config")

    def set_arith(self, filter: int, arith: int):
        _check(load().mpf_profile_set_arith(self.handle, int(filter), int(arith)),
               "mpf_profile_set_arith")

    def set_shard_factor(self, filter: int, factor: int):
        _check(load().mpf_profile_set_shard_factor(self.handle, int(filter), int(factor)),
               "mpf_profile_set_shard_factor")

    def get_shard_factor(self, filter: int) -> int:
        w = ctypes.c_int()
        _check(load().mpf_profile_get_shard_factor(self.handle, int(filter), ctypes.byref(w)),
               "mpf_profile_get_shard_factor")
        return w.value

    def set_table_memory(self, filter: int, where: int):
        _check(load().mpf_profile_set_table_memory(self.handle, int(filter), int(where)),
               "mpf_profile_set_table_memory")

    def get_table_memory(self, filter: int) -> int:
        w = ctypes.c_int()
        _check(load().mpf_profile_get_table_memory(self.handle, int(filter), ctypes.byref(w)),
               "mpf_profile_get_table_memory")
        return w.value

    def get_config(self, filter: int):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().mpf_profile_get_config(self.handle, int(filter), ctypes.byref(a),
                                             ctypes.byref(b)), "mpf_profile_get_config")
        return a.value, b.value

    def footprint(self, filter: int):
        """(shared memory per block, device bytes of the score tables) of
        this profile's scans with one filter (``mpf_profile_footprint``)."""
        sm, tb = ctypes.c_uint32(), ctypes.c_uint64()
        _check(load().mpf_profile_footprint(self.handle, int(filter), ctypes.byref(sm), ctypes.byref(tb)),
               "mpf_profile_footprint")
        return sm.value, tb.value

    def close(self):
        if getattr(self, "handle", None):
            if self.ctx._release(self.handle):
                load().mpf_profile_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Database:
    """``mpf_db``: residues resident in device memory."""

    def __init__(self, ctx: Context, residues, offsets, lengths):
        lib = load()
        residues = np.ascontiguousarray(residues, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
        if offsets.size != lengths.size:
            raise ValueError("offsets and lengths differ in size")
        h = ctypes.c_void_p()
        _check(lib.mpf_db_upload(ctx.handle, residues.ctypes.data if residues.size else None,
                                 int(residues.size), offsets.ctypes.data if offsets.size else None,
                                 lengths.ctypes.data if lengths.size else None, int(lengths.size),
                                 ctypes.byref(h)), "mpf_db_upload")
        self.handle = h
        self.ctx = ctx
        ctx._own(h, "mpf_db_destroy")

    @property
    def n_seqs(self) -> int:
        return int(load().mpf_db_n_seqs(self.handle))

    @property
    def n_residues(self) -> int:
        return int(load().mpf_db_n_residues(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            if self.ctx._release(self.handle):
                load().mpf_db_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _scan1(fn_name, ctx, prof, db, raw, flag, nat):
    _check(getattr(load(), fn_name)(ctx.handle, prof.handle, db.handle, _ptr(raw), _ptr(flag),
                                    _ptr(nat)), fn_name)


def msv_scan(ctx: Context, prof: Profile, db: Database, raw, overflow, nat=None):
    """``mpf_msv_scan`` into caller buffers (host numpy or device tensors)."""
    _scan1("mpf_msv_scan", ctx, prof, db, raw, overflow, nat)


def ssv_scan(ctx: Context, prof: Profile, db: Database, raw, overflow, nat=None):
    """``mpf_ssv_scan`` into caller buffers (host numpy or device tensors)."""
    _scan1("mpf_ssv_scan", ctx, prof, db, raw, overflow, nat)


def _handles(profs: Sequence[Profile]):
    arr = (ctypes.c_void_p * len(profs))(*[p.handle.value for p in profs])
    return arr


def scan_batch(ctx: Context, filter: int, profs: Sequence[Profile], db: Database, raw, overflow,
               nat=None):
    """``mpf_scan_batch``: outputs are [n_q][n_seqs]; with filter MSV_SSV
    [2][n_q][n_seqs] (the MSV block, then the SSV block)."""
    arr = _handles(profs)
    _check(load().mpf_scan_batch(ctx.handle, int(filter), arr, len(profs), db.handle, _ptr(raw),
                                 _ptr(overflow), _ptr(nat)), "mpf_scan_batch")


class Plan:
    """``mpf_plan``: a reusable (optionally graph-captured) batch launch."""

    def __init__(self, ctx: Context, filter: int, profs: Sequence[Profile], db: Database, raw,
                 overflow, nat=None):
        self._arr = _handles(profs)
        self._keep = (list(profs), db, raw, overflow, nat)
        h = ctypes.c_void_p()
        _check(load().mpf_plan_create(ctx.handle, int(filter), self._arr, len(profs), db.handle,
                                      _ptr(raw), _ptr(overflow), _ptr(nat), ctypes.byref(h)),
               "mpf_plan_create")
        self.handle = h
        self.ctx = ctx
        ctx._own(h, "mpf_plan_destroy")

    def launch(self):
        _check(load().mpf_plan_launch(self.handle), "mpf_plan_launch")

    def capture_graph(self):
        _check(load().mpf_plan_capture_graph(self.handle), "mpf_plan_capture_graph")

    @property
    def kernel_launches(self) -> int:
        return int(load().mpf_plan_kernel_launches(self.handle))

    def groups(self):
        """Per launch group: dict(lanes, words, table, queries_per_warp,
        n_queries, filters), as ``mpf_plan_group_info`` reports them
        (filters: 1 MSV, 2 SSV, 3 both in one sweep)."""
        lib = load()
        out = []
        for i in range(int(lib.mpf_plan_group_count(self.handle))):
            v = [ctypes.c_int() for _ in range(6)]
            _check(lib.mpf_plan_group_info(self.handle, i, *[ctypes.byref(x) for x in v]),
                   "mpf_plan_group_info")
            out.append(dict(zip(("lanes", "words", "table", "queries_per_warp", "n_queries", "filters"),
                                (x.value for x in v))))
        return out

    def close(self):
        if getattr(self, "handle", None):
            if self.ctx._release(self.handle):
                load().mpf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_sets(lanes: int, words, max_smem: int = 232448):
    """``mpf_plan_pack_sets``: per query (words ascending) the index of the
    first query of its packed set, or -1 for a query left to its one-query
    kernel."""
    w = np.ascontiguousarray(words, dtype=np.int32)
    out = np.full(w.size, -2, dtype=np.int32)
    _check(load().mpf_plan_pack_sets(int(lanes), w.ctypes.data if w.size else None, int(w.size),
                                     int(max_smem), out.ctypes.data if w.size else None),
           "mpf_plan_pack_sets")
    return out


def scan_noalloc(ctx: Context, filter: int, prof: Profile, db: Database, raw, overflow, nat=None):
    """``mpf_scan_noalloc``: a scan into device buffers that allocates no
    device memory (scratch lives in a fixed device array inside the library;
    calls overlapping on the GPU race)."""
    _check(load().mpf_scan_noalloc(ctx.handle, int(filter), prof.handle, db.handle, _ptr(raw),
                                   _ptr(overflow), _ptr(nat)), "mpf_scan_noalloc")


def pipeline_scan(ctx: Context, profs: Sequence[Profile], db: Database, ssv_min_nat: float,
                  ssv_out, msv_out, n_pass):
    """``mpf_pipeline_scan``: SSV over every sequence, MSV over the ones whose
    SSV nat score is >= ssv_min_nat (or overflowed).  ``ssv_out`` and
    ``msv_out`` are (raw, flag, nat) device tensors of n_q * n_seqs; MSV
    entries of filtered sequences read raw 0, flag 2, nat NaN."""
    arr = _handles(profs)
    _check(load().mpf_pipeline_scan(ctx.handle, arr, len(profs), db.handle, float(ssv_min_nat),
                                    *[_ptr(t) for t in ssv_out], *[_ptr(t) for t in msv_out],
                                    _ptr(n_pass)), "mpf_pipeline_scan")


def pvalues(ctx: Context, nat, mu: float, lam: float, out):
    """``mpf_pvalues``: Gumbel P-values of device nat scores into ``out``."""
    _check(load().mpf_pvalues(ctx.handle, _ptr(nat), int(nat.numel()), float(mu), float(lam),
                              _ptr(out)), "mpf_pvalues")


class VitProfile:
    """``mpf_vprofile`` built from a Viterbi profile record (``synth.VitProfile``
    or any object with ``M, K, msc, trans, special, base, scale``)."""

    def __init__(self, ctx: Context, vprof):
        lib = load()
        msc = np.ascontiguousarray(vprof.msc, dtype=np.int16)
        trans = np.ascontiguousarray(vprof.trans, dtype=np.int16)
        special = np.ascontiguousarray(vprof.special, dtype=np.int16)
        K, M = msc.shape
        if trans.shape != (8, M) or special.shape != (8,):
            raise ValueError("trans must be 8 x M and special 8 values")
        h = ctypes.c_void_p()
        _check(lib.mpf_vit_profile_create(ctx.handle, int(M), int(K), msc.ctypes.data,
                                          trans.ctypes.data, special.ctypes.data, int(vprof.base),
                                          float(vprof.scale), ctypes.byref(h)),
               "mpf_vit_profile_create")
        self.handle = h
        self.ctx = ctx
        self.M = int(M)
        ctx._own(h, "mpf_vit_profile_destroy")

    def close(self):
        if getattr(self, "handle", None):
            if self.ctx._release(self.handle):
                load().mpf_vit_profile_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def viterbi_scan(ctx: Context, vprofs: Sequence[VitProfile], db: Database, score, overflow,
                 nat=None):
    """``mpf_viterbi_scan``: int16 scores, overflow bytes and nat scores,
    [n_q][n_seqs] (host numpy or device tensors)."""
    arr = _handles(vprofs)
    _check(load().mpf_viterbi_scan(ctx.handle, arr, len(vprofs), db.handle, _ptr(score),
                                   _ptr(overflow), _ptr(nat)), "mpf_viterbi_scan")


def viterbi_rescore(ctx: Context, vprofs: Sequence[VitProfile], db: Database, msv_flag, msv_nat,
                    msv_min_nat: float, score, overflow, nat, n_pass):
    """``mpf_viterbi_rescore``: Viterbi over the sequences whose MSV flag is 1
    or MSV nat >= msv_min_nat; the others read score -32768, flag 2, nat NaN.
    Device tensors."""
    arr = _handles(vprofs)
    _check(load().mpf_viterbi_rescore(ctx.handle, arr, len(vprofs), db.handle, _ptr(msv_flag),
                                      _ptr(msv_nat), float(msv_min_nat), _ptr(score),
                                      _ptr(overflow), _ptr(nat), _ptr(n_pass)),
           "mpf_viterbi_rescore")


def debug_check_selftest(ctx: Context):
    """``mpf_debug_check_selftest``: one failing index check (debug library);
    the next ``ctx.sync()`` raises MpfError(MPF_EDEVICE)."""
    _check(load().mpf_debug_check_selftest(ctx.handle), "mpf_debug_check_selftest")
