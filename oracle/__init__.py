"""Scalar MSV/SSV and P7Viterbi oracle (test infrastructure).

This package is the checker, not the product: only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It wraps ``mpf_oracle.c`` (plain C, one scalar loop per cell, every byte
saturation of Alg. 2 / Alg. 7 written out) and ``mpf_vit_oracle.c`` (the same
for the 16-bit Viterbi recurrence of Eq. 1) through ctypes.  It imports
nothing from the CUDA library and the library imports nothing from here.

``build()`` compiles the C file with gcc into ``oracle/_build/``;
``scan()`` scores sequences of a database against one profile.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpf_oracle.c")
_VIT_SRC = os.path.join(_HERE, "mpf_vit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmpf_oracle.so")
_lib = None

MSV = 0
SSV = 1


def compile_source(src, out: str) -> str:
    """Compile oracle C source file(s) into the shared library ``out``."""
    srcs = [src] if isinstance(src, str) else list(src)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library and return its path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_VIT_SRC))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    return compile_source([_SRC, _VIT_SRC], _LIB_PATH)


def load_library(path: str):
    """Open a compiled oracle library (the default one, or a test build)."""
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.oracle_scan.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p,
        ctypes.c_uint8, ctypes.c_uint8, ctypes.c_uint8, ctypes.c_uint8,
        u8p, ctypes.c_uint32, ctypes.c_float, ctypes.c_uint8,
        u8p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
        ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
        u8p, u8p, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.oracle_scan.restype = ctypes.c_int
    if hasattr(lib, "oracle_viterbi"):
        i16p = ctypes.POINTER(ctypes.c_int16)
        lib.oracle_viterbi.argtypes = [
            ctypes.c_int, ctypes.c_int, i16p, i16p, i16p, ctypes.c_int, ctypes.c_float,
            u8p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
            ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
            i16p, u8p, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        lib.oracle_viterbi.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def scan(filter: int, prof, residues, offsets, lengths, index=None, nthreads: int = 1):
    """Score sequences against one profile with the scalar oracle.

    ``prof`` is any object with the profile fields ``M, K, cost (K x M
    uint8), bias, tbm, tec, tjb_fixed, tjb_by_len (uint8 array or None),
    scale, base``.  ``residues`` (uint8), ``offsets`` (uint64) and ``lengths``
    (uint32) describe the database; ``index`` optionally selects sequences.
    Returns ``(raw uint8, flag uint8, nat float32)`` arrays.
    """
    lib = _load()
    cost = np.ascontiguousarray(prof.cost, dtype=np.uint8)
    K, M = cost.shape
    assert M == prof.M and K == prof.K
    tjb = None
    n_tjb = 0
    if getattr(prof, "tjb_by_len", None) is not None:
        tjb = np.ascontiguousarray(prof.tjb_by_len, dtype=np.uint8)
        n_tjb = int(tjb.size)
    residues = np.ascontiguousarray(residues, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    if index is not None:
        index = np.ascontiguousarray(index, dtype=np.uint64)
        n = int(index.size)
    else:
        n = int(lengths.size)
    raw = np.zeros(n, np.uint8)
    flag = np.zeros(n, np.uint8)
    nat = np.zeros(n, np.float32)
    if residues.size == 0:
        residues = np.zeros(1, np.uint8)
    rc = lib.oracle_scan(
        int(filter), int(M), int(K), _ptr(cost, ctypes.c_uint8),
        int(prof.bias), int(prof.tbm), int(prof.tec), int(prof.tjb_fixed),
        _ptr(tjb, ctypes.c_uint8), n_tjb, float(prof.scale), int(prof.base),
        _ptr(residues, ctypes.c_uint8), _ptr(offsets, ctypes.c_uint64),
        _ptr(lengths, ctypes.c_uint32), _ptr(index, ctypes.c_uint64), n,
        _ptr(raw, ctypes.c_uint8), _ptr(flag, ctypes.c_uint8), _ptr(nat, ctypes.c_float),
        int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_scan failed with status {rc}")
    return raw, flag, nat


def msv(prof, residues, offsets, lengths, index=None, nthreads: int = 1):
    """MSV scores (Alg. 2 with the J/B special-state update)."""
    return scan(MSV, prof, residues, offsets, lengths, index, nthreads)


def ssv(prof, residues, offsets, lengths, index=None, nthreads: int = 1):
    """SSV scores (Alg. 7, single segment, no J state)."""
    return scan(SSV, prof, residues, offsets, lengths, index, nthreads)


def gumbel_pvalue(x, mu: float, lam: float):
    """P(S > x) for a Gumbel (type I extreme-value) score distribution with
    location mu and slope lam, the per-sequence P-value the filters record
    (Alg. 2, Alg. 7): 1 - exp(-exp(-lam (x - mu))), in float64; +inf -> 0,
    NaN stays NaN."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(over="ignore", invalid="ignore"):
        p = -np.expm1(-np.exp(-lam * (x - mu)))
    p = np.where(np.isposinf(x), 0.0, p)
    return p


def ssv_passes(flag, nat, ssv_min_nat: float):
    """The SSV -> MSV hand-off rule of Sec. 2.1, as a boolean mask: a
    sequence goes on to MSV when its SSV score overflowed (flag != 0; it
    certainly scores high) or its SSV nat score is at least ssv_min_nat
    (inclusive), compared in float32."""
    flag = np.asarray(flag)
    nat = np.asarray(nat, dtype=np.float32)
    with np.errstate(invalid="ignore"):
        return (flag != 0) | (nat >= np.float32(ssv_min_nat))


def pipeline(prof, residues, offsets, lengths, ssv_min_nat: float, nthreads: int = 1):
    """SSV over every sequence, MSV over those whose SSV nat score is
    >= ssv_min_nat or whose SSV score overflowed (Sec. 2.1).  Returns
    (ssv (raw, flag, nat), msv (raw, flag, nat) with raw 0 / flag 2 / NaN for
    filtered sequences, number passing)."""
    sr, sf, sn = ssv(prof, residues, offsets, lengths, nthreads=nthreads)
    keep = ssv_passes(sf, sn, ssv_min_nat)
    idx = np.flatnonzero(keep).astype(np.uint64)
    n = sr.size
    mr = np.zeros(n, np.uint8)
    mf = np.full(n, 2, np.uint8)
    mn = np.full(n, np.nan, np.float32)
    if idx.size:
        r, f, nt = msv(prof, residues, offsets, lengths, index=idx, nthreads=nthreads)
        mr[idx.astype(np.int64)] = r
        mf[idx.astype(np.int64)] = f
        mn[idx.astype(np.int64)] = nt
    return (sr, sf, sn), (mr, mf, mn), int(idx.size)


VIT_TRANSITIONS = ("BM", "MM", "IM", "DM", "MI", "II", "MD", "DD")
VIT_SPECIALS = ("NN", "NB", "EC", "CC", "CT", "EJ", "JJ", "JB")


def viterbi(vprof, residues, offsets, lengths, index=None, nthreads: int = 1):
    """P7Viterbi filter scores (Eq. 1 with the Plan-7 special states, 16-bit
    saturating word arithmetic).  ``vprof`` has ``M, K, msc (K x M int16),
    trans (8 x M int16, order VIT_TRANSITIONS), special (8 int16, order
    VIT_SPECIALS), base, scale``.  Returns (score int16, flag uint8, nat float32)."""
    lib = _load()
    msc = np.ascontiguousarray(vprof.msc, dtype=np.int16)
    trans = np.ascontiguousarray(vprof.trans, dtype=np.int16)
    special = np.ascontiguousarray(vprof.special, dtype=np.int16)
    K, M = msc.shape
    assert trans.shape == (8, M) and special.shape == (8,)
    residues = np.ascontiguousarray(residues, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint32)
    if index is not None:
        index = np.ascontiguousarray(index, dtype=np.uint64)
        n = int(index.size)
    else:
        n = int(lengths.size)
    score = np.zeros(n, np.int16)
    flag = np.zeros(n, np.uint8)
    nat = np.zeros(n, np.float32)
    if residues.size == 0:
        residues = np.zeros(1, np.uint8)
    i16 = ctypes.c_int16
    rc = lib.oracle_viterbi(int(M), int(K), _ptr(msc, i16), _ptr(trans, i16), _ptr(special, i16),
                            int(vprof.base), float(vprof.scale), _ptr(residues, ctypes.c_uint8),
                            _ptr(offsets, ctypes.c_uint64), _ptr(lengths, ctypes.c_uint32),
                            _ptr(index, ctypes.c_uint64), n, _ptr(score, i16),
                            _ptr(flag, ctypes.c_uint8), _ptr(nat, ctypes.c_float), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_viterbi failed with status {rc}")
    return score, flag, nat


def viterbi_stage(vprof, residues, offsets, lengths, msv_flag, msv_nat, msv_min_nat: float,
                  nthreads: int = 1):
    """Third pipeline stage (Sec. 2.1): Viterbi over the sequences whose MSV
    flag is 1 (overflow) or whose MSV nat score is >= msv_min_nat; flag 2
    (filtered by SSV, nat NaN) never passes.  Returns (score, flag, nat) with
    score -32768, flag 2, nat NaN for the others, and the number passing."""
    msv_flag = np.asarray(msv_flag)
    msv_nat = np.asarray(msv_nat, dtype=np.float32)
    with np.errstate(invalid="ignore"):
        keep = (msv_flag == 1) | (msv_nat >= np.float32(msv_min_nat))
    idx = np.flatnonzero(keep).astype(np.uint64)
    n = msv_flag.size
    vs = np.full(n, -32768, np.int16)
    vf = np.full(n, 2, np.uint8)
    vn = np.full(n, np.nan, np.float32)
    if idx.size:
        s, f, nt = viterbi(vprof, residues, offsets, lengths, index=idx, nthreads=nthreads)
        vs[idx.astype(np.int64)] = s
        vf[idx.astype(np.int64)] = f
        vn[idx.astype(np.int64)] = nt
    return (vs, vf, vn), int(idx.size)
