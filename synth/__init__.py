"""Seeded synthetic key columns shaped like the paper's workloads.

These generators only produce inputs (they hold none of the compressed key
sort's arithmetic); the CPU oracle tests, the CUDA parity tests and the bench
all draw from here.  The generation itself is C (``synth.c``, counter-based
SplitMix64 draws, OpenMP when available) so that the 64M-200M-row columns are
ready in seconds on the host.

Workload recipes (the datasets of the paper's evaluation are not available;
these stand in for them):

* ``varying_bits_u64``   -- integer column with 24 seeded varying bit positions
* ``urls``               -- URL keys, stand-in for the ExURL / WikiURL tables
* ``titles``             -- Zipf-prefixed strings, stand-in for Wikititle
* ``dna``                -- {A,C,G,T} strings, stand-in for the Human EST keys
* ``uniform_u32`` / ``sequential_noise_u64`` -- plain integer columns
* ``zipf_tagged_u64``    -- Zipf(s) over 2^40 values under a 12-bit tag
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
BASE_SEED = 20200924
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, U64, U32, D = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        lib.synth_draw.argtypes = [U64, U64, U64]
        lib.synth_draw.restype = U64
        lib.synth_threads.restype = ctypes.c_int
        lib.synth_zipf_table.argtypes = [U64, U64, U64, D, P]
        lib.synth_zipf_rejinv.argtypes = [U64, U64, D, D, P]
        lib.synth_varying_bits_u64.argtypes = [U64, U64, U32, P, P]
        lib.synth_urls.argtypes = [U64, U64, U32, U32, D, P]
        lib.synth_dna.argtypes = [U64, U64, U32, D, U32, U32, P]
        lib.synth_titles.argtypes = [U64, U64, U32, U32, D, P]
        lib.synth_uniform_u32.argtypes = [U64, U64, P]
        lib.synth_sequential_noise_u64.argtypes = [U64, U64, P]
        lib.synth_zipf_tagged_u64.argtypes = [U64, U64, D, P]
        lib.synth_zipf_letters.argtypes = [U64, U64, U32, U32, D, P]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().synth_threads())


def draw(seed: int, stream: int, i: int) -> int:
    return int(_load().synth_draw(seed, stream, i))


def zipf_table(n: int, seed: int, N: int, s: float) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _load().synth_zipf_table(n, seed, N, s, _p(out))
    return out


def zipf_rejinv(n: int, seed: int, N: float, s: float) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().synth_zipf_rejinv(n, seed, float(N), s, _p(out))
    return out


def varying_bits_u64(n: int, seed: int, nvary: int = 24):
    """uint64 keys where only ``nvary`` seeded bit positions vary (rest fixed)."""
    pos = np.empty(nvary, np.uint32)
    out = np.empty(n, np.uint64)
    _load().synth_varying_bits_u64(n, seed, nvary, _p(pos), _p(out))
    return out, [int(p) for p in pos]


def zipf_letters(n: int, seed: int, key_bytes: int, m: int, s: float) -> np.ndarray:
    """The paper's Zipf(s, n, m) datasets: [n, key_bytes] uint8 keys whose
    8-byte words start with m fixed characters followed by lowercase letters
    drawn from Zipf(s) over 26 letters."""
    out = np.empty((n, key_bytes), np.uint8)
    _load().synth_zipf_letters(n, seed, key_bytes, m, s, _p(out))
    return out


def urls(n: int, seed: int, W: int = 32, nnames: int = 100_000, s: float = 1.1) -> np.ndarray:
    out = np.empty((n, W), np.uint8)
    _load().synth_urls(n, seed, W, nnames, s, _p(out))
    return out


def dna(n: int, seed: int, W: int = 32, frac_prefixed: float = 0.2, groups: int = 65536,
        prefix_len: int = 24) -> np.ndarray:
    out = np.empty((n, W), np.uint8)
    _load().synth_dna(n, seed, W, frac_prefixed, groups, prefix_len, _p(out))
    return out


def titles(n: int, seed: int, W: int, nwords: int = 10_000, s: float = 1.0) -> np.ndarray:
    out = np.empty((n, W), np.uint8)
    _load().synth_titles(n, seed, W, nwords, s, _p(out))
    return out


def uniform_u32(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _load().synth_uniform_u32(n, seed, _p(out))
    return out


def sequential_noise_u64(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().synth_sequential_noise_u64(n, seed, _p(out))
    return out


def zipf_tagged_u64(n: int, seed: int, s: float = 0.9) -> np.ndarray:
    out = np.empty(n, np.uint64)
    _load().synth_zipf_tagged_u64(n, seed, s, _p(out))
    return out


def table_columns(n: int, seed: int) -> list:
    """One table, six index columns of widths 4, 8, 12, 16, 32 and 64 bytes."""
    return [
        uniform_u32(n, seed),
        sequential_noise_u64(n, seed + 1),
        titles(n, seed + 2, 12),
        titles(n, seed + 3, 16),
        titles(n, seed + 4, 32),
        titles(n, seed + 5, 64),
    ]
