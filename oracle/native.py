"""Build and load the oracle's C core (fth_oracle.c).  Test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fth_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfth_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fth_oracle.c with plain gcc (-O2, OpenMP over replicas)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


P = ctypes.c_void_p
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
D = ctypes.c_double
INT = ctypes.c_int


def _declare(L):
    L.oracle_philox4x32_10.argtypes = [P, P, P]
    L.oracle_philox4x32_10.restype = None
    L.oracle_normals.argtypes = [U64, U32, U32, U32, INT, P]
    L.oracle_normals.restype = None
    L.oracle_replica_normals.argtypes = [U64, U32, U32, U32, INT, INT, P]
    L.oracle_replica_normals.restype = None
    L.oracle_prologue.argtypes = [I64, I64, INT, INT, P, P, P, P, P, P, D, U64, U32, U32, P, P, P]
    L.oracle_prologue.restype = INT
    L.oracle_steps.argtypes = ([I64, I64, INT, INT, P, P, P, P, P, P, P, P, D, U64, U32, U32, I64, P,
                                P, P, INT, P, I64, P, I64, I64, P, P, P, P, P, P])
    L.oracle_steps.restype = INT
    L.oracle_force.argtypes = [I64, I64, INT, P, P, P, P, P, P]
    L.oracle_force.restype = None


def ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(ptr(c), ptr(k), ptr(out))
    return out


def normals(seed: int, kappa: int, i: int, j: int, count: int) -> np.ndarray:
    """The first `count` normals of the stream of counter word j (a replica pair):
    Philox calls k = 0, 1, ... with counter (kappa, i, j, k), four normals per call."""
    out = np.zeros(((count + 3) // 4) * 4, dtype=np.float64)
    lib().oracle_normals(U64(seed), U32(kappa), U32(i), U32(j), INT(count), ptr(out))
    return out[:count]


def replica_normals(seed: int, kappa: int, i: int, r: int, width: int, count: int) -> np.ndarray:
    """The first `count` of the `width` normals of global replica r: positions
    (r mod 2) * width + t of the stream of its pair r // 2."""
    out = np.zeros(count, dtype=np.float64)
    lib().oracle_replica_normals(U64(seed), U32(kappa), U32(i), U32(r), INT(width), INT(count),
                                 ptr(out))
    return out
