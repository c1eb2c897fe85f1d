"""CPU oracle for syndrome-based normalized min-sum decoding (Algorithm 1, Sec. 2).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The decoder library and its Python binding never import it,
and it imports nothing from them: inputs (H in CSR, syndromes, priors) arrive as plain arrays.

The arithmetic lives in ``qldpc_oracle.c`` (plain scalar C, compiled with gcc on first use, no
floating-point contraction).  This module only compiles it, marshals numpy arrays and, for timing,
splits a batch over host threads (ctypes releases the GIL during the call).

Parity pins (see tests/test_oracle_pins.py): the hand-worked single-check update, the Eq. (1)
trace against its closed-form recurrence, tree codes against brute-force max-product, loopy tiny
codes against brute-force minimum weight, and the exact symmetries of min-sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qldpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
NO_EARLY_STOP = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qldpc_oracle.c into liboracle.so beside it (gcc, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i32 = ctypes.c_int32
            u32 = ctypes.c_uint32
            for name, real in (("oracle_msa_f64", ctypes.c_double), ("oracle_msa_f32", ctypes.c_float)):
                f = getattr(lib, name)
                f.argtypes = [p, p, i32, i32, p, i32, p, i32, real, u32, p, p, p, p, p]
                f.restype = ctypes.c_int
            lib.oracle_msa_i16.argtypes = [p, p, i32, i32, p, i32, p, i32, ctypes.c_float, u32,
                                           p, p, p, p, p]
            lib.oracle_msa_i16.restype = ctypes.c_int
            lib.oracle_alpha_q.argtypes = [ctypes.c_float]
            lib.oracle_alpha_q.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def alpha_q(alpha: float) -> int:
    """Fixed-point scale round_half_away(alpha * 2^15) used by the i16 mode (-1 if out of (0, 1])."""
    return _load().oracle_alpha_q(float(alpha))


def msa(row_ptr, col_idx, m: int, n: int, syndromes, prior, max_iter: int, alpha: float,
        precision: str = "f64", early_stop: bool = True, threads: int = 1) -> dict:
    """Decode a batch with Algorithm 1.

    row_ptr/col_idx: H in CSR (int32).  syndromes: uint8 [B, m].  prior: [n] LLRs gamma_n.
    precision: "f64", "f32" or "i16".  Returns a dict with
      err   uint8 [B, n]  decisions e_hat
      iters int32 [B]     CN+VN rounds run
      ok    uint8 [B]     1 iff H e_hat^T = s
      post  [B, n]        a-posteriori LLR Q_n of the last iteration (float64 / float32; for i16
                          the raw 32-bit fixed-point value, LLR = post / 256)
      margin float64 [B]  smallest |q| or |Q| the shot produced (near-tie diagnostic)
    """
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8).reshape(-1, m)
    batch = syn.shape[0]
    if precision == "f64":
        fn, pdt, post_dt, alpha_c = lib.oracle_msa_f64, np.float64, np.float64, float(alpha)
    elif precision == "f32":
        fn, pdt, post_dt, alpha_c = lib.oracle_msa_f32, np.float32, np.float32, float(np.float32(alpha))
    elif precision == "i16":
        fn, pdt, post_dt, alpha_c = lib.oracle_msa_i16, np.float32, np.int32, float(np.float32(alpha))
    else:
        raise ValueError(f"unknown precision {precision!r}")
    prior = np.ascontiguousarray(prior, dtype=pdt).reshape(n)
    err = np.zeros((batch, n), dtype=np.uint8)
    iters = np.zeros(batch, dtype=np.int32)
    ok = np.zeros(batch, dtype=np.uint8)
    post = np.zeros((batch, n), dtype=post_dt)
    margin = np.zeros(batch, dtype=np.float64)
    flags = 0 if early_stop else NO_EARLY_STOP

    def run(lo, hi):
        if hi <= lo:
            return 0
        return fn(_ptr(row_ptr), _ptr(col_idx), m, n, _ptr(syn[lo:hi]), hi - lo, _ptr(prior),
                  int(max_iter), alpha_c, flags, _ptr(err[lo:hi]), _ptr(iters[lo:hi]),
                  _ptr(ok[lo:hi]), _ptr(post[lo:hi]), _ptr(margin[lo:hi]))

    threads = max(1, min(int(threads), max(batch, 1)))
    if threads == 1:
        rcs = [run(0, batch)]
    else:
        bounds = np.linspace(0, batch, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(lambda i: run(bounds[i], bounds[i + 1]), range(threads)))
    bad = [rc for rc in rcs if rc != 0]
    if bad:
        raise ValueError(f"oracle rejected the input (code {bad[0]})")
    return {"err": err, "iters": iters, "ok": ok, "post": post, "margin": margin}
