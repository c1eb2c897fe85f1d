"""CPU oracle for syndrome-based normalized min-sum decoding (Algorithm 1, Sec. 2).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The decoder library and its Python binding never import it,
and it imports nothing from them: inputs (H in CSR, syndromes, priors) arrive as plain arrays.

The arithmetic lives in ``qldpc_oracle.c`` (plain scalar C, compiled with gcc on first use, no
floating-point contraction).  This module only compiles it, marshals numpy arrays and, for timing,
splits a batch over host threads (ctypes releases the GIL during the call).

Parity pins (see tests/test_oracle_pins.py): the hand-worked single-check update, the Eq. (1)
trace against its closed-form recurrence, tree codes against brute-force max-product, loopy tiny
codes against brute-force minimum weight, and the exact symmetries of min-sum.  The layered
(row-serial) schedule (tests/test_oracle_layered.py): a hand-worked two-check trace, schedule
independence when no variable is shared, tree exactness, and bit-identical results under any
reordering that keeps checks sharing a variable in order.  The neural
min-sum functions (tests/test_oracle_nms.py): constant weights reduce them to the plain decoder,
the reverse-mode gradient matches central finite differences and a closed form for one check.
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
            for name in ("oracle_msa_i16", "oracle_msa_i8"):
                f = getattr(lib, name)
                f.argtypes = [p, p, i32, i32, p, i32, p, i32, ctypes.c_float, u32, p, p, p, p, p]
                f.restype = ctypes.c_int
            for name, real in (("oracle_layered_f64", ctypes.c_double), ("oracle_layered_f32", ctypes.c_float)):
                f = getattr(lib, name)
                f.argtypes = [p, p, i32, i32, p, i32, p, i32, real, u32, p, p, p, p]
                f.restype = ctypes.c_int
            for name in ("oracle_layered_i16", "oracle_layered_i8"):
                f = getattr(lib, name)
                f.argtypes = [p, p, i32, i32, p, i32, p, i32, ctypes.c_float, u32, p, p, p, p]
                f.restype = ctypes.c_int
            lib.oracle_alpha_q.argtypes = [ctypes.c_float]
            lib.oracle_alpha_q.restype = ctypes.c_int
            for name in ("oracle_nms_train_f64", "oracle_nms_train_f32"):
                f = getattr(lib, name)
                f.argtypes = [p, p, i32, i32, p, p, i32, p, p, i32, p, i32, p, p, p, p]
                f.restype = ctypes.c_int
            lib.oracle_nms_decode_f32.argtypes = [p, p, i32, i32, p, i32, p, p, i32, i32, ctypes.c_float,
                                                  p, p, p, p, p]
            lib.oracle_nms_decode_f32.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def alpha_q(alpha: float) -> int:
    """Fixed-point scale round_half_away(alpha * 2^15) used by the i16 mode (-1 if out of (0, 1])."""
    return _load().oracle_alpha_q(float(alpha))


def msa(row_ptr, col_idx, m: int, n: int, syndromes, prior, max_iter: int, alpha: float,
        precision: str = "f64", early_stop: bool = True, threads: int = 1, schedule: str = "flooding") -> dict:
    """Decode a batch with Algorithm 1 (schedule "flooding") or its row-serial variant ("layered").

    row_ptr/col_idx: H in CSR (int32).  syndromes: uint8 [B, m].  prior: [n] LLRs gamma_n.
    precision: "f64", "f32", "i16" or "i8".  Returns a dict with
      err   uint8 [B, n]  decisions e_hat
      iters int32 [B]     CN+VN rounds run
      ok    uint8 [B]     1 iff H e_hat^T = s
      post  [B, n]        a-posteriori LLR Q_n of the last iteration (float64 / float32; for i16
                          and i8 the raw 32-bit fixed-point value, LLR = post / 256 or post / 4)
      margin float64 [B]  smallest |q| or |Q| the shot produced (near-tie diagnostic; flooding only)
    """
    if schedule == "layered":
        return _layered(row_ptr, col_idx, m, n, syndromes, prior, max_iter, alpha, precision, early_stop, threads)
    if schedule != "flooding":
        raise ValueError(f"unknown schedule {schedule!r}")
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
    elif precision == "i8":
        fn, pdt, post_dt, alpha_c = lib.oracle_msa_i8, np.float32, np.int32, float(np.float32(alpha))
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


def _layered(row_ptr, col_idx, m, n, syndromes, prior, max_iter, alpha, precision, early_stop, threads):
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8).reshape(-1, m)
    batch = syn.shape[0]
    if precision == "f64":
        fn, pdt, post_dt, alpha_c = lib.oracle_layered_f64, np.float64, np.float64, float(alpha)
    elif precision == "f32":
        fn, pdt, post_dt, alpha_c = lib.oracle_layered_f32, np.float32, np.float32, float(np.float32(alpha))
    elif precision == "i16":
        fn, pdt, post_dt, alpha_c = lib.oracle_layered_i16, np.float32, np.int32, float(np.float32(alpha))
    elif precision == "i8":
        fn, pdt, post_dt, alpha_c = lib.oracle_layered_i8, np.float32, np.int32, float(np.float32(alpha))
    else:
        raise ValueError(f"unknown precision {precision!r}")
    prior = np.ascontiguousarray(prior, dtype=pdt).reshape(n)
    err = np.zeros((batch, n), dtype=np.uint8)
    iters = np.zeros(batch, dtype=np.int32)
    ok = np.zeros(batch, dtype=np.uint8)
    post = np.zeros((batch, n), dtype=post_dt)
    flags = 0 if early_stop else NO_EARLY_STOP

    def run(lo, hi):
        if hi <= lo:
            return 0
        return fn(_ptr(row_ptr), _ptr(col_idx), m, n, _ptr(syn[lo:hi]), hi - lo, _ptr(prior), int(max_iter),
                  alpha_c, flags, _ptr(err[lo:hi]), _ptr(iters[lo:hi]), _ptr(ok[lo:hi]), _ptr(post[lo:hi]))

    threads = max(1, min(int(threads), max(batch, 1)))
    bounds = np.linspace(0, batch, threads + 1).astype(int)
    if threads == 1:
        rcs = [run(0, batch)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(lambda i: run(bounds[i], bounds[i + 1]), range(threads)))
    bad = [rc for rc in rcs if rc != 0]
    if bad:
        raise ValueError(f"oracle rejected the input (code {bad[0]})")
    return {"err": err, "iters": iters, "ok": ok, "post": post}


# ------------------------------------------------------------------------------------------------
# Neural normalized min-sum (learned weights w[t][e], CSR edge order)
# ------------------------------------------------------------------------------------------------
def nms_train(row_ptr, col_idx, m, n, syndromes, targets, prior, weights, grad_loss=None,
              precision: str = "f64", post: bool = False, threads: int = 1, loss_weights=None,
              loss: str = "error"):
    """Training pass of the neural min-sum decoder: T iterations, no stop test.

    weights: [T, E] (E = nnz, CSR edge order).  precision "f64" or "f32" is the type the forward
    runs in; losses and gradients are always float64.  loss_weights: [T] per-iteration weights
    lambda_t (None: 1/T each).  loss "error": BCE of sigma(-Q) against the sampled error;
    "syndrome": BCE of the soft syndrome against s (targets unused).  Returns a dict with
      loss [B]          sum_t lambda_t / n sum_v BCE(sigma(-Q^t_v), y_v)   ("error"), or
                        sum_t lambda_t / m sum_c -log P^t_c                 ("syndrome")
      post [B, T, n]    Q^t of every iteration (only with post=True)
      grad [T, E]       sum_b grad_loss[b] d loss_b / d w (only when grad_loss is given)
    """
    lib = _load()
    kind = {"error": 0, "syndrome": 1}[loss]
    if precision == "f64":
        fn, real = lib.oracle_nms_train_f64, np.float64
    elif precision == "f32":
        fn, real = lib.oracle_nms_train_f32, np.float32
    else:
        raise ValueError(f"unknown precision {precision!r}")
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8).reshape(-1, m)
    y = np.ascontiguousarray(targets, dtype=np.uint8).reshape(-1, n)
    w = np.ascontiguousarray(weights, dtype=real)
    T = w.shape[0]
    pr = np.ascontiguousarray(prior, dtype=real).reshape(n)
    B = syn.shape[0]
    out_loss = np.zeros(B, dtype=np.float64)
    posts = np.zeros((B, T, n), dtype=real) if post else None
    g = None if grad_loss is None else np.ascontiguousarray(grad_loss, dtype=np.float64).reshape(B)
    lw = None if loss_weights is None else np.ascontiguousarray(loss_weights, dtype=np.float64).reshape(T)
    threads = max(1, min(int(threads), max(B, 1)))
    bounds = np.linspace(0, B, threads + 1).astype(int)
    parts = [np.zeros_like(w, dtype=np.float64) for _ in range(threads)] if g is not None else None

    def run(i):
        lo, hi = bounds[i], bounds[i + 1]
        if hi <= lo:
            return 0
        return fn(_ptr(rp), _ptr(ci), m, n, _ptr(syn[lo:hi]), _ptr(y[lo:hi]), hi - lo, _ptr(pr), _ptr(w), T,
                  _ptr(lw), kind, _ptr(g[lo:hi]) if g is not None else None, _ptr(out_loss[lo:hi]),
                  _ptr(posts[lo:hi]) if posts is not None else None, _ptr(parts[i]) if parts else None)

    if threads == 1:
        rcs = [run(0)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(run, range(threads)))
    bad = [rc for rc in rcs if rc != 0]
    if bad:
        raise ValueError(f"oracle rejected the input (code {bad[0]})")
    out = {"loss": out_loss}
    if posts is not None:
        out["post"] = posts
    if parts is not None:
        out["grad"] = np.sum(parts, axis=0)
    return out


def nms_decode(row_ptr, col_idx, m, n, syndromes, prior, weights, max_iter_plain, alpha, threads: int = 1):
    """FP32 learned decoding with plain min-sum fallback; dict like msa() plus 'fallback'."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8).reshape(-1, m)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    T = w.shape[0]
    pr = np.ascontiguousarray(prior, dtype=np.float32).reshape(n)
    B = syn.shape[0]
    err = np.zeros((B, n), dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    ok = np.zeros(B, dtype=np.uint8)
    post = np.zeros((B, n), dtype=np.float32)
    fb = np.zeros(B, dtype=np.uint8)
    threads = max(1, min(int(threads), max(B, 1)))
    bounds = np.linspace(0, B, threads + 1).astype(int)

    def run(i):
        lo, hi = bounds[i], bounds[i + 1]
        if hi <= lo:
            return 0
        return lib.oracle_nms_decode_f32(_ptr(rp), _ptr(ci), m, n, _ptr(syn[lo:hi]), hi - lo, _ptr(pr), _ptr(w), T,
                                         int(max_iter_plain), float(np.float32(alpha)), _ptr(err[lo:hi]),
                                         _ptr(iters[lo:hi]), _ptr(ok[lo:hi]), _ptr(post[lo:hi]), _ptr(fb[lo:hi]))

    if threads == 1:
        rcs = [run(0)]
    else:
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(run, range(threads)))
    if any(rcs):
        raise ValueError("oracle rejected the input")
    return {"err": err, "iters": iters, "ok": ok, "post": post, "fallback": fb}
