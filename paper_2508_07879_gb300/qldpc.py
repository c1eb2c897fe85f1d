"""Python binding of libqldpc.so (include/qldpc.h) -- argument marshalling only.

The functions named ``qldpc_*`` mirror the C ABI one to one and take raw integers for pointers.
``Graph``, ``decode``, ``decode_pair`` and ``decode_host`` wrap them for torch tensors and numpy
arrays.  Every step of the decoder runs in the library's CUDA kernels; this module never computes
a message, a decision or a syndrome check, and there is no CPU fallback: if the library is missing
or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqldpc.so")

QLDPC_OK = 0
QLDPC_PENDING = 1
QLDPC_BUSY = 2
QLDPC_ERR_INVALID_ARG = -1
QLDPC_ERR_UNSUPPORTED = -2
QLDPC_ERR_OOM = -3
QLDPC_ERR_CUDA = -4
QLDPC_ERR_TIMEOUT = -5
QLDPC_FP32 = 0
QLDPC_INT16 = 1
QLDPC_INT8 = 2
QLDPC_NO_EARLY_STOP = 1
QLDPC_LEARNED = 2
QLDPC_LAYERED = 4
QLDPC_LOSS_ERROR = 0
QLDPC_LOSS_SYNDROME = 1
LOSSES = {"error": QLDPC_LOSS_ERROR, "syndrome": QLDPC_LOSS_SYNDROME}
QLDPC_MAX_ROW_DEGREE = 32
QLDPC_MAX_COL_DEGREE = 16
QLDPC_MAX_CHECKS = 65535
QLDPC_KERNEL_AUTO = 0
QLDPC_KERNEL_BATCH = 1
QLDPC_KERNEL_LATENCY = 2
QLDPC_KERNEL_PACKED = 3
KERNELS = {"auto": QLDPC_KERNEL_AUTO, "batch": QLDPC_KERNEL_BATCH, "latency": QLDPC_KERNEL_LATENCY,
           "packed": QLDPC_KERNEL_PACKED}

PRECISIONS = {"fp32": QLDPC_FP32, "int16": QLDPC_INT16, "int8": QLDPC_INT8}


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                          f"g.build()'` (or paper_2508_07879_gb300/build.py) first")
    return ctypes.CDLL(LIB_PATH)


_lib = _load()


class ServerConfig(ctypes.Structure):
    """qldpc_server_config (include/qldpc.h)."""
    _fields_ = [("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("ring_capacity", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("blocks", ctypes.c_int32 * 4),
                ("idle_timeout_ns", ctypes.c_int64), ("max_runtime_ns", ctypes.c_int64)]

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_f32 = ctypes.c_float

_SIGNATURES = {
    "qldpc_graph_create": ([_p, _p, _i32, _i32, ctypes.POINTER(_p)], ctypes.c_int),
    "qldpc_graph_create_csc": ([_p, _p, _i32, _i32, ctypes.POINTER(_p)], ctypes.c_int),
    "qldpc_graph_destroy": ([_p], None),
    "qldpc_graph_dims": ([_p, _p, _p, _p, _p, _p], ctypes.c_int),
    "qldpc_graph_layers": ([_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], ctypes.c_int),
    "qldpc_graph_footprint": ([_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "qldpc_graph_set_launch": ([_p, _i32, _i32, _i32], ctypes.c_int),
    "qldpc_graph_reserve": ([_p, _i32], ctypes.c_int),
    "qldpc_decode": ([_p, _p, _i32, _p, _i32, _f32, _p, _p, _p], ctypes.c_int),
    "qldpc_decode_ex": ([_p, _p, _i32, _p, _i32, _f32, _p, _p, _p, _p, _i32, _u32, _p], ctypes.c_int),
    "qldpc_decode_pair": ([_p, _p, _p, _p, _i32, _p, _p, _i32, _f32, _p, _p, _p, _p, _p, _p, _p, _p,
                           _i32, _u32, _p], ctypes.c_int),
    "qldpc_decode_host": ([_p, _p, _i32, _p, _i32, _f32, _p, _p, _p, _i32, _u32, _p], ctypes.c_int),
    "qldpc_decode_pair_host": ([_p, _p, _p, _p, _i32, _p, _p, _i32, _f32, _p, _p, _p, _p, _p, _p, _i32, _u32, _p],
                               ctypes.c_int),
    "qldpc_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "qldpc_decode_host_noalloc": ([_p, _p, _i32, _p, _i32, _f32, _p, _p, _p, _i32, _u32, _p], ctypes.c_int),
    "qldpc_noalloc_scratch_bytes": ([], ctypes.c_size_t),
    "qldpc_server_create": ([_p, _p, _i32, ctypes.POINTER(ServerConfig), ctypes.POINTER(_p)], ctypes.c_int),
    "qldpc_server_submit": ([_p, _i32, _p, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "qldpc_server_poll": ([_p, _i32, ctypes.c_uint64, _p, _p, _p], ctypes.c_int),
    "qldpc_server_replay": ([_p, _i32, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, ctypes.c_int64], ctypes.c_int),
    "qldpc_server_status": ([_p, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "qldpc_server_info": ([_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_size_t)],
                          ctypes.c_int),
    "qldpc_server_destroy": ([_p], None),
    "qldpc_graph_set_weights": ([_p, _p, _i32], ctypes.c_int),
    "qldpc_nms_workspace_bytes": ([_p, _i32, _i32, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "qldpc_nms_forward": ([_p, _p, _p, _i32, _p, _p, _i32, _p, _i32, _p, _p, _p, ctypes.c_size_t, _p], ctypes.c_int),
    "qldpc_nms_backward": ([_p, _p, _p, _i32, _p, _i32, _p, _i32, _p, _p, _p, ctypes.c_size_t, _p], ctypes.c_int),
    "qldpc_adam_step": ([_p, _p, _p, _p, ctypes.c_int64, _i32, _f32, _f32, _f32, _f32, _p], ctypes.c_int),
    "qldpc_sample_errors": ([_p, ctypes.c_uint64, ctypes.c_int64, _i32, ctypes.c_double, ctypes.c_double, _p, _p,
                             _p], ctypes.c_int),
    "qldpc_logical_failures": ([_p, _i32, _i32, _p, _p, _p, _i32, _p, _p], ctypes.c_int),
}
for _name, (_args, _res) in _SIGNATURES.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

# Raw C entry points, same names as include/qldpc.h.
qldpc_graph_create = _lib.qldpc_graph_create
qldpc_graph_create_csc = _lib.qldpc_graph_create_csc
qldpc_graph_destroy = _lib.qldpc_graph_destroy
qldpc_graph_dims = _lib.qldpc_graph_dims
qldpc_graph_footprint = _lib.qldpc_graph_footprint
qldpc_graph_layers = _lib.qldpc_graph_layers
qldpc_graph_set_launch = _lib.qldpc_graph_set_launch
qldpc_graph_reserve = _lib.qldpc_graph_reserve
qldpc_decode = _lib.qldpc_decode
qldpc_decode_ex = _lib.qldpc_decode_ex
qldpc_decode_pair = _lib.qldpc_decode_pair
qldpc_decode_host = _lib.qldpc_decode_host
qldpc_decode_pair_host = _lib.qldpc_decode_pair_host
qldpc_status_string = _lib.qldpc_status_string
qldpc_decode_host_noalloc = _lib.qldpc_decode_host_noalloc
qldpc_noalloc_scratch_bytes = _lib.qldpc_noalloc_scratch_bytes
qldpc_server_create = _lib.qldpc_server_create
qldpc_server_submit = _lib.qldpc_server_submit
qldpc_server_poll = _lib.qldpc_server_poll
qldpc_server_replay = _lib.qldpc_server_replay
qldpc_server_status = _lib.qldpc_server_status
qldpc_server_info = _lib.qldpc_server_info
qldpc_server_destroy = _lib.qldpc_server_destroy
qldpc_graph_set_weights = _lib.qldpc_graph_set_weights
qldpc_nms_workspace_bytes = _lib.qldpc_nms_workspace_bytes
qldpc_nms_forward = _lib.qldpc_nms_forward
qldpc_nms_backward = _lib.qldpc_nms_backward
qldpc_adam_step = _lib.qldpc_adam_step
qldpc_sample_errors = _lib.qldpc_sample_errors
qldpc_logical_failures = _lib.qldpc_logical_failures
QLDPC_NOALLOC_SCRATCH_BYTES = qldpc_noalloc_scratch_bytes()   # as compiled into the library


class QldpcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = qldpc_status_string(status).decode()
        super().__init__(f"{what}: {msg}" if what else msg)


def check(status: int, what: str = "") -> None:
    if status != QLDPC_OK:
        raise QldpcError(status, what)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data            # an int: ctypes passes it as the void* the signature declares


def _dev_ptr(t, dtype, shape, name):
    """Device pointer of a contiguous CUDA tensor of the given dtype and shape (validation only)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Graph:
    """A Tanner graph uploaded to the current CUDA device (owns a qldpc_graph)."""

    def __init__(self, row_ptr, col_idx, m: int, n: int):
        self._h = None
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        if rp.shape != (m + 1,):
            raise ValueError("row_ptr must have m+1 entries")
        h = ctypes.c_void_p()
        check(qldpc_graph_create(_np_ptr(rp), _np_ptr(ci) if ci.size else None, int(m), int(n),
                                 ctypes.byref(h)), "qldpc_graph_create")
        self._h = h
        self.m, self.n, self.nnz = int(m), int(n), int(rp[-1])
        self.learned_iters = 0

    @classmethod
    def from_csr(cls, csr) -> "Graph":
        return cls(csr.row_ptr, csr.col_idx, csr.m, csr.n)

    @classmethod
    def from_dense(cls, h) -> "Graph":
        h = np.asarray(h, dtype=np.uint8) & 1
        rows, cols = np.nonzero(h)
        rp = np.zeros(h.shape[0] + 1, dtype=np.int32)
        np.add.at(rp, rows + 1, 1)
        return cls(np.cumsum(rp), cols, h.shape[0], h.shape[1])

    @property
    def handle(self):
        return self._h

    def dims(self):
        vals = [ctypes.c_int32() for _ in range(5)]
        check(qldpc_graph_dims(self._h, *[ctypes.byref(v) for v in vals]), "qldpc_graph_dims")
        return tuple(v.value for v in vals)

    def layers(self, widest: bool = False):
        """Number of layers of the layered schedule in this row order (and the widest layer)."""
        n_l, w_l = _i32(), _i32()
        check(qldpc_graph_layers(self._h, ctypes.byref(n_l), ctypes.byref(w_l)), "qldpc_graph_layers")
        return (n_l.value, w_l.value) if widest else n_l.value

    def footprint(self, precision: str = "fp32"):
        """(variable lanes, shared-memory bytes of one shot in the throughput kernel)."""
        lanes, nbytes = ctypes.c_int32(), ctypes.c_size_t()
        check(qldpc_graph_footprint(self._h, PRECISIONS[precision], ctypes.byref(lanes), ctypes.byref(nbytes)),
              "qldpc_graph_footprint")
        return lanes.value, nbytes.value

    def set_launch(self, kernel: str = "auto", threads_per_block: int = 0, blocks_per_sm: int = 0) -> None:
        """Force a kernel ("batch" / "latency") and optionally its shape; "auto" restores the default."""
        check(qldpc_graph_set_launch(self._h, KERNELS[kernel], int(threads_per_block), int(blocks_per_sm)),
              "qldpc_graph_set_launch")

    def reserve(self, max_batch: int) -> None:
        check(qldpc_graph_reserve(self._h, int(max_batch)), "qldpc_graph_reserve")

    def set_weights(self, weights) -> None:
        """Learned weights float32 [T, nnz] (CSR edge order; numpy, or a torch tensor on the host
        or this device) for decodes with learned=True; None clears them."""
        if weights is None:
            check(qldpc_graph_set_weights(self._h, None, 0), "qldpc_graph_set_weights")
            self.learned_iters = 0
            return
        try:
            import torch
            is_tensor = isinstance(weights, torch.Tensor)
        except ImportError:
            is_tensor = False
        if is_tensor:
            w = weights.detach()
            if w.dtype != torch.float32 or w.dim() != 2 or w.shape[1] != self.nnz:
                raise ValueError(f"weights must be float32 [T, {self.nnz}]")
            w = w.contiguous()
            T = int(w.shape[0])
            check(qldpc_graph_set_weights(self._h, ctypes.c_void_p(w.data_ptr()) if T else None, T),
                  "qldpc_graph_set_weights")
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            if w.ndim != 2 or w.shape[1] != self.nnz:
                raise ValueError(f"weights must be float32 [T, {self.nnz}]")
            T = int(w.shape[0])
            check(qldpc_graph_set_weights(self._h, _np_ptr(w) if T else None, T), "qldpc_graph_set_weights")
        self.learned_iters = T

    def close(self) -> None:
        if self._h:
            qldpc_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _flags(early_stop: bool, learned: bool, layered: bool = False) -> int:
    return ((0 if early_stop else QLDPC_NO_EARLY_STOP) | (QLDPC_LEARNED if learned else 0)
            | (QLDPC_LAYERED if layered else 0))


def decode(graph: Graph, syndromes, prior, max_iter: int, alpha: float = 0.75,
           precision: str = "fp32", early_stop: bool = True, want_post: bool = False,
           out=None, stream=None, learned: bool = False, layered: bool = False):
    """Decode syndromes (CUDA uint8 [B, m]) with prior LLRs (CUDA float32 [n]).

    Returns (err uint8 [B, n], iters int32 [B], ok uint8 [B], post float32 [B, n] or None), all
    CUDA tensors, enqueued on ``stream`` (default: torch's current stream).  ``out`` may supply
    the four output tensors to avoid allocation.  ``learned``: the graph's learned weights first,
    then plain min-sum for up to ``max_iter`` iterations on shots not yet decoded.  ``layered``:
    the row-serial schedule instead of flooding.
    """
    import torch
    batch = int(syndromes.shape[0]) if syndromes.dim() == 2 else 0
    dev = syndromes.device
    if out is None:
        err = torch.empty((batch, graph.n), dtype=torch.uint8, device=dev)
        iters = torch.empty(batch, dtype=torch.int32, device=dev)
        ok = torch.empty(batch, dtype=torch.uint8, device=dev)
        post = torch.empty((batch, graph.n), dtype=torch.float32, device=dev) if want_post else None
    else:
        err, iters, ok, post = out
    flags = _flags(early_stop, learned, layered)
    check(qldpc_decode_ex(graph.handle,
                          _dev_ptr(syndromes, torch.uint8, (batch, graph.m), "syndromes"), batch,
                          _dev_ptr(prior, torch.float32, (graph.n,), "prior"), int(max_iter),
                          float(alpha),
                          _dev_ptr(err, torch.uint8, (batch, graph.n), "err"),
                          _dev_ptr(iters, torch.int32, (batch,), "iters"),
                          _dev_ptr(ok, torch.uint8, (batch,), "ok"),
                          _dev_ptr(post, torch.float32, (batch, graph.n), "post") if post is not None else None,
                          PRECISIONS[precision], flags, _stream_handle(stream)),
          "qldpc_decode_ex")
    return err, iters, ok, post


def decode_soft(graph: Graph, syndromes, prior, syndrome_llr, max_iter: int, alpha: float = 0.75,
                precision: str = "fp32", early_stop: bool = True, want_post: bool = False, stream=None,
                layered: bool = False):
    """Soft-syndrome decoding: ``graph`` is the data-syndrome Tanner graph [H | I_m]
    (``workloads.data_syndrome_csr``), ``syndromes`` the measured bits (CUDA uint8 [B, m]),
    ``prior`` the data LLRs (CUDA float32 [n]) and ``syndrome_llr`` the LLRs that each measured bit
    is right (CUDA float32 [m], ln((1 - q)/q) for a read error rate q).  Runs the ordinary decode
    on that graph with the priors side by side; returns (err [B, n], syndrome errors [B, m], iters,
    ok, post [B, n + m] or None)."""
    import torch
    n = graph.n - graph.m
    if n < 1 or prior.shape != (n,) or syndrome_llr.shape != (graph.m,):
        raise ValueError("decode_soft expects a data-syndrome graph, prior [n] and syndrome_llr [m]")
    full = torch.cat([prior.float(), syndrome_llr.float()]).contiguous()
    err, iters, ok, post = decode(graph, syndromes, full, max_iter, alpha, precision, early_stop, want_post,
                                  stream=stream, layered=layered)
    return err[:, :n], err[:, n:], iters, ok, post


def decode_pair(g_z: Graph, g_x: Graph, s_x, s_z, prior_x, prior_z, max_iter: int,
                alpha: float = 0.75, precision: str = "fp32", early_stop: bool = True,
                want_post: bool = False, stream=None, learned: bool = False, layered: bool = False):
    """X and Z halves of a CSS syndrome round in one launch; returns two (err, iters, ok, post)."""
    import torch
    batch = int(s_x.shape[0])
    dev = s_x.device
    outs = []
    for g in (g_z, g_x):
        outs.append((torch.empty((batch, g.n), dtype=torch.uint8, device=dev),
                     torch.empty(batch, dtype=torch.int32, device=dev),
                     torch.empty(batch, dtype=torch.uint8, device=dev),
                     torch.empty((batch, g.n), dtype=torch.float32, device=dev) if want_post else None))
    (ex, ix, ox, px), (ez, iz, oz, pz) = outs
    flags = _flags(early_stop, learned, layered)
    check(qldpc_decode_pair(g_z.handle, g_x.handle,
                            _dev_ptr(s_x, torch.uint8, (batch, g_z.m), "s_x"),
                            _dev_ptr(s_z, torch.uint8, (batch, g_x.m), "s_z"), batch,
                            _dev_ptr(prior_x, torch.float32, (g_z.n,), "prior_x"),
                            _dev_ptr(prior_z, torch.float32, (g_x.n,), "prior_z"),
                            int(max_iter), float(alpha),
                            _dev_ptr(ex, torch.uint8, (batch, g_z.n), "err_x"),
                            _dev_ptr(ez, torch.uint8, (batch, g_x.n), "err_z"),
                            _dev_ptr(ix, torch.int32, (batch,), "iters_x"),
                            _dev_ptr(iz, torch.int32, (batch,), "iters_z"),
                            _dev_ptr(ox, torch.uint8, (batch,), "ok_x"),
                            _dev_ptr(oz, torch.uint8, (batch,), "ok_z"),
                            _dev_ptr(px, torch.float32, (batch, g_z.n), "post_x") if want_post else None,
                            _dev_ptr(pz, torch.float32, (batch, g_x.n), "post_z") if want_post else None,
                            PRECISIONS[precision], flags, _stream_handle(stream)),
          "qldpc_decode_pair")
    return (ex, ix, ox, px), (ez, iz, oz, pz)


def decode_host(graph: Graph, syndromes: np.ndarray, prior: np.ndarray, max_iter: int,
                alpha: float = 0.75, precision: str = "fp32", early_stop: bool = True,
                out=None, stream=None, layered: bool = False):
    """End-to-end decode from host (numpy) buffers; synchronous.  Returns (err, iters, ok) numpy.

    Pass page-locked arrays (e.g. ``torch.empty(..., pin_memory=True).numpy()``) for fast copies.
    """
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8)
    batch = syn.shape[0]
    if syn.shape != (batch, graph.m):
        raise ValueError(f"syndromes must have shape (B, {graph.m})")
    pr = np.ascontiguousarray(prior, dtype=np.float32)
    if pr.shape != (graph.n,):
        raise ValueError(f"prior must have shape ({graph.n},)")
    if out is None:
        err = np.empty((batch, graph.n), dtype=np.uint8)
        iters = np.empty(batch, dtype=np.int32)
        ok = np.empty(batch, dtype=np.uint8)
    else:
        err, iters, ok = out
    flags = _flags(early_stop, False, layered)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    check(qldpc_decode_host(graph.handle, _np_ptr(syn), batch, _np_ptr(pr), int(max_iter),
                            float(alpha), _np_ptr(err), _np_ptr(iters), _np_ptr(ok),
                            PRECISIONS[precision], flags, sh), "qldpc_decode_host")
    return err, iters, ok


def decode_pair_host(graph_z: Graph, graph_x: Graph, s_x: np.ndarray, s_z: np.ndarray, prior_x: np.ndarray,
                     prior_z: np.ndarray, max_iter: int, alpha: float = 0.75, precision: str = "fp32",
                     early_stop: bool = True, out=None, stream=None, layered: bool = False):
    """X+Z pair decode (one launch) end to end from host (numpy) buffers; synchronous.  s_x [B, m_z]
    is decoded with graph_z, s_z [B, m_x] with graph_x.  Returns ((err_x, iters_x, ok_x), (err_z,
    iters_z, ok_z)); out, if given, is that pair of triples (page-locked arrays avoid all copies)."""
    sx = np.ascontiguousarray(s_x, dtype=np.uint8)
    sz = np.ascontiguousarray(s_z, dtype=np.uint8)
    batch = sx.shape[0]
    if sx.shape != (batch, graph_z.m) or sz.shape != (batch, graph_x.m):
        raise ValueError("s_x must be (B, m_z) and s_z (B, m_x)")
    px = np.ascontiguousarray(prior_x, dtype=np.float32)
    pz = np.ascontiguousarray(prior_z, dtype=np.float32)
    if out is None:
        out = tuple((np.empty((batch, graph_z.n), np.uint8), np.empty(batch, np.int32), np.empty(batch, np.uint8))
                    for _ in range(2))
    (ex, ix, ox), (ez, iz, oz) = out
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    check(qldpc_decode_pair_host(graph_z.handle, graph_x.handle, _np_ptr(sx), _np_ptr(sz), batch, _np_ptr(px),
                                 _np_ptr(pz), int(max_iter), float(alpha), _np_ptr(ex), _np_ptr(ez), _np_ptr(ix),
                                 _np_ptr(iz), _np_ptr(ox), _np_ptr(oz), PRECISIONS[precision],
                                 _flags(early_stop, False, layered), sh), "qldpc_decode_pair_host")
    return out


class Server:
    """Persistent decoding server over up to four codes (qldpc_server_*).

    graphs: list of Graph; priors: list of float32 [n] numpy arrays (host).  The worker kernel starts
    on the first request and leaves after `idle_timeout_s` without requests (restarted on demand).
    layered=True: workers on the layered schedule (rows of degree <= 8, at most 256 checks per layer).
    """

    def __init__(self, graphs, priors, max_iter: int, alpha: float = 0.75, precision: str = "fp32",
                 early_stop: bool = True, ring_capacity: int = 256, blocks=None,
                 idle_timeout_s: float = 0.5, max_runtime_s: float = 600.0, threads_per_block: int = 0,
                 learned: bool = False, layered: bool = False):
        self._h = None
        self.graphs = list(graphs)
        self._priors = [np.ascontiguousarray(p, dtype=np.float32) for p in priors]
        cfg = ServerConfig()
        cfg.precision = PRECISIONS[precision]
        cfg.max_iter = int(max_iter)
        cfg.alpha = float(alpha)
        cfg.flags = _flags(early_stop, learned, layered)
        cfg.ring_capacity = int(ring_capacity)
        cfg.threads_per_block = int(threads_per_block)
        for i, b in enumerate(blocks or []):
            cfg.blocks[i] = int(b)
        cfg.idle_timeout_ns = int(idle_timeout_s * 1e9)
        cfg.max_runtime_ns = int(max_runtime_s * 1e9)
        garr = (ctypes.c_void_p * len(self.graphs))(*[g.handle.value for g in self.graphs])
        parr = (ctypes.c_void_p * len(self._priors))(*[p.ctypes.data for p in self._priors])
        h = ctypes.c_void_p()
        check(qldpc_server_create(garr, parr, len(self.graphs), ctypes.byref(cfg), ctypes.byref(h)),
              "qldpc_server_create")
        self._h = h

    def submit(self, code: int, syndrome) -> int:
        """Returns a ticket, or None when the code's ring is full."""
        syn = np.ascontiguousarray(syndrome, dtype=np.uint8)
        if syn.shape != (self.graphs[code].m,):
            raise ValueError("syndrome must have shape (m,)")
        t = ctypes.c_uint64()
        rc = qldpc_server_submit(self._h, int(code), _np_ptr(syn), ctypes.byref(t))
        if rc == QLDPC_BUSY:
            return None
        check(rc, "qldpc_server_submit")
        return t.value

    def poll(self, code: int, ticket: int):
        """(err, iters, ok) when done, else None."""
        err = np.empty(self.graphs[code].n, dtype=np.uint8)
        it = ctypes.c_int32()
        ok = ctypes.c_uint8()
        rc = qldpc_server_poll(self._h, int(code), ctypes.c_uint64(ticket), _np_ptr(err), ctypes.byref(it),
                               ctypes.byref(ok))
        if rc == QLDPC_PENDING:
            return None
        check(rc, "qldpc_server_poll")
        return err, it.value, ok.value

    def replay(self, codes, syndromes, arrival_ns, timeout_s: float = 10.0, want_workers: bool = False):
        """Open-loop replay: request i = (codes[i], syndromes[i]) submitted at arrival_ns[i].

        Returns (errs list of uint8 arrays, iters int32 [R], ok uint8 [R], latency_ns int64 [R]), plus
        workers int32 [R] (the worker block that decoded each request) with want_workers=True.
        """
        codes = np.ascontiguousarray(codes, dtype=np.int32)
        nreq = len(codes)
        syn_parts = [np.ascontiguousarray(x, dtype=np.uint8) for x in syndromes]
        syn_off = np.zeros(nreq, dtype=np.int64)
        err_off = np.zeros(nreq, dtype=np.int64)
        if nreq:
            syn_off[1:] = np.cumsum([len(x) for x in syn_parts])[:-1]
            ns = np.array([self.graphs[c].n for c in codes], dtype=np.int64)
            err_off[1:] = np.cumsum(ns)[:-1]
            syn_flat = np.concatenate(syn_parts)
            # written once here, so that its pages are in place before the replay's clock starts
            err_flat = np.empty(int(ns.sum()), dtype=np.uint8)
            err_flat.fill(0)
        else:
            syn_flat = np.zeros(1, dtype=np.uint8)
            err_flat = np.zeros(1, dtype=np.uint8)
        arrival = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        iters = np.full(nreq, 0, dtype=np.int32)      # np.full writes every page, unlike np.zeros
        ok = np.full(nreq, 0, dtype=np.uint8)
        lat = np.full(nreq, 0, dtype=np.int64)
        workers = np.full(max(nreq, 1), -1, dtype=np.int32)
        check(qldpc_server_replay(self._h, nreq, _np_ptr(codes), _np_ptr(syn_flat), _np_ptr(syn_off),
                                  _np_ptr(arrival), _np_ptr(err_flat), _np_ptr(err_off), _np_ptr(iters),
                                  _np_ptr(ok), _np_ptr(lat), _np_ptr(workers), int(timeout_s * 1e9)),
              "qldpc_server_replay")
        errs = [err_flat[err_off[i]:err_off[i] + self.graphs[codes[i]].n] for i in range(nreq)]
        if want_workers:
            return errs, iters, ok, lat, workers[:nreq]
        return errs, iters, ok, lat

    def info(self) -> dict:
        """The worker pool: {"workers", "threads_per_block", "smem_per_block"}."""
        wk, th, sm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
        check(qldpc_server_info(self._h, ctypes.byref(wk), ctypes.byref(th), ctypes.byref(sm)), "qldpc_server_info")
        return {"workers": wk.value, "threads_per_block": th.value, "smem_per_block": sm.value}

    def status(self) -> int:
        st = ctypes.c_uint32()
        check(qldpc_server_status(self._h, ctypes.byref(st)), "qldpc_server_status")
        return st.value

    def close(self) -> None:
        if self._h:
            qldpc_server_destroy(self._h)
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


# ------------------------------------------------------------------------------------------------
# Learned decoder training and evaluation helpers (device tensors in, device tensors out)
# ------------------------------------------------------------------------------------------------
def nms_workspace_bytes(graph: Graph, batch: int, T: int) -> int:
    out = ctypes.c_size_t()
    check(qldpc_nms_workspace_bytes(graph.handle, int(batch), int(T), ctypes.byref(out)), "qldpc_nms_workspace_bytes")
    return out.value


def nms_forward(graph: Graph, syndromes, targets, prior, weights, workspace, want_post: bool = False, stream=None,
                loss_weights=None, loss: str = "error"):
    """Training forward (qldpc_nms_forward).  workspace: CUDA uint8 tensor of at least
    nms_workspace_bytes(graph, B, T) bytes; loss_weights: CUDA float32 [T] or None (1/T each);
    loss "error" or "syndrome" (targets may be None for "syndrome").
    Returns (loss float32 [B], post float32 [B, n] or None)."""
    import torch
    kind = LOSSES[loss]
    batch = int(syndromes.shape[0])
    T = int(weights.shape[0])
    out = torch.empty(batch, dtype=torch.float32, device=syndromes.device)
    post = torch.empty((batch, graph.n), dtype=torch.float32, device=syndromes.device) if want_post else None
    check(qldpc_nms_forward(graph.handle, _dev_ptr(syndromes, torch.uint8, (batch, graph.m), "syndromes"),
                            _dev_ptr(targets, torch.uint8, (batch, graph.n), "targets")
                            if targets is not None else None, batch,
                            _dev_ptr(prior, torch.float32, (graph.n,), "prior"),
                            _dev_ptr(weights, torch.float32, (T, graph.nnz), "weights"), T,
                            _dev_ptr(loss_weights, torch.float32, (T,), "loss_weights")
                            if loss_weights is not None else None, kind,
                            _dev_ptr(out, torch.float32, (batch,), "loss"),
                            _dev_ptr(post, torch.float32, (batch, graph.n), "post") if post is not None else None,
                            ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel() * workspace.element_size()),
                            _stream_handle(stream)), "qldpc_nms_forward")
    return out, post


def nms_backward(graph: Graph, syndromes, targets, prior, T: int, grad_loss, workspace, stream=None,
                 loss_weights=None, loss: str = "error"):
    """Training backward (qldpc_nms_backward) after nms_forward on the same workspace (same loss).
    Returns the weight gradient float32 [T, nnz]."""
    import torch
    kind = LOSSES[loss]
    batch = int(syndromes.shape[0])
    grad = torch.empty((int(T), graph.nnz), dtype=torch.float32, device=syndromes.device)
    check(qldpc_nms_backward(graph.handle, _dev_ptr(syndromes, torch.uint8, (batch, graph.m), "syndromes"),
                             _dev_ptr(targets, torch.uint8, (batch, graph.n), "targets")
                             if targets is not None else None, batch,
                             _dev_ptr(prior, torch.float32, (graph.n,), "prior"), int(T),
                             _dev_ptr(loss_weights, torch.float32, (int(T),), "loss_weights")
                             if loss_weights is not None else None, kind,
                             _dev_ptr(grad_loss, torch.float32, (batch,), "grad_loss"),
                             _dev_ptr(grad, torch.float32, (int(T), graph.nnz), "grad"),
                             ctypes.c_void_p(workspace.data_ptr()), int(workspace.numel() * workspace.element_size()),
                             _stream_handle(stream)), "qldpc_nms_backward")
    return grad


def adam_step(params, grads, exp_avg, exp_avg_sq, step: int, lr: float = 1e-3, betas=(0.9, 0.999),
              eps: float = 1e-8, stream=None) -> None:
    """In-place Adam update of CUDA float32 tensors of one shape (qldpc_adam_step)."""
    import torch
    shape = tuple(params.shape)
    count = int(params.numel())
    check(qldpc_adam_step(_dev_ptr(params, torch.float32, shape, "params"),
                          _dev_ptr(grads, torch.float32, shape, "grads"),
                          _dev_ptr(exp_avg, torch.float32, shape, "exp_avg"),
                          _dev_ptr(exp_avg_sq, torch.float32, shape, "exp_avg_sq"), count, int(step), float(lr),
                          float(betas[0]), float(betas[1]), float(eps), _stream_handle(stream)), "qldpc_adam_step")


def sample_errors(graph: Graph, seed: int, first_shot: int, batch: int, p_lo: float, p_hi=None, device=None,
                  stream=None):
    """Device-side seeded errors and syndromes (qldpc_sample_errors).  Returns (err [B, n], syn [B, m])."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    p_hi = p_lo if p_hi is None else p_hi
    err = torch.empty((int(batch), graph.n), dtype=torch.uint8, device=dev)
    syn = torch.empty((int(batch), graph.m), dtype=torch.uint8, device=dev)
    check(qldpc_sample_errors(graph.handle, ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(first_shot),
                              int(batch), float(p_lo), float(p_hi),
                              _dev_ptr(err, torch.uint8, (int(batch), graph.n), "err") if batch else None,
                              _dev_ptr(syn, torch.uint8, (int(batch), graph.m), "syn") if batch else None,
                              _stream_handle(stream)), "qldpc_sample_errors")
    return err, syn


def logical_failures(logicals, errors, decisions, ok, stream=None):
    """fail uint8 [B] (qldpc_logical_failures); logicals: CUDA uint8 [k, n]."""
    import torch
    k, n = int(logicals.shape[0]), int(logicals.shape[1])
    batch = int(errors.shape[0])
    fail = torch.empty(batch, dtype=torch.uint8, device=errors.device)
    check(qldpc_logical_failures(_dev_ptr(logicals, torch.uint8, (k, n), "logicals"), k, n,
                                 _dev_ptr(errors, torch.uint8, (batch, n), "errors"),
                                 _dev_ptr(decisions, torch.uint8, (batch, n), "decisions"),
                                 _dev_ptr(ok, torch.uint8, (batch,), "ok"), batch,
                                 _dev_ptr(fail, torch.uint8, (batch,), "fail"), _stream_handle(stream)),
          "qldpc_logical_failures")
    return fail
