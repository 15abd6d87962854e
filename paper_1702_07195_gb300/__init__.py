"""Smith-Waterman protein database search on NVIDIA GB300 (sm_103a).

Thin ctypes binding over ``libswgb.so`` (C ABI in ``include/swgb.h``): argument marshalling
only, every step of the search runs in the library's CUDA kernels.  There is no CPU path:
if the library is missing or cannot be loaded, importing this package raises.

Names follow the C ABI: ``sw_db_load``, ``sw_search``, ``sw_search_batch``,
``sw_search_batch_device`` (also exported as ``sw_search_async``), ``sw_get_stats``,
``sw_topk``, ``sw_search_noalloc``, ``Server`` (``sw_server_*``), ``sw_last_error``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB


class SwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"swgb status {status}: {msg}")
        self.status = status


STATUS = {0: "SW_OK", -1: "SW_ERR_ARG", -2: "SW_ERR_CODE", -3: "SW_ERR_OOM", -4: "SW_ERR_CUDA",
          -5: "SW_ERR_TIMEOUT", -6: "SW_ERR_BUSY", -7: "SW_ERR_STATE"}


class DbOptions(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("long_cutoff", ctypes.c_int32),
                ("flag_cap", ctypes.c_int32), ("placement", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


PLACE_DEVICE, PLACE_HOST = 0, 1


class Stats(ctypes.Structure):
    _fields_ = [("inter_ms", ctypes.c_float), ("intra_ms", ctypes.c_float),
                ("rescore_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("cells", ctypes.c_int64), ("inter_cells", ctypes.c_int64),
                ("flagged", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("inter_grid", ctypes.c_int32), ("inter_block", ctypes.c_int32),
                ("graph_replay", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("multi_query", ctypes.c_int32), ("score_profile", ctypes.c_int32),
                ("intra_packed", ctypes.c_int32), ("wave_lanes", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("rows_per_strip", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("num_variants", ctypes.c_int32), ("gcups", ctypes.c_float * 8)]

    def as_dict(self) -> dict:
        return {"variant": self.variant, "rows_per_strip": self.rows_per_strip,
                "warps_per_block": self.warps_per_block, "from_cache": bool(self.from_cache),
                "gcups": [round(float(x), 1) for x in self.gcups[:self.num_variants]]}


class ServerOptions(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("max_query_len", ctypes.c_int32),
                ("state_budget_bytes", ctypes.c_int64), ("slices", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("in_flight", ctypes.c_int32), ("max_in_flight", ctypes.c_int32),
                ("joined_while_running", ctypes.c_int64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
                ("gcups", ctypes.c_double), ("cells", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_u8p = ctypes.POINTER(ctypes.c_uint8)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libswgb.so not built ({LIB_PATH}); run __graft_entry__.build() "
                          "or python paper_1702_07195_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "sw_db_load": (ctypes.c_int, [_u8p, _i64p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_vp)]),
        "sw_db_load_ex": (ctypes.c_int, [_u8p, _i64p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.POINTER(DbOptions), ctypes.POINTER(_vp)]),
        "sw_db_free": (None, [_vp]),
        "sw_db_num_seqs": (ctypes.c_int64, [_vp]),
        "sw_db_num_residues": (ctypes.c_int64, [_vp]),
        "sw_search": (ctypes.c_int, [_vp, _u8p, ctypes.c_int32, _i8p, ctypes.c_int32,
                                     ctypes.c_int32, _i32p]),
        "sw_search_batch": (ctypes.c_int, [_vp, ctypes.POINTER(_u8p), _i32p, ctypes.c_int32, _i8p,
                                           ctypes.c_int32, ctypes.c_int32, _i32p]),
        "sw_search_batch_device": (ctypes.c_int, [_vp, _vp, _i64p, ctypes.c_int32, _i8p,
                                                  ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
        "sw_search_async": (ctypes.c_int, [_vp, _vp, _i64p, ctypes.c_int32, _i8p,
                                           ctypes.c_int32, ctypes.c_int32, _vp, _vp]),
        "sw_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(Stats)]),
        "sw_search_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _i8p, ctypes.c_int32,
                                             ctypes.c_int32, _vp, _vp]),
        "sw_layout_sizes": (ctypes.c_int, [_i64p, ctypes.c_int64, ctypes.c_int32, _i64p, _i64p, _i64p]),
        "sw_layout_build": (ctypes.c_int, [_u8p, _i64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           _i64p, _i32p, _i32p, _u8p, _i32p]),
        "sw_db_tune": (ctypes.c_int, [_vp, ctypes.POINTER(_u8p), _i32p, ctypes.c_int32, _i8p,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                      ctypes.c_int32, ctypes.POINTER(TuneResult)]),
        "sw_db_set_variant": (ctypes.c_int, [_vp, ctypes.c_int32]),
        "sw_server_create": (ctypes.c_int, [_vp, _i8p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(ServerOptions), ctypes.POINTER(_vp)]),
        "sw_server_submit": (ctypes.c_int, [_vp, _u8p, ctypes.c_int32, _i64p]),
        "sw_server_poll": (ctypes.c_int, [_vp, ctypes.c_int64, _i32p, _i32p]),
        "sw_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, _i32p, ctypes.c_int32]),
        "sw_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ServerStats), ctypes.c_int32]),
        "sw_server_destroy": (None, [_vp]),
        "sw_topk": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                   _vp]),
        "sw_last_error": (ctypes.c_char_p, []),
        "sw_version": (ctypes.c_char_p, []),
        "sw_launch_count": (ctypes.c_int64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def sw_last_error() -> str:
    return lib.sw_last_error().decode()


def _check(status: int):
    if status != 0:
        raise SwError(status, f"{STATUS.get(status, status)}: {sw_last_error()}")


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)[:0]
    return a


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _matrix(matrix):
    m = np.ascontiguousarray(matrix, dtype=np.int8)
    if m.ndim != 2 or m.shape[0] != m.shape[1]:
        raise ValueError("matrix must be square (A x A)")
    return m


class Database:
    """A database resident on the GPU (``sw_db``).  Free with ``close()`` or a ``with`` block."""

    def __init__(self, handle, alphabet_size):
        self._h = handle
        self.alphabet_size = alphabet_size

    @property
    def handle(self):
        if not self._h:
            raise ValueError("database is closed")
        return self._h

    @property
    def num_seqs(self) -> int:
        return int(lib.sw_db_num_seqs(self.handle))

    @property
    def num_residues(self) -> int:
        return int(lib.sw_db_num_residues(self.handle))

    def close(self):
        if self._h:
            lib.sw_db_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Residue encoding (the C ABI takes codes in [0, alphabet_size)): NCBI protein order, the order
# of the usual BLOSUM/PAM tables -- 20 standard amino acids, then B, Z, X and the stop symbol.
NCBI_PROTEIN_ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"


def encode(seq: str, alphabet: str = NCBI_PROTEIN_ALPHABET) -> np.ndarray:
    """Letters -> uint8 codes (the letter's position in `alphabet`, case-insensitive).  A letter
    outside the alphabet raises ValueError (the C ABI would answer SW_ERR_CODE)."""
    table = np.full(256, 255, dtype=np.uint8)
    for i, c in enumerate(alphabet):
        table[ord(c.upper())] = i
        table[ord(c.lower())] = i
    raw = np.frombuffer(seq.encode("ascii"), dtype=np.uint8)
    codes = table[raw]
    bad = np.nonzero(codes == 255)[0]
    if bad.size:
        raise ValueError(f"letter {seq[int(bad[0])]!r} at position {int(bad[0])} is not in the alphabet")
    return codes


def encode_database(seqs, alphabet: str = NCBI_PROTEIN_ALPHABET):
    """Sequences (strings) -> (residues uint8, offsets int64) as sw_db_load takes them."""
    codes = [encode(q, alphabet) for q in seqs]
    offsets = np.zeros(len(codes) + 1, dtype=np.int64)
    np.cumsum([c.shape[0] for c in codes], out=offsets[1:])
    residues = np.concatenate(codes) if codes else np.zeros(0, dtype=np.uint8)
    return residues, offsets


def sw_db_load(residues, offsets, alphabet_size: int = 24, long_cutoff: int = 0,
               device: int = 0, flag_cap: int = 0, placement: int = PLACE_DEVICE) -> Database:
    """Preprocess and upload a database (residues uint8 codes, offsets int64[N+1]).

    placement=PLACE_HOST keeps it in pinned host memory that the kernels stream over the
    CPU-GPU link (databases larger than device memory)."""
    r = _u8(residues)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    n = int(o.shape[0] - 1)
    opts = DbOptions()
    opts.device = int(device)
    opts.long_cutoff = int(long_cutoff)
    opts.flag_cap = int(flag_cap)
    opts.placement = int(placement)
    h = _vp()
    _check(lib.sw_db_load_ex(_ptr(r, _u8p), _ptr(o, _i64p), n, int(alphabet_size),
                             ctypes.byref(opts), ctypes.byref(h)))
    return Database(h, alphabet_size)


def sw_search(db: Database, query, matrix, gap_open: int, gap_extend: int) -> np.ndarray:
    """Scores of one query against every database sequence (int32, original order)."""
    q = _u8(query)
    m = _matrix(matrix)
    out = np.empty(db.num_seqs, dtype=np.int32)
    _check(lib.sw_search(db.handle, _ptr(q, _u8p), int(q.shape[0]), _ptr(m, _i8p), int(gap_open),
                         int(gap_extend), _ptr(out, _i32p)))
    return out


def sw_search_batch(db: Database, queries, matrix, gap_open: int, gap_extend: int) -> np.ndarray:
    """Scores of several queries, shape (num_queries, num_seqs), int32."""
    qs = [_u8(q) for q in queries]
    m = _matrix(matrix)
    arr = (_u8p * max(1, len(qs)))(*[_ptr(q, _u8p) for q in qs])
    lens = np.array([q.shape[0] for q in qs] or [0], dtype=np.int32)
    out = np.empty((len(qs), db.num_seqs), dtype=np.int32)
    _check(lib.sw_search_batch(db.handle, arr, _ptr(lens, _i32p), len(qs), _ptr(m, _i8p),
                               int(gap_open), int(gap_extend), _ptr(out, _i32p)))
    return out


def sw_search_batch_device(db: Database, d_queries, query_offsets, matrix, gap_open: int,
                           gap_extend: int, d_scores, stream=None) -> None:
    """Device-resident batch search on torch CUDA tensors; enqueued on ``stream``.

    d_queries: uint8 CUDA tensor of concatenated queries; query_offsets: host int64 array
    (num_queries + 1); d_scores: int32 CUDA tensor of num_queries * num_seqs elements.
    ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None for torch's current stream.
    """
    import torch
    o = np.ascontiguousarray(query_offsets, dtype=np.int64)
    nq = int(o.shape[0] - 1)
    if d_scores.dtype != torch.int32 or not d_scores.is_cuda or not d_scores.is_contiguous():
        raise ValueError("d_scores must be a contiguous int32 CUDA tensor")
    if d_scores.numel() < nq * db.num_seqs:
        raise ValueError("d_scores too small")
    if d_queries.dtype != torch.uint8 or not d_queries.is_cuda or not d_queries.is_contiguous():
        raise ValueError("d_queries must be a contiguous uint8 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream(d_scores.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    m = _matrix(matrix)
    _check(lib.sw_search_batch_device(db.handle, _vp(d_queries.data_ptr()), _ptr(o, _i64p), nq,
                                      _ptr(m, _i8p), int(gap_open), int(gap_extend),
                                      _vp(d_scores.data_ptr()), _vp(s)))


# The boundary's name for the asynchronous device-pointer search; same call.
sw_search_async = sw_search_batch_device


def sw_search_noalloc(db: Database, d_query, matrix, gap_open: int, gap_extend: int, d_scores,
                      stream=None) -> None:
    """One query, no device allocation inside the library (see include/swgb.h).

    For callers that cannot let a library call cudaMalloc at search time.  d_query: uint8
    CUDA tensor; d_scores: int32 CUDA tensor of num_seqs elements.  Calls that overlap on the
    GPU share one fixed scratch array and race: keep them on one stream.
    """
    import torch
    if d_scores.dtype != torch.int32 or not d_scores.is_cuda or not d_scores.is_contiguous():
        raise ValueError("d_scores must be a contiguous int32 CUDA tensor")
    if d_scores.numel() < db.num_seqs:
        raise ValueError("d_scores too small")
    if d_query.dtype != torch.uint8 or not d_query.is_cuda or not d_query.is_contiguous():
        raise ValueError("d_query must be a contiguous uint8 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream(d_scores.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    m = _matrix(matrix)
    _check(lib.sw_search_noalloc(db.handle, _vp(d_query.data_ptr()), int(d_query.numel()),
                                 _ptr(m, _i8p), int(gap_open), int(gap_extend),
                                 _vp(d_scores.data_ptr()), _vp(s)))


def sw_db_tune(db: Database, queries, matrix, gap_open: int, gap_extend: int,
               cache_path: str | None = None, force: bool = False) -> dict:
    """Times every inter-task kernel variant on the probe queries and keeps the fastest."""
    qs = [_u8(q) for q in queries]
    m = _matrix(matrix)
    arr = (_u8p * max(1, len(qs)))(*[_ptr(q, _u8p) for q in qs])
    lens = np.array([q.shape[0] for q in qs] or [0], dtype=np.int32)
    res = TuneResult()
    _check(lib.sw_db_tune(db.handle, arr, _ptr(lens, _i32p), len(qs), _ptr(m, _i8p),
                          int(gap_open), int(gap_extend),
                          cache_path.encode() if cache_path else None, int(force),
                          ctypes.byref(res)))
    return res.as_dict()


def sw_db_set_variant(db: Database, variant: int) -> None:
    _check(lib.sw_db_set_variant(db.handle, int(variant)))


def sw_topk(d_scores, num_seqs: int, num_queries: int, k: int, stream=None):
    """Sorting stage: per query, the k best (score, index) pairs, descending score, ties by
    ascending index.  d_scores: int32 CUDA tensor (num_queries * num_seqs).  Returns two int32
    CUDA tensors of shape (num_queries, k)."""
    import torch
    if d_scores.dtype != torch.int32 or not d_scores.is_cuda or not d_scores.is_contiguous():
        raise ValueError("d_scores must be a contiguous int32 CUDA tensor")
    if d_scores.numel() < num_queries * num_seqs:
        raise ValueError("d_scores too small")
    top_s = torch.empty((num_queries, k), dtype=torch.int32, device=d_scores.device)
    top_i = torch.empty((num_queries, k), dtype=torch.int32, device=d_scores.device)
    if stream is None:
        stream = torch.cuda.current_stream(d_scores.device)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.sw_topk(_vp(d_scores.data_ptr()), int(num_seqs), int(num_queries), int(k),
                       _vp(top_s.data_ptr()), _vp(top_i.data_ptr()), _vp(s)))
    return top_s, top_i


def sw_get_stats(db: Database) -> dict:
    st = Stats()
    _check(lib.sw_get_stats(db.handle, ctypes.byref(st)))
    return st.as_dict()


def sw_launch_count() -> int:
    return int(lib.sw_launch_count())


def sw_layout(residues, offsets, alphabet_size: int = 24, long_cutoff: int = 3072) -> dict:
    """Host-only preprocessing stage (no GPU): the interleaved layout the kernels read."""
    r = _u8(residues)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    n = int(o.shape[0] - 1)
    ng, nb, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.sw_layout_sizes(_ptr(o, _i64p), n, int(long_cutoff), ctypes.byref(ng),
                               ctypes.byref(nb), ctypes.byref(nl)))
    goff = np.zeros(max(1, ng.value), np.int64)
    glen = np.zeros(max(1, ng.value), np.int32)
    perm = np.zeros(max(1, ng.value * 64), np.int32)
    inter = np.zeros(max(1, nb.value), np.uint8)
    lids = np.zeros(max(1, nl.value), np.int32)
    _check(lib.sw_layout_build(_ptr(r, _u8p), _ptr(o, _i64p), n, int(alphabet_size),
                               int(long_cutoff), _ptr(goff, _i64p), _ptr(glen, _i32p),
                               _ptr(perm, _i32p), _ptr(inter, _u8p), _ptr(lids, _i32p)))
    return {"group_off": goff[:ng.value], "group_len": glen[:ng.value],
            "perm": perm[:ng.value * 64], "inter": inter[:nb.value], "long_ids": lids[:nl.value]}


class Server:
    """Continuous-batching search server over a resident database (``sw_server_*``)."""

    def __init__(self, db: Database, matrix, gap_open: int, gap_extend: int,
                 max_inflight: int = 0, max_query_len: int = 0, state_budget_bytes: int = 0,
                 slices: int = 0, max_pending: int = 0):
        self.db = db
        m = _matrix(matrix)
        opts = ServerOptions()
        opts.max_inflight, opts.max_query_len = int(max_inflight), int(max_query_len)
        opts.state_budget_bytes, opts.slices = int(state_budget_bytes), int(slices)
        opts.max_pending = int(max_pending)
        h = _vp()
        _check(lib.sw_server_create(db.handle, _ptr(m, _i8p), int(gap_open), int(gap_extend),
                                    ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    def submit(self, query) -> int:
        q = _u8(query)
        t = ctypes.c_int64()
        _check(lib.sw_server_submit(self._h, _ptr(q, _u8p), int(q.shape[0]), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int):
        out = np.empty(self.db.num_seqs, dtype=np.int32)
        done = ctypes.c_int32()
        _check(lib.sw_server_poll(self._h, int(ticket), _ptr(out, _i32p), ctypes.byref(done)))
        return out if done.value else None

    def wait(self, ticket: int, timeout_ms: int = 60000) -> np.ndarray:
        out = np.empty(self.db.num_seqs, dtype=np.int32)
        _check(lib.sw_server_wait(self._h, int(ticket), _ptr(out, _i32p), int(timeout_ms)))
        return out

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(lib.sw_server_get_stats(self._h, ctypes.byref(st), int(reset)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib.sw_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
