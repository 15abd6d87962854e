"""sw_search_noalloc: the search entry point for callers that cannot let the library
allocate device memory at search time (services overlapping many streams, where cudaMalloc
may synchronise the device; processes whose device memory belongs to another allocator;
code that must not allocate after start-up).

The entry point is called directly through the C ABI (ctypes) and its scores are compared,
element by element (integer scores: tolerance 0, as in every parity test here), with the
existing entry point sw_search_batch_device on two calls in a row.  The database mixes
short subjects (int16x2 inter-task kernel), planted hits that saturate int16 lanes (int32
rescore) and subjects above the intra-task cutoff.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

MAX_QUERY = 8192     # SW_NOALLOC_MAX_QUERY in include/swgb.h
SW_ERR_ARG = -1


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_lib()
    import paper_1702_07195_gb300 as m
    return m


def _c_entry(sw):
    fn = ctypes.CDLL(sw.LIB_PATH).sw_search_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_int8), ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _database():
    wl = w.plain(seed=31, scale=0.05)
    db2, q_sat, _ = w.plant_saturating(wl.db, wl.queries[0][:60], count=4, run=3200)
    rng = np.random.default_rng(77)
    longs = [w.draw_residues(rng, n) for n in (4500, 5200, 6100)]
    seqs = [db2.seq(i) for i in range(db2.num_seqs)] + longs
    return w.from_sequences(seqs), [wl.queries[0], q_sat], wl.matrix


def test_noalloc_matches_existing_entry_point(sw):
    import torch
    db, queries, matrix = _database()
    fn = _c_entry(sw)
    mat = np.ascontiguousarray(matrix, np.int8)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE, long_cutoff=4096) as h:
        n = h.num_seqs
        stream = torch.cuda.current_stream()
        free_delta = []
        for q in queries:                                   # two calls in a row
            dq = torch.from_numpy(q).cuda()
            ref = torch.empty(n, dtype=torch.int32, device="cuda")
            sw.sw_search_batch_device(h, dq, np.array([0, len(q)], np.int64), matrix, 10, 2, ref)
            got = torch.full((n,), -9, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            st = fn(h.handle, dq.data_ptr(), len(q),
                    mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), 10, 2, got.data_ptr(),
                    stream.cuda_stream)
            assert st == 0, sw.sw_last_error()
            torch.cuda.synchronize()
            free_delta.append(free0 - torch.cuda.mem_get_info()[0])
            r, g = ref.cpu().numpy(), got.cpu().numpy()
            bad = np.nonzero(r != g)[0]
            assert bad.size == 0, f"{bad.size} mismatches, first at {bad[0]}: {g[bad[0]]} vs {r[bad[0]]}"
        assert int(ref.max()) > 32767          # the second query saturates int16 lanes
        assert free_delta[1] == 0               # the second call allocated nothing


def test_noalloc_rejects_oversized_query(sw):
    import torch
    db, _, matrix = _database()
    fn = _c_entry(sw)
    mat = np.ascontiguousarray(matrix, np.int8)
    with sw.sw_db_load(db.residues, db.offsets, w.ALPHABET_SIZE) as h:
        dq = torch.zeros(MAX_QUERY + 1, dtype=torch.uint8, device="cuda")
        out = torch.empty(h.num_seqs, dtype=torch.int32, device="cuda")
        st = fn(h.handle, dq.data_ptr(), MAX_QUERY + 1,
                mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), 10, 2, out.data_ptr(), None)
        assert st == SW_ERR_ARG
        assert "SW_NOALLOC_MAX_QUERY" in sw.sw_last_error()
