"""CPU-only checks of the C ABI library: it loads, exports every symbol include/*.h
declares, and its host-side preprocessing stage (paper Section 4: sort by length, group,
pad with a dummy code) produces the layout the kernels read.  No compute call needs a GPU.
"""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*"
                             r"([a-z][A-Za-z0-9_]*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def sw():
    import __graft_entry__
    __graft_entry__.build_lib()
    import paper_1702_07195_gb300 as m
    return m


def test_exports_every_declared_symbol(sw):
    names = _declared_functions()
    assert "sw_db_load" in names and "sw_search" in names and len(names) >= 12
    lib = ctypes.CDLL(sw.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert sw.lib.sw_version().decode().startswith("swgb")


def _declaration_docs():
    """(function name, the last column-0 comment before its declaration) for include/*.h."""
    out = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        comments = [(m.start(), m.group(0)) for m in re.finditer(r"^/\*.*?\*/", text, flags=re.S | re.M)
                    if not m.group(0).startswith("/* ----")]
        bare = re.sub(r"/\*.*?\*/", lambda m: " " * len(m.group(0)), text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*"
                             r"([a-z][A-Za-z0-9_]*)\s*\(", bare, flags=re.M):
            doc = [c for pos, c in comments if pos < m.start(1)]
            out.append((m.group(1), doc[-1] if doc else ""))
    return out


def test_every_declaration_cites_its_passage():
    """Each entry point's comment names the paper passage that defines it (a section or an
    equation) or says that the paper has none (serving, housekeeping, no-allocation search)."""
    docs = _declaration_docs()
    assert len(docs) >= 25
    cite = re.compile(r"Section \d|Eq\. |Eqs\. |[Nn]ot in the paper|no counterpart")
    missing = [name for name, doc in docs if not cite.search(doc)]
    assert not missing, f"declarations without a citation: {missing}"
    names = {n for n, _ in docs}
    assert {"sw_search_async", "sw_search_batch_device", "sw_db_tune", "sw_server_create"} <= names


def _reconstruct(lay, num_seqs):
    goff, glen, perm, inter = lay["group_off"], lay["group_len"], lay["perm"], lay["inter"]
    seqs = {}
    for g in range(len(glen)):
        L = int(glen[g])
        j = np.arange(L)
        for s in range(64):
            sid = int(perm[g * 64 + s])
            t, lane = s // 2, s % 2
            idx = goff[g] + (j // 8) * 512 + t * 16 + (j % 8) * 2 + lane
            seqs[(g, s)] = (sid, inter[idx] if L else np.zeros(0, np.uint8))
    return seqs


@pytest.mark.parametrize("cutoff", [64, 3072])
def test_layout_roundtrip(sw, cutoff):
    rng = np.random.default_rng(5)
    lens = np.concatenate([rng.integers(0, 300, size=150), [0, 0, 1, 7, 8, 9, 63, 64, 65],
                           rng.integers(3000, 3300, size=3)])
    rng.shuffle(lens)
    db = w.database_from_lengths(rng, lens)
    A = w.ALPHABET_SIZE
    lay = sw.sw_layout(db.residues, db.offsets, A, long_cutoff=cutoff)
    n = db.num_seqs
    short = [k for k in range(n) if lens[k] <= cutoff]
    longs = [k for k in range(n) if lens[k] > cutoff]
    assert sorted(lay["long_ids"].tolist()) == sorted(longs)
    ll = [int(lens[k]) for k in lay["long_ids"]]
    assert ll == sorted(ll, reverse=True)
    assert len(lay["group_len"]) == (len(short) + 63) // 64
    seen = []
    prev_max = -1
    for (g, s), (sid, data) in sorted(_reconstruct(lay, n).items()):
        L = int(lay["group_len"][g])
        assert L % 8 == 0
        if sid < 0:
            assert (data == A).all()
            continue
        seen.append(sid)
        ln = int(lens[sid])
        assert ln <= L < ln + 8 or L == 0 or ln < L
        assert np.array_equal(data[:ln], db.seq(sid))
        assert (data[ln:] == A).all()
    assert sorted(seen) == short
    # ascending length order across slots and groups
    order_lens = [int(lens[sid]) for sid in lay["perm"] if sid >= 0]
    assert order_lens == sorted(order_lens)
    # group padding = max length rounded to 8
    for g in range(len(lay["group_len"])):
        ids = [int(x) for x in lay["perm"][g * 64:(g + 1) * 64] if x >= 0]
        assert int(lay["group_len"][g]) == (max(int(lens[i]) for i in ids) + 7) // 8 * 8
    # fillers only in the last group's tail
    p = lay["perm"]
    assert (p[: len(short)] >= 0).all() and (p[len(short):] == -1).all()


def test_layout_rejects_bad_input(sw):
    with pytest.raises(sw.SwError) as e:
        sw.sw_layout(np.array([0, 1, 30], np.uint8), np.array([0, 3], np.int64), 24)
    assert e.value.status == -2
    with pytest.raises(sw.SwError) as e:
        sw.sw_layout(np.zeros(4, np.uint8), np.array([0, 3, 2], np.int64), 24)
    assert e.value.status == -1
    with pytest.raises(sw.SwError) as e:
        sw.sw_layout(np.zeros(4, np.uint8), np.array([1, 4], np.int64), 24)
    assert e.value.status == -1
    with pytest.raises(sw.SwError):
        sw.sw_layout(np.zeros(4, np.uint8), np.array([0, 4], np.int64), 24, long_cutoff=12)


def test_layout_empty_database(sw):
    lay = sw.sw_layout(np.zeros(0, np.uint8), np.array([0], np.int64), 24)
    assert len(lay["group_len"]) == 0 and len(lay["long_ids"]) == 0


def test_product_package_has_no_cpu_path():
    """The product package never imports the oracle (a CPU fallback would void parity)."""
    pkg = os.path.join(ROOT, "paper_1702_07195_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "sw_oracle" not in text, path


def test_encoding_helpers(sw):
    """Letters -> codes in the NCBI protein order, the same codes as the BLOSUM62 table's."""
    assert sw.NCBI_PROTEIN_ALPHABET == w.ALPHABET
    seq = "MKTAYIAKQRqisfvkshfsrqLEERLGLIEVQAPILSRVGDGTQDNLSGAEKAVQVKVKALPDAQFEVVHSLAKWKRQTLGQHDFSAGEGLYTHMKALRPDEDRLSPLHSVYVDQWDWERVMGDGERQFSTLKSTVEAIWAGIKATEAAVSEEFGLAPFLPDQIHFVHSQELLSRYPDLDAKGRERAIAKDLGAVFLVGIGGKLSDGHRHDVRAPDYDDWSTPSELGHAGLNGDILVWNPVLEDAFELSSMGIRVDADTLKHQLALTGDEDRLELEWHQALLRGEMPQTIGGGIGQSRLTMLLLQLPHIGQVQAGVWPAACRERVPLY*BZX"
    np.testing.assert_array_equal(sw.encode(seq), w.encode(seq))
    with pytest.raises(ValueError):
        sw.encode("ACGTJ")
    res, off = sw.encode_database(["ARN", "", "W*"])
    np.testing.assert_array_equal(res, [0, 1, 2, 17, 23])
    np.testing.assert_array_equal(off, [0, 3, 3, 5])
    res, off = sw.encode_database(["ACGT", "GG"], alphabet="ACGT")
    np.testing.assert_array_equal(res, [0, 1, 2, 3, 2, 2])
