"""The C-ABI library builds, loads and exports every function include/ob.h declares.
No compute calls: this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ob.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ob_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ob_price_ask_bid", "ob_price_ask_bid_plain", "ob_crr_american",
              "ob_price_ask_bid_host", "ob_get_stats", "ob_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1110_2477_gb300 import _build
    lib_path = _build.build()
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n), n
    import paper_1110_2477_gb300 as ob
    assert set(_declared()) <= set(ob.EXPORTS)


def test_strerror_without_gpu():
    import paper_1110_2477_gb300 as ob
    from paper_1110_2477_gb300 import _build
    _build.build()
    assert ob.ob_strerror(0) == "ok"
    assert "capacity" in ob.ob_strerror(-3) or "outgrew" in ob.ob_strerror(-3)
    assert ob.ob_strerror(12345) == "unknown status code"


def test_option_record_layout_matches_header():
    import workloads as W
    assert W.OPTION_DTYPE.itemsize == 64
    assert [W.OPTION_DTYPE.fields[f][1] for f in ("S0", "K", "K2", "sigma", "R", "T", "k", "N", "payoff")] == \
        [0, 8, 16, 24, 32, 40, 48, 56, 60]


def test_stats_record_matches_header():
    """The binding's ob_stats_t mirrors the header's fields, in order."""
    import re
    from paper_1110_2477_gb300 import ObStats
    text = open(os.path.join(ROOT, "include", "ob.h")).read()
    body = text[text.index("typedef struct {", text.index("Counters of the most recent")):]
    body = body[:body.index("} ob_stats_t;")]
    fields = re.findall(r"^\s*(int64_t|int32_t)\s+(\w+);", body, re.M)
    assert [n for _, n in fields] == [n for n, _ in ObStats._fields_]
    sizes = {"int64_t": 8, "int32_t": 4}
    packed = sum(sizes[t] for t, _ in fields)
    assert ctypes.sizeof(ObStats) == (packed + 7) // 8 * 8  # tail padding to the int64 alignment
