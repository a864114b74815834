"""The autotune cache file (rdct_autotune_cache_save / _load / _clear): host logic, no GPU needed.

A loaded file contributes exactly its well-formed lines with valid launch shapes; saving writes every
entry back in the same form; clearing empties the cache."""
import ctypes
import os

from paper_1402_6034_gb300 import rdct

LINE = ('{{"key": "{key}", "warps_per_cta": {w}, "ctas_per_sm": {c}, "items_per_chunk": {i}, '
        '"blocks_per_thread": {b}, "staging": {s}}}')


def _entries(path):
    with open(path) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip()]


def test_round_trip_skips_malformed_and_invalid_lines(tmp_path):
    rdct.autotune_cache_clear()
    good = [LINE.format(key="GPU-A/sm103/152:n12:b20:3:3:4", w=4, c=4, i=32, b=2, s=0),
            LINE.format(key="GPU-A/sm103/152:n4096:b26:2:5:3", w=8, c=0, i=8, b=1, s=0)]
    bad = [LINE.format(key="GPU-A/sm103/152:n1:b3:10:0:0", w=0, c=4, i=32, b=2, s=0),   # warps_per_cta 0
           LINE.format(key="GPU-A/sm103/152:n2:b3:10:0:0", w=4, c=4, i=32, b=3, s=0),   # blocks_per_thread 3
           '{"key": "x", "warps_per_cta": 4}',                                          # truncated
           "not json at all"]
    src = tmp_path / "cache_in.jsonl"
    src.write_text("\n".join(bad[:2] + good[:1] + bad[2:] + good[1:]) + "\n")
    assert rdct.autotune_cache_load(str(src)) == 2
    out = tmp_path / "cache_out.jsonl"
    rdct.autotune_cache_save(str(out))
    assert sorted(_entries(out)) == sorted(good)
    # loading the saved file again changes nothing
    assert rdct.autotune_cache_load(str(out)) == 2
    rdct.autotune_cache_save(str(out))
    assert sorted(_entries(out)) == sorted(good)
    rdct.autotune_cache_clear()
    rdct.autotune_cache_save(str(out))
    assert _entries(out) == []


def test_errors(tmp_path):
    lib = rdct.load()
    assert lib.rdct_autotune_cache_load(os.fsencode(str(tmp_path / "missing.jsonl")), None) == 8
    assert lib.rdct_autotune_cache_load(None, None) == 1
    assert lib.rdct_autotune_cache_save(None) == 1
    assert lib.rdct_autotune_cache_save(os.fsencode(str(tmp_path / "no_such_dir" / "x.jsonl"))) == 1
    n = ctypes.c_int32(-1)
    empty = tmp_path / "empty.jsonl"
    empty.write_text("")
    assert lib.rdct_autotune_cache_load(os.fsencode(str(empty)), ctypes.byref(n)) == 0 and n.value == 0
