"""The server's device-budget arena (host logic; runs without a GPU).

Checks first-fit placement, alignment, coalescing of neighbours on free, OOM
without side effects, and a long random alloc/free sequence against a plain
Python model of the free space.
"""
import numpy as np
import pytest

from paper_1402_6034_gb300 import rdct


@pytest.fixture(scope="module")
def lib():
    return rdct.load()


def test_alignment_and_first_fit(lib):
    a = rdct.Arena(1 << 16, 256)
    x = a.alloc(1)
    y = a.alloc(257)
    z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768)
    assert a.used == 1024
    a.free(y)
    assert a.alloc(300) == 256  # first fit reuses the hole
    a.close()


def test_coalescing_restores_one_block(lib):
    a = rdct.Arena(4096, 256)
    offs = [a.alloc(256) for _ in range(16)]
    assert a.alloc(1) is None  # full: OOM, nothing changes
    assert a.used == 4096
    for o in offs[::2]:
        a.free(o)
    assert a.largest_free == 256
    for o in offs[1::2]:
        a.free(o)
    assert a.used == 0 and a.largest_free == 4096
    a.close()


def test_errors(lib):
    a = rdct.Arena(4096, 256)
    with pytest.raises(rdct.RdctError) as e:
        a.free(123)
    assert e.value.status == 8
    assert a.alloc(8192) is None
    with pytest.raises(rdct.RdctError):
        rdct.Arena(4096, 100)  # alignment must be a power of two
    a.close()


def test_random_sequence_matches_model(lib):
    size, align = 1 << 20, 256
    a = rdct.Arena(size, align)
    rng = np.random.default_rng(0)
    live = {}  # offset -> aligned size
    for step in range(4000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 40000))
            off = a.alloc(n)
            need = (n + align - 1) // align * align
            if off is None:
                # model: no gap of `need` bytes may exist
                edges = sorted(live.items())
                pos, biggest = 0, 0
                for o, s in edges:
                    biggest = max(biggest, o - pos)
                    pos = o + s
                biggest = max(biggest, size - pos)
                assert biggest < need
            else:
                assert off % align == 0 and off + need <= size
                for o, s in live.items():  # no overlap
                    assert off + need <= o or o + s <= off
                live[off] = need
        assert a.used == sum(live.values())
    for off in list(live):
        a.free(off)
    assert a.used == 0 and a.largest_free == size
    a.close()
