"""The allocation-free (key, value) sort (pgs_sort_pairs_static), called through the C ABI,
against the tile lists of pgs_render and against numpy's stable sort.

Some callers cannot allocate device memory themselves (their memory belongs to another
allocator's pool, or a cudaMalloc would synchronise a latency-critical loop); this entry point
keeps its scratch in a fixed device array instead.  The test feeds it the render's pairs in
canonical order (canonical index, then tile) and expects the render's lists (the stable sort of
the pairs by tile and depth) bit for bit, on two calls in a row with different inputs, so the second call also checks that what
the first left in the shared scratch does not leak into the result.

This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2601_17354_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _render_pairs(g, cam):
    from paper_2601_17354_gb300 import _lib as L
    from paper_2601_17354_gb300 import rasterizer as R
    rast = R.Rasterizer()
    rast.render(R.GaussianBuffer.from_arrays(g), cam)
    assert rast.status()[0] == 0
    keys = rast.read_buffer(L.PGS_BUF_KEYS)
    vals = rast.read_buffer(L.PGS_BUF_VALUES)
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    return keys, vals, 32 + max(1, int(np.ceil(np.log2(tiles))))


def _status():
    from paper_2601_17354_gb300 import _lib as L
    return L.lib().pgs_sort_pairs_static_status(C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _static_sort(keys_in, vals_in, key_bits):
    from paper_2601_17354_gb300 import _lib as L
    lib = L.lib()
    kin = torch.from_numpy(keys_in.view(np.int64)).cuda()
    vin = torch.from_numpy(vals_in.view(np.int32)).cuda()
    kout = torch.empty_like(kin)
    vout = torch.empty_like(vin)
    stream = torch.cuda.current_stream()
    rc = lib.pgs_sort_pairs_static(C.c_void_p(kin.data_ptr()), C.c_void_p(vin.data_ptr()),
                                   C.c_void_p(kout.data_ptr()), C.c_void_p(vout.data_ptr()),
                                   len(keys_in), key_bits, C.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.pgs_strerror(rc)
    torch.cuda.synchronize()
    return kout.cpu().numpy().view(np.uint64), vout.cpu().numpy().view(np.uint32)


def _emission_order(keys, vals):
    order = np.lexsort((keys >> np.uint64(32), vals))  # by canonical index, then tile
    return keys[order], vals[order]


def test_static_sort_matches_render_sort_twice():
    scenes = [S.tiny_scene(0)[:2], S.tiny_scene(5, n=3000, width=150, height=90)[:2]]
    for g, cam in scenes:
        keys, vals, bits = _render_pairs(g, cam)
        assert 0 < len(keys) <= 1 << 18
        ek, ev = _emission_order(keys, vals)
        assert not np.array_equal(ek, keys)
        sk, sv = _static_sort(ek, ev, bits)
        assert np.array_equal(sk, keys)
        assert np.array_equal(sv, vals)
        assert _status() == 0


@pytest.mark.parametrize("key_bits", [40, 48, 64, 5])
def test_static_sort_key_bits_and_pass_parity(key_bits):
    """Odd (40 bits: 5 passes; 5 bits: 1 pass) and even (48 bits: 6 passes; 64 bits: 8 passes)
    pass counts, with key bits above key_bits set at random: they take no part in the order (a
    stable sort by the low key_bits bits, checked against numpy's stable argsort), and keys_out
    keeps them."""
    rng = np.random.default_rng(key_bits)
    n = 70_001
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    low = keys & mask
    m = n // 3
    low[0:3 * m:3] = low[1:3 * m:3]  # every third key repeats its neighbour's low bits: ties
    keys = (keys & ~mask) | low
    sort_key = keys & mask
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    order = np.argsort(sort_key, kind="stable")
    for _ in range(2):  # twice: the shared scratch keeps the first call's contents
        sk, sv = _static_sort(keys, vals, key_bits)
        assert np.array_equal(sv, vals[order])
        assert np.array_equal(sk, keys[order])
        assert _status() == 0


def test_static_sort_rejects_sizes_beyond_its_scratch():
    from paper_2601_17354_gb300 import _lib as L
    lib = L.lib()
    rc = lib.pgs_sort_pairs_static(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                   (1 << 18) + 1, 40, None)
    assert rc == L.PGS_ERR_TOO_LARGE
    assert "262144" in lib.pgs_strerror(rc).decode()
