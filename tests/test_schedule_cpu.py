"""Host logic of the static schedule (no GPU): every cell of every instance is
owned by exactly one warp segment, blocks get equal cell counts, and warps
inside a block get equal strip-rows to within one row."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_1309_1720_gb300 import build, _lib
    build.build()
    return _lib.lib()


def schedule(L, nxs, nys, cx, G, NW):
    n = len(nxs)
    a = (ctypes.c_int32 * n)(*nxs)
    b = (ctypes.c_int32 * n)(*nys)
    ws = (ctypes.c_int32 * (G * NW + 1))()
    ns = ctypes.c_int64()
    assert L.cg_static_schedule(a, b, n, cx, G, NW, None, 0, ws, ctypes.byref(ns)) == 0
    segs = (ctypes.c_int32 * (10 * max(1, ns.value)))()
    assert L.cg_static_schedule(a, b, n, cx, G, NW, segs, ns.value, ws, ctypes.byref(ns)) == 0
    return np.array(segs[:10 * ns.value]).reshape(-1, 10), np.array(ws[:])


@pytest.mark.parametrize("nxs,nys,cx,G,NW", [
    ([1024], [1024], 2, 152, 16),
    ([128], [128], 2, 152, 16),
    ([2], [2], 1, 152, 16),
    ([67], [45], 1, 7, 4),
    ([150, 97, 2, 64, 300], [97, 150, 3, 64, 11], 2, 13, 8),
    ([2048], [2048], 2, 152, 16),
])
def test_exact_cover_and_balance(L, nxs, nys, cx, G, NW):
    segs, ws = schedule(L, nxs, nys, cx, G, NW)
    own = [np.zeros((ny, nx), dtype=np.int32) for nx, ny in zip(nxs, nys)]
    tw = 32 * cx
    per_warp = np.zeros(G * NW, dtype=np.int64)
    per_block = np.zeros(G, dtype=np.int64)
    for w in range(G * NW):
        for k in range(ws[w], ws[w + 1]):
            inst, x0, y0, y1, ra, a0, a1, rb, b0, b1 = segs[k]
            nx = nxs[inst]
            assert x0 % tw == 0 and 0 <= y0 <= y1 < nys[inst]
            per_warp[w] += y1 - y0 + 1
            for y in range(y0, y1 + 1):
                for x in range(x0, min(x0 + tw, nx)):
                    if y == ra and not (a0 <= x < a1):
                        continue
                    if y == rb and not (b0 <= x < b1):
                        continue
                    own[inst][y, x] += 1
                    per_block[w // NW] += 1
    for o in own:
        assert np.all(o == 1)
    total = sum(nx * ny for nx, ny in zip(nxs, nys))
    assert per_block.max() - per_block.min() <= 1 + (0 if total >= G else 1)
    for b in range(G):
        pw = per_warp[b * NW:(b + 1) * NW]
        assert pw.max() - pw.min() <= 1
