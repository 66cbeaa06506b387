"""Host logic of the static schedule (no GPU): every cell of every instance is
owned by exactly one warp segment, blocks own consecutive ranges that start
at strip-row starts and hold equal numbers of strip-rows (to within one),
warps inside a block get equal strip-rows to within one row, and each
block's dependency range covers the owners of its whole one-cell halo."""
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
    assert L.cg_static_schedule(a, b, n, cx, G, NW, None, 0, ws, ctypes.byref(ns), None) == 0
    segs = (ctypes.c_int32 * (10 * max(1, ns.value)))()
    deps = (ctypes.c_int32 * (2 * G))()
    assert L.cg_static_schedule(a, b, n, cx, G, NW, segs, ns.value, ws, ctypes.byref(ns), deps) == 0
    return (np.array(segs[:10 * ns.value]).reshape(-1, 10), np.array(ws[:]),
            np.array(deps[:]).reshape(G, 2))


CASES = [
    ([1024], [1024], 2, 152, 16),
    ([128], [128], 2, 152, 16),
    ([2], [2], 1, 152, 16),
    ([67], [45], 1, 7, 4),
    ([150, 97, 2, 64, 300], [97, 150, 3, 64, 11], 2, 13, 8),
    ([2048], [2048], 2, 152, 16),
]


@pytest.mark.parametrize("nxs,nys,cx,G,NW", CASES)
def test_exact_cover_and_balance(L, nxs, nys, cx, G, NW):
    segs, ws, deps = schedule(L, nxs, nys, cx, G, NW)
    own = [np.full((ny, nx), -1, dtype=np.int64) for nx, ny in zip(nxs, nys)]
    tw = 32 * cx
    per_warp = np.zeros(G * NW, dtype=np.int64)
    per_block = np.zeros(G, dtype=np.int64)
    for w in range(G * NW):
        for k in range(ws[w], ws[w + 1]):
            inst, x0, y0, y1, ra, a0, a1, rb, b0, b1 = segs[k]
            nx = nxs[inst]
            assert x0 % tw == 0 and 0 <= y0 <= y1 < nys[inst]
            per_warp[w] += y1 - y0 + 1
            x1 = min(x0 + tw, nx)
            blk = np.zeros((y1 - y0 + 1, x1 - x0), dtype=bool)
            blk[:] = True
            xs = np.arange(x0, x1)
            if y0 <= ra <= y1:
                blk[ra - y0] = (xs >= a0) & (xs < a1)
            if y0 <= rb <= y1:
                blk[rb - y0] = (xs >= b0) & (xs < b1)
            sub = own[inst][y0:y1 + 1, x0:x1]
            assert np.all(sub[blk] == -1)
            sub[blk] = w // NW
            per_block[w // NW] += int(blk.sum())
    for o in own:
        assert np.all(o >= 0)
    # blocks own whole strip-rows, consecutive in plan order, equal in
    # number to within one
    flat = np.concatenate([o.reshape(-1) for o in own])
    assert np.all(np.diff(flat) >= 0)
    strips = np.zeros(G, dtype=np.int64)
    for o in own:
        ny, nx = o.shape
        for x0 in range(0, nx, tw):
            blk = o[:, x0:x0 + tw]
            assert np.all(blk == blk[:, :1])
            np.add.at(strips, blk[:, 0], 1)
    assert strips.max() - strips.min() <= 1
    assert per_block.sum() == flat.size
    for b in range(G):
        pw = per_warp[b * NW:(b + 1) * NW]
        assert pw.max() - pw.min() <= 1
    # every block owning a cell within one row/column of block b's cells lies
    # in b's dependency range
    for o in own:
        ny, nx = o.shape
        lo = np.full((ny, nx), np.iinfo(np.int64).max)
        hi = np.full((ny, nx), -1)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                src = o[max(0, dy):ny + min(0, dy), max(0, dx):nx + min(0, dx)]
                dst = (slice(max(0, -dy), ny + min(0, -dy)), slice(max(0, -dx), nx + min(0, -dx)))
                lo[dst] = np.minimum(lo[dst], src)
                hi[dst] = np.maximum(hi[dst], src)
        assert np.all(deps[o, 0] <= lo) and np.all(hi <= deps[o, 1])


def adjoint_schedule(L, nx, ny, cx, G, NW):
    ws = (ctypes.c_int32 * (G * NW + 1))()
    ns = ctypes.c_int64()
    assert L.cg_adjoint_schedule(nx, ny, cx, G, NW, None, 0, ws, ctypes.byref(ns)) == 0
    segs = (ctypes.c_int32 * (10 * max(1, ns.value)))()
    assert L.cg_adjoint_schedule(nx, ny, cx, G, NW, segs, ns.value, ws, ctypes.byref(ns)) == 0
    return np.array(segs[:10 * ns.value]).reshape(-1, 10), np.array(ws[:])


def _scaled(nx, ny, tw):
    """Cells on the adjoint's scaled boundary path: rows 0, 1, ny-2, ny-1 and
    the column strips starting at column <= 1 or reaching column nx-2."""
    m = np.zeros((ny, nx), dtype=bool)
    m[:2] = True
    m[max(0, ny - 2):] = True
    for x0 in range(0, nx, tw):
        if x0 <= 1 or x0 + tw >= nx - 1:
            m[:, x0:x0 + tw] = True
    return m


@pytest.mark.parametrize("nx,ny,cx,G,NW", [
    (512, 512, 2, 152, 16), (1024, 1024, 2, 152, 16), (129, 65, 2, 152, 16), (67, 45, 1, 7, 4),
    (2, 2, 1, 152, 16), (3, 7, 2, 5, 4), (4096, 3, 2, 152, 16), (65, 300, 1, 13, 8),
])
def test_adjoint_schedule_cover_and_cost_balance(L, nx, ny, cx, G, NW):
    """Exact cover by warp segments, no segment mixing the first or last two
    rows with interior rows, warps inside a block within one
    strip-row of each other, blocks owning whole strip-rows, and block costs
    (1.4 per strip-row on the scaled boundary path, 1 otherwise) equal to
    within one strip-row at each end of a block (2 x 1.4)."""
    segs, ws = adjoint_schedule(L, nx, ny, cx, G, NW)
    tw = 32 * cx
    own = np.full((ny, nx), -1, dtype=np.int64)
    per_warp = np.zeros(G * NW, dtype=np.int64)
    for w in range(G * NW):
        for k in range(ws[w], ws[w + 1]):
            inst, x0, y0, y1, ra, a0, a1, rb, b0, b1 = segs[k]
            assert inst == 0 and x0 % tw == 0 and 0 <= y0 <= y1 < ny
            # rows 0, 1, ny-2, ny-1 never share a segment with interior rows
            edge = [y <= 1 or y >= ny - 2 for y in range(y0, y1 + 1)]
            assert all(edge) or not any(edge), (y0, y1, ny)
            per_warp[w] += y1 - y0 + 1
            x1 = min(x0 + tw, nx)
            blk = np.ones((y1 - y0 + 1, x1 - x0), dtype=bool)
            xs = np.arange(x0, x1)
            if y0 <= ra <= y1:
                blk[ra - y0] = (xs >= a0) & (xs < a1)
            if y0 <= rb <= y1:
                blk[rb - y0] = (xs >= b0) & (xs < b1)
            sub = own[y0:y1 + 1, x0:x1]
            assert np.all(sub[blk] == -1)
            sub[blk] = w // NW
    assert np.all(own >= 0)
    for b in range(G):
        pw = per_warp[b * NW:(b + 1) * NW]
        assert pw.max() - pw.min() <= 1
    # blocks own consecutive row-major ranges, in block order
    flat = own.reshape(-1)
    assert np.all(np.diff(flat) >= 0)
    scaled = _scaled(nx, ny, tw)
    per_block = np.zeros(G)
    for x0 in range(0, nx, tw):
        blk = own[:, x0:x0 + tw]
        assert np.all(blk == blk[:, :1])
        np.add.at(per_block, blk[:, 0], np.where(scaled[:, x0], 1.4, 1.0))
    if ny * ((nx + tw - 1) // tw) >= 4 * G:
        assert per_block.max() - per_block.min() <= 2.8 + 1e-9


# ---------------------------------------------------------------------------
# Temporally blocked kernel (cg_tblock.cuh): the index arithmetic of its
# stage rounds and of its neighbour waits, restated here and checked before
# it runs on a GPU.

def _stage_round_cells(threads, m):
    """Cell of each thread in a round of m cells (-1: surplus lane, -2: warp
    skips the round), as the stage loop of k_tblock assigns them."""
    tid = np.arange(threads)
    wid = tid >> 5
    out = np.where(tid < m, tid, -1)
    out[(wid << 5) >= m] = -2
    return out


@pytest.mark.parametrize("threads", [64, 96, 128, 256, 384, 512])
def test_tblock_stage_rounds_cover_once(threads):
    """Every cell of a round goes to exactly one active lane, packed into
    ceil(m/32) warps (the FP64 pipe costs a whole warp per instruction
    however many lanes are active); the other warps skip the round."""
    for m in range(1, threads + 1):
        cells = _stage_round_cells(threads, m)
        act = cells[cells >= 0]
        assert np.array_equal(np.sort(act), np.arange(m)), m
        running = [w for w in range(threads // 32) if not (cells[32 * w:32 * w + 32] == -2).all()]
        assert len(running) == (m + 31) // 32, m
        for w in running:
            assert (cells[32 * w:32 * w + 32] >= 0).any(), (m, w)


def _tb_window(t0, t1, n, h):
    return (-1 if t0 - h <= 0 else t0 - h), (n + 1 if t1 + h >= n else t1 + h)


@pytest.mark.parametrize("n", [2, 3, 7, 45, 128, 301])
@pytest.mark.parametrize("tx", [1, 2, 5, 11, 16, 64])
@pytest.mark.parametrize("H", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("bc", [0, 1])
def test_tblock_neighbour_ranges(n, tx, H, bc):
    """A tile's window (tile plus H cells, ghosts at the edges read from the
    cells they mirror or repeat) lies in the tiles within ceil(H/tx) of it,
    the range a block waits for between passes."""
    tiles = (n + tx - 1) // tx
    r = (H + tx - 1) // tx
    for b in range(tiles):
        w0, w1 = _tb_window(b * tx, min(b * tx + tx, n), n, H)
        for g in range(w0, w1):
            if g < 0:
                src = (1 if n > 1 else 0) if bc == 0 else 0
            elif g >= n:
                src = (n - 2 if n > 1 else 0) if bc == 0 else n - 1
            else:
                src = g
            assert abs(src // tx - b) <= r, (b, g, src)
