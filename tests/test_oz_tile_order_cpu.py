"""The tile order of the complex128 tensor-core update for one problem (`OzSingleSrc::range`,
`first` and `next` in csrc/gf_update_tc.cu), restated in Python.

The tiles are the (row tile, column tile) grid, nrt x nct, in row-major order.  When a tile row
holds at least one tile per CTA and its B digit blocks (6208 bytes per column tile) fit in
16 MB, CTA c walks tiles c, c + g, c + 2g, ...  Otherwise CTA c walks the contiguous range
[T c / g, T (c + 1) / g).  Both must visit every tile exactly once, through the cursor's
incremental steps, and each CTA's tiles come in row-major order (the A digit tile is reloaded
only when the row tile changes)."""
import random

B_BLOCK = 6 * 32 * 8 * 4 + 64          # kOzBBlock: six digit slices of 32 x 8 TF32 + 16 exponents
MAX_B = 16 << 20                        # kOzInterleaveMaxB


def tile_range(nrt, nct, c, g):
    T = nrt * nct
    if nct >= g and nct * B_BLOCK <= MAX_B:
        return c, T, g
    return T * c // g, T * (c + 1) // g, 1


def walk(nrt, nct, c, g):
    tb, te, ts = tile_range(nrt, nct, c, g)
    out = []
    if tb < te:
        rt, ct = divmod(tb, nct)                      # first()
        t = tb
        while t < te:
            out.append((rt, ct))
            t += ts
            ct += ts                                  # next()
            while ct >= nct:
                ct -= nct
                rt += 1
    return out


def _check(nrt, nct, g):
    seen = []
    for c in range(g):
        tiles = walk(nrt, nct, c, g)
        assert tiles == sorted(tiles)                 # row-major within a CTA
        seen += tiles
    assert sorted(seen) == [(r, k) for r in range(nrt) for k in range(nct)]


def test_every_tile_once_in_both_orders():
    rng = random.Random(3)
    cases = [(1, 1, 1), (1, 5, 152), (3, 151, 152), (2, 152, 152), (4, 153, 152), (7, 2305, 152),
             (1, 2702, 152), (2, 2703, 152), (5, 300, 7)]
    cases += [(rng.randint(1, 40), rng.randint(1, 3000), rng.choice([1, 2, 7, 76, 152])) for _ in range(60)]
    for nrt, nct, g in cases:
        _check(nrt, nct, g)


def test_order_chosen_for_the_measured_sizes():
    g = 152
    # 128x128 (n = 16385) and 192x192 (n = 36865) brushes: interleaved; 320x320 (n = 102401): contiguous
    for n, interleaved in ((16385, True), (36865, True), (102401, False), (4097, True), (50, False)):
        nct = (n + 15) // 16
        nrt = (n + 127) // 128
        assert (tile_range(nrt, nct, 0, g)[2] == g) == interleaved, n
    # the limit sits between n = 43,232 (2702 column tiles) and the next tile
    assert 2702 * B_BLOCK <= MAX_B < 2703 * B_BLOCK
