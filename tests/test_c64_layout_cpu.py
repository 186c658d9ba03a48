"""The operand-block layout of the complex64 update (`c64_off`, `c64_padP` and the LBO/SBO of
its shared-memory descriptors in csrc/gf_update_c64.cu), restated in Python: a 128-row x 16-deep
FP16 chunk is stored K-major as 8-row x 16-byte core matrices, the K neighbour core matrix at
+128 bytes (LBO) and the next 8-row group at +256 bytes (SBO).  Every (row, k) must own a
distinct 2-byte slot of the 4 KB half-chunk, rows of one core matrix must be 16 bytes apart and
the two 128-row halves of a 256-row operand must continue with the same strides."""

LBO, SBO = 128, 256


def c64_off(r: int, k: int) -> int:
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2


def c64_padP(p: int) -> int:
    return (p + 15) // 16 * 16


def test_half_chunk_is_a_bijection_onto_4kb():
    offs = sorted(c64_off(r, k) for r in range(128) for k in range(16))
    assert offs == list(range(0, 4096, 2))


def test_core_matrix_strides():
    for r in range(0, 128, 8):
        for k in (0, 8):
            base = c64_off(r, k)
            # one core matrix: 8 rows of 16 contiguous bytes (8 FP16 along K)
            assert [c64_off(r + i, k + j) - base for i in range(8) for j in range(8)] == \
                [16 * i + 2 * j for i in range(8) for j in range(8)]
            if k == 0:
                assert c64_off(r, 8) - base == LBO
            if r + 8 < 128:
                assert c64_off(r + 8, k) - base == SBO
    # a second 128-row part placed right after the first (at +4 KB) continues the SBO progression
    assert c64_off(128, 0) - c64_off(120, 0) == SBO
    assert c64_off(128, 0) - c64_off(0, 0) == 4096


def test_padded_rank_holds_whole_groups_of_four_per_quarter():
    for p in range(1, 129):
        P = c64_padP(p)
        assert P >= p and P % 16 == 0 and P - p < 16
        assert (P // 4) % 4 == 0          # each of the S GEMM's four u-quarters is a multiple of 4
