"""Index and bank arithmetic of the pack transpositions, restated on the CPU.

The producers of the fused pack + filter (and the streaming pack) stage a
block of 256 rows (row r at byte r*m) and hand out LANES x J items, item =
(lane l, position quad j), to the threads in order: thread tid takes items
tid, tid + nthreads, ...  These tests restate that arithmetic from
csrc/shouji_pack.cuh and csrc/shouji_pack_filter.cu and check:
  - the blocks of both producer groups and their items cover every (tile,
    lane, quad) of both sequence sets exactly once, and every output word
    index stays inside the packed array;
  - every shared-memory word read stays inside the staged buffer;
  - within a warp, at every step of the unrolled loop, the odd-word
    transposition (m % 8 == 4) reads 32 distinct banks, and so does the
    general one whenever its rotation step exists.
"""
import pytest

TILE, BLOCK_SEQS, LANES, GROUPS = 1024, 256, 8, 2
HALF_BLOCKS = TILE // BLOCK_SEQS
BLOCKS_PER_TILE = 2 * HALF_BLOCKS


def buf_bytes(m):
    return (BLOCK_SEQS * m + 16 + 127) // 128 * 128


def rotation_step(rs, lanes=LANES):
    """Restated from shouji_pack.cuh: c with c * (rs/4) = 32/lanes (mod 32)."""
    if rs % 4:
        return 0
    W, target = rs // 4, 32 // lanes
    for c in range(32):
        if (c * W) % 32 == target:
            return c
    return 0


def odd_word_rows(l):
    """Row (within the block) that step k = 4q + v reads for lane l."""
    return [32 * l + 4 * ((q + l) % 8) + v for q in range(8) for v in range(4)]


def general_rows(l, rot_step):
    rot = (rot_step * l) % 32
    return [32 * l + (k + rot) % 32 for k in range(32)]


def items(m):
    J = (m + 3) // 4
    return [(item % LANES, item // LANES) for item in range(LANES * J)]


def cta_ranges(n_tiles, sms=152):
    grid = min(n_tiles, sms)
    return [(n_tiles * b // grid, n_tiles * (b + 1) // grid) for b in range(grid)]


@pytest.mark.parametrize("m", [1, 3, 4, 33, 100, 199])
@pytest.mark.parametrize("n", [1, 5000, 300_001])
def test_blocks_and_items_cover_every_output_word_once(m, n):
    tiles = (n + TILE - 1) // TILE
    seen = [bytearray(tiles * m * 32), bytearray(tiles * m * 32)]  # uint2 words of reads, refs
    for T0, T1 in cta_ranges(tiles):
        nblk = (T1 - T0) * BLOCKS_PER_TILE
        for g in range(GROUPS):
            for i in range(g, nblk, GROUPS):
                t = T0 + i // BLOCKS_PER_TILE
                which = (i // HALF_BLOCKS) % 2
                lane0 = (i % HALF_BLOCKS) * LANES
                for l, j in items(m):
                    for q in range(4):
                        p = 4 * j + q
                        if p < m:
                            wi = (t * m + p) * 32 + lane0 + l
                            assert wi < tiles * m * 32
                            seen[which][wi] += 1
    assert all(c == 1 for s in seen for c in s)


@pytest.mark.parametrize("m", list(range(1, 256)))
def test_staged_reads_stay_in_the_buffer(m):
    # the one-block-per-CTA pack stages 256 m + 16 bytes; the rings round that up
    words = (BLOCK_SEQS * m + 16) // 4
    assert buf_bytes(m) // 4 >= words
    rs = m
    for l, j in items(m):
        if m % 8 == 4:  # odd-word transposition
            W = m // 4
            top = max(r * W + j for r in odd_word_rows(l))
        else:
            rows = general_rows(l, rotation_step(rs))
            # the unaligned form reads the word after the first one too
            top = max((r * rs + 4 * j) // 4 + (0 if m % 4 == 0 else 1) for r in rows)
        assert top < words, (m, l, j)


def warp_banks(m, rows_of, W):
    its = items(m)
    for w0 in range(0, len(its) - 31, 32):
        warp = its[w0:w0 + 32]
        for k in range(32):
            yield {(rows_of(l)[k] * W + j) % 32 for l, j in warp}


@pytest.mark.parametrize("m", list(range(4, 256, 8)))
def test_odd_word_transposition_reads_32_banks(m):
    W = m // 4
    for banks in warp_banks(m, odd_word_rows, W):
        assert len(banks) == 32, m


@pytest.mark.parametrize("m", [m for m in range(4, 256, 4) if rotation_step(m)])
def test_rotated_transposition_reads_32_banks(m):
    c = rotation_step(m)
    for banks in warp_banks(m, lambda l: general_rows(l, c), m // 4):
        assert len(banks) == 32, m


# The batched form's persistent pack (csrc/shouji_batch.cu, pack_async_kernel)
# stages 128 rows (4 lanes) at a row stride of m rounded up to 16 bytes (and
# off multiples of 32), leaving `gap` free rows after each lane's 32 rows, and
# pack_transpose_spaced reads each lane's rows in order.

BATCH_SEQS, BATCH_LANES = 128, 4


def batch_row_stride(m):
    rs = (m + 15) & ~15
    return rs + 16 if rs % 32 == 0 else rs


def lane_gap(m):
    return rotation_step(batch_row_stride(m), BATCH_LANES)


def spaced_word(l, k, j, m):
    """Shared-memory word that lane l's item of quad j reads at step k."""
    ws = batch_row_stride(m) // 4
    return (l * (32 + lane_gap(m)) + k) * ws + j


@pytest.mark.parametrize("m", range(1, 256))
def test_spaced_rows_read_32_distinct_banks_and_stay_in_the_buffer(m):
    rs, gap = batch_row_stride(m), lane_gap(m)
    assert gap in (2, 6)  # the step exists for every staged row stride
    # the smallest buffer that holds length m with its gaps (the kernel uses
    # gaps only when its buffer is at least this large)
    buf_words = ((BATCH_SEQS + (BATCH_LANES - 1) * gap) * rs + 16) // 4
    J = (m + 3) // 4
    its = [(item % BATCH_LANES, item // BATCH_LANES) for item in range(BATCH_LANES * J)]
    for w0 in range(0, len(its), 32):
        warp = its[w0:w0 + 32]
        for k in range(32):
            banks = [spaced_word(l, k, j, m) % 32 for l, j in warp]
            assert len(set(banks)) == len(banks), (m, w0, k)
    for l, j in its:
        for k in range(32):
            assert 0 <= spaced_word(l, k, j, m) < buf_words
    # every staged row (where the copies put it) is a row the lanes read
    staged = {r + (r // 32) * gap for r in range(BATCH_SEQS)}
    read = {l * (32 + gap) + k for l in range(BATCH_LANES) for k in range(32)}
    assert staged == read
