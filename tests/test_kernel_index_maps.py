"""CPU checks of kernel index arithmetic (the maps written out again here, with
the kernels' constants): every staged element lands in exactly one in-bounds
shared-memory slot and every read finds the element it means; MMA widths stay
valid; output coordinates cover each block exactly once."""
import itertools


# --- pre_add3_bt_kernel: 8 (n) x 32 (k) patch, 256 threads, 16 float4 each ----

BT_N, BT_K, BT_PITCH, THREADS = 8, 32, 9, 256
SMEM_FLOATS = 64 * BT_K * BT_PITCH


def bt_stage(t, j):
    """(sub-block ab, row kr, first column) and the shared offset of the float4."""
    L = t + THREADS * j
    ab, kr, q = L >> 6, (L & 63) >> 1, L & 1
    return ab, kr, 4 * q, (ab * BT_K + kr) * BT_PITCH + 4 * q


def test_bt_staging_is_a_bijection_onto_the_tile():
    seen = {}
    for t, j in itertools.product(range(THREADS), range(16)):
        ab, kr, c0, off = bt_stage(t, j)
        assert 0 <= ab < 64 and 0 <= kr < BT_K and c0 in (0, 4)
        for c in range(4):
            key = (ab, kr, c0 + c)
            assert key not in seen
            seen[key] = off + c
            assert 0 <= off + c < SMEM_FLOATS
    assert len(seen) == 64 * BT_K * BT_N
    # each thread's reads: X[a][b] at position (tn, tk) is element (8a + b, tk, tn)
    for t in range(THREADS):
        tn, tk = t >> 5, t & 31
        for a, b in itertools.product(range(8), range(8)):
            assert ((a * 8 + b) * BT_K + tk) * BT_PITCH + tn == seen[(a * 8 + b, tk, tn)]


def test_bt_reads_are_bank_conflict_free_per_warp():
    for warp in range(THREADS // 32):
        for a, b in itertools.product(range(8), range(8)):
            banks = {(((a * 8 + b) * BT_K + (t & 31)) * BT_PITCH + (t >> 5)) % 32
                     for t in range(32 * warp, 32 * warp + 32)}
            assert len(banks) == 32


def test_bt_global_coordinates_follow_the_sub_block_layout():
    # element (ab, kr, c) of the patch at (n0, k0) is B[b * w + k][a * h + n],
    # i.e. B^T sub-block (a, b) at leaf position (n, k)
    h, w, n0, k0 = 24, 40, 16, 32
    for t, j in itertools.product(range(THREADS), range(16)):
        ab, kr, c0, _ = bt_stage(t, j)
        a, b = ab >> 3, ab & 7
        k, n = k0 + kr, n0 + c0
        row, col = b * w + k, a * h + n
        assert (row // w, row % w) == (b, k) or k >= w
        assert (col // h, col % h) == (a, n) or n >= h


# --- narrow last tile column (tile_cols) --------------------------------------

def tile_cols(n_total, tn, width):
    rem = n_total - tn * width
    return width if rem >= width else (rem + 31) & ~31


def test_tile_cols_gives_valid_mma_widths():
    for width in (128, 256):
        for n in range(1, 3 * width + 1):
            tiles = (n + width - 1) // width
            for tn in range(tiles):
                c = tile_cols(n, tn, width)
                assert c % 32 == 0 and 32 <= c <= width
                assert tn * width + c >= min(n, (tn + 1) * width)   # covers every valid column
                if width == 256:   # CTA pair: each CTA stages c / 2 rows of B, a multiple of 16
                    assert (c // 2) % 16 == 0


def test_pair_b_halves_meet_for_narrow_tiles():
    # CTA 0 stages tile rows [0, 128), CTA 1 rows [c / 2, c / 2 + 128); the MMA
    # reads [0, c / 2) from CTA 0 and [c / 2, c) from CTA 1
    for c in range(32, 257, 32):
        cta0 = set(range(0, c // 2))
        cta1 = set(range(c // 2, c))
        assert cta0 | cta1 == set(range(c)) and not (cta0 & cta1)
        assert c // 2 <= 128 and c - c // 2 <= 128


# --- post_add3_kernel output blocks --------------------------------------------

def test_post_add3_writes_each_node_block_once():
    seen = set()
    for q0 in range(4):
        for s in range(16):
            q1, q2 = s >> 2, s & 3
            rb = 4 * (q0 >> 1) + 2 * (q1 >> 1) + (q2 >> 1)
            cb = 4 * (q0 & 1) + 2 * (q1 & 1) + (q2 & 1)
            assert (rb, cb) not in seen
            seen.add((rb, cb))
    assert seen == set(itertools.product(range(8), range(8)))


# --- batched maxima: one 32 x 128 block per CTA, 4 float4 per thread -----------

def test_batched_absmax_block_covers_every_element_once():
    seen = set()
    for t, j in itertools.product(range(256), range(4)):
        g = t + 256 * j
        r, c = g >> 5, 4 * (g & 31)
        for d in range(4):
            assert (r, c + d) not in seen
            seen.add((r, c + d))
    assert seen == set(itertools.product(range(32), range(128)))
