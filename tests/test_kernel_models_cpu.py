"""CPU models of kernel index arithmetic that must hold for every access to
stay in bounds and every element to be counted once.  Each test restates one
kernel's rule in Python and checks it exhaustively or on random cases, so a
change to the rule can be checked here before it runs on a GPU."""
import random

import numpy as np

def test_engine_fp4_slot_ring_waits_cover_every_alias():
    """k_xcorr_mma4's slot ring per item: super-chunk j (4 chunks) reads
    [64 j, 64 j + 76) and writes [64 j + 12, 64 j + 76) (from 0 when j = 0)
    on a ring of 256 slots, after waiting for super-chunk j - 3.  Every
    earlier super-chunk of the item whose reads alias those writes is j - 3
    or older, and reads stay inside the ring and its 32-slot mirror."""
    ring = 256
    for nchunks in range(1, 193):
        nsc = -(-nchunks // 4)
        reads = {}
        for j in range(nsc):
            c_last = min(4 * j + 3, nchunks - 1)
            lo = 0 if j == 0 else 64 * j + 12
            writes = {e % ring for e in range(lo, 16 * c_last + 28)}
            for jp, rd in reads.items():
                if rd & writes:
                    assert jp <= j - 3, (nchunks, j, jp)
            rd = set()
            for c in range(4 * j, c_last + 1):
                assert (16 * c) % ring + 28 <= ring + 32
                rd |= {(16 * c + i) % ring for i in range(28)}
            reads[j] = rd


def _argmax32_visits(addr, n, gx, threads=256):
    """k_argmax32's partition of one pair's n int32 correlations at byte
    address addr (4-byte aligned) over gx CTAs: `head` scalars up to the first
    16-byte boundary, int4 vectors (four per thread per step), the scalar
    tail.  Returns how often each element is read; asserts every vector load
    is 16-byte aligned and inside the array."""
    nthr = gx * threads
    head = min(((16 - (addr & 15)) & 15) >> 2, n)
    nv = (n - head) >> 2
    tail0 = head + 4 * nv
    seen = [0] * n
    for tid in range(nthr):
        if tid < head:
            seen[tid] += 1
        if tid < n - tail0:
            seen[tail0 + tid] += 1
        v0 = tid
        while v0 < nv:
            for k in range(4):
                v = v0 + k * nthr
                if v < nv:
                    i = head + 4 * v
                    assert (addr + 4 * i) % 16 == 0 and i + 3 < n
                    for e in range(4):
                        seen[i + e] += 1
            v0 += 4 * nthr
    return seen


def test_argmax32_reads_every_element_once_with_aligned_vectors():
    for addr in (0, 4, 8, 12):
        for n in (1, 2, 3, 4, 5, 7, 8, 15, 16, 17, 63, 64, 65, 1023, 1024, 1025):
            for gx in (1, 2):
                assert all(c == 1 for c in _argmax32_visits(addr, n, gx)), (addr, n, gx)
    rng = random.Random(1)
    for _ in range(60):
        addr, n, gx = 4 * rng.randrange(4), rng.randrange(1, 12000), rng.randrange(1, 4)
        assert all(c == 1 for c in _argmax32_visits(addr, n, gx)), (addr, n, gx)
    # the bench's layout: pair p's 131071 lags start at element 131071 p
    for p in range(4):
        assert all(c == 1 for c in _argmax32_visits((4 * 131071 * p) % 16, 131071, 32))


def _conv_tc_model(X, W, b):
    """k_conv_tc's operand arithmetic for one layer (32 -> 32 channels,
    kernel 9, padding 4, + bias, ReLU, max-pool 2), on float arrays standing
    for the BF16 bytes.  The input is split by position parity into 8
    arrays of 8 channels (even array j holds channels 8j..8j+7 of positions
    2r - 4, odd array of 2r - 3, row r); the weights are staged as 11 tap
    blocks per 8-channel group (taps -1 .. 9, the ends zero).  A tile of 128
    pooled outputs is 10 shifted row windows x 2 channel halves of
    128 x 64 x 16 products read through the descriptors' strides (core
    matrices of 8 rows x 16 bytes, stride byte offset 128, leading byte
    offset one array), columns 0..31 the odd pre-pool output, 32..63 the
    even one."""
    C, K = 32, 9
    L = X.shape[0]
    Lo = L // 2
    R = (L // 2 + 127) // 128 * 128 + 4
    G = np.zeros((8, R, 8))
    for r in range(R):
        for par in range(2):
            pos = 2 * r - 4 + par
            if 0 <= pos < L:
                for j in range(4):
                    G[par * 4 + j, r] = X[pos, 8 * j:8 * j + 8]
    Ws = np.zeros((4, 11, 32, 8))
    for j in range(4):
        for t in range(11):
            if 0 <= t - 1 < K:
                for co in range(32):
                    Ws[j, t, co] = W[co, 8 * j:8 * j + 8, t - 1]
    wflat = Ws.reshape(-1)
    out = np.zeros((Lo, C))
    arr = 132 * 16  # bytes per parity array in a tile (128 + 4 rows of 16 bytes)

    def rd(flat, start, lbo, sbo, rows, kk):
        byte = start + (rows // 8) * sbo + (rows % 8) * 16 + (kk // 8) * lbo + (kk % 8) * 2
        assert (byte >= 0).all() and (byte // 2 < flat.size).all()
        return flat[byte // 2]
    m, n, kk = np.arange(128)[:, None], np.arange(64)[:, None], np.arange(16)[None, :]
    for tile in range((Lo + 127) // 128):
        P0 = tile * 128
        tflat = G[:, P0:P0 + 132].copy().reshape(-1)
        D = np.zeros((128, 64))
        for w in range(10):
            par, dd = w // 5, w % 5
            for h in range(2):
                A = rd(tflat, (par * 4 + 2 * h) * arr + 16 * dd, arr, 128, m, kk)
                B = rd(wflat, ((2 * h) * 11 + 2 * dd + par) * 512, 11 * 512, 128, n, kk)
                D += A @ B.T
        for mm in range(128):
            if P0 + mm < Lo:
                out[P0 + mm] = np.maximum(np.maximum(D[mm, 32:], D[mm, :32]) + b, 0)
    return out


def test_conv_parity_layout_computes_conv_relu_pool():
    rng = np.random.default_rng(1)
    C, K = 32, 9
    for L in (256, 288, 520, 1024):
        X = rng.standard_normal((L, C))
        W = rng.standard_normal((C, C, K))
        b = rng.standard_normal(C)
        Xp = np.zeros((L + 8, C))
        Xp[4:4 + L] = X
        z = np.zeros((L, C))
        for k in range(K):
            z += Xp[k:k + L] @ W[:, :, k].T
        z = np.maximum(z + b, 0)
        ref = np.maximum(z[0::2], z[1::2])
        assert np.abs(_conv_tc_model(X, W, b) - ref).max() < 1e-9, L


def _scores_pair_model(fx, fy, Lf, alpha, G=16, pad=32, warps=16):
    """k_scores_pair's walk: x features in rows [0, Lf + 16) and y in rows
    [0, Lf + 2 pad) of shared memory (zero outside the signal); warp w takes
    bin groups w and w + ceil(ngroups / 2); a group walks only the blocks of
    16 positions where its 16 bins overlap.  Asserts every shared-memory row
    it reads is inside its array; returns the scores."""
    nb = 2 * Lf - 1
    out = np.full(nb, np.nan)
    xs = np.zeros((Lf + 16, 32))
    xs[:Lf] = fx.T
    ys = np.zeros((Lf + 2 * pad, 32))
    ys[pad:pad + Lf] = fy.T
    ng = (nb + G - 1) // G
    half = (ng + 1) // 2
    for w in range(warps):
        for gi in range(2):
            g = w + gi * half
            if w >= half or g >= ng:
                continue
            lg = G * g - (Lf - 1)
            wlo = max(0, -(lg + G - 1)) & ~(G - 1)
            whi = (min(Lf, Lf - lg) + G - 1) & ~(G - 1)
            acc = np.zeros((32, G))
            for ib in range(wlo, whi, G):
                for s2 in range(G):
                    xr = ib + s2
                    assert 0 <= xr < Lf + 16
                    for t in range(G):
                        yr = ib + lg + pad + s2 + t
                        assert 0 <= yr < Lf + 2 * pad
                        acc[:, t] += xs[xr] * ys[yr]
            for t in range(G):
                if G * g + t < nb:
                    out[G * g + t] = alpha * acc[:, t].sum()
    return out


def test_scores_pair_walk_stays_in_bounds_and_scores_every_bin():
    rng = np.random.default_rng(0)
    for Lf in (8, 64, 136, 256):
        fx, fy = rng.standard_normal((32, Lf)), rng.standard_normal((32, Lf))
        ref = np.array([sum((fx[:, i] * fy[:, i + l]).sum() for i in range(Lf) if 0 <= i + l < Lf)
                        for l in range(-(Lf - 1), Lf)]) * 0.5
        got = _scores_pair_model(fx, fy, Lf, 0.5)
        assert not np.isnan(got).any(), Lf
        assert np.abs(got - ref).max() < 1e-9, Lf


def _qone_table_model(pre, kqte=16):
    """k_qone's level table built the kernel's way: thread t owns first
    digits [16 t, 16 t + 16) as four words of bytes, starts every byte at the
    count of threshold digits below its range, adds 1 to the bytes above each
    threshold digit inside its range and marks that digit's byte; negative
    levels are (0x80 - l) ^ 0x80 per byte; a marked byte is 0x80 in both
    halves.  Returns the 8192 table bytes (index = float bits >> 19)."""
    tab = np.zeros(8192, np.uint8)
    for t in range(4096 // kqte):
        h0 = kqte * t
        lv0 = sum(1 for p in pre if p < h0)
        w = [lv0 * 0x01010101] * (kqte // 4)
        cm = 0
        for p in pre:
            d = (p - h0) & 0xFFFFFFFF
            if d < kqte:
                cm |= 1 << d
                for j in range(kqte):
                    if j > d:
                        w[j >> 2] += 1 << (8 * (j & 3))
        for k in range(kqte // 4):
            mk = 0
            for e in range(4):
                if (cm >> (4 * k + e)) & 1:
                    mk |= 0xFF << (8 * e)
            neg = ((0x80808080 - w[k]) & 0xFFFFFFFF) ^ 0x80808080
            pos_w = (w[k] & ~mk & 0xFFFFFFFF) | (0x80808080 & mk)
            neg_w = (neg & ~mk & 0xFFFFFFFF) | (0x80808080 & mk)
            for e in range(4):
                tab[h0 + 4 * k + e] = (pos_w >> (8 * e)) & 0xFF
                tab[4096 + h0 + 4 * k + e] = (neg_w >> (8 * e)) & 0xFF
    return tab


def test_qone_level_table_matches_the_first_digit_rule():
    """Every table byte equals its definition: 0x80 where the first digit is
    a threshold's (the sample is a candidate), else sign * #{m : digit >
    digit of t_m} as a two's-complement byte -- for sorted threshold digits
    drawn at random, with repeats, at range edges and several in one
    thread's range."""
    rng = np.random.default_rng(5)
    cases = [[0], [4095], [15, 16], [16, 16, 16, 17, 31, 32, 47], [0, 0, 0, 0, 0, 0, 0]]
    for _ in range(40):
        M = int(rng.choice([1, 7]))
        cases.append(sorted(int(v) for v in rng.integers(0, 4096, M)))
    for _ in range(20):  # clustered, like the thresholds of Gaussian data
        base = int(rng.integers(900, 1100))
        cases.append(sorted(base + int(v) for v in rng.integers(0, 40, 7)))
    hi = np.arange(4096)
    for pre in cases:
        tab = _qone_table_model(pre)
        pa = np.array(pre)
        cand = (hi[:, None] == pa[None, :]).any(1)
        lv = (hi[:, None] > pa[None, :]).sum(1)
        want_pos = np.where(cand, 0x80, lv).astype(np.uint8)
        want_neg = np.where(cand, 0x80, (-lv) & 0xFF).astype(np.uint8)
        assert np.array_equal(tab[:4096], want_pos), pre
        assert np.array_equal(tab[4096:], want_neg), pre


def test_qone_marks_flag_exactly_the_candidate_bytes():
    """qone_marks: p & ~(p << 1) & 0x80808080 has bit 7 of a byte set iff
    the byte is 0x80, over every byte a table holds (levels -7..7 and the
    mark) in every position of a word, with the neighbouring bytes'
    carries."""
    vals = [v & 0xFF for v in range(-7, 8)] + [0x80]
    rng = np.random.default_rng(9)
    for _ in range(4000):
        b = [int(rng.choice(vals)) for _ in range(4)]
        p = b[0] | b[1] << 8 | b[2] << 16 | b[3] << 24
        m = p & ~((p << 1) & 0xFFFFFFFF) & 0x80808080
        for e in range(4):
            assert bool((m >> (8 * e + 7)) & 1) == (b[e] == 0x80), b


def test_qone_candidate_columns_hold_every_sample_a_thread_sees():
    """k_qone's candidate list is column-major, qone_rows(n) = n // 256 + 8
    rows of 256 threads: no thread sees more samples than that in either
    pass (float4 i = 1024 c + 256 k + t below n4, four samples each, then
    the tail j = 4 n4 + t + 256 m, or every sample when x is unaligned), and
    the two columns fit the list's 2 (n + 2048) words."""
    T, V = 256, 4
    ns = list(range(0, 3000)) + [65536, 65536 + 123, 262144, 262143, 9007]
    for n in ns:
        rows = n // T + 8
        assert 2 * T * rows <= 2 * (n + 2048)
        for vec in (True, False):
            n4 = n >> 2 if vec else 0
            per = np.zeros(T, np.int64)
            idx = np.arange(n4)
            np.add.at(per, idx % T, 4)
            tail = np.arange(4 * n4, n)
            np.add.at(per, (tail - 4 * n4) % T, 1)
            assert per.max(initial=0) <= rows, (n, vec, per.max())


def _scores_tc_drain_model(G, Lf):
    """k_scores_tc's diagonal sums restated: warp w (quadrant q = w % 4, half
    w // 4) takes its 32 x 32 blocks of G (rows 128 mt + 32 q + r, columns
    128 half + 32 cb + c) in the kernel's order; lane t sums the block's
    diagonals d1 = t - 31 (rows 31 - t .. 31) and d2 = t + 1 (rows 0 .. 30 - t)
    of the skewed copy S[r][c] (row stride 33) and adds them to its warp's
    row at lag + 255; bin b = l + Lf - 1 is then the sum of the 8 rows in
    warp order.  Asserts every read stays in the copy and every write in the
    row."""
    part = np.zeros((8, 512))
    for w in range(8):
        q, half = w & 3, w >> 2
        for mt in range(2):
            for cb in range(4):
                j0, i0 = 128 * half + 32 * cb, 128 * mt + 32 * q
                S = np.zeros(32 * 33)
                for r in range(32):
                    S[r * 33:r * 33 + 32] = G[i0 + r, j0:j0 + 32]
                for t in range(32):
                    s1 = s2 = 0.0
                    for r in range(32):
                        if r >= 31 - t:
                            a = r * 33 + r + t - 31
                            assert r * 33 <= a < r * 33 + 32
                            s1 += S[a]
                        if r <= 30 - t:
                            a = r * 33 + r + t + 1
                            assert r * 33 <= a < r * 33 + 32
                            s2 += S[a]
                    i1 = j0 - i0 + t - 31 + 255
                    assert 0 <= i1 < 512
                    part[w, i1] += s1
                    if t < 31:
                        i2 = j0 - i0 + t + 1 + 255
                        assert 0 <= i2 < 512
                        part[w, i2] += s2
    nb = 2 * Lf - 1
    return np.array([part[:, b - (Lf - 1) + 255].sum() for b in range(nb)])


def test_scores_tc_diagonal_sums_cover_every_entry_once():
    """The drain's block diagonals add up to score[l] = sum_i G[i][i + l] for
    every bin, with rows past Lf zero (as the kernel's operands are), for the
    full length and a shorter one."""
    rng = np.random.default_rng(12)
    for Lf in (256, 200, 8):
        X = np.zeros((256, 32)); Y = np.zeros((256, 32))
        X[:Lf] = rng.random((Lf, 32)); Y[:Lf] = rng.random((Lf, 32))
        G = X @ Y.T
        got = _scores_tc_drain_model(G, Lf)
        want = np.array([np.trace(G, offset=l) for l in range(-(Lf - 1), Lf)])
        assert np.allclose(got, want, rtol=1e-12, atol=1e-9), Lf


def _st_key(s, l):
    """k_scores_tc's bin key (float32 score, lag) as a Python int."""
    s = np.float32(s)
    if s == 0:
        s = np.float32(0.0)
    u = int(np.array(s, np.float32).view(np.uint32))
    u = (~u & 0xFFFFFFFF) if u & 0x80000000 else (u | 0x80000000)
    rank = 2 * abs(l) + (1 if l > 0 else 0)
    return (u << 32) | (0xFFFFFFFF - rank)


def test_scores_key_orders_bins_like_better():
    """The key's order is `better`'s: higher score, then smaller |l|, then
    negative l; -0 ties +0; the score and lag decode back."""
    def better(s, l, bs, bl):
        if s != bs:
            return s > bs
        return abs(l) < abs(bl) if abs(l) != abs(bl) else l < bl
    rng = np.random.default_rng(4)
    vals = [0.0, -0.0, 1.5, -1.5, 3.0, -7.25, 1e-30, -1e-30, 2.0 ** 100]
    for _ in range(3000):
        s1, s2 = (float(rng.choice(vals)) if rng.random() < 0.5 else float(np.float32(rng.normal())) for _ in range(2))
        l1, l2 = (int(v) for v in rng.integers(-255, 256, 2))
        if l1 == l2:
            continue
        k1, k2 = _st_key(s1, l1), _st_key(s2, l2)
        assert (k1 > k2) == better(np.float32(s1), l1, np.float32(s2), l2), (s1, l1, s2, l2)
        rank = 0xFFFFFFFF - (k1 & 0xFFFFFFFF)
        assert ((rank >> 1) if rank & 1 else -(rank >> 1)) == l1
        u = k1 >> 32
        bits = (u ^ 0x80000000) if u & 0x80000000 else (~u & 0xFFFFFFFF)
        assert np.array(bits, np.uint32).view(np.float32) == np.float32(s1)


def test_conv12_unit_builds_layer2_tile_and_owns_each_level_once():
    """k_conv12_tc's unit (layer-2 tile P0, 128 outputs): the decimated
    window d[4 P0 - 12 + i] (i < 536), layer-1 outputs t < 256 from the
    im2col rows (tile t // 128, parity, taps 2 t + par + k) and t = 256..263
    from the halo formula, written to E/O rows t // 2 of parity t % 2, equal
    the direct conv + bias + ReLU + pool of layer 1 at u = 2 P0 - 4 + t (zero
    outside [0, Ld / 2)); and the units' owned samples [4 P0, 4 P0 + 512)
    cover the decimated signal once."""
    rng = np.random.default_rng(8)
    for Ld in (1024, 4096, 512):
        d = rng.integers(-16, 17, Ld) / 4.0
        w = rng.normal(size=(32, 9))
        b = rng.normal(size=32)
        L2 = Ld // 2
        # direct layer 1: z[v] = sum_k d[v + k - 4] w[k], pooled pairs (2u, 2u + 1)
        dp = np.concatenate([np.zeros(4), d, np.zeros(4)])
        z = np.stack([dp[v:v + 9] @ w.T for v in range(Ld)])
        x2 = np.maximum(np.maximum(z[0::2], z[1::2]) + b, 0)  # [L2][32]
        Lo = L2 // 2
        tps = -(-Lo // 128)
        owned = np.zeros(Ld, int)
        for unit in range(tps):
            P0 = unit * 128
            ds = np.array([d[j] if 0 <= j < Ld else 0.0 for j in range(4 * P0 - 12, 4 * P0 - 12 + 536)])
            for i in range(12, 12 + 512):
                j = 4 * P0 - 12 + i
                if 0 <= j < Ld:
                    owned[j] += 1
            E = np.full((132, 32), np.nan); O = np.full((132, 32), np.nan)
            for t in range(264):
                zz = [ds[2 * t + par:2 * t + par + 9] @ w.T for par in (0, 1)]
                uu = 2 * P0 - 4 + t
                y = np.maximum(np.maximum(zz[0], zz[1]) + b, 0) if 0 <= uu < L2 else np.zeros(32)
                (E if t % 2 == 0 else O)[t // 2] = y
            for r in range(132):
                for arr, pos in ((E, 2 * (P0 + r) - 4), (O, 2 * (P0 + r) - 3)):
                    want = x2[pos] if 0 <= pos < L2 else np.zeros(32)
                    assert np.allclose(arr[r], want), (Ld, unit, r)
        assert (owned == 1).all(), Ld


def test_conv12_e4m3_bytes_of_unit_levels():
    """k_conv12_tc's E4M3 copy of levels in {-1, 0, 1}: per word
    ((w & 0x01010101) * 0x38) | (w & 0x80808080) gives 0x00 for 0, 0x38 (1.0)
    for 1 and 0xB8 (-1.0) for -1 in every byte of every combination."""
    import itertools
    enc = {0: 0x00, 1: 0x38, -1: 0xB8}
    for lv in itertools.product((-1, 0, 1), repeat=4):
        w = 0
        for k, v in enumerate(lv):
            w |= (v & 0xFF) << (8 * k)
        e = (((w & 0x01010101) * 0x38) | (w & 0x80808080)) & 0xFFFFFFFF
        assert all(((e >> (8 * k)) & 0xFF) == enc[v] for k, v in enumerate(lv)), lv
