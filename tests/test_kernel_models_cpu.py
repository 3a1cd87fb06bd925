"""CPU models of kernel index arithmetic that must hold for every access to
stay in bounds and every element to be counted once.  Each test restates one
kernel's rule in Python and checks it exhaustively or on random cases, so a
change to the rule can be checked here before it runs on a GPU."""
import random

import numpy as np

RING = 256          # k_xcorr_mma_win: slot ring of 256 (+ a 32-slot mirror)
SC_SLOTS = 46       # slots a super-chunk reads: [R, R + 46)


def _ring_rule(nchunks_per_segment):
    """k_xcorr_mma_win's slot ring.  Super-chunk S (two 128-sample chunks,
    counted over the CTA's run; g = its segment's index in the run) has
    origin R(S) = 32 (S + g).  Chunk c of a segment reads ring positions
    [16 c, 16 c + 30) from the segment origin; a super-chunk writes
    [32 sc + 14, 16 c_last + 30) (all of [0, 16 c_last + 30) at a segment
    start).  Before writing, the producers wait for the newest earlier
    super-chunk S' with R(S) - R(S') > RING - 46 (at most 8 back).  Checks:
    every earlier super-chunk whose reads alias this one's writes is one the
    producers waited for."""
    S, origins, reads = 0, [], {}
    for g, nch in enumerate(nchunks_per_segment):
        nsc = -(-nch // 2)
        r0 = 32 * (S + g)
        for sc in range(nsc):
            R = r0 + 32 * sc
            waited = -1
            for k in range(8, 0, -1):
                rk = origins[-k] if len(origins) >= k else -10 ** 18
                if R - rk > RING - SC_SLOTS:
                    waited = S - k
            c_last = min(2 * sc + 1, nch - 1)
            lo = 0 if sc == 0 else 32 * sc + 14
            writes = {(r0 + e) % RING for e in range(lo, 16 * c_last + 30)}
            for s_prev, rd in reads.items():
                if rd & writes:
                    assert s_prev <= waited, (nchunks_per_segment, S, s_prev, waited)
            rd = set()
            for c in range(2 * sc, c_last + 1):
                rd |= {(r0 + 16 * c + i) % RING for i in range(30)}
            reads[S] = rd
            origins.append(R)
            S += 1


def test_windows_slot_ring_never_overwrites_unread_slots():
    _ring_rule([24] * 20)
    _ring_rule([1] * 30)
    _ring_rule([2, 3, 24, 1, 24, 9, 24])
    rng = random.Random(0)
    for _ in range(300):
        _ring_rule([rng.randint(1, 24) for _ in range(rng.randint(1, 30))])


def _ring_rule_fp4(nchunks_per_segment, sc_chunks=4, ring=512):
    """k_xcorr_mma_win4's slot ring: a chunk reads [16 c, 16 c + 28) (two
    K = 64 steps over slots e0 + g + 4 h, e0 = 16 c + 8 s); a super-chunk of
    sc_chunks chunks has origin R(S) = 16 sc_chunks (S + g), reads
    16 sc_chunks + 12 slots, writes [step sc + 12, 16 c_last + 28) (from 0 at
    a segment start), and the producers wait for the newest earlier
    super-chunk with R - R' > ring - reads.  Checks that every earlier
    super-chunk whose reads alias this one's writes is one they waited for,
    and that a super-chunk's reads stay inside the ring and its 32-slot
    mirror."""
    step = 16 * sc_chunks
    nread = step + 12
    S, origins, reads = 0, [], {}
    for g, nch in enumerate(nchunks_per_segment):
        nsc = -(-nch // sc_chunks)
        r0 = step * (S + g)
        for sc in range(nsc):
            R = r0 + step * sc
            assert R % ring + nread <= ring + 32
            waited = -1
            for k in range(8, 0, -1):
                rk = origins[-k] if len(origins) >= k else -10 ** 18
                if R - rk > ring - nread:
                    waited = S - k
            c_last = min(sc_chunks * sc + sc_chunks - 1, nch - 1)
            lo = 0 if sc == 0 else step * sc + 12
            writes = {(r0 + e) % ring for e in range(lo, 16 * c_last + 28)}
            for s_prev, rd in reads.items():
                if rd & writes:
                    assert s_prev <= waited, (nchunks_per_segment, S, s_prev, waited)
            rd = set()
            for c in range(sc_chunks * sc, c_last + 1):
                for st in range(2):
                    rd |= {(r0 + 16 * c + 8 * st + gg + 4 * h) % ring for gg in range(16) for h in range(2)}
            reads[S] = rd
            origins.append(R)
            S += 1


def test_windows_fp4_slot_ring_never_overwrites_unread_slots():
    for scc in (4, 8):
        _ring_rule_fp4([24] * 20, scc)
        _ring_rule_fp4([1] * 30, scc)
        _ring_rule_fp4([2, 3, 24, 1, 24, 9, 24], scc)
        rng = random.Random(scc)
        for _ in range(150):
            _ring_rule_fp4([rng.randint(1, 24) for _ in range(rng.randint(1, 30))], scc)


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


def _funnel_r(lo, hi, sh):
    return (((hi << 32) | lo) >> (sh & 31)) & 0xFFFFFFFF


def test_windows_fp4_slots_hold_the_hankel_operand():
    """k_xcorr_mma_win4's producers: the x segment as TMA stages it (packed
    nibbles from sample 32 floor((ks - 127) / 32), 2048 bytes, zeros outside
    the signal), each lane's two slot rows from five funnel-shifted words of
    four aligned 8-byte loads; every read stays in the 2048-byte buffer, and
    the core matrices an MMA's descriptor names (slot e0 + g + 4 h, e0 =
    16 c + 8 s) hold A[m][k] = x[ks - 127 + 128 c + 64 s + m + k]."""
    rng = np.random.default_rng(3)
    n = 9000
    x = rng.integers(0, 16, size=n)      # nibble values stand for the levels
    for ks in (0, 128, 3072, 6144, 8832):
        nch = min(24, (-(-(n + 254) // 128) * 128 - ks) // 128)
        x0 = 32 * ((ks - 127) // 32)
        nib = np.zeros(4096, np.int64)
        for i in range(4096):
            if 0 <= x0 + i < n:
                nib[i] = x[x0 + i]
        buf = [int(nib[2 * j]) | (int(nib[2 * j + 1]) << 4) for j in range(2048)]
        bp = (ks - 127) - x0
        slots = {}
        e_hi = 16 * (nch - 1) + 28
        for e0 in range(0, e_hi, 2):
            for r in range(8):
                pn = bp + 8 * e0 + r
                a8 = (pn >> 1) & ~7
                sbit = 4 * pn - 8 * a8
                assert 0 <= sbit <= 60 and a8 + 32 <= 2048
                u = [int.from_bytes(bytes(buf[a8 + 4 * i: a8 + 4 * i + 4]), "little") for i in range(8)]
                wo, sh = sbit >= 32, sbit & 31
                w = [_funnel_r(u[j + 1] if wo else u[j], u[j + 2] if wo else u[j + 1], sh) for j in range(5)]
                for k in range(2):
                    if e0 + k < e_hi:
                        slots.setdefault(e0 + k, {})[r] = w[k:k + 4]
        for c in range(nch):
            for st in range(2):
                e0 = 16 * c + 8 * st
                for m in range(0, 128, 7):
                    for kk in range(64):
                        g, r, h, cc = m // 8, m % 8, kk // 32, kk % 32
                        words = slots[e0 + g + 4 * h][r]
                        v = (words[cc // 8] >> (4 * (cc % 8))) & 0xF
                        t = ks - 127 + 128 * c + 64 * st + m + kk
                        want = x[t] if 0 <= t < n else 0
                        assert v == want, (ks, c, st, m, kk)


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
