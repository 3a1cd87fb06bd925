"""CPU models of kernel index arithmetic that must hold for every access to
stay in bounds and every element to be counted once.  Each test restates one
kernel's rule in Python and checks it exhaustively or on random cases, so a
change to the rule can be checked here before it runs on a GPU."""
import random

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
