"""CPU model of the polyphase windows kernel (k_xcorr_win_pp in
csrc/winpp.cu): its job plan, the order in which its TMA role fills and its
MMA role releases the x-tile and y-chunk rings, and its arithmetic (blocks
D_u over 128-sample rows, diagonals, windows, segments).  The model follows
the kernel's rules step by step so that a change to them is checked here,
against a direct correlation, before it runs on a GPU."""
import random

import numpy as np

SEG_ROWS = 512       # rows summed per accumulator
TILE_ROWS = 32       # K rows per MMA
HALF_ROWS = 256      # x rows per load and release
X_HALVES = 3         # x ring
UNIT_ROWS = 64       # y rows per load and release
Y_UNITS = 11         # y ring
MIRROR_ROWS = 32     # rows of unit slot 0 mirrored past the ring's end
GROUP_UNITS = Y_UNITS - 2
WIN_LEN = 257


def fdiv128(a):
    return a // 128  # Python's floor division


def pp_plan(wins):
    """Blocks the windows [lo, hi] need (floor(lo/128) .. floor((hi+127)/128)),
    merged into sorted runs (adjacent runs join), cut into jobs of 2 blocks."""
    iv = sorted((fdiv128(lo), fdiv128(hi + 127)) for lo, hi in wins if hi >= lo)
    jobs, i = [], 0
    while i < len(iv):
        r0, r1 = iv[i]
        i += 1
        while i < len(iv) and iv[i][0] <= r1 + 1:
            r1 = max(r1, iv[i][1])
            i += 1
        for u in range(r0, r1 + 1, 2):
            jobs.append((u, 2 if r1 - u >= 1 else 1))
    return jobs


def visits(plans, nseg, rows_total, J0, J1):
    """The kernel's walk over jobs [J0, J1) in (pair, segment, job) order:
    yields (p, s, tiles, groups) with groups a list of (first logical y
    unit, units, [(u, nb), ...])."""
    flat = [(p, s, k) for p, pl in enumerate(plans) for s in range(nseg) for k in range(len(pl))]
    run = flat[J0:J1]
    yu = 0
    i = 0
    while i < len(run):
        p, s, _ = run[i]
        ks = []
        while i < len(run) and run[i][0] == p and run[i][1] == s:
            ks.append(run[i][2])
            i += 1
        rows = min(SEG_ROWS, rows_total - SEG_ROWS * s)
        tiles = -(-rows // TILE_ROWS)
        jl = [plans[p][k] for k in ks]

        def units(g0, k):
            r = jl[k][0] + jl[k][1] - 1 - jl[g0][0] + TILE_ROWS * tiles
            return -(-r // UNIT_ROWS)

        groups, ge = [], 0
        while ge < len(jl):
            gb = ge
            ge = gb + 1
            while ge < len(jl) and units(gb, ge) <= GROUP_UNITS:
                ge += 1
            gun = units(gb, ge - 1)
            groups.append((yu, gun, jl[gb:ge]))
            yu += gun
        yield p, s, tiles, groups


class _Bar:
    """An mbarrier: `count` arrivals complete a phase; a wait for parity p
    passes once the phase counter's parity differs from p."""

    def __init__(self, count):
        self.count, self.pending, self.phase = count, 0, 0

    def arrive(self):
        self.pending += 1
        if self.pending == self.count:
            self.pending, self.phase = 0, self.phase + 1

    def ready(self, parity):
        return (self.phase & 1) != parity


def simulate(plans, nseg, rows_total, J0, J1, lanes=4, seed=0, by_slot=True):
    """Runs the kernel's TMA role (a slot's loads by lane slot % lanes) and its
    two MMA issuers (alternate jobs; a slot released by both: the last job's
    issuer after each batch, the other after its own last job of the group or
    visit, once the group's units or visit's halves are loaded) in a random
    interleaving, with the slots' full and empty barriers modelled as
    mbarriers (waits by parity).  Checks that the run finishes (no circular
    wait, no barrier lapped) and that every MMA finds in its x half and y rows
    (through the mirror past the ring's end) the data it expects."""
    rng = random.Random(seed)
    V = list(visits(plans, nseg, rows_total, J0, J1))
    tph = HALF_ROWS // TILE_ROWS
    # ---- the TMA role's loads, as in the kernel
    loads = []  # ('x', slot, lap, (p, first row)) / ('y', ...)
    xh = yu = 0
    for p, s, tiles, groups in V:
        nh = -(-tiles * TILE_ROWS // HALF_ROWS)
        rowbase = s * SEG_ROWS
        for gi, (gyu, gun, jl) in enumerate(groups):
            ubase = rowbase + jl[0][0]
            c = 0
            if gi == 0:
                for h in range(nh):
                    loads.append(('x', (xh + h) % X_HALVES, (xh + h) // X_HALVES, (p, rowbase + HALF_ROWS * h)))
                    need = (HALF_ROWS * (h + 1) + TILE_ROWS) // UNIT_ROWS
                    while c < gun and c <= need:
                        loads.append(('y', (gyu + c) % Y_UNITS, (gyu + c) // Y_UNITS, (p, ubase + UNIT_ROWS * c)))
                        c += 1
            while c < gun:
                loads.append(('y', (gyu + c) % Y_UNITS, (gyu + c) // Y_UNITS, (p, ubase + UNIT_ROWS * c)))
                c += 1
        xh += nh
    # ---- each issuer's program: ('wait', kind, slot, parity) / ('mma', ...) / ('rel', kind, slot)
    progs = [[], []]
    jc = 0
    xh = 0
    nmma = 0
    for p, s, tiles, groups in V:
        nh = -(-tiles * TILE_ROWS // HALF_ROWS)
        nj = sum(len(jl) for _, _, jl in groups)
        vlast = (jc + nj - 1) & 1
        xwaited = [False, False]
        for gi, (gyu, gun, jl) in enumerate(groups):
            glast = (jc + len(jl) - 1) & 1
            ywaited = [-1, -1]
            freed = 0
            for k, (u, nb) in enumerate(jl):
                me = jc & 1
                prog = progs[me]
                urel = u - jl[0][0]
                last_visit = gi == len(groups) - 1 and k == len(jl) - 1
                last_group = k == len(jl) - 1
                for h in range(nh):
                    t0, t1 = tph * h, min(tiles, tph * (h + 1))
                    if not xwaited[me]:
                        prog.append(('wait', 'x', (xh + h) % X_HALVES, ((xh + h) // X_HALVES) & 1))
                        if t1 == tiles:
                            xwaited[me] = True
                    need = (urel + TILE_ROWS * t1 + nb - 2) // UNIT_ROWS
                    while ywaited[me] < need:
                        ywaited[me] += 1
                        U = gyu + ywaited[me]
                        prog.append(('wait', 'y', U % Y_UNITS, (U // Y_UNITS) & 1))
                    for t in range(t0, t1):
                        want_x = [(p, s * SEG_ROWS + TILE_ROWS * t + r) for r in range(TILE_ROWS)]
                        want_y = [(p, s * SEG_ROWS + u + TILE_ROWS * t + r) for r in range(TILE_ROWS + nb - 1)]
                        pos = UNIT_ROWS * gyu + urel + TILE_ROWS * t
                        prog.append(('mma', (xh + h) % X_HALVES, t - t0, want_x, pos, want_y))
                        nmma += 1
                    if last_visit:
                        prog.append(('rel', 'x', (xh + h) % X_HALVES))
                    if last_group:
                        upto = gun if t1 == tiles else (urel + TILE_ROWS * t1) // UNIT_ROWS
                        while freed < upto:
                            prog.append(('rel', 'y', (gyu + freed) % Y_UNITS))
                            freed += 1
                jc += 1
            other = 1 - glast
            while ywaited[other] < gun - 1:
                ywaited[other] += 1
                U = gyu + ywaited[other]
                progs[other].append(('wait', 'y', U % Y_UNITS, (U // Y_UNITS) & 1))
            for i in range(gun):
                progs[other].append(('rel', 'y', (gyu + i) % Y_UNITS))
        other = 1 - vlast
        for h in range(nh):
            if not xwaited[other]:
                progs[other].append(('wait', 'x', (xh + h) % X_HALVES, ((xh + h) // X_HALVES) & 1))
        for h in range(nh):
            progs[other].append(('rel', 'x', (xh + h) % X_HALVES))
        xh += nh
    # ---- run
    full = {'x': [_Bar(1) for _ in range(X_HALVES)], 'y': [_Bar(1) for _ in range(Y_UNITS)]}
    empty = {'x': [_Bar(2) for _ in range(X_HALVES)], 'y': [_Bar(2) for _ in range(Y_UNITS)]}
    xrows = [None] * X_HALVES
    yrows = [None] * (Y_UNITS * UNIT_ROWS + MIRROR_ROWS)
    if by_slot:  # slot s by lane s % lanes (the kernel's rule)
        lane_loads = [[ld for ld in loads if ld[1] % lanes == l] for l in range(lanes)]
    else:  # load i by lane i % lanes
        lane_loads = [[ld for i, ld in enumerate(loads) if i % lanes == l] for l in range(lanes)]
    pcs = {('L', l): 0 for l in range(lanes)}
    pcs.update({('I', 0): 0, ('I', 1): 0})
    done_mma = 0

    def step(actor):
        nonlocal done_mma
        kind_, idx = actor
        if kind_ == 'L':
            q = lane_loads[idx]
            if pcs[actor] >= len(q):
                return False
            kind, slot, lap, (p, row) = q[pcs[actor]]
            if lap > 0 and not empty[kind][slot].ready((lap - 1) & 1):
                return False
            if kind == 'x':
                xrows[slot] = [(p, row + r) for r in range(HALF_ROWS)]
            else:
                for r in range(UNIT_ROWS):
                    yrows[slot * UNIT_ROWS + r] = (p, row + r)
                if slot == 0:
                    for r in range(MIRROR_ROWS):
                        yrows[Y_UNITS * UNIT_ROWS + r] = (p, row + r)
            full[kind][slot].arrive()
            pcs[actor] += 1
            return True
        prog = progs[idx]
        if pcs[actor] >= len(prog):
            return False
        op = prog[pcs[actor]]
        if op[0] == 'wait':
            if not full[op[1]][op[2]].ready(op[3]):
                return False
        elif op[0] == 'mma':
            _, xs, tin, want_x, pos, want_y = op
            assert xrows[xs][TILE_ROWS * tin:TILE_ROWS * (tin + 1)] == want_x
            phys = pos % (Y_UNITS * UNIT_ROWS)
            assert yrows[phys:phys + len(want_y)] == want_y, (pos, yrows[phys], want_y[0])
            done_mma += 1
        else:
            empty[op[1]][op[2]].arrive()
        pcs[actor] += 1
        return True

    actors = list(pcs)
    while True:
        live = [a for a in actors if pcs[a] < (len(lane_loads[a[1]]) if a[0] == 'L' else len(progs[a[1]]))]
        if not live:
            break
        rng.shuffle(live)
        if not any(step(a) for a in live):
            info = []
            for a in live:
                if a[0] == 'L':
                    info.append((a, lane_loads[a[1]][pcs[a]][:3]))
                else:
                    info.append((a, progs[a[1]][pcs[a]][:4]))
            raise AssertionError(f"circular wait: {info} x-empty {[(b.phase, b.pending) for b in empty['x']]} "
                                 f"y-empty {[(b.phase, b.pending) for b in empty['y']]} "
                                 f"x-full {[b.phase for b in full['x']]} y-full {[b.phase for b in full['y']]}")
    assert done_mma == nmma
    return nmma


def _windows_adjacent(n, centre_bin, rng):
    """8 windows of 257 lags around bins 256 l (adjacent bins)."""
    out = []
    for w in range(8):
        c = 256 * (centre_bin + w - 4)
        lo, hi = max(c - 128, -(n - 1)), min(c + 128, n - 1)
        out.append((lo, hi))
    return out


def _windows_random(n, rng):
    lf = n // 256
    bins = rng.sample(range(-(lf - 1), lf), 8)
    return [(max(256 * l - 128, -(n - 1)), min(256 * l + 128, n - 1)) for l in bins]


def _runs(J, G):
    return [(J * c // G, J * (c + 1) // G) for c in range(G)]


def test_plan_blocks_cover_every_window_lag():
    rng = random.Random(1)
    for _ in range(300):
        n = rng.choice([4096, 65536, 100000])
        wins = _windows_random(n, rng) if rng.random() < 0.5 else _windows_adjacent(n, rng.randint(-200, 200), rng)
        blocks = {u + i for u, nb in pp_plan(wins) for i in range(nb)}
        for lo, hi in wins:
            for tau in range(lo, hi + 1, 7):
                # the blocks holding terms of c[tau]: floor((b + tau) / 128), b < 128
                need = {(b + tau) // 128 for b in range(128)}
                assert need <= blocks
    # adjacent bins: 17 blocks (9 jobs) for 8 windows of 257 lags
    wins = _windows_adjacent(65536, 0, rng)
    pl = pp_plan(wins)
    assert sum(nb for _, nb in pl) == 17 and len(pl) == 9


def _ring_cases(seed, trials):
    rng = random.Random(seed)
    for trial in range(trials):
        n = rng.choice([65536, 65536, 4096, 3000, 100000, 140000])
        rows_total = -(-n // 128)
        nseg = -(-rows_total // SEG_ROWS)
        npairs = rng.randint(1, 12)
        plans = []
        for _ in range(npairs):
            r = rng.random()
            if r < 0.4:
                wins = _windows_adjacent(n, rng.randint(-(n // 256) + 5, n // 256 - 5), rng)
            elif r < 0.65:
                wins = _windows_random(n, rng)
            elif r < 0.8:  # windows on no 128-lag boundary (four blocks each)
                wins = [(lo, lo + 256) for lo in rng.sample(range(-(n - 1), n - 257), 8)]
            else:
                wins = []  # a pair without jobs (all windows empty)
            plans.append(pp_plan(wins))
        J = sum(len(pl) for pl in plans) * nseg
        G = rng.choice([1, 2, 3, 7])
        for J0, J1 in _runs(J, G):
            if J1 > J0:
                yield trial, plans, nseg, rows_total, J0, J1


def test_rings_fill_before_read_and_release_after_last_read():
    cases = 0
    for trial, plans, nseg, rows_total, J0, J1 in _ring_cases(2, 40):
        for seed in range(3):  # interleavings of the loader lanes and the two issuers
            cases += simulate(plans, nseg, rows_total, J0, J1, seed=100 * trial + seed)
    assert cases > 3000


def test_ring_model_catches_a_lane_lapping_its_slot():
    # loads dealt to lanes in turn (not by slot) let one lane fill a slot's
    # next lap before another lane's fill of the previous one: the model must
    # see it (a wrong operand or a circular wait)
    failures = 0
    for trial, plans, nseg, rows_total, J0, J1 in _ring_cases(2, 40):
        try:
            simulate(plans, nseg, rows_total, J0, J1, seed=trial, by_slot=False)
        except AssertionError:
            failures += 1
    assert failures > 0


def _pp_windows(x, y, wins, n):
    """The kernel's arithmetic, visit by visit (one per segment here): each
    job's blocks D_u over the segment's rows, value D[b][j] added to diagonal
    j - b + 127 of its block's slot; then per window lag tau = lo + t, with
    q = floor(tau / 128) and r = tau - 128 q, diagonal r + 127 of block q plus
    (r >= 1) diagonal r - 1 of block q + 1, the blocks found by their slots."""
    rows_total = -(-n // 128)
    xp = np.zeros(rows_total * 128, np.int64)
    yp = np.zeros(rows_total * 128, np.int64)
    xp[:n], yp[:n] = x, y
    X = xp.reshape(rows_total, 128)
    Y = yp.reshape(rows_total, 128)
    nseg = -(-rows_total // SEG_ROWS)
    out = [np.zeros(WIN_LEN, np.int64) for _ in wins]
    diag_idx = (np.arange(128)[None, :] - np.arange(128)[:, None] + 127).ravel()
    plan = pp_plan(wins)
    assert len(plan) <= 16 and sum(nb for _, nb in plan) <= 32
    for s in range(nseg):
        a0, a1 = s * SEG_ROWS, min((s + 1) * SEG_ROWS, rows_total)
        diag = np.zeros((32, 256), np.int64)
        slot = 0
        for u, nb in plan:
            for blk in range(nb):
                rows = np.arange(a0, a1) + u + blk
                ok = (rows >= 0) & (rows < rows_total)
                Yb = np.zeros((a1 - a0, 128), np.int64)
                Yb[ok] = Y[rows[ok]]
                D = X[a0:a1].T @ Yb                      # D[b][j]
                assert np.abs(D).max(initial=0) < 2 ** 24  # exact in FP32
                diag[slot + blk, :255] += np.bincount(diag_idx, weights=D.ravel().astype(np.float64),
                                                      minlength=255).astype(np.int64)
            slot += nb
        for w, (lo, hi) in enumerate(wins):
            if hi < lo:
                continue
            wslot = []
            for i in range(4):  # slot of block floor(lo / 128) + i, or -1
                ub, sl, acc = fdiv128(lo) + i, -1, 0
                for u, nb in plan:
                    if u <= ub < u + nb:
                        sl = acc + ub - u
                    acc += nb
                wslot.append(sl)
            for t in range(hi - lo + 1):
                tau = lo + t
                q = fdiv128(tau)
                r, i0 = tau - 128 * q, q - fdiv128(lo)
                v = diag[wslot[i0], r + 127] if wslot[i0] >= 0 else 0
                if r >= 1 and wslot[i0 + 1] >= 0:
                    v += diag[wslot[i0 + 1], r - 1]
                out[w][t] += v
    return out


def test_polyphase_arithmetic_equals_direct_correlation():
    rng = np.random.default_rng(3)
    for n, kb in ((3000, 1), (8192, 7), (70000, 7)):
        x = rng.integers(-kb, kb + 1, n)
        y = rng.integers(-kb, kb + 1, n)
        full = np.correlate(y, x, mode="full")  # full[k] = sum_i x[i] y[i + k - (n - 1)]
        prng = random.Random(n)
        unaligned = [(lo, lo + 256) for lo in prng.sample(range(-(n - 1), n - 257), 8)]
        for wins in (_windows_adjacent(n, prng.randint(-3, 3), prng), _windows_random(n, prng), unaligned,
                     [(-(n - 1), -(n - 1) + 100), (n - 1 - 256, n - 1), (5, 4)]):
            got = _pp_windows(x, y, wins, n)
            for (lo, hi), o in zip(wins, got):
                want = full[np.arange(lo, hi + 1) + n - 1]
                assert np.array_equal(o[:hi - lo + 1], want)
                assert not o[hi - lo + 1:].any()


def _drain_16x256b(D, qd, h, cols):
    """The epilogue's drain of one warp's share as pp_drain does it: lanes
    32 qd .. + 31, `cols` columns from 64 h (one block) or the whole block
    (cols = 128); thread t holds rows 32 qd + t // 4 + 8 k and columns
    8 g + 2 (t % 4) + e, sums each chain of equal g - k and adds it at
    diagonal index 8 s + e + 2 (t % 4) - t // 4 - 32 qd + 127 (+ 64 h)."""
    G = cols // 8
    c0 = 64 * h if cols == 64 else 0
    out = np.zeros(256, np.int64)
    seen = np.zeros((128, 128), np.int64)
    for t in range(32):
        r, m = t // 4, t % 4
        acc = np.zeros((2, G + 3), np.int64)
        for k in range(4):
            for g in range(G):
                for e in range(2):
                    b, j = 32 * qd + r + 8 * k, c0 + 8 * g + 2 * m + e
                    acc[e, g - k + 3] += D[b, j]
                    seen[b, j] += 1
        for i in range(G + 3):
            for e in range(2):
                idx = 8 * (i - 3) + e + 2 * m - r - 32 * qd + 127 + c0
                assert 0 <= idx <= 254
                out[idx] += acc[e, i]
    return out, seen


def test_epilogue_chains_sum_every_value_on_its_diagonal():
    rng = np.random.default_rng(5)
    D = rng.integers(-1000, 1000, (128, 128))
    want = np.zeros(256, np.int64)
    for b in range(128):
        for j in range(128):
            want[j - b + 127] += D[b, j]
    for cols, halves in ((128, (0,)), (64, (0, 1))):
        got = np.zeros(256, np.int64)
        seen = np.zeros((128, 128), np.int64)
        for qd in range(4):
            for h in halves:
                o, sn = _drain_16x256b(D, qd, h, cols)
                got += o
                seen += sn
        assert (seen == 1).all()  # every value read once
        assert np.array_equal(got, want)
