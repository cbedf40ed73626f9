"""CPU emulation of the tile kernels' index arithmetic (no GPU).

Replays, for every thread of every CTA, the global and shared-memory
addresses that the tile kernels compute (same formulas, written again in
Python from the kernel design: x y z split, rows at rev(x) in shared memory,
XOR swizzle, V x V register transpose, pair/self unit enumeration) and
checks that

  * every global access stays inside the 2^k-element buffer and every
    shared-memory access inside the CTA's allocation,
  * each source element is loaded exactly once and each destination
    element written exactly once,
  * shared-memory rows are written without bank conflicts and read without
    bank conflicts (per 128-byte wavefront),
  * the resulting permutation equals the CPU oracle.

This is the check run before any kernel goes to a GPU.
"""
import numpy as np
import pytest

import pins


def brev(v, w):
    return pins.brute_rev(v, w) if w else 0


def count_lt(w):
    return (1 << (w - 1)) - (1 << ((w + 1) // 2 - 1)) if w >= 1 else 0


def count_self(w):
    return 1 << ((w + 1) // 2)


def unrank_lt(q, w):
    outer = 0
    d = 0
    while 2 * d + 2 <= w:
        rem = w - 2 * d
        c01 = 1 << (rem - 2)
        if q < c01:
            return outer | (q << (d + 1)) | (1 << d)
        q -= c01
        r2 = count_lt(rem - 2)
        if q >= r2:
            q -= r2
            outer |= (1 << (w - 1 - d)) | (1 << d)
        d += 1
    return outer


def unrank_self(p, w):
    a = (w + 1) // 2
    lw = w - a
    return (p << lw) | brev(p >> (a - lw), lw)


def blocked_tile(t, w):
    lo, hi, mid = t & 7, (t >> 3) & 7, t >> 6
    return (hi << (w - 3)) | (mid << 3) | lo


def blocked_unit(q, w):
    mw = w - 6
    full = count_lt(mw) << 6
    if q < full:
        mid, hi, lo = unrank_lt(q >> 6, mw), (q >> 3) & 7, q & 7
    else:
        q2 = q - full
        mid, r = unrank_self(q2 // 36, mw), q2 % 36
        if r < 28:
            lo = 0
            while r >= brev(lo, 3):
                r -= brev(lo, 3)
                lo += 1
            hi = r
        else:
            lo = r - 28
            hi = brev(lo, 3)
    y = (hi << (w - 3)) | (mid << 3) | lo
    return y, brev(y, w)


class Geom:
    def __init__(self, E, W, BX, BZ):
        self.E, self.W, self.BX, self.BZ = E, W, BX, BZ
        self.V = W // E
        self.CIN = (1 << BZ) // self.V
        self.COUT = (1 << BX) // self.V
        assert self.CIN * W >= 128 and self.COUT * W >= 128
        self.CHUNKS = (1 << BX) * self.CIN
        self.UNITS = self.CIN * self.COUT
        self.THREADS = min(self.UNITS, 256)
        self.PHASE = 128 // W
        self.SWZ = self.PHASE - 1


def emulate_tile(G, k, nthr, src_tiles, dst_tiles, row_stride_in, row_stride_out,
                 n_elems, loads, stores, conflicts):
    """One CTA: load NT tiles (element offsets of their (x=0, z=0) corner),
    then store tile t to dst_tiles[t].  Records element moves."""
    smem = {}
    per = (G.CHUNKS + nthr - 1) // nthr
    for t, base in enumerate(src_tiles):
        # load phase, per warp instruction: lanes of one i
        for i in range(per):
            slots = []
            for tid in range(nthr):
                q = tid + i * nthr
                if q >= G.CHUNKS:
                    continue
                x, c = q // G.CIN, q % G.CIN
                for e in range(G.V):
                    g = base + x * row_stride_in + c * G.V + e
                    assert 0 <= g < n_elems
                    loads.append(g)
                X = brev(x, G.BX)
                pc = c ^ ((X // G.V) & G.SWZ)
                assert 0 <= pc < G.CIN
                s = t * G.CHUNKS + X * G.CIN + pc
                assert 0 <= s < len(src_tiles) * G.CHUNKS
                smem[s] = [(base + x * row_stride_in + c * G.V + e) for e in range(G.V)]
                slots.append((tid, s))
            conflicts.append(_wavefront_conflicts(slots, G.W))
    for t, dbase in enumerate(dst_tiles):
        per_u = (G.UNITS + nthr - 1) // nthr
        for i in range(per_u):
            for j in range(G.V):
                slots = []
                for tid in range(nthr):
                    u = tid + i * nthr
                    if u >= G.UNITS:
                        continue
                    c, d = u // G.COUT, u % G.COUT
                    pc = c ^ (d & G.SWZ)
                    s = t * G.CHUNKS + (d * G.V + j) * G.CIN + pc
                    slots.append((tid, s))
                conflicts.append(_wavefront_conflicts(slots, G.W))
            for tid in range(nthr):
                u = tid + i * nthr
                if u >= G.UNITS:
                    continue
                c, d = u // G.COUT, u % G.COUT
                pc = c ^ (d & G.SWZ)
                blk = [smem[t * G.CHUNKS + (d * G.V + j) * G.CIN + pc] for j in range(G.V)]
                for e in range(G.V):
                    Z = brev(c * G.V + e, G.BZ)
                    for j in range(G.V):
                        g = dbase + Z * row_stride_out + d * G.V + j
                        assert 0 <= g < n_elems
                        stores.append((g, blk[j][e]))


def _wavefront_conflicts(slots, W):
    """Extra wavefronts beyond the minimum for one warp-wide shared access of
    W bytes per lane (slots: (lane, chunk index)), per warp."""
    extra = 0
    by_warp = {}
    for tid, s in slots:
        by_warp.setdefault(tid // 32, []).append(s)
    for chunks in by_warp.values():
        # bank of each 4-byte word touched
        words = {}
        for s in chunks:
            b0 = s * W
            for w in range(max(1, W // 4)):
                addr = b0 + 4 * w
                words.setdefault((addr // 4) % 32, set()).add(addr // 4)
        need = max(len(v) for v in words.values())
        minimum = max(1, (len(chunks) * W + 127) // 128)
        extra += max(0, need - minimum)
    return extra


SHAPES = {
    16: [(3, 3), (4, 4), (5, 5), (6, 6), (4, 5), (5, 4), (5, 6), (6, 5)],
    8: [(4, 4), (5, 5), (6, 6), (4, 5), (5, 4), (5, 6), (6, 5)],
    4: [(5, 5), (6, 6), (7, 7), (5, 6), (6, 5), (6, 7), (7, 6)],
    2: [(6, 6), (7, 7)],
    1: [(7, 7), (8, 8)],
}
WIDE = {8: [(4, 4), (5, 5)], 4: [(5, 5), (6, 6)], 2: [(6, 6)], 1: [(7, 7)]}


def run_oop(E, W, bx, bz, k, nthr=None, order=0):
    G = Geom(E, W, bx, bz)
    nthr = nthr or G.THREADS
    n = 1 << k
    wy = k - bx - bz
    loads, stores, conflicts = [], [], []
    for t in range(1 << wy):
        y = blocked_tile(t, wy) if (order == 1 and wy >= 6) else t
        assert 0 <= y < (1 << wy)
        ry = brev(y, wy)
        emulate_tile(G, k, nthr, [y << bz], [ry << bx], 1 << (k - bx), 1 << (k - bz), n,
                     loads, stores, conflicts)
    return G, loads, stores, conflicts


def run_inplace(E, W, b, k, nthr=None, order=0):
    G = Geom(E, W, b, b)
    nthr = nthr or G.THREADS
    n = 1 << k
    w = k - 2 * b
    loads, stores, conflicts = [], [], []
    units = count_lt(w) + count_self(w)
    seen = set()
    for q in range(units):
        if order == 1 and w >= 6:
            y, ry = blocked_unit(q, w)
            assert 0 <= y < (1 << w) and ry == brev(y, w)
            src, dst = ([y << b, ry << b], [ry << b, y << b]) if y != ry else ([y << b], [y << b])
        elif q < count_lt(w):
            y = unrank_lt(q, w)
            ry = brev(y, w)
            assert y < ry
            src, dst = [y << b, ry << b], [ry << b, y << b]
        else:
            y = unrank_self(q - count_lt(w), w)
            assert y == brev(y, w)
            src, dst = [y << b], [y << b]
        y0 = src[0] >> b
        assert y0 not in seen and brev(y0, w) not in seen
        seen.add(y0)
        seen.add(brev(y0, w))
        emulate_tile(G, k, nthr, src, dst, 1 << (k - b), 1 << (k - b), n, loads, stores,
                     conflicts)
    assert len(seen) == 1 << w  # every tile covered exactly once
    return G, loads, stores, conflicts


def check_result(k, loads, stores):
    n = 1 << k
    assert sorted(loads) == list(range(n)), "each source element loaded once"
    dsts = sorted(g for g, _ in stores)
    assert dsts == list(range(n)), "each destination element written once"
    perm = np.empty(n, dtype=np.int64)
    for g, s in stores:
        perm[g] = s
    exp = np.array([brev(j, k) for j in range(n)])
    assert np.array_equal(perm, exp)


@pytest.mark.parametrize("E", sorted(SHAPES))
def test_oop_index_math(E):
    for bx, bz in SHAPES[E]:
        for k in sorted({bx + bz, bx + bz + 1, bx + bz + 2}):
            if (1 << k) > (1 << 17):
                continue
            G, loads, stores, conf = run_oop(E, 16, bx, bz, k)
            check_result(k, loads, stores)
            assert sum(conf) == 0, (E, bx, bz, k)


@pytest.mark.parametrize("E", sorted(SHAPES))
def test_inplace_index_math(E):
    for b in sorted({bx for bx, bz in SHAPES[E] if bx == bz}):
        for k in sorted({2 * b, 2 * b + 1, 2 * b + 2, 2 * b + 3}):
            if (1 << k) > (1 << 17):
                continue
            G, loads, stores, conf = run_inplace(E, 16, b, k)
            check_result(k, loads, stores)
            assert sum(conf) == 0, (E, b, k)


@pytest.mark.parametrize("E", sorted(WIDE))
def test_element_wide_index_math(E):
    for b, _ in WIDE[E]:
        k = 2 * b + 1
        G, loads, stores, conf = run_oop(E, E, b, b, k)
        check_result(k, loads, stores)
        G, loads, stores, conf = run_inplace(E, E, b, k)
        check_result(k, loads, stores)


def batched_stage_bytes(k, E, b):
    raw = (E << k) if b == 0 else 2 * (1 << b) * ((E << b) + 16)
    return (raw + 127) & ~127


def emulate_staged_unit(E, b, k, u, nthr=256, transpose=False, copy=0):
    """Replay one unit of the TMA-staged batched kernel: the copies the
    producer warp issues (row x of each tile to padded row rev(x), or x for
    a transposition; copy 0: one bulk copy per row, copy 1: the rows'
    16-byte chunks spread over the 32 lanes) and the store phase of the
    consumer threads.
    Bit reversal: an array of 2^k elements; transposition: a 2^k x 2^k
    matrix.  Returns (copied source elements, stores as (destination
    element, source element), read-slot conflicts)."""
    n = 1 << (2 * k if transpose else k)
    stage = batched_stage_bytes(2 * b if transpose else k, E, b)
    smem = {}  # byte offset of an element in the stage -> source element
    loads, stores, conflicts = [], [], 0
    if b == 0:
        nbytes = E << k
        assert nbytes % 16 == 0 and nbytes <= stage
        for i in range(n):
            smem[i * E] = i
            loads.append(i)
        for j in range(n):
            stores.append((j, smem[brev(j, k) * E]))
        return loads, stores, 0
    rowb, rows = E << b, 1 << b
    pitch = rowb + 16
    if transpose:
        T = 1 << (k - b)
        npairs = T * (T - 1) // 2
        if T >= 8:
            tr, tc = blocked_upper(u, T)
        elif u < npairs:
            tr, tc = unrank_upper(u)
        else:
            tr = tc = u - npairs
        nt = 1 if tr == tc else 2
        stride = E << k
        a_off = ((tr << (b + k)) + (tc << b)) * E
        r_off = ((tc << (b + k)) + (tr << b)) * E
        rmap = lambda x: x
    else:
        wy = k - 2 * b
        npairs = count_lt(wy)
        if u < npairs:
            y = unrank_lt(u, wy)
            ry, nt = brev(y, wy), 2
        else:
            y = unrank_self(u - npairs, wy)
            ry, nt = y, 1
        stride = E << (k - b)
        a_off, r_off = (y << b) * E, (ry << b) * E
        rmap = lambda x: brev(x, b)
    tx = 0
    if copy == 0:
        for q in range(nt * rows):
            t, x = q >> b, q & (rows - 1)
            dst = t * rows * pitch + rmap(x) * pitch
            src = (r_off if t else a_off) + x * stride
            assert dst % 16 == 0 and src % 16 == 0 and rowb % 16 == 0
            assert 0 <= dst and dst + rowb <= stage and 0 <= src and src + rowb <= n * E
            for o in range(0, rowb, E):
                assert dst + o not in smem
                smem[dst + o] = (src + o) // E
                loads.append((src + o) // E)
            tx += rowb
        assert tx == nt * rows * rowb  # the byte count lane 0 expects
    else:
        cpr = rowb // 16
        log_cpr = cpr.bit_length() - 1
        assert cpr == 1 << log_cpr
        chunks = nt * (rows << log_cpr)
        assert chunks % 32 == 0  # every lane issues the same number of copies
        for lane in range(32):
            for q in range(lane, chunks, 32):
                c = q & (cpr - 1)
                tx_ = q >> log_cpr
                t, x = tx_ >> b, tx_ & (rows - 1)
                dst = t * rows * pitch + rmap(x) * pitch + c * 16
                src = (r_off if t else a_off) + x * stride + c * 16
                assert dst % 16 == 0 and src % 16 == 0
                assert 0 <= dst and dst + 16 <= stage and 0 <= src and src + 16 <= n * E
                for o in range(0, 16, E):
                    assert dst + o not in smem
                    smem[dst + o] = (src + o) // E
                    loads.append((src + o) // E)
    V = 16 // E
    log_v = V.bit_length() - 1
    log_c = b - log_v
    cmask = (1 << log_c) - 1
    units = 1 << (2 * log_c)
    for t, dst_tile in ((0, r_off), (1, a_off))[:nt]:
        base = t * rows * pitch
        reads = {}
        for q in range(units):
            cl = q & (V - 1)
            rest = q >> log_v
            d = rest & cmask
            c = ((rest >> log_c) << log_v) | cl
            blk = []
            for j in range(V):
                addr = base + (d * V + j) * pitch + c * 16
                assert addr % 16 == 0 and addr + 16 <= stage
                blk.append([smem[addr + e * E] for e in range(V)])
                reads.setdefault((q // 32, j), []).append((q % nthr, addr // 16))
            for e in range(V):
                Z = rmap(c * V + e)
                g = dst_tile + Z * stride + d * 16
                assert g % 16 == 0 and g + 16 <= n * E
                for j in range(V):
                    stores.append((g // E + j, blk[j][e]))
        conflicts += sum(_wavefront_conflicts(sl, 16) for sl in reads.values())
    return loads, stores, conflicts


BATCHED_SHAPES = {16: (3, 4, 5), 8: (4, 5), 4: (5, 6)}
BATCHED_BMIN = {16: 3, 8: 4, 4: 5}


@pytest.mark.parametrize("nthr", (128, 256))
@pytest.mark.parametrize("copy", (0, 1))
@pytest.mark.parametrize("E", sorted(BATCHED_SHAPES))
def test_batched_staged_index_math(E, copy, nthr):
    """TMA-staged batched kernel with 4 or 8 consumer warps (nthr), tile
    rows staged as bulk copies (copy 0) or as per-thread 16-byte chunks
    (copy 1): copies in bounds, 16-byte
    aligned and counted in the expected bytes; every staged chunk read once
    per tile without bank conflicts; every element moved once to rev(i)."""
    cases = [(k, 0) for k in range(2, 16)
             if k < 2 * BATCHED_BMIN[E] or (E << k) <= 32768]   # whole array staged
    cases += [(k, b) for b in BATCHED_SHAPES[E] for k in range(2 * b, 2 * b + 4)
              if k <= 17]
    for k, b in cases:
        units = 1 if b == 0 else count_lt(k - 2 * b) + count_self(k - 2 * b)
        loads, stores, conf = [], [], 0
        for u in range(units):
            lo, st, c = emulate_staged_unit(E, b, k, u, nthr=nthr, copy=copy)
            loads += lo
            stores += st
            conf += c
        check_result(k, loads, stores)
        assert conf == 0, (E, b, k)
    # the same pipeline as an in-place square transposition (2^a x 2^a)
    b = {16: 5, 8: 5, 4: 6}[E]
    for a in (b, b + 1, b + 3, b + 4):
        T = 1 << (a - b)
        loads, stores, conf = [], [], 0
        for u in range(T * (T - 1) // 2 + T):
            lo, st, c = emulate_staged_unit(E, b, a, u, nthr=nthr, transpose=True, copy=copy)
            loads += lo
            stores += st
            conf += c
        n = 1 << (2 * a)
        assert sorted(loads) == list(range(n))
        assert sorted(g for g, _ in stores) == list(range(n))
        side = 1 << a
        assert all(src == (g % side) * side + g // side for g, src in stores), (E, a)
        assert conf == 0
    # two stages of the largest unit leave room for three CTAs per SM
    worst = max(batched_stage_bytes(2 * b, E, b) for b in BATCHED_SHAPES[E])
    assert 3 * (2 * worst + 1024 + 128) <= 228 * 1024


def test_unranking_enumerates_pairs_and_palindromes():
    for w in range(0, 15):
        lt = [unrank_lt(q, w) for q in range(count_lt(w))]
        assert sorted(lt) == [y for y in range(1 << w) if y < brev(y, w)]
        pal = [unrank_self(p, w) for p in range(count_self(w))]
        assert sorted(pal) == [y for y in range(1 << w) if y == brev(y, w)]


def find_array(first_ticket, t):
    """Warp-parallel search of the batched kernel, lane by lane."""
    lo, hi = 0, len(first_ticket)
    rounds = 0
    while hi - lo > 1:
        span = hi - lo
        pos = [lo + ((span * lane) >> 5) for lane in range(32)]
        ok = [first_ticket[p] <= t for p in pos]
        assert all(0 <= p < len(first_ticket) for p in pos)
        last = max(l for l in range(32) if ok[l])
        nlo = pos[last]
        nhi = pos[last + 1] if last < 31 else hi
        lo, hi = nlo, nhi
        rounds += 1
        assert rounds < 10
    return lo


def test_batched_array_search():
    rng = np.random.default_rng(3)
    for count in (1, 2, 3, 31, 32, 33, 100, 4096):
        sizes = rng.integers(1, 50, size=count)
        first = np.concatenate([[0], np.cumsum(sizes)[:-1]]).tolist()
        total = int(sizes.sum())
        for t in list(range(0, min(total, 300))) + rng.integers(0, total, 300).tolist():
            a = find_array(first, int(t))
            assert first[a] <= t < (first[a + 1] if a + 1 < count else total)


def guided_schedule(arrays, ctas, guide=4, ticket_bytes=262144, extra_max=24):
    """Host-side ticket schedule of the batched launch, restated: arrays
    (units, unit_bytes), largest first; the grain (units per ticket) is
    about ticket_bytes of tiles and is halved, down to one unit, whenever the
    work left falls below guide x ctas x the ticket's bytes, splitting an
    array across descriptors (unit0, units, grain, first_ticket)."""
    order = sorted(range(len(arrays)), key=lambda i: -arrays[i][0] * arrays[i][1])
    left = sum(u * ub for u, ub in arrays)
    t, extra, desc = 0, 0, []
    for a in order:
        units, ub = arrays[a]
        gmax = min(max(1, ticket_bytes // ub), units)
        u = 0
        while u < units:
            want = left // (guide * ctas * ub)
            g = gmax
            while g > 1 and g > want:
                g = (g + 1) // 2
            n = units - u
            if g > 1 and extra < extra_max:
                keep = g * guide * ctas * ub
                m = (left - keep) // ub + 1
                n = min(n, (m + g - 1) // g * g)
            elif g > 1:
                g = gmax
            desc.append((a, u, n, g, t, left, extra < extra_max))
            t += -(-n // g)
            if u > 0:
                extra += 1
            u += n
            left -= n * ub
    return desc, t


def test_batched_guided_schedule():
    """Every unit of every array in exactly one ticket; descriptors in
    ticket order; while descriptors are left for splits, no ticket holds
    more than the work left at its start / (guide x CTAs), or one unit;
    at most 24 descriptors beyond one per array."""
    rng = np.random.default_rng(11)
    cases = [[(count_lt(w) + count_self(w), 32768)] * c for w, c in ((14, 2), (12, 8), (10, 64))]
    cases += [[(int(rng.integers(1, 2000)), int(rng.choice([2048, 8192, 16384, 32768])))
               for _ in range(int(rng.integers(1, 200)))] for _ in range(15)]
    for arrays in cases:
        for ctas in (1, 152, 456):
            desc, tickets = guided_schedule(arrays, ctas)
            covered = {}
            seen_t = 0
            for a, u0, n, g, ft, left, split_ok in desc:
                if split_ok:
                    assert g == 1 or g * arrays[a][1] * 4 * ctas <= left
                assert ft == seen_t and n >= 1 and g >= 1
                seen_t += -(-n // g)
                for tk in range(-(-n // g)):
                    lo, hi = u0 + tk * g, min(u0 + (tk + 1) * g, u0 + n)
                    for u in range(lo, hi):
                        assert (a, u) not in covered
                        covered[(a, u)] = ft + tk
            assert seen_t == tickets
            assert len(covered) == sum(u for u, _ in arrays)
            assert len(desc) <= len(arrays) + 24
            if desc[-1][6]:
                assert desc[-1][3] == 1  # the last tickets are single units


@pytest.mark.parametrize("E", (16, 8, 4))
def test_blocked_order_index_math(E):
    """The blocked launch order (runs of 8 adjacent tiles) is a bijection
    of the tiles / units and keeps every access in bounds."""
    b = {16: 3, 8: 4, 4: 5}[E]
    for k in (2 * b + 6, 2 * b + 7, 2 * b + 8):
        if (1 << k) > (1 << 17):
            continue
        G, loads, stores, conf = run_oop(E, 16, b, b, k, order=1)
        check_result(k, loads, stores)
        G, loads, stores, conf = run_inplace(E, 16, b, k, order=1)
        check_result(k, loads, stores)
        assert sum(conf) == 0


def test_blocked_unit_covers_all_tiles_large_w():
    for w in range(6, 17):
        seen = set()
        for q in range(count_lt(w) + count_self(w)):
            y, ry = blocked_unit(q, w)
            assert y not in seen and ry not in seen
            seen.add(y)
            seen.add(ry)
        assert len(seen) == 1 << w
        assert sorted({blocked_tile(t, w) for t in range(1 << w)}) == list(range(1 << w))


# ----------------------------------------------- runtime-geometry tiles --
def emulate_g(E, W, nthr, rev, srcs, dsts, stride_in, stride_out, bx, bz, n, loads, stores):
    """load_tiles_g / store_tile_g of one CTA (run-time bx, bz; rev maps on
    or off).  srcs/dsts: element offsets of the tiles' corners."""
    V = W // E
    lv = V.bit_length() - 1
    phase = 128 // W
    log_cin = bz - lv
    log_cout = bx - lv
    assert log_cin >= 0 and log_cout >= 0
    cin = 1 << log_cin
    mask = min(cin, phase) - 1
    chunks = 1 << (bx + log_cin)
    smem = {}
    for t, base in enumerate(srcs):
        for q in range(chunks):
            x, c = q >> log_cin, q & (cin - 1)
            X = brev(x, bx) if rev else x
            pc = c ^ ((X >> lv) & mask)
            assert 0 <= pc < cin
            s = t * chunks + (X << log_cin) + pc
            assert s not in smem and 0 <= s < len(srcs) * chunks
            els = []
            for e in range(V):
                g = base + x * stride_in + c * V + e
                assert 0 <= g < n
                loads.append(g)
                els.append(g)
            smem[s] = els
    units = 1 << (log_cin + log_cout)
    for t, dbase in enumerate(dsts):
        for u in range(units):
            c, d = u >> log_cout, u & ((1 << log_cout) - 1)
            pc = c ^ (d & mask)
            blk = [smem[t * chunks + ((d * V + j) << log_cin) + pc] for j in range(V)]
            for e in range(V):
                z = c * V + e
                Z = brev(z, bz) if rev else z
                for j in range(V):
                    g = dbase + Z * stride_out + d * V + j
                    assert 0 <= g < n
                    stores.append((g, blk[j][e]))


TARGET_B = {16: 5, 8: 5, 4: 6, 2: 7, 1: 8}


def transpose_tiles(a, c, E, vec16=True):
    """The host's tile choice for an out-of-place transposition."""
    B = TARGET_B[E]
    T = 2 * B
    lv = (16 // E).bit_length() - 1
    bz0 = min(c, B)
    bx = min(a, T - bz0)
    bz = min(c, T - bx)
    W = 16 if (vec16 and bx >= lv and bz >= lv) else E
    return bx, bz, W


def check_perm(n, loads, stores, expected_src_of_dst):
    assert sorted(loads) == list(range(n))
    assert sorted(g for g, _ in stores) == list(range(n))
    for g, s in stores:
        assert s == expected_src_of_dst[g]


def transpose_src_of_dst(a, c):
    R, C = 1 << a, 1 << c
    out = np.empty(R * C, dtype=np.int64)
    for i in range(R):
        for j in range(C):
            out[j * R + i] = i * C + j
    return out


@pytest.mark.parametrize("E", (16, 8, 4, 2, 1))
def test_transpose_oop_index_math(E):
    for a, c in ((0, 0), (0, 5), (5, 0), (1, 9), (9, 1), (3, 4), (6, 6), (7, 2), (2, 11),
                 (11, 3)):
        for vec in (True, False):
            bx, bz, W = transpose_tiles(a, c, E, vec)
            n = 1 << (a + c)
            loads, stores = [], []
            for t in range(1 << ((a - bx) + (c - bz))):
                tr, tc = t >> (c - bz), t & ((1 << (c - bz)) - 1)
                emulate_g(E, W, 256, False, [(tr << (bx + c)) + (tc << bz)],
                          [(tc << (bz + a)) + (tr << bx)], 1 << c, 1 << a, bx, bz, n,
                          loads, stores)
            check_perm(n, loads, stores, transpose_src_of_dst(a, c))


def blocked_upper(q, T):
    Tb = T >> 3
    off = Tb * (Tb - 1) // 2 * 64
    if q < off:
        bi, bj = unrank_upper(q >> 6)
        return (bi << 3) + ((q >> 3) & 7), (bj << 3) + (q & 7)
    q2 = q - off
    blk, u = q2 // 36, q2 % 36
    if u < 28:
        r, c = unrank_upper(u)
        return (blk << 3) + r, (blk << 3) + c
    return (blk << 3) + (u - 28), (blk << 3) + (u - 28)


def test_blocked_upper_covers_each_pair_once():
    for T in (8, 16, 64):
        seen = [blocked_upper(q, T) for q in range(T * (T + 1) // 2)]
        assert sorted(seen) == sorted((r, c) for c in range(T) for r in range(c + 1))


def unrank_upper(q):
    import math
    col = int((1.0 + math.sqrt(1.0 + 8.0 * q)) * 0.5)
    while col * (col - 1) // 2 > q:
        col -= 1
    while (col + 1) * col // 2 <= q:
        col += 1
    return q - col * (col - 1) // 2, col


def test_upper_triangle_unranking():
    for T in (1, 2, 3, 8, 33, 256):
        got = [unrank_upper(q) for q in range(T * (T - 1) // 2)]
        assert got == [(r, c) for c in range(T) for r in range(c)]
    # large indices: consistency at the column boundaries
    for col in (1 << 12, (1 << 14) - 1, 1 << 15):
        q0 = col * (col - 1) // 2
        assert unrank_upper(q0) == (0, col)
        assert unrank_upper(q0 - 1) == (col - 2, col - 1)


@pytest.mark.parametrize("E", (16, 8, 4, 1))
def test_transpose_inplace_index_math(E):
    lv = (16 // E).bit_length() - 1
    for a in (0, 1, 2, 5, 7, 8, 9):
        b = min(a, TARGET_B[E])
        W = 16 if b >= lv else E
        Tn = 1 << (a - b)
        n = 1 << (2 * a)
        loads, stores = [], []
        npairs = Tn * (Tn - 1) // 2
        for q in range(npairs + Tn):
            if Tn >= 8:
                tr, tc = blocked_upper(q, Tn)
                assert tr <= tc < Tn
            elif q < npairs:
                tr, tc = unrank_upper(q)
            else:
                tr = tc = q - npairs
            if tr < tc:
                A = (tr << (b + a)) + (tc << b)
                B_ = (tc << (b + a)) + (tr << b)
                emulate_g(E, W, 256, False, [A, B_], [B_, A], 1 << a, 1 << a, b, b, n,
                          loads, stores)
            else:
                A = (tr << (b + a)) + (tc << b)
                emulate_g(E, W, 256, False, [A], [A], 1 << a, 1 << a, b, b, n, loads, stores)
        if a:
            check_perm(n, loads, stores, transpose_src_of_dst(a, a))


def segment_choice(m, E):
    b_min = {16: 3, 8: 4, 4: 5, 2: 6, 1: 7}[E]
    if m < 2 * b_min:
        return 0
    return min(TARGET_B[E] - (1 if E <= 2 else 0), m // 2)


@pytest.mark.parametrize("E", (16, 8, 4, 2))
def test_segments_index_math(E):
    for s_log, m in ((0, 12), (3, 10), (4, 13), (2, 15)):
        b = segment_choice(m, E)
        if b == 0:
            continue
        n = 1 << (s_log + m)
        w = m - 2 * b
        units = count_lt(w) + count_self(w)
        loads, stores = [], []
        for qq in range(units << s_log):
            seg, q = qq // units, qq % units
            base = seg << m
            if q < count_lt(w):
                y = unrank_lt(q, w)
                ry = brev(y, w)
                srcs, dsts = [base + (y << b), base + (ry << b)], [base + (ry << b),
                                                                   base + (y << b)]
            else:
                y = unrank_self(q - count_lt(w), w)
                srcs = dsts = [base + (y << b)]
            emulate_g(E, 16, 256, True, srcs, dsts, 1 << (m - b), 1 << (m - b), b, b, n,
                      loads, stores)
        exp = np.array([((g >> m) << m) + brev(g & ((1 << m) - 1), m) for g in range(n)])
        check_perm(n, loads, stores, exp)


def test_recursive_composition_math():
    """The three passes of the recursive ablation compose to the full
    permutation (even k), and the odd-k route with its even-odd step too."""
    def seg_rev(v, h):
        s = 1 << h
        return np.concatenate([v[r * s:(r + 1) * s][[brev(j, h) for j in range(s)]]
                               for r in range(len(v) // s)])

    def transpose_sq(v, h):
        s = 1 << h
        return v.reshape(s, s).T.reshape(-1)

    for k in (2, 4, 6, 8, 10):
        h = k // 2
        v = np.arange(1 << k)
        out = seg_rev(transpose_sq(seg_rev(v, h), h), h)
        assert out.tolist() == [brev(j, k) for j in range(1 << k)]
    for k in (3, 5, 7, 9):
        v = np.arange(1 << k)
        eo = np.concatenate([v[0::2], v[1::2]])
        h = (k - 1) // 2
        halves = [seg_rev(transpose_sq(seg_rev(part, h), h), h)
                  for part in (eo[: 1 << (k - 1)], eo[1 << (k - 1):])]
        assert np.concatenate(halves).tolist() == [brev(j, k) for j in range(1 << k)]


def test_fused_fft_butterfly_indexing():
    """dit_stages' thread -> (column z, pair X0, twiddle index) mapping applies
    every stage to every output row (a shared-memory column) exactly as the
    textbook stage, with table index j * 2^(B-s) < 2^(B-1)."""
    rng = np.random.default_rng(0)
    for B in (3, 4, 5, 6):
        BZ = B
        table = np.exp(-2j * np.pi * np.arange(1 << (B - 1)) / (1 << B))
        for S in range(0, B + 1):
            cols = rng.normal(size=(1 << BZ, 1 << B)) + 1j * rng.normal(size=(1 << BZ, 1 << B))
            got = cols.copy()
            NB = 1 << (B + BZ - 1)
            for s in range(1, S + 1):
                h = 1 << (s - 1)
                touched = set()
                for u in range(NB):
                    z = u & ((1 << BZ) - 1)
                    p = u >> BZ
                    j = p & (h - 1)
                    X0 = ((p >> (s - 1)) << s) + j
                    ti = j << (B - s)
                    assert 0 <= X0 < X0 + h < (1 << B) and 0 <= ti < (1 << (B - 1))
                    assert (z, X0) not in touched and (z, X0 + h) not in touched
                    touched |= {(z, X0), (z, X0 + h)}
                    a, b = got[z, X0], got[z, X0 + h] * table[ti]
                    got[z, X0], got[z, X0 + h] = a + b, a - b
                assert len(touched) == (1 << BZ) << B
            exp = cols.copy()
            for s in range(1, S + 1):
                m, h = 1 << s, 1 << (s - 1)
                for base in range(0, 1 << B, m):
                    for j in range(h):
                        w = np.exp(-2j * np.pi * j / m)
                        a, b = exp[:, base + j].copy(), exp[:, base + j + h] * w
                        exp[:, base + j], exp[:, base + j + h] = a + b, a - b
            assert np.allclose(got, exp, atol=1e-12)


def test_fused_fft_register_passes():
    """dit_pass: groups of 2^R elements X = base + j + t 2^s0 per column, R
    stages in registers, passes of up to three stages -- same result as the
    textbook stages, every element in exactly one group per pass."""
    rng = np.random.default_rng(1)
    for B in (3, 4, 5, 6):
        BZ = B
        table = np.exp(-2j * np.pi * np.arange(1 << (B - 1)) / (1 << B))
        for S in range(0, B + 1):
            cols = rng.normal(size=(1 << BZ, 1 << B)) + 1j * rng.normal(size=(1 << BZ, 1 << B))
            got = cols.copy()
            s0 = 0
            while s0 < S:
                R = min(3, S - s0)
                seen = set()
                for g in range(1 << (B + BZ - R)):
                    z = g & ((1 << BZ) - 1)
                    q = g >> BZ
                    j = q & ((1 << s0) - 1)
                    base = (q >> s0) << (s0 + R)
                    Xs = [base + j + (t << s0) for t in range(1 << R)]
                    assert all(0 <= X < (1 << B) for X in Xs)
                    for X in Xs:
                        assert (z, X) not in seen
                        seen.add((z, X))
                    v = [got[z, X] for X in Xs]
                    for r in range(R):
                        s = s0 + r + 1
                        hmask = (1 << (s - 1)) - 1
                        for t in range(1 << R):
                            if t & (1 << r):
                                continue
                            jj = (j + (t << s0)) & hmask
                            w = table[jj << (B - s)]
                            a, b = v[t], v[t + (1 << r)] * w
                            v[t], v[t + (1 << r)] = a + b, a - b
                    for X, val in zip(Xs, v):
                        got[z, X] = val
                assert len(seen) == (1 << BZ) << B
                s0 += R
            exp = cols.copy()
            for s in range(1, S + 1):
                m, h = 1 << s, 1 << (s - 1)
                for base in range(0, 1 << B, m):
                    for j in range(h):
                        w = np.exp(-2j * np.pi * j / m)
                        a, b = exp[:, base + j].copy(), exp[:, base + j + h] * w
                        exp[:, base + j], exp[:, base + j + h] = a + b, a - b
            assert np.allclose(got, exp, atol=1e-12), (B, S)


def _bfly_multiply_add(a, b, w):
    """butterfly(): a' from two multiply-adds per component, b' = 2a - a'."""
    px = b.real * w.real + (-b.imag * w.imag + a.real)
    py = b.real * w.imag + (b.imag * w.real + a.imag)
    return px + 1j * py, (2 * a.real - px) + 1j * (2 * a.imag - py)


def _bfly_const(a, b, S, JJ):
    """butterfly_const<S, JJ>(), forward: w = 1, the quarter turn -i, or an
    eighth turn as sqrt(1/2) (re, im) from s = b.x + b.y, d = b.y - b.x."""
    if JJ == 0 or 2 * JJ == 1 << (S - 1):
        t = b if JJ == 0 else -1j * b
        return a + t, a - t
    assert S == 3 and JJ in (1, 3)
    c = np.sqrt(0.5)
    s, d = b.real + b.imag, b.imag - b.real
    re, im = (s, d) if JJ == 1 else (d, -s)
    px, py = c * re + a.real, c * im + a.imag
    return px + 1j * py, (2 * a.real - px) + 1j * (2 * a.imag - py)


def _radix4_table():
    """kRadix4Fma as written in brev_fft.cu: row j = {t1, t2, t3, c1, c2,
    c3 / c1}."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_1708_01873_gb300", "csrc", "brev_fft.cu")).read()
    body = re.search(r"kRadix4Fma\[8\]\[6\] = \{(.*?)\};", src, re.S).group(1)
    rows = re.findall(r"\{([^{}]*)\}", body)
    return [[float(x) for x in r.split(",")] for r in rows]


def _radix4_fma(v, K):
    """radix4_fma restated: stages 4 and 5 of a group v0..v3 (positions j +
    8 t) in the tangent form w^m = c_m (1 + i t_m)."""
    t1, t2, t3, c1, c2, r = K
    u = v[1] + 1j * t2 * v[1]
    A, Bv = v[0] + c2 * u, v[0] - c2 * u
    p2, p3 = v[2] + 1j * t1 * v[2], v[3] + 1j * t3 * v[3]
    qp, qm = p2 + r * p3, p2 - r * p3
    return [A + c1 * qp, Bv - 1j * c1 * qm, A - c1 * qp, Bv + 1j * c1 * qm]


def test_radix4_constants_are_the_closed_forms():
    """Each entry of the kernels' radix-4 table is the double nearest its
    definition (exactly, against 50-digit arithmetic when mpmath is there;
    within 1e-15 relative of numpy's libm values in any case), rows 0 and 4 are
    unused, and the tangent form reproduces w^m: c_m (1 + i t_m) = w^m."""
    K = _radix4_table()
    assert len(K) == 8 and all(len(r) == 6 for r in K)
    assert K[0] == [0.0] * 6 and K[4] == [0.0] * 6
    try:
        import mpmath as mp
    except ImportError:
        mp = None
    for j in (1, 2, 3, 5, 6, 7):
        th = -np.pi * j / 16
        if mp is not None:
            with mp.workdps(50):
                a = -mp.pi * j / 16
                exact = [mp.tan(a), mp.tan(2 * a), mp.tan(3 * a), mp.cos(a), mp.cos(2 * a),
                         mp.cos(3 * a) / mp.cos(a)]
                assert K[j] == [float(x) for x in exact], j
        want = [np.tan(th), np.tan(2 * th), np.tan(3 * th), np.cos(th), np.cos(2 * th),
                np.cos(3 * th) / np.cos(th)]
        for got, w in zip(K[j], want):  # numpy's angle 3 th is itself rounded
            assert abs(got - w) <= 1e-15 * max(1.0, abs(w)), (j, got, w)
        w = np.exp(1j * th)
        t1, t2, t3, c1, c2, r = K[j]
        assert abs(c1 * (1 + 1j * t1) - w) < 1e-15
        assert abs(c2 * (1 + 1j * t2) - w ** 2) < 1e-15
        assert abs(r * c1 * (1 + 1j * t3) - w ** 3) < 1e-15


def test_fused_fft_multiply_add_butterflies():
    """The kernels' arithmetic forms -- forward butterflies only, with
    compile-time twiddles in the first pass (w = 1, quarter and eighth turns)
    and table twiddles with the double-precision multiply-add butterfly after
    it, or, for the second pass's radix-4 groups with j not 0 or 4, the
    22-operation tangent form (complex<float> keeps the textbook butterfly
    emulated above); the
    inverse conjugates the imaginary parts on the first pass's loads and the
    last pass's stores -- give the textbook DIT stages with
    w = exp(-+2 pi i j / 2^s) for every B and S, both directions."""
    rng = np.random.default_rng(7)
    for B in (3, 4, 5, 6):
        BZ = B
        table = np.exp(-2j * np.pi * np.arange(1 << (B - 1)) / (1 << B))
        for S in range(1, B + 1):
            for inverse in (0, 1):
                cols = rng.normal(size=(1 << BZ, 1 << B)) + 1j * rng.normal(size=(1 << BZ, 1 << B))
                got = cols.copy()
                conj = np.conj if inverse else (lambda x: x)
                R0 = min(3, S)
                last = conj if S == R0 else (lambda x: x)
                for base in range(0, 1 << B, 1 << R0):  # dit_first_pass, all columns at once
                    v = [conj(got[:, base + t]) for t in range(1 << R0)]
                    for r in range(R0):
                        for t in range(1 << R0):
                            if t & (1 << r):
                                continue
                            v[t], v[t + (1 << r)] = _bfly_const(v[t], v[t + (1 << r)], r + 1,
                                                                t & ((1 << r) - 1))
                    for t in range(1 << R0):
                        got[:, base + t] = last(v[t])
                s0 = R0
                while s0 < S:  # dit_pass
                    R = min(3, S - s0)
                    last = conj if s0 + R == S else (lambda x: x)
                    for q in range(1 << (B - R)):
                        j = q & ((1 << s0) - 1)
                        base = (q >> s0) << (s0 + R)
                        Xs = [base + j + (t << s0) for t in range(1 << R)]
                        v = [got[:, X].copy() for X in Xs]
                        if R == 2 and j not in (0, 4):  # radix4_fma (double precision)
                            v = _radix4_fma(v, _radix4_table()[j])
                            for X, val in zip(Xs, v):
                                got[:, X] = last(val)
                            continue
                        for r in range(R):
                            s = s0 + r + 1
                            hmask = (1 << (s - 1)) - 1
                            for t in range(1 << R):
                                if t & (1 << r):
                                    continue
                                jj = (j + (t << s0)) & hmask
                                if j in (0, 4) and (jj * 8) % (1 << s) == 0:
                                    # dit_group<J = 0, 4>: whole eighth turns take
                                    # butterfly_const's compile-time form
                                    v[t], v[t + (1 << r)] = _bfly_const(
                                        v[t], v[t + (1 << r)], 3, (jj * 8) >> s)
                                    continue
                                w = table[jj << (B - s)]
                                v[t], v[t + (1 << r)] = _bfly_multiply_add(v[t], v[t + (1 << r)],
                                                                           w)
                        for X, val in zip(Xs, v):
                            got[:, X] = last(val)
                    s0 += R
                exp = cols.copy()
                sign = 1 if inverse else -1
                for s in range(1, S + 1):
                    m, h = 1 << s, 1 << (s - 1)
                    for base in range(0, 1 << B, m):
                        for j in range(h):
                            w = np.exp(sign * 2j * np.pi * j / m)
                            a, b = exp[:, base + j].copy(), exp[:, base + j + h] * w
                            exp[:, base + j], exp[:, base + j + h] = a + b, a - b
                assert np.allclose(got, exp, atol=1e-12), (B, S, inverse)


def test_fused_fft_pair_passes_cover_both_tiles():
    """In place, one pass loop runs the groups of both staged tiles of a
    pair: index gt -> tile gt >> LOG_GROUPS (at gt's tile offset), group
    gt & (groups - 1); each (tile, group) exactly once for any thread count."""
    for B in (3, 4, 5, 6):
        for R in (1, 2, 3):
            log_groups = 2 * B - R
            for nt in (1, 2):
                for nthr in (64, 256, 512):
                    seen = set()
                    for tid in range(nthr):
                        for gt in range(tid, nt << log_groups, nthr):
                            tile, g = gt >> log_groups, gt & ((1 << log_groups) - 1)
                            assert 0 <= tile < nt
                            assert (tile, g) not in seen
                            seen.add((tile, g))
                    assert len(seen) == nt << log_groups


def _streaming_claims(units, grid, rng, buffers):
    """The streaming complex<double> FFT kernels' schedule, one CTA per
    resident slot, run under a random interleaving of the CTAs.  CTA c
    starts at unit c and claims grid + (the counter's old value) for the
    unit after it before its first unit is processed; in the loop, while
    the next unit is valid, thread 0 claims the one after it (an atomic on
    the shared counter), the CTA processes the current unit, and the claim
    becomes the next unit (units >= `units` end the loop).  With two
    buffers (out of place) the next unit's tiles are loaded before the
    current one is processed; with one (in place) after it.  Returns the
    units each CTA processed in order, the counter's final value and the
    load/process log of every CTA."""
    counter = [0]

    def claim():
        v = counter[0]
        counter[0] += 1
        return grid + v

    def cta(c):
        log = []
        q = c
        qn = claim()  # prologue: thread 0, published by the barrier
        log.append(("load", q))
        yield
        while q < units:
            nxt = qn < units
            if nxt and buffers == 2:
                log.append(("load", qn))
            cl = claim() if nxt else None
            yield  # other CTAs run between the claim and its use
            log.append(("process", q))
            q, qn = qn, (cl if nxt else units)
            if q < units and buffers == 1:
                log.append(("load", q))
            yield
        return log

    gens = {c: cta(c) for c in range(grid)}
    logs = {}
    while gens:
        c = int(rng.choice(list(gens)))
        try:
            next(gens[c])
        except StopIteration as stop:
            logs[c] = stop.value
            del gens[c]
    return logs, counter[0]


@pytest.mark.parametrize("buffers", (1, 2))
def test_streaming_fft_claims_cover_each_unit_once(buffers):
    """Every unit (tile, or tile pair in place) is processed by exactly one
    CTA, every CTA ends, each CTA loads a unit before processing it and
    processes what it loaded in the same order.  The counter ends at exactly
    `units`: the units past the first `grid` are claimed once each, and every
    CTA makes one failing claim, so grid + counter stays below units + grid
    and a 32-bit counter cannot wrap for any array the kernels accept."""
    rng = np.random.default_rng(3)
    for units, grid in ((913, 912), (1024, 912), (2048, 912), (5000, 456), (40, 7), (8, 7)):
        for _ in range(3):
            logs, final = _streaming_claims(units, grid, rng, buffers)
            assert sorted(logs) == list(range(grid))
            done = [q for log in logs.values() for op, q in log if op == "process"]
            assert sorted(done) == list(range(units))
            for log in logs.values():
                loaded = [q for op, q in log if op == "load" and q < units]
                processed = [q for op, q in log if op == "process"]
                assert loaded == processed
                for i, (op, q) in enumerate(log):  # loaded before processed
                    if op == "process":
                        assert ("load", q) in log[:i]
            assert final == units


class _MBar:
    """mbarrier phase semantics: a phase completes when its pending
    arrivals reach 0 and its transaction bytes are all in; try_wait(P) is
    true while the barrier's current phase parity differs from P."""

    def __init__(self, count):
        self.count, self.pending, self.tx, self.completed = count, count, 0, 0

    def _check(self):
        if self.pending == 0 and self.tx == 0:
            self.completed += 1
            self.pending = self.count

    def arrive(self, expect_tx=0):
        self.tx += expect_tx
        self.pending -= 1
        assert self.pending >= 0
        self._check()

    def complete_tx(self, n):
        self.tx -= n
        self._check()

    def async_arrive_register(self):
        """cp.async.mbarrier.arrive (no .noinc): pending rises now and
        falls when the thread's copies land (async_arrive_done)."""
        self.pending += 1

    def async_arrive_done(self):
        self.pending -= 1
        assert self.pending >= 0
        self._check()

    def try_wait(self, parity):
        return (self.completed & 1) != parity


def simulate_batched_pipeline(n_units, S, n_consumers, seed, lanes=0):
    """Random interleavings of the batched kernel's producer warp, its
    consumer warps and the copy engine, following the kernel's waits and
    arrivals; fails on a read before the bytes land, a stage overwritten
    while read, a lost or repeated unit, or a wait that can never end.
    lanes = 0: bulk copies (lane 0's arrival carries the byte count);
    lanes > 0: that many lanes' per-thread copies, each lane tied to the
    barrier by an asynchronous arrival, then lane 0's plain arrival."""
    rng = np.random.default_rng(seed)
    full = [_MBar(1) for _ in range(S)]
    empty = [_MBar(n_consumers) for _ in range(S)]
    info = [None] * S
    owner = [None] * S
    landed = set()
    inflight = []
    consumed = [[] for _ in range(n_consumers)]

    def producer():
        i = 0
        while True:
            st = i % S
            if i >= S:
                par = (i // S - 1) & 1
                yield lambda st=st, par=par: empty[st].try_wait(par)
            if i >= n_units:
                info[st] = -1
                full[st].arrive()
                break
            owner[st] = i
            if lanes == 0:
                info[st] = i
                full[st].arrive(expect_tx=64)
                inflight.append((st, i, None))
            else:
                for lane in range(lanes):  # copies issued, then the async arrivals
                    full[st].async_arrive_register()
                    inflight.append((st, i, lane))
                yield lambda: True  # __syncwarp: the lanes' copies may land meanwhile
                info[st] = i
                full[st].arrive()
            i += 1
        for m in range(1, S):
            if m > i:
                break
            j = i - m
            yield lambda j=j: full[j % S].try_wait((j // S) & 1)

    def consumer(w):
        i = 0
        while True:
            st = i % S
            yield lambda st=st, par=(i // S) & 1: full[st].try_wait(par)
            u = info[st]
            if u == -1:
                return
            assert u in landed and owner[st] == u
            consumed[w].append(u)
            yield lambda: True  # reading the stage takes time
            assert owner[st] == u, "stage overwritten while being read"
            empty[st].arrive()
            i += 1

    actors = {"p": producer()}
    actors.update({w: consumer(w) for w in range(n_consumers)})
    waits = {}
    for name, g in actors.items():
        waits[name] = next(g, None)
    live = {n for n, wt in waits.items() if wt is not None}
    steps = 0
    while live or inflight:
        ready = [n for n in live if waits[n]()]
        choices = ready + (["copy"] if inflight else [])
        assert choices, "deadlock: no actor can proceed"
        c = choices[rng.integers(len(choices))]
        if c == "copy":
            st, u, lane = inflight.pop(rng.integers(len(inflight)))
            if lane is None:
                landed.add(u)
                full[st].complete_tx(64)
            else:
                if not any(x[1] == u for x in inflight):
                    landed.add(u)  # the unit's last lane landed
                full[st].async_arrive_done()
        else:
            nxt = next(actors[c], None)
            if nxt is None:
                live.discard(c)
            else:
                waits[c] = nxt
        steps += 1
        assert steps < 200000
    for w in range(n_consumers):
        assert consumed[w] == list(range(n_units))


@pytest.mark.parametrize("lanes", [0, 3])
@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_batched_pipeline_protocol(S, lanes):
    for n_units in (0, 1, 2, S, S + 1, 7, 23):
        for seed in range(12):
            simulate_batched_pipeline(n_units, S, 8, seed * 31 + n_units, lanes)
