"""An index-level model of the recursion kernel's schedule (csrc/delta.cu), run on the CPU.

The model follows the kernel step by step: the host-made min-max partition of each degree's rows
over the CTAs (optimal_cuts, with the owners of the rows a step reads), the per-CTA flags, the
chunking of a CTA's rows to fit its shared memory, the padded row layouts, the warp split of
32-column segments, the half and integer steps with the divided half rows and the neighbour
partial sums passed between lanes (including the carry across a warp's segments), the pads, the
slab double buffer and the table writes by warps 1-15.  Every shared-memory access is checked
against the chunk's allocation (and must read a written slot), every slab read against the degree
it must hold, under random and adversarial interleavings of the CTAs; the resulting table is
compared with the oracle's.  A change to the kernel's index arithmetic or its waits that breaks
one of these shows up here, on the CPU, before any GPU run."""
import bisect
import math
import random

import numpy as np
import pytest

from oracle import transforms as T

def po(m): return m * (m + 5) // 2
def tri(m): return m * (m + 1) // 2
def segF(n):
    q, r = n >> 5, n & 31
    return 16 * q * (q + 1) + r * (q + 1)
def segF_inv(t):
    q = int((math.sqrt(1.0 + 0.25 * t) - 1.0) * 0.5)
    q = max(q, 0)
    while q > 0 and 16 * q * (q + 1) > t: q -= 1
    while 16 * (q + 1) * (q + 2) <= t: q += 1
    r = (t - 16 * q * (q + 1)) // (q + 1)
    n = 32 * q + min(r, 31)
    assert segF(n) <= t and segF(n + 1) > t
    return n
def row_cost(m): return segF(m + 2) - 2 + segF(m + 1) - 1
def cut_row(rows, o, nb):
    x = row_cost(rows) * o // nb
    a, b = 0, rows
    while a < b:
        mid = (a + b) >> 1
        if row_cost(mid) >= x: b = mid
        else: a = mid + 1
    return a
# device-made partition (no host table: the no-allocation entry point)
def cta_rows_device(lp, c, nb): return cut_row(lp + 1, c, nb), cut_row(lp + 1, c + 1, nb)
def owner_device(l, row, nb):
    S = row_cost(l + 1)
    return min(((row_cost(row) + 1) * nb + S - 1) // S - 1, nb - 1)

def optimal_cuts(l, nb):
    rows = l + 2
    seg = lambda n: (n + 31) // 32
    pre = [0]
    for m in range(rows): pre.append(pre[-1] + (seg(m + 3) if m <= l else 0) + seg(m + 2) + 1)
    share = lambda a, b: pre[b] - pre[a] + (seg(a + 2) if a > 0 else 0)
    def pack(T):
        out = []; a = 0; c = 0
        while a < rows:
            if c == nb: return None
            b = a + 1
            if share(a, b) > T: return None
            while b < rows and share(a, b + 1) <= T: b += 1
            out.append(a); a = b; c += 1
        out += [rows] * (nb + 1 - len(out))
        return out
    lo, hi = 1, share(0, rows)
    while lo < hi:
        mid = (lo + hi) // 2
        if pack(mid) is not None: hi = mid
        else: lo = mid + 1
    return pack(lo)
CUTS = {}
def cuts_of(l, nb):
    if (l, nb) not in CUTS: CUTS[(l, nb)] = optimal_cuts(l, nb)
    return CUTS[(l, nb)]
# host-made partition (a plan's table)
def cta_rows_host(lp, c, nb):
    cu = cuts_of(lp - 1, nb); return cu[c], cu[c + 1]
def owner_host(l, row, nb):
    if l == 0: return 0
    cu = cuts_of(l - 1, nb)
    c = bisect.bisect_right(cu, row) - 1
    return max(0, min(c, nb - 1))

def slab_doubles(L): return (L + 2) * (L + 7) // 2 + 2
def chunk_need(l, c0, c1):
    Alo = c0 - 1 if c0 > 0 else 0
    Ahi = min(c1 - 1, l)
    return (po(Ahi + 2) - po(Alo)) + 2 + (po(c1) - po(Alo)) + (tri(c1) - tri(c0)) + 2 * (Ahi - Alo + 1) + 2 * (c1 - c0)
def warp_segments(lo, hi, add, warp, nw):
    base = segF(lo + add - 1); S = segF(hi + add) - base
    s0 = S * warp // nw; s1 = S * (warp + 1) // nw
    x = segF_inv(base + s0) - add + 1
    x = max(lo, min(x, hi))
    seg = s0 - (segF(x + add - 1) - base)
    if s1 > s0:
        assert 0 <= seg and seg * 32 <= x + add - 1, (lo, hi, add, warp, x, seg)
    return x, seg, s1 - s0

class Smem:
    def __init__(self, n): self.v = np.full(n, np.nan); self.w = np.zeros(n, bool)
    def rd(self, i):
        assert 0 <= i < len(self.v), ('smem read oob', i, len(self.v)); assert self.w[i], ('smem unwritten', i)
        return self.v[i]
    def wr(self, i, x):
        assert 0 <= i < len(self.v), ('smem write oob', i, len(self.v)); self.v[i] = x; self.w[i] = True

def run(L, nb, cap, seed, strategy, nwarps=16, partition="host"):
    cta_rows, owner_of = (cta_rows_host, owner_host) if partition == "host" else (cta_rows_device, owner_device)
    rng = random.Random(seed)
    sq = np.sqrt(np.arange(2 * L + 4, dtype=float))
    p = 1 / math.sqrt(2)
    SD = slab_doubles(L)
    slabs = [np.zeros(SD), np.zeros(SD)]; tags = [np.full(SD, -9), np.full(SD, -9)]
    slabs[0][:3] = [0, 1, 0]; tags[0][:3] = 0
    off = lambda l: l * (l + 1) * (2 * l + 1) // 6
    table = np.full(off(L), np.nan); table[0] = 1.0
    done = [0] * nb; prog = [0] * nb
    for m in range(L): assert chunk_need(max(L - 2, 0), m, m + 1) <= cap
    def proc(c):
        for l in range(L - 1):
            lp = l + 1
            r0, r1 = cta_rows(lp, c, nb)
            if r0 >= r1:
                done[c] = lp; yield ('x',); continue
            a, b = max(r0 - 2, 0), min(r1 + 1, l)
            o0, o1 = owner_of(l, a, nb), owner_of(l, b, nb)
            yield ('wait', o0, o1, l)
            Yg, Tg = slabs[l & 1], tags[l & 1]; Yn, Tn = slabs[lp & 1], tags[lp & 1]
            sc = p / (2 * l + 1); sc2 = p / (2 * lp)
            c0 = r0
            while c0 < r1:
                c1 = r1
                if chunk_need(l, c0, r1) > cap:
                    lo, hi = c0 + 1, r1
                    while lo < hi:
                        mid = (lo + hi + 1) >> 1
                        if chunk_need(l, c0, mid) <= cap: lo = mid
                        else: hi = mid - 1
                    c1 = lo
                Alo = c0 - 1 if c0 > 0 else 0; Ahi = min(c1 - 1, l); Ytop = min(Ahi + 1, l)
                ybase = po(Alo); ycount = po(Ytop + 1) - ybase; z0 = tri(c0)
                sm = Smem(cap)
                Xs = po(Ahi + 2) - ybase; Zs = Xs + 2 + po(c1) - ybase; Rh = Zs + tri(c1) - z0; Ri = Rh + 2 * (Ahi - Alo + 1)
                assert Ri + 2 * (c1 - c0) == chunk_need(l, c0, c1)
                for i in range(ycount):
                    assert Tg[ybase + i] == l, ('stale', c, l, ybase + i, Tg[ybase + i])
                    sm.wr(i, Yg[ybase + i])
                yield ('staged',)
                if Ytop < Ahi + 1:
                    for i in range(l + 4): sm.wr(po(l + 1) - ybase + i, 0.0)
                if c1 - 1 > l:
                    for i in range(l + 4): sm.wr(Xs + 2 + po(l + 1) - ybase + i, 0.0)
                # half row A is stored divided by ra(A) = sq[l+A+1] sc (row -1 by ra(0)); factors:
                # kappa_A = rb/ra, rat_A = ra(A)/ra(A-1); integer row m: alpha_m = ia(m) ra(m-1), kappa_m
                for A in range(Alo, Ahi + 1):
                    sm.wr(Rh + 2 * (A - Alo), sq[l - A] / sq[l + A + 1])
                    sm.wr(Rh + 2 * (A - Alo) + 1, sq[l + A + 1] / sq[l + A] if A > 0 else 1.0)
                for m in range(c0, c1):
                    rho_prev = (sq[l + m] if m > 0 else sq[l + 1]) * sc
                    sm.wr(Ri + 2 * (m - c0), sq[lp + m] * sc2 * rho_prev)
                    sm.wr(Ri + 2 * (m - c0) + 1, (sq[lp - m] * sq[l + m + 1]) / (sq[lp + m] * sq[l + m]) if m > 0 else 1.0)
                cnt = {}
                for warp in range(nwarps):
                    A, seg, count = warp_segments(Alo, Ahi, 3, warp, nwarps)
                    yo = po(A) - ybase
                    carry = 0.0
                    if count > 0 and seg > 0:
                        kap = sm.rd(Rh + 2 * (A - Alo)); idx = seg * 32 - 1
                        carry = kap * sm.rd(yo + A + 3 + idx) + sm.rd(yo + idx)
                    for k in range(count):
                        kap, rat = sm.rd(Rh + 2 * (A - Alo)), sm.rd(Rh + 2 * (A - Alo) + 1)
                        P = [0.0] * 32; Q = [0.0] * 32
                        for lane in range(32):
                            idx = seg * 32 + lane
                            if idx <= A + 2:
                                y0 = sm.rd(yo + idx); y1 = sm.rd(yo + A + 3 + idx)
                                P[lane] = kap * y1 + y0; Q[lane] = kap * y1 - y0
                        Pm = [carry] + P[:31]; carry = P[31]
                        for lane in range(32):
                            idx = seg * 32 + lane
                            if 1 <= idx <= A + 2:
                                B = idx - 1
                                cnt[(A, B)] = cnt.get((A, B), 0) + 1
                                sb, smb = sq[l + B], sq[l + 1 - B]
                                v = smb * Q[lane] + sb * Pm[lane]
                                xr = Xs + 2 + yo
                                sm.wr(xr + B, v)
                                if B == A:
                                    if A > Alo: sm.wr(xr - 1, -v * rat)
                                    elif A == 0: sm.wr(Xs + 1, -v)
                                if A == 0 and B == 1: sm.wr(Xs, v)
                        seg += 1
                        if seg * 32 > A + 2:
                            yo += A + 3; A += 1; seg = 0
                assert all(v == 1 for v in cnt.values()) and len(cnt) == sum(A + 2 for A in range(Alo, Ahi + 1))
                if c1 - 1 > l: sm.wr(Xs + 2 + po(l) - ybase + l + 2, 0.0)
                cnt = {}
                for warp in range(nwarps):
                    m, seg, count = warp_segments(c0, c1 - 1, 2, warp, nwarps)
                    xo = 2 + po(m) - ybase; zo = tri(m) - z0; yr = po(m)
                    carry = 0.0
                    if count > 0 and seg > 0:
                        kap = sm.rd(Ri + 2 * (m - c0) + 1); idx = seg * 32 - 1
                        carry = kap * sm.rd(Xs + xo + idx) + sm.rd(Xs + (xo - (m + 2) if m > 0 else 0) + idx)
                    for k in range(count):
                        alpha, kap = sm.rd(Ri + 2 * (m - c0)), sm.rd(Ri + 2 * (m - c0) + 1)
                        P = [0.0] * 32; Q = [0.0] * 32
                        for lane in range(32):
                            cc = seg * 32 + lane
                            if cc <= m + 1:
                                x0 = sm.rd(Xs + (xo - (m + 2) if m > 0 else 0) + cc); x1 = sm.rd(Xs + xo + cc)
                                P[lane] = kap * x1 + x0; Q[lane] = kap * x1 - x0
                        Pm = [carry] + P[:31]; carry = P[31]
                        for lane in range(32):
                            cc = seg * 32 + lane
                            if 1 <= cc <= m + 1:
                                n = cc - 1
                                cnt[(m, n)] = cnt.get((m, n), 0) + 1
                                sb, smb = sq[lp + n], sq[lp - n]
                                v = alpha * (smb * Q[lane] + sb * Pm[lane])
                                def W(i, x):
                                    assert 0 <= i < SD; Yn[i] = x; Tn[i] = lp
                                W(yr + n + 1, v)
                                if n == 1: W(yr, -v if (lp + m) & 1 else v)
                                if n + 1 == m:
                                    W(yr - 1, -v)
                                    if m == 1: W(yr - 3, v if lp & 1 else -v)
                                if n == m and m == lp: W(yr + m + 2, 0.0)
                                sm.wr(Zs + zo + n, v)
                        seg += 1
                        if seg * 32 > m + 1:
                            xo += m + 3; zo += m + 1; yr += m + 3; m += 1; seg = 0
                assert all(v == 1 for v in cnt.values()) and len(cnt) == sum(m + 1 for m in range(c0, c1))
                yield ('computed',)
                if c1 == r1: done[c] = lp
                Tb = off(lp)
                for warp in range(1, nwarps):
                    m, seg, count = warp_segments(c0, c1 - 1, 1, warp - 1, nwarps - 1)
                    zo = tri(m) - z0; trow = Tb + m * (lp + 1)
                    for k in range(count):
                        for lane in range(32):
                            n = seg * 32 + lane
                            if n <= m: table[trow + n] = sm.rd(Zs + zo + n)
                        seg += 1
                        if seg * 32 > m: zo += m + 1; trow += lp + 1; m += 1; seg = 0
                width = c1 - c0; items = (c1 - 1) * width
                inv_w = np.float32(1.0) / np.float32(width)
                for i in range(items):
                    n = int(np.float32(np.float32(i) + np.float32(0.5)) * inv_w)
                    j = i - n * width
                    if j < 0: n -= 1; j += width
                    elif j >= width: n += 1; j -= width
                    assert 0 <= j < width and n == i // width
                    m = c0 + j
                    if m > n:
                        vv = sm.rd(Zs + tri(m) - z0 + n)
                        table[Tb + n * (lp + 1) + m] = -vv if (m - n) & 1 else vv
                yield ('tabled',)
                c0 = c1
    procs = {c: proc(c) for c in range(nb)}
    pend = {c: next(procs[c], None) for c in range(nb)}
    while any(v is not None for v in pend.values()):
        ready = [c for c, ev in pend.items() if ev is not None and (ev[0] != 'wait' or all(done[o] >= ev[3] for o in range(ev[1], ev[2] + 1)))]
        assert ready, 'deadlock'
        if strategy == 'random': c = rng.choice(ready)
        elif strategy == 'fast': c = max(ready, key=lambda q: (prog[q], rng.random()))
        else: c = min(ready, key=lambda q: (prog[q], rng.random()))
        prog[c] += 1
        pend[c] = next(procs[c], None)
    ref = T.delta_quadrant(L)
    assert not np.isnan(table).any()
    return np.abs(table - ref).max()



@pytest.mark.parametrize("strategy", ["random", "fast", "slow"])
@pytest.mark.parametrize("L,nb,tight", [(1, 2, False), (2, 3, False), (5, 2, True), (12, 5, False), (30, 7, True),
                                         (40, 9, True), (45, 16, False), (64, 152, False)])
def test_schedule_model_matches_oracle(L, nb, tight, strategy):
    """tight: the shared memory holds only the widest single-row chunk, so shares split into
    chunks; otherwise every share fits one chunk."""
    need = max(chunk_need(max(L - 2, 0), m, m + 1) for m in range(L))
    err = run(L, nb, need if tight else 10 ** 6, L + nb, strategy)
    assert err < 1e-13


@pytest.mark.parametrize("L,nb", [(3, 2), (20, 6), (33, 40)])
def test_schedule_model_with_device_partition(L, nb):
    """The partition the kernel makes itself when it has no host table."""
    for strategy in ("random", "fast", "slow"):
        assert run(L, nb, 10 ** 6, L, strategy, partition="device") < 1e-13


def test_segment_inverse():
    for t in range(0, 20000, 7):
        segF_inv(t)
