"""A lane-level model of the column recursion kernel (csrc/delta_column.cu), run on the CPU.

The model follows the kernel warp step by warp step: the task list (degree l, block b of 32
columns, longest first), the first row from the lanes' factor products and the warp's suffix
scan with split-off exponents, the chunk coefficients a(m'), b(m') made from the sqrt tables,
the update in the kernel's rounding order (the coefficient 2m a(m') rounded once: the kernel's
integer-pipe product is the exactly rounded one), the direct row writes and the transposed
entries staged in a 32 x 33 block and flushed a chunk at a time, and the per-lane exponent of the
scaled variant (band-limits above 1024).  The tile output's rescaled relation (Delta = p y,
y_{m'-1} = m alpha y_{m'} - y_{m'+1}, with the plan-time tables made as rescale_tables_kernel
makes them) runs through the same model.  Every table write is checked against
the table's bounds and must land on an entry not written before; at the end every entry must
have been written once, and the table must equal the oracle's (the Risbo recursion) to the
tolerance the GPU tests use.  A change to the kernel's index arithmetic that breaks coverage or
bounds shows up here before any GPU run."""
import math

import numpy as np
import pytest

from oracle import transforms as T


def offset(l):
    return l * (l + 1) * (2 * l + 1) // 6


def tasks(L):
    t = [(l, b) for l in range(L) for b in range(l // 32 + 1)]
    t.sort(key=lambda x: -(x[0] - 32 * x[1]))  # Python's sort is stable, as std::stable_sort
    return t


def exp_of(v):
    return math.frexp(v)[1] - 1  # unbiased exponent of a normal double


def with_exp(v, e):
    return math.ldexp(math.frexp(v)[0] * 2.0, e)


def rescale_tables(L, sq, rsq):
    """alpha(l, m') and p(l, m') of the rescaled relation, per degree, in the order and rounding of
    rescale_tables_kernel: p(l, l) = p(l, l-1) = 1, p(l, m'-1) = b(m') p(l, m'+1),
    alpha(l, m') = 2 a(m') p(l, m') / p(l, m'-1)."""
    al, p = [], []
    for l in range(L):
        a_l, p_l = np.zeros(l + 1), np.zeros(l + 1)
        p_up = p_cur = 1.0
        for mp in range(l, -1, -1):
            p_dn = x = 0.0
            if mp >= 1:
                a = rsq[l - mp + 1] * rsq[l + mp]
                b = (sq[l - mp] * sq[l + mp + 1]) * a
                p_dn = 1.0 if mp == l else b * p_up
                x = (2.0 * a * p_cur) / p_dn
            a_l[mp], p_l[mp] = x, p_cur
            p_up, p_cur = p_cur, p_dn
        al.append(a_l)
        p.append(p_l)
    return al, p


def run_task(l, b, sq, rsq, table, written, scaled, resc=None):
    m0 = 32 * b
    lanes = np.arange(32)
    m = m0 + lanes
    act = m <= l
    # first row: lanes' products of every 32nd factor g(k), k >= m0 + 33
    gm = np.ones(32)
    for j in range(32):
        k = m0 + 33 + j
        while k <= l:
            gm[j] = gm[j] * (sq[l + k] * rsq[l - k + 1])
            k += 32
    ge = np.array([exp_of(x) for x in gm])
    gm = np.array([with_exp(x, 0) for x in gm])
    for d in (16, 8, 4, 2, 1):
        om, oe = gm[lanes ^ d], ge[lanes ^ d]
        gm = gm * om
        ge = ge + oe + np.array([exp_of(x) for x in gm])
        gm = np.array([with_exp(x, 0) for x in gm])
    h = np.where(m + 1 <= l, sq[np.minimum(l + m + 1, len(sq) - 1)] * rsq[np.maximum(l - m, 1)], 1.0)
    for d in (1, 2, 4, 8, 16):
        o = np.concatenate([h[d:], np.zeros(d)])
        h = np.where(lanes + d < 32, h * o, h)
    v = h * gm
    E = np.zeros(32, dtype=np.int64)
    cur = np.zeros(32)
    for i in range(32):
        if not act[i]:
            continue
        sgn = -1.0 if (l - m[i]) & 1 else 1.0
        if not scaled or exp_of(v[i]) + ge[i] - l >= -1021:
            cur[i] = sgn * math.ldexp(v[i], int(ge[i]) - l)
        else:
            cur[i] = sgn * v[i]
            E[i] = ge[i] - l
    prev = np.zeros(32)
    m2 = 2.0 * m
    base, row = offset(l), l + 1
    stage = np.full((32, 33), np.nan)
    coef = np.zeros(64)

    def put(idx, val):
        assert offset(l) <= idx < offset(l + 1), (l, idx)
        assert not written[idx], ("written twice", l, idx)
        written[idx] = True
        table[idx] = val

    pl = None if resc is None else resc[1][l]
    for mp in range(l, m0 - 1, -1):
        j = mp & 31
        if mp == l or j == 31:
            k = (mp & ~31) + lanes
            if resc is not None:  # alpha(l, m') and p(l, m') of the chunk from the tables
                ok = k <= l
                kk = np.minimum(k, l)
                coef[:32] = np.where(ok, resc[0][l][kk], 0.0)
                coef[32:] = np.where(ok, pl[kk], 0.0)
            else:
                ok = (k >= 1) & (k <= l)
                kk = np.clip(k, 1, l if l >= 1 else 1)
                a = np.where(ok, rsq[np.maximum(l - kk + 1, 1)] * rsq[l + kk], 0.0)
                bb = np.where(ok, (sq[np.maximum(l - kk, 0)] * sq[l + kk + 1]) * a, 0.0)
                coef[:32], coef[32:] = a, bb
        out = np.where(E != 0, 0.0, cur) if scaled else cur.copy()
        for i in range(32):
            if act[i]:
                put(base + mp * row + m[i], out[i] if resc is None else pl[mp] * out[i])
        if mp >= m0 + 32:
            for i in range(32):
                stage[i, j] = -out[i] if (mp - m[i]) & 1 else out[i]
            if j == 0:
                for r in range(32):
                    if m0 + r > l:
                        break
                    for c in range(32):
                        col = mp + c
                        if col <= l:
                            assert not math.isnan(stage[r, c]), "flush reads an unstaged slot"
                            put(base + (m0 + r) * row + col, stage[r, c] if resc is None else pl[col] * stage[r, c])
                stage[:] = np.nan
        if mp > m0:
            if resc is not None:
                nxt = (m * coef[j]) * cur - prev  # the kernel fuses this into one FMA; the model rounds twice
            else:
                c = m2 * coef[j]
                t2 = coef[32 + j] * prev
                nxt = c * cur - t2  # the kernel fuses this into one FMA; the model rounds twice
            prev, cur = cur, nxt
            if scaled:
                for i in range(32):
                    if E[i] == 0:
                        continue
                    x = exp_of(cur[i]) if cur[i] != 0 else -1100
                    if x + E[i] >= -1021:
                        cur[i] = math.ldexp(cur[i], int(E[i]))
                        prev[i] = math.ldexp(prev[i], int(E[i]))
                        E[i] = 0
                    elif x > 512:
                        cur[i] *= 2.0 ** -512
                        prev[i] *= 2.0 ** -512
                        E[i] += 512


def model_table(L, scaled=None, degrees=None, rescaled=False):
    scaled = L > 1024 if scaled is None else scaled
    nsq = 2 * L + 4
    sq = np.sqrt(np.arange(nsq, dtype=np.float64))
    rsq = np.zeros(nsq)
    rsq[1:] = 1.0 / np.sqrt(np.arange(1, nsq, dtype=np.float64))
    resc = rescale_tables(L, sq, rsq) if rescaled else None
    n = offset(L)
    table = np.zeros(n)
    written = np.zeros(n, dtype=bool)
    for l, b in tasks(L):
        if degrees is None or l in degrees:
            run_task(l, b, sq, rsq, table, written, scaled, resc)
    return table, written


@pytest.mark.parametrize("L", [1, 2, 3, 31, 32, 33, 65, 97])
def test_column_model_covers_table_once_and_matches_oracle(L):
    table, written = model_table(L)
    assert written.all()
    want = T.delta_quadrant(L)
    assert np.abs(table - want).max() < 1e-13


def test_column_model_scaled_variant_matches_oracle_at_small_L():
    """The per-lane exponent path (used above L = 1024) gives the same table where nothing is out of range."""
    L = 70
    table, written = model_table(L, scaled=True)
    assert written.all()
    assert np.abs(table - T.delta_quadrant(L)).max() < 1e-13


@pytest.mark.parametrize("L,scaled", [(33, False), (97, False), (70, True)])
def test_rescaled_relation_matches_oracle(L, scaled):
    """The tile output's relation: Delta = p y with y from the rescaled three-term relation and the
    plan-time alpha, p gives the oracle's table (the Risbo recursion) to the FP64 tolerance."""
    table, written = model_table(L, scaled=scaled, rescaled=True)
    assert written.all()
    assert np.abs(table - T.delta_quadrant(L)).max() < 1e-13


def test_rescale_factors_stay_in_range():
    """p(l, m') in [0.15, 1] up to l = 2047, so p y and the FP32 output keep Delta's range."""
    L = 2048
    nsq = 2 * L + 4
    sq = np.sqrt(np.arange(nsq, dtype=np.float64))
    rsq = np.zeros(nsq)
    rsq[1:] = 1.0 / sq[1:]
    lo, hi = 1.0, 0.0
    for l in (1, 2, 3, 100, 1023, 1024, 2047):
        p_up = p_cur = 1.0
        for mp in range(l, 0, -1):
            a = rsq[l - mp + 1] * rsq[l + mp]
            b = (sq[l - mp] * sq[l + mp + 1]) * a
            p_dn = 1.0 if mp == l else b * p_up
            lo, hi = min(lo, p_dn), max(hi, p_dn)
            p_up, p_cur = p_cur, p_dn
    assert 0.15 < lo and hi <= 1.0


def test_task_list_is_longest_first_and_complete():
    L = 300
    t = tasks(L)
    lengths = [l - 32 * b + 1 for l, b in t]
    assert lengths == sorted(lengths, reverse=True)
    assert len(t) == sum(l // 32 + 1 for l in range(L))
    assert len(set(t)) == len(t)


@pytest.mark.slow
def test_column_model_scaled_high_degree_matches_oracle():
    """Degree 1500 of a band-limit above 1024: first-row entries below 2^-1022 start with an exponent."""
    l = 1500
    L = l + 1
    table, written = model_table(L, degrees={l})
    got = table[offset(l):offset(l + 1)].reshape(l + 1, l + 1)
    assert written[offset(l):offset(l + 1)].all()
    full = T.wigner_full(2 * l)
    assert np.abs(got - full[l:, l:]).max() < 5e-13


# ---- the tile output of 3xTF32 plans ---------------------------------------------------------

def a_layout(L):
    """The forward A-tile layout of the tensor-core plans (contract_tc.cu tc_setup): per m the
    index of tile (m, m // 128, 0), and the forward items (m, i, c1, first tile)."""
    nC, nI = (L + 31) // 32, (L + 127) // 128
    abase, items, ft = [], [], 0
    for m in range(L):
        abase.append(ft)
        for i in range(m // 128, nI):
            items.append((m, i, min(nC, 4 * i + 4), ft))
            ft += 4 * i + 4
    return abase, items, ft


def tile_index(abase, M, il, c):
    im = M // 128
    assert il >= im and 0 <= c < 4 * il + 4
    return abase[M] + 2 * il * (il + 1) - 2 * im * (im + 1) + c


def test_tile_index_matches_the_plan_layout():
    for L in (1, 64, 129, 300, 1024):
        abase, items, total = a_layout(L)
        # the column recursion's per-M base (tile_base_kernel): ab2[M] = abase[M] - 2 i (i + 1)
        ab2 = [abase[M] - 2 * (M >> 7) * ((M >> 7) + 1) for M in range(L)]
        seen = set()
        for m, i, c1, first in items:
            assert tile_index(abase, m, i, 0) == first
            for c in range(4 * i + 4):
                t = tile_index(abase, m, i, c)
                assert t == ab2[m] + 2 * i * (i + 1) + c
                assert 0 <= t < total and t not in seen
                seen.add(t)
        assert len(seen) == total


def model_tiles(L, s):
    """Every A entry the tile-mode kernel writes: (tile, row, k) -> value, following its two
    write paths (the row of 32 K values across the warp, and the flushed transposition block)."""
    tab = T.delta_quadrant(L)
    off = T.delta_offsets(L)
    abase, _, _ = a_layout(L)
    U = {}
    for l in range(L):
        D = tab[off[l]:off[l + 1]].reshape(l + 1, l + 1)
        for mp in range(l + 1):
            d = 0.0 if l < abs(s) else D[mp, abs(s)] * (-1.0 if (s > 0 and (l + mp) & 1) else 1.0)
            U[l, mp] = np.float32(np.sqrt((2 * l + 1) / (4 * np.pi)) * d)
    out = {}

    def put(key, val):
        assert key not in out, ("written twice", key)
        out[key] = val

    for l, b in tasks(L):
        D = tab[off[l]:off[l + 1]].reshape(l + 1, l + 1)
        m0, il, row = 32 * b, l // 128, l % 128
        for mp in range(l, m0 - 1, -1):
            for lane in range(32):
                m = m0 + lane
                if m > l:
                    continue
                x = D[mp, m]  # Delta_{m' m}, lane m at step m'
                sgn = -1.0 if (mp - m) & 1 else 1.0
                put((tile_index(abase, mp, il, m0 // 32), row, lane), U[l, m] * np.float32(sgn * x))
            if mp >= m0 + 32 and (mp & 31) == 0:
                for r in range(32):
                    M = m0 + r
                    if M > l:
                        break
                    for lane in range(32):
                        c = mp + lane
                        if c <= l:
                            put((tile_index(abase, M, il, mp // 32), row, lane), U[l, c] * np.float32(D[c, M]))
    return out, U


@pytest.mark.parametrize("L,s", [(40, 2), (97, -1), (150, 0)])
def test_tile_mode_writes_every_entry_of_A_once(L, s):
    """A_m[l][m'] = U_l[m'] Delta^l_{m'm} for every 0 <= m, m' <= l < L lands exactly once at
    row l mod 128, K = m' mod 32 of tile (m, l // 128, m' // 32); nothing else is written."""
    out, U = model_tiles(L, s)
    tab = T.delta_quadrant(L)
    off = T.delta_offsets(L)
    abase, _, _ = a_layout(L)
    want = {}
    for l in range(L):
        D = tab[off[l]:off[l + 1]].reshape(l + 1, l + 1)
        for m in range(l + 1):
            for mp in range(l + 1):
                key = (tile_index(abase, m, l // 128, mp // 32), l % 128, mp % 32)
                want[key] = U[l, mp] * np.float32(D[mp, m])
    assert set(out) == set(want)
    # the oracle's full-matrix table is symmetric only to rounding: compare to FP32 rounding
    keys = sorted(want)
    a = np.array([out[k] for k in keys], dtype=np.float64)
    b = np.array([want[k] for k in keys], dtype=np.float64)
    assert np.abs(a - b).max() <= 2e-7 * np.abs(b).max()


def inv_layout(L, s):
    """The inverse A-tile layout (contract_tc.cu tc_setup): item (m, i) holds chunks kc in
    [c0, nC), c0 = max(max(m, |s|) // 32, 4i); the tile of chunk kc is ibase[m, i] + kc."""
    nC, nI, at = (L + 31) // 32, (L + 127) // 128, 0
    ibase = {}
    for m in range(L):
        lmin = max(m, abs(s))
        for i in range(nI):
            c0 = max(lmin // 32, 4 * i)
            if c0 < nC:
                ibase[m, i] = at - c0
                at += nC - c0
    return ibase, at


def lane_tasks(L, s):
    nC = (L + 31) // 32
    t = [(m, kc) for m in range(L) for kc in range(max(m, abs(s)) // 32, nC)]
    t.sort(key=lambda x: -(min(32 * x[1] + 31, L - 1) - x[0]))
    return t


@pytest.mark.parametrize("L,s", [(40, 2), (97, -1), (150, 0), (140, 35)])
def test_degree_lane_mode_writes_every_entry_of_the_inverse_A_once(L, s):
    """The recursion with one lane per degree (the inverse's tiles), followed step by step with the
    kernel's index arithmetic -- the triangle index and the tile-base pointer moved by additions,
    the tile of row m' of column m reloaded at each 128-row boundary -- and its rescaled relation
    (Delta = p y): A_m[m'][l] = U_l[m'] Delta^l_{m'm} for every 0 <= m, m' <= l < L with l >= |s|
    lands once at row m' mod 128, K = l mod 32 of the tile of chunk l // 32 of item (m, m' // 128),
    each such tile exists, and the values match the oracle's table rounded to FP32."""
    tab = T.delta_quadrant(L)
    off = T.delta_offsets(L)
    ibase, total = inv_layout(L, s)
    nI = (L + 127) // 128
    ib = [-10 ** 9] * (L * nI)  # the plan's ibase array; entries of items that do not exist are never used
    for (mm, i), v in ibase.items():
        ib[mm * nI + i] = v
    nsq = 2 * L + 4
    sq = np.sqrt(np.arange(nsq, dtype=np.float64))
    rsq = np.zeros(nsq)
    rsq[1:] = 1.0 / sq[1:]
    alpha, pp = rescale_tables(L, sq, rsq)
    Ds = [tab[off[l]:off[l + 1]].reshape(l + 1, l + 1) for l in range(L)]
    U = {}
    for l in range(L):
        for mp in range(l + 1):
            d = 0.0 if l < abs(s) else Ds[l][mp, abs(s)] * (-1.0 if (s > 0 and (l + mp) & 1) else 1.0)
            U[l, mp] = np.float32(np.sqrt((2 * l + 1) / (4 * np.pi)) * d)

    def tri(r, l):
        return r * L - r * (r - 1) // 2 + (l - r)

    f32 = np.float32
    out = {}
    for m, kc in lane_tasks(L, s):
        top = min(32 * kc + 31, L - 1)
        ls = [32 * kc + lane for lane in range(32)]
        inl = [l < L and l >= m for l in ls]
        wr = [inl[i] and ls[i] >= abs(s) for i in range(32)]
        kidx = [top * L - top * (top - 1) // 2 + (l - top) for l in ls]
        ibr = top * nI + (m >> 7)
        ct, tb = ib[ibr], None
        cur, prev = [0.0] * 32, [0.0] * 32
        for mp in range(top, m - 1, -1):
            nt = None
            if mp > m:
                ibr -= nI
                nt = ib[ibr]
                for i in range(32):
                    kidx[i] -= L - mp
                    if inl[i] and mp - 1 <= ls[i]:
                        assert kidx[i] == tri(mp - 1, ls[i])
            if mp == top or (mp & 127) == 127:
                tb = ib[m * nI + (mp >> 7)] + kc
            for i in range(32):
                l = ls[i]
                if mp == l and inl[i]:
                    cur[i], prev[i] = Ds[l][l, m], 0.0  # y_l = Delta_{l m}
                if not (inl[i] and mp <= l):
                    continue
                if wr[i]:
                    x = f32(cur[i])
                    pf = f32(pp[l][mp])
                    key = (tb, mp % 128, i)
                    assert tb == ibase[m, mp // 128] + kc and 0 <= tb < total and key not in out
                    out[key] = (U[l, mp] * pf) * x
                    if mp > m:
                        key = (ct + kc, m % 128, i)
                        assert ct + kc == ibase[mp, m // 128] + kc and 0 <= key[0] < total and key not in out
                        out[key] = (U[l, m] * pf) * (-x if (mp - m) & 1 else x)
                if mp > m:
                    cur[i], prev[i] = (m * alpha[l][mp]) * cur[i] - prev[i], cur[i]
            ct = nt
    want = {}
    for l in range(abs(s), L):
        for m in range(l + 1):
            for mp in range(l + 1):
                want[(ibase[m, mp // 128] + l // 32, mp % 128, l % 32)] = U[l, mp] * np.float32(Ds[l][mp, m])
    assert set(out) == set(want)
    keys = sorted(want)
    a = np.array([out[k] for k in keys], dtype=np.float64)
    b = np.array([want[k] for k in keys], dtype=np.float64)
    assert np.abs(a - b).max() <= 3e-7 * np.abs(b).max()
