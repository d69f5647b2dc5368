"""Index models of two tiled kernels (test helper, no GPU).

Each function restates, in Python, the index arithmetic of one CUDA kernel
of the library -- which element goes where, per thread and per loop -- so
that a CPU test can check it before a GPU runs it: every access inside its
buffer, every output written exactly once, and the result equal to the
stage's plain definition.  The arithmetic itself (sums, products) is done in
double precision; only the indexing follows the kernels.

row_split_stage: `dfb_b_tile` (csrc/dfb_tile.cuh), one row-split stage s >= 3
  of the directional filter bank (§2.1) on an R2 x C pair of coset arrays,
  cut into tiles of 16 rows: the straightened shared-memory frame (tile row r
  holds array column c0 + x - r - i q), the two ladder passes over quads of
  targets, both staging paths (row-major arrays and transposed ones) and
  both store paths.
rle_tile: `k_rle_count_b` / `k_rle_write_b` (csrc/k_codec.cu), the tokens of
  one tile of whole rows (§3.8) from the per-chunk bit masks and block scans.
lp_level_tile: `lp_level_tile` (csrc/lp_tile.cuh), one 64 x 64 tile of a
  single-precision Laplacian-pyramid level (§2.1, Fig. 1), analysis or
  synthesis, centred on the tile's rounded mean: the staged window, the four
  passes with a run of outputs per thread read from one window, the lowpass
  share stored from the column pass.
"""
import numpy as np

from plan_emulator import _fan_taps

ROWS = 16


def _cmod(a, n):
    """C's truncating remainder"""
    r = abs(a) % n
    return -r if a < 0 else r


def _wrap_fast(v, C, CB):
    assert 0 <= v < C + CB, (v, C, CB)
    return v if v < C else (v - C if C >= CB else _cmod(v, C))


def geometry(NT):
    """BGeo<NT>: reach, staged columns, row stride, outputs per row, staged rows, margin, floats, offset"""
    R = NT - 1
    CB, CBS = 128, 132
    COLS = (CB - 2 * R) & ~3
    RB = ROWS + 2 * R
    MARGIN = 8
    return dict(R=R, CB=CB, CBS=CBS, COLS=COLS, RB=RB, MARGIN=MARGIN, SMB=RB * CBS + 2 * MARGIN,
                D=2 if NT == 4 else 0)


def passes(NT, FO):
    """BPass<NT, FO>: row offsets, row ranges, quad origins and counts, window misalignments"""
    g = geometry(NT)
    R, COLS, D = g["R"], g["COLS"], g["D"]
    DB1 = -((NT - 2) // 2) if FO else -(NT // 2)
    DB2 = -(NT // 2) if FO else -((NT - 2) // 2)
    X1 = (R + DB2) & ~3
    X2 = R - (R + D) % 4
    return dict(DB1=DB1, DB2=DB2, R10=R + DB2, R11=R + DB2 + ROWS + R, X1=X1, NQ1=(2 * R + DB2 + COLS - X1 + 3) // 4,
                M1=(D + X1 + DB1) % 4, X2=X2, NQ2=(R + COLS - X2 + 3) // 4, M2=(X2 + DB2) % 4)


def _ladder(T, offT, S, offS, NT, R0, R1, X, NQ, DB, M, alpha, gamma, nwarps, g):
    """ladder_quads: lane k -> quad X + 4k, warp w -> rows [R0 + w KC, ...); updates applied after the pass"""
    taps = [w for _, w in _fan_taps(NT)]
    CBS, SMB = g["CBS"], g["SMB"]
    KC = (R1 - R0 + nwarps - 1) // nwarps
    nch = (M + NT + 6) // 4
    upd = []
    for w in range(nwarps):
        r0 = R0 + w * KC
        if r0 >= R1:
            continue
        for q in range(NQ):
            x = X + 4 * q
            assert (offT + x) % 4 == 0, "target quads on 16-byte boundaries"
            for rho in range(r0 + DB, min(r0 + KC, R1) + DB + NT - 1):
                base = offS + rho * CBS + x + DB - M
                assert base % 4 == 0 and base >= 0 and base + 4 * nch <= SMB, "window chunks inside the buffer"
            for r in range(r0, min(r0 + KC, R1)):
                tb = offT + r * CBS + x
                assert 0 <= tb and tb + 4 <= SMB
                for j in range(4):
                    acc = sum(taps[ia] * taps[b] * S[offS + (r + DB + ia) * CBS + x + j + DB + b]
                              for ia in range(NT) for b in range(NT))
                    upd.append((tb + j, alpha * T[tb + j] + gamma * acc))
    for idx, v in upd:
        T[idx] = v


def row_split_stage(E, O, i, NT, fo, alphas, transposed_in, transposed_out, nwarps):
    """the outputs (E', O') of one stage on coset arrays E, O (R2 x C), slope index i, computed tile by
    tile with the kernel's indexing; every output must be written exactly once (asserted)"""
    g = geometry(NT)
    R, CB, CBS, COLS, RB, MARGIN, SMB, D = (g[k] for k in ("R", "CB", "CBS", "COLS", "RB", "MARGIN", "SMB", "D"))
    P = passes(NT, fo)
    a1, g1, a2, g2 = alphas
    R2, C = E.shape
    offE, offO = MARGIN + (D if fo else 0), MARGIN + (0 if fo else D)
    out = [np.full((R2, C), np.nan), np.full((R2, C), np.nan)]
    count = [np.zeros((R2, C), int), np.zeros((R2, C), int)]
    for t0 in range(0, R2, ROWS):
        for c0 in range(0, C, COLS):
            buf = [np.full(SMB, np.nan), np.full(SMB, np.nan)]
            off = [offE, offO]
            for par, A in enumerate((E, O)):
                if not transposed_in:
                    for r in range(RB):
                        tu = t0 - R + r
                        vs = (c0 - r - i * (2 * tu + par)) % C
                        for x in range(CB):
                            col = vs + x if vs + CB <= C else _wrap_fast(vs + x, C, CB)
                            buf[par][off[par] + r * CBS + x] = A[tu % R2, col]
                else:
                    assert RB <= 32
                    for w in range(nwarps):
                        for lane in range(RB):
                            tu = t0 - R + lane
                            vr = (c0 - lane - i * (2 * tu + par)) % C
                            sh = ((2 * i + 1) * lane) & (CB - 1)
                            for j in range(w, CB, nwarps):
                                x = (j + sh) & (CB - 1)
                                buf[par][off[par] + lane * CBS + x] = A[tu % R2, _wrap_fast(vr + x, C, CB)]
            F, oF, Sx, oS = (buf[1], off[1], buf[0], off[0]) if fo else (buf[0], off[0], buf[1], off[1])
            _ladder(F, oF, Sx, oS, NT, P["R10"], P["R11"], P["X1"], P["NQ1"], P["DB1"], P["M1"], a1, g1, nwarps, g)
            _ladder(Sx, oS, F, oF, NT, R, R + ROWS, P["X2"], P["NQ2"], P["DB2"], P["M2"], a2, g2, nwarps, g)
            ncol = min(COLS, C - c0)
            for par in range(2):
                for rr in range(ROWS):
                    t = t0 + rr
                    if t >= R2:
                        break
                    if not transposed_out:
                        vs = (c0 - rr - i * (2 * t + par)) % C
                        cols = [(xx, vs + xx if vs + ncol <= C else _wrap_fast(vs + xx, C, CB)) for xx in range(ncol)]
                    else:
                        vr = (c0 - rr - i * (2 * t + par)) % C
                        sh = ((2 * i + 1) * rr) % COLS
                        cols = []
                        for j in range(COLS):
                            xx = j + sh - (COLS if j + sh >= COLS else 0)
                            if xx < ncol:
                                cols.append((xx, _wrap_fast(vr + xx, C, COLS)))
                    for xx, col in cols:
                        out[par][t, col] = buf[par][off[par] + (R + rr) * CBS + R + xx]
                        count[par][t, col] += 1
    assert (count[0] == 1).all() and (count[1] == 1).all(), "every output written exactly once"
    return out[0], out[1]


# ------------------------------------------------------------------ RLE tiles
RLE_THREADS, RLE_CHUNK = 256, 2048


def _popc(x):
    return bin(x).count("1")


def _rle_chunk(res, g, e0, e1, w):
    """rle_chunk: the 8 codes g .. g+7 as (values, non-zero, run-start, run-end) bit masks"""
    vals = [int(res[g + j]) for j in range(8)]
    rel = g - e0
    jf = -rel if rel < 0 else 0
    jl = min(8, e1 - g)
    valid = ((1 << jl) - (1 << jf)) if jl > jf else 0
    zero = sum(1 << j for j in range(8) if vals[j] == 0) & valid
    p0 = (rel + jf) % w
    rstart = rend = 0
    if w >= 8:
        js, je = jf + (0 if p0 == 0 else w - p0), jf + w - 1 - p0
        rstart = (1 << js) if js < 8 else 0
        rend = (1 << je) if je < 8 else 0
    else:
        p = p0
        for j in range(jf, 8):
            rstart |= (p == 0) << j
            rend |= (p == w - 1) << j
            p = 0 if p + 1 == w else p + 1
    zprev = int(bool(jf == 0 and rel > 0 and res[g - 1] == 0))
    znext = bool(g + 8 < e1 and res[g + 8] == 0)
    zp = ((zero << 1) | zprev) & 0xFF
    zn = (zero >> 1) | (0x80 if znext else 0)
    return vals, valid & ~zero & 0xFF, zero & (rstart | (~zp & 0xFF)), zero & (rend | (~zn & 0xFF))


def rle_tile(res, e0, n, w):
    """the tokens of the tile [e0, e0 + n) (rows of width w) as the two kernels place them: the count
    kernel's total, then the writer's chunks with their block scans (token offsets and the latest
    zero-run start before each thread); asserts that the positions fill [0, count) exactly once"""
    e1 = e0 + n
    count = 0
    for tid in range(RLE_THREADS):
        g = (e0 & ~7) + 8 * tid
        while g < e1:
            _, nz, rs, _ = _rle_chunk(res, g, e0, e1, w)
            count += _popc(nz) + 2 * _popc(rs)
            g += RLE_CHUNK
    tok, carry, carry_s = {}, 0, -1
    for gb in range(e0 & ~7, e1, RLE_CHUNK):
        ks = [_rle_chunk(res, gb + 8 * t, e0, e1, w) if gb + 8 * t < e1 else ([0] * 8, 0, 0, 0)
              for t in range(RLE_THREADS)]
        cn = [_popc(k[1]) + 2 * _popc(k[2]) for k in ks]
        ls = [(gb + 8 * t - e0) + k[2].bit_length() - 1 if k[2] else -1 for t, k in enumerate(ks)]
        excl = np.concatenate([[0], np.cumsum(cn)[:-1]]).astype(int)
        exmax = [-1] + list(np.maximum.accumulate(ls)[:-1])
        for t, (vals, nz, rs, re) in enumerate(ks):
            rel = gb + 8 * t - e0
            tpos, sprev = carry + int(excl[t]), max(carry_s, int(exmax[t]))
            for j in range(8):
                bit = 1 << j
                if not (nz | rs | re) & bit:
                    continue
                below = bit - 1
                pj = tpos + _popc(nz & below) + 2 * _popc(rs & below)
                writes = []
                if nz & bit or rs & bit:
                    writes.append((pj, vals[j] if nz & bit else 0))
                if re & bit:
                    le = rs & (below | bit)
                    sr = rel + le.bit_length() - 1 if le else sprev
                    writes.append((pj + 1 if sr == rel + j else pj - 1, rel + j - sr + 1))
                for p, v in writes:
                    assert p not in tok, "a token position written twice"
                    tok[p] = v
        carry += sum(cn)
        carry_s = max(carry_s, max(ls))
    assert sorted(tok) == list(range(count)), "token positions fill the tile's count exactly"
    return [tok[i] for i in range(count)]


# ------------------------------------------------------------------ LP level tile
LP_T = 64


def lp_geometry(RA, RS):
    """LevelGeo<RA, RS>: half-resolution window, staged window, strides, runs per thread"""
    MLO = -(RS // 2)
    VN = (LP_T - 1 + RS) // 2 - MLO + 1
    MN = 2 * (VN - 1) + 2 * RA + 1
    run = 7 if VN % 7 == 0 else 6 if VN % 6 == 0 else 5
    return dict(MLO=MLO, VN=VN, MN=MN, Y0=2 * MLO - RA, MNS=MN + (MN & 1), TS=LP_T + 2,
                NA=max(MN * VN, VN * (LP_T + 2)), KR=run, KC=run, KP=8, SLO=RS // 2, SHI=(RS + 1) // 2)


def _rd(buf, i):
    assert 0 <= i < buf.size, ("shared read out of its array", i, buf.size)
    assert not np.isnan(buf[i]), ("shared read before write", i)
    return buf[i]


def lp_level_tile(RA, RS, syn, fa, fs, main, ty, tx, cin=None, cin_lo=None):
    """one tile (ty, tx) of a level: analysis (cout, out) of the periodic image main, or synthesis out
    from the detail main and the coarse lowpass cin (+ cin_lo); returns (out 64 x 64, cout 32 x 32 or
    None) with the kernel's indexing, every shared access checked in bounds and initialised"""
    g = lp_geometry(RA, RS)
    MLO, VN, MN, Y0, MNS, TS, NA = (g[k] for k in ("MLO", "VN", "MN", "Y0", "MNS", "TS", "NA"))
    H, W = main.shape
    y0, x0 = ty * LP_T, tx * LP_T
    m0, n0 = y0 // 2, x0 // 2
    ta = lambda b: fa[b + RA]
    ts = lambda t: fs[t + RS]
    s_main = np.full(MN * MNS, np.nan)
    for r in range(MN):
        for c in range(MN):
            s_main[r * MNS + c] = main[(y0 + Y0 + r) % H, (x0 + Y0 + c) % W]
    s_v = np.full(VN * VN, np.nan)
    if syn:
        for m in range(VN):
            for n in range(VN):
                s_v[m * VN + n] = cin[(m0 + MLO + m) % (H // 2), (n0 + MLO + n) % (W // 2)]
        mu = float(np.rint(s_v.sum() / (2 * VN * VN)))
        for m in range(VN):
            for n in range(VN):
                e = s_v[m * VN + n] - 2 * mu
                if cin_lo is not None:
                    e += cin_lo[(m0 + MLO + m) % (H // 2), (n0 + MLO + n) % (W // 2)]
                s_v[m * VN + n] = e
    else:
        mu = float(np.rint(np.nansum(s_main[:MN * MNS]) / (MN * MN)))
    sub = mu if not syn else 0.0
    # decimating row pass
    s_a = np.full(NA, np.nan)
    KR = g["KR"]
    for i in range(MN * (VN // KR)):
        run, r = divmod(i, MN)
        w = r * MNS + 2 * KR * run
        assert w % 2 == 0, "pair loads"
        x = [_rd(s_main, w + j) - sub for j in range(2 * KR + 2 * RA - 1)]
        for k in range(KR):
            s_a[r * VN + KR * run + k] = sum(ta(b) * x[2 * k + RA - b] for b in range(-RA, RA + 1))
    # decimating column pass, the lowpass share
    KC = g["KC"]
    cout = None if syn else np.full((LP_T // 2, LP_T // 2), np.nan)
    for i in range(VN * (VN // KC)):
        run, n = divmod(i, VN)
        mr = KC * run
        y = [_rd(s_a, (2 * mr + j) * VN + n) for j in range(2 * KC + 2 * RA - 1)]
        for k in range(KC):
            acc = sum(ta(a) * y[2 * k + RA - a] for a in range(-RA, RA + 1))
            m = mr + k
            if syn:
                s_v[m * VN + n] = _rd(s_v, m * VN + n) - acc
            else:
                s_v[m * VN + n] = acc
                if 0 <= m + MLO < LP_T // 2 and 0 <= n + MLO < LP_T // 2:
                    assert np.isnan(cout[m + MLO, n + MLO])
                    cout[m + MLO, n + MLO] = acc + 2 * mu
    # expanding passes, pairs of outputs, runs of KP pairs
    KP, SLO, SHI = g["KP"], g["SLO"], g["SHI"]
    NWE = KP + SLO + SHI

    def pairs(z, k):
        ev = sum(ts(t) * z[k + SLO - t // 2] for t in range(-RS, RS + 1) if t % 2 == 0)
        od = sum(ts(t) * z[k + SLO + (1 - t) // 2] for t in range(-RS, RS + 1) if t % 2)
        return ev, od

    s_a = np.full(NA, np.nan)
    for i in range(VN * (LP_T // 2 // KP)):
        run, m = divmod(i, VN)
        p0 = KP * run
        vb = m * VN + p0 - MLO - SLO
        assert vb >= m * VN and vb + NWE <= (m + 1) * VN, "a window inside its row"
        z = [_rd(s_v, vb + j) for j in range(NWE)]
        for k in range(KP):
            d = m * TS + 2 * (p0 + k)
            assert d + 1 < NA
            s_a[d], s_a[d + 1] = pairs(z, k)
    out = np.full((LP_T, LP_T), np.nan)
    for i in range(LP_T * (LP_T // 2 // KP)):
        run, x = divmod(i, LP_T)
        p0 = KP * run
        z = [_rd(s_a, (p0 - MLO - SLO + j) * TS + x) for j in range(NWE)]
        for k in range(KP):
            ev, od = pairs(z, k)
            for h, acc in ((0, ev), (1, od)):
                yy = 2 * (p0 + k) + h
                mv = _rd(s_main, (2 * p0 - Y0) * MNS + (x - Y0) + (2 * k + h) * MNS)
                assert np.isnan(out[yy, x]), "an output written twice"
                out[yy, x] = (mv + acc) + mu if syn else (mv - sub) - acc
    assert not np.isnan(out).any()
    return out, cout
