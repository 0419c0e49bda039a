"""CPU emulations of the three 3D interior-sweep kernels (k_rb_zmarch,
k_rb_stream3d, k_rb_span3d): the same work items, the same pipelines of planes (ring
slots, loads issued ahead, register rotations), the same per-lane and
per-warp indexing, the same shuffles at the warp edges and the same clamped
or zero-filled loads outside the box.  Each must give bitwise the result of
the red half-sweep followed by the black half-sweep in place (Eq. jac2d in
Gauss-Seidel red-black order, Sec. 2.4) and write every unknown exactly
once.  Host logic only: no GPU."""
import numpy as np
import pytest

import oracle
from paper_1111_0983_gb300 import inputs



def plane_items(T, TY, TX, seg):
    """Tiles of TY rows x TX columns, the runs of planes holding unknowns
    (gaps of up to 2 idle planes merged), cut into at most seg planes."""
    n = T.shape[0]
    ty, tx = (n + TY - 1) // TY, (n + TX - 1) // TX
    act = np.zeros((ty * tx, n), bool)
    I, J, K = np.nonzero((T == 1) | (T == 2))
    act[(J // TY) * tx + K // TX, I] = True
    out = []
    for t in range(ty * tx):
        a, i = act[t], 0
        while i < n:
            if not a[i]:
                i += 1
                continue
            end = i + 1
            for k in range(end, n):
                if a[k]:
                    end = k + 1
                elif k - end >= 2:
                    break
            for s0 in range(i, end, seg):
                out.append((t // tx, t % tx, s0, min(end, s0 + seg)))
            i = end
    return out


def red_black_in_place(u, f, T, h2):
    u = u.copy()
    for colour in (0, 1):
        I, J, K = np.nonzero(T == 1)
        for i, j, k in zip(I, J, K):
            if (i + j + k) % 2 != colour:
                continue
            nb = (((u[i, j, k - 1] + u[i, j, k + 1]) + u[i - 1, j, k]) + u[i + 1, j, k]) + (u[i, j - 1, k] + u[i, j + 1, k])
            u[i, j, k] = (np.float32(h2) * f[i, j, k] + nb) * np.float32(1 / 6)
    return u


def red_black_in_place_fast(u, f, T, h2):
    """The same in-place sweep vectorised per colour (nodes of one colour are
    not neighbours of each other), the same sums in the same order."""
    u = u.copy()
    I, J, K = np.nonzero(T == 1)
    for colour in (0, 1):
        m = (I + J + K) % 2 == colour
        i, j, k = I[m], J[m], K[m]
        nb = (((u[i, j, k - 1] + u[i, j, k + 1]) + u[i - 1, j, k]) + u[i + 1, j, k]) + (u[i, j - 1, k] + u[i, j + 1, k])
        u[i, j, k] = (np.float32(h2) * f[i, j, k] + nb) * np.float32(1 / 6)
    return u


def emulate_zmarch(u, f, T, h2, TY=16, TX=64):
    n = u.shape[0]
    UX, US, RX, RS = TX + 4, (TY + 4) * (TX + 4), TX + 2, (TY + 2) * (TX + 2)
    MROW, MPL = 3, 56
    out, written = np.zeros_like(u), np.zeros(u.shape, int)
    uf, ff, tf = u.ravel(), f.ravel(), T.ravel()
    for (ty_, tx_, a, b) in plane_items(T, TY, TX, 32):
        r0, c0 = ty_ * TY, tx_ * TX
        assert 1 <= a < b <= n - 1
        su = np.full((6, US), np.nan, np.float32)
        sf = np.full((5, RS), np.nan, np.float32)
        sh = np.full((3, RS), np.nan, np.float32)
        sm = np.zeros((5, MPL), np.uint64)
        mask = np.zeros((b - a + 2, MPL), np.uint64)   # host-built inside-node masks
        for ii in range(a - 1, b + 1):
            for ry in range(TY + 2):
                for rx in range(TX + 2):
                    gj, gk = r0 - 1 + ry, c0 - 1 + rx
                    if 0 <= ii < n and 0 <= gj < n and 0 <= gk < n and tf[(ii * n + gj) * n + gk] == 1:
                        mask[ii - a + 1, ry * MROW + (rx >> 5)] |= np.uint64(1 << (rx & 31))

        def load_u(i):
            for idx in range(US):
                ry, rx = divmod(idx, UX)
                gj, gk = r0 - 2 + ry, c0 - 2 + rx
                ok = 0 <= i < n and 0 <= gj < n and 0 <= gk < n
                su[(i + 6) % 6, idx] = uf[(i * n + gj) * n + gk] if ok else 0

        def load_f(i):
            for idx in range(RS):
                ry, rx = divmod(idx, RX)
                gj, gk = r0 - 1 + ry, c0 - 1 + rx
                ok = 0 <= i < n and 0 <= gj < n and 0 <= gk < n
                sf[i % 5, idx] = ff[(i * n + gj) * n + gk] if ok else 0
            sm[i % 5] = mask[i - a + 1]

        def inside(i, ry, rx):
            return (int(sm[i % 5, ry * MROW + (rx >> 5)]) >> (rx & 31)) & 1

        load_u(a - 2), load_u(a - 1), load_u(a), load_f(a - 1)
        load_u(a + 1), load_f(a)
        if a + 2 <= b + 1:
            load_u(a + 2)
        if a + 1 <= b:
            load_f(a + 1)
        for j in range(a - 1, b + 1):
            if j + 4 <= b + 1:
                load_u(j + 4)
            if j + 3 <= b:
                load_f(j + 3)
            um, uc, up = su[(j + 5) % 6], su[(j + 6) % 6], su[(j + 7) % 6]
            for idx in range(RS):
                ry, rx = divmod(idx, RX)
                ui = (ry + 1) * UX + rx + 1
                val = uc[ui]
                if inside(j, ry, rx) and (j + ry + rx) % 2 == 0:
                    nb = (((uc[ui - 1] + uc[ui + 1]) + um[ui]) + up[ui]) + (uc[ui - UX] + uc[ui + UX])
                    val = (np.float32(h2) * sf[j % 5, idx] + nb) * np.float32(1 / 6)
                sh[j % 3, idx] = val
            if j - 1 >= a:
                i = j - 1
                hm, hc, hp = sh[(i - 1) % 3], sh[i % 3], sh[(i + 1) % 3]
                for idx in range(TY * TX):
                    oy, ox = divmod(idx, TX)
                    gj, gk = r0 + oy, c0 + ox
                    if gj >= n or gk >= n:
                        continue
                    ri = (oy + 1) * RX + ox + 1
                    val = hc[ri]
                    if inside(i, oy + 1, ox + 1) and (i + oy + ox) % 2 == 1:
                        nb = (((hc[ri - 1] + hc[ri + 1]) + hm[ri]) + hp[ri]) + (hc[ri - RX] + hc[ri + RX])
                        val = (np.float32(h2) * sf[i % 5, ri] + nb) * np.float32(1 / 6)
                    out[i, gj, gk] = val
                    written[i, gj, gk] += 1
    return out, written


def emulate_stream3d(u, f, T, h2, TY=12, W=28):
    n = u.shape[0]
    NW = TY + 4
    out, written = np.zeros_like(u), np.zeros(u.shape, int)
    wv, lv = np.meshgrid(np.arange(NW), np.arange(32), indexing="ij")
    zero_row = np.zeros((1, 32), np.float32)
    for (ty_, tx_, a, b) in plane_items(T, TY, W, 64):
        r0, k0 = ty_ * TY, tx_ * W
        row, col = r0 - 2 + wv, k0 - 2 + lv
        ok = (row >= 0) & (row < n) & (col >= 0) & (col < n)
        offr, offc = np.where(ok, row, 0), np.where(ok, col, 0)   # lanes outside the box read node 0
        red_here = (wv >= 1) & (wv <= NW - 2) & (lv >= 1) & (lv <= 30)
        owner = ok & (wv >= 2) & (wv <= NW - 3) & (lv >= 2) & (lv <= W + 1)
        par = (row + col) & 1

        def ld(arr, i):   # clamped plane, as the kernel
            return arr[min(max(i, 0), n - 1)][offr, offc]

        def up(x):     # __shfl_up_sync(., 1): lane 0 keeps its own value
            return np.concatenate([x[:, :1], x[:, :-1]], 1)

        def down(x):   # __shfl_down_sync(., 1): lane 31 keeps its own value
            return np.concatenate([x[:, 1:], x[:, -1:]], 1)

        def rows(x):   # the rows of the adjacent warps (0 beyond the CTA)
            return np.concatenate([zero_row, x[:-1]], 0), np.concatenate([x[1:], zero_row], 0)

        om, oc, op = ld(u, a - 2), ld(u, a - 1), ld(u, a)
        hm = np.zeros((NW, 32), np.float32)
        hc = hm.copy()
        fc, fm = ld(f, a - 1), np.zeros((NW, 32), np.float32)
        tc, tm = ld(T, a - 1), np.zeros((NW, 32), T.dtype)
        q = [[ld(u, a + 1 + s), ld(f, a + s), ld(T, a + s)] for s in range(3)]
        j, s = a - 1, 0
        while True:
            uq, fq, tq = q[s]
            oym, oyp = rows(oc)
            cond = red_here & ok & (j >= 0) & ((tc & 3) == 1) & (((j + par) & 1) == 0)
            nb = (((up(oc) + down(oc)) + om) + op) + (oym + oyp)
            hn = np.where(cond, (np.float32(h2) * fc + nb) * np.float32(1 / 6), oc).astype(np.float32)
            hym, hyp = rows(hc)
            if j - 1 >= a:
                condb = ((tm & 3) == 1) & (((j - 1 + par) & 1) == 1)
                nbb = (((up(hc) + down(hc)) + hm) + hn) + (hym + hyp)
                o = np.where(condb, (np.float32(h2) * fm + nbb) * np.float32(1 / 6), hc).astype(np.float32)
                out[j - 1][row[owner], col[owner]] = o[owner]
                written[j - 1][row[owner], col[owner]] += 1
            om, oc, op = oc, op, uq
            hm, hc = hc, hn
            fm, fc = fc, fq
            tm, tc = tc, tq
            if j + 5 <= b + 1:     # no load past the last plane the item reads
                q[s][0] = ld(u, j + 5)
            if j + 4 <= b:
                q[s][1], q[s][2] = ld(f, j + 4), ld(T, j + 4)
            j, s = j + 1, (s + 1) % 3
            if j > b:
                break
    return out, written


def row_spans(T):
    """Per (plane, row): the span of the unknowns and of the inside nodes
    (lo, hi; lo > hi when empty), and whether the inside nodes are one
    interval."""
    n = T.shape[0]
    kind = T & 3
    kk = np.arange(n)
    unk, ins = (kind == 1) | (kind == 2), kind == 1
    lo, hi = np.where(unk, kk, n).min(-1), np.where(unk, kk, -1).max(-1)
    ilo, ihi = np.where(ins, kk, n).min(-1), np.where(ins, kk, -1).max(-1)
    cnt = ins.sum(-1)
    simple = bool(((cnt == 0) | (cnt == ihi - ilo + 1)).all())
    return lo, hi, ilo, ihi, simple


def span_items(lo, hi, C, J=12, seg=32):
    """Row blocks of J rows; per block the runs of planes with unknowns (gaps
    of up to 2 idle planes merged) cut into at most seg planes; per piece the
    windows k0 = kmin - 1 + m (32 C - 2) covering [kmin, kmax]."""
    n = lo.shape[0]
    W = 32 * C - 2
    out = []
    for jb in range((n + J - 1) // J):
        rs = slice(jb * J, min(n, jb * J + J))
        l = np.where(lo[:, rs] <= hi[:, rs], lo[:, rs], n).min(1)
        h = np.where(lo[:, rs] <= hi[:, rs], hi[:, rs], -1).max(1)
        act = l <= h
        i = 0
        while i < n:
            if not act[i]:
                i += 1
                continue
            end = i + 1
            for k in range(end, n):
                if act[k]:
                    end = k + 1
                elif k - end >= 2:
                    break
            for s0 in range(i, end, seg):
                s1 = min(end, s0 + seg)
                kmin, kmax = l[s0:s1][act[s0:s1]].min(), h[s0:s1][act[s0:s1]].max()
                k0 = kmin - 1
                while k0 + 1 <= kmax:
                    out.append((jb, k0, s0, s1))
                    k0 += W
            i = end
    return out


def emulate_span3d(u, f, T, h2, C, J=12):
    n = u.shape[0]
    NW = J + 4
    lo, hi, ilo, ihi, simple = row_spans(T)
    assert simple
    out, written = np.zeros_like(u), np.zeros(u.shape, int)
    wv = np.arange(NW)[:, None, None]
    cv = np.arange(C)[None, :, None]
    lv = np.arange(32)[None, None, :]
    sixth, h2 = np.float32(1 / 6), np.float32(h2)
    for (jb, k0, a, b) in span_items(lo, hi, C, J):
        r0 = jb * J
        row = r0 - 2 + wv                      # (NW, 1, 1)
        k = k0 + lv + 32 * cv                  # (1, C, 32)
        rok = (row >= 0) & (row < n)
        rowc = np.clip(row, 0, n - 1)
        redrow = (wv >= 1) & (wv <= NW - 2)
        owner = (wv >= 2) & (wv <= NW - 3)
        par = (row + k0 + lv) & 1
        own = ~(((lv == 0) & (cv == 0)) | ((lv == 31) & (cv == C - 1)))

        def meta(p):   # spans of the CTA's rows in plane p (empty outside the box)
            if p < 0 or p >= n:
                e = np.full((NW, 1, 1), 0xFFFF), np.zeros((NW, 1, 1), int)
                return e + e
            m = [x[p, rowc[:, 0, 0]].reshape(NW, 1, 1) for x in (lo, hi, ilo, ihi)]
            return [np.where(rok, m[0], 0xFFFF), np.where(rok, m[1], 0),
                    np.where(rok, m[2], 0xFFFF), np.where(rok, m[3], 0)]

        def has(l_, h_, kk):
            return (kk >= l_) & (kk <= h_)

        def ld_u(p):
            l_, h_, _, _ = meta(p)
            pc = min(max(p, 0), n - 1)
            x = np.where(has(l_, h_, k), u[pc, rowc, np.clip(k, 0, n - 1)], 0).astype(np.float32)
            ke = np.where(np.arange(32) == 31, k0 - 1, k0 + 32 * C)[None, :]
            me = ((np.arange(32) == 0) | (np.arange(32) == 31))[None, :] & has(l_[:, 0], h_[:, 0], ke)
            e = np.where(me, u[pc, rowc[:, 0], np.clip(ke, 0, n - 1)], 0).astype(np.float32)
            return [x, e]

        def ld_f(p):
            _, _, l_, h_ = meta(p)
            pc = min(max(p, 0), n - 1)
            m = redrow & has(l_, h_, k)
            return np.where(m, f[pc, rowc, np.clip(k, 0, n - 1)], 0).astype(np.float32)

        def shl(x, e):   # __shfl_sync(., lane - 1) of the kernel's source values
            s = x.copy()
            for c in range(C):
                s[:, c, 31] = e[:, 31] if c == 0 else x[:, c - 1, 31]
            return np.roll(s, 1, axis=2)

        def shr(x, e):   # __shfl_sync(., lane + 1)
            s = x.copy()
            for c in range(C):
                s[:, c, 0] = e[:, 0] if c == C - 1 else x[:, c + 1, 0]
            return np.roll(s, -1, axis=2)

        def rows(x):     # the rows of the adjacent warps (0 beyond the CTA)
            z = np.zeros_like(x[:1])
            return np.concatenate([z, x[:-1]], 0), np.concatenate([x[1:], z], 0)

        zero = np.zeros((NW, C, 32), np.float32)
        om = ld_u(a - 2)[0]
        oc, op = ld_u(a - 1), ld_u(a)
        uq = [ld_u(a + 1 + s) if a + 1 + s <= b + 1 else [zero, np.zeros((NW, 32), np.float32)] for s in range(3)]
        hm, hc = zero, zero
        fc, fm = ld_f(a - 1), zero
        fq = [ld_f(a + s) if a + s <= b else zero for s in range(3)]
        j, s = a - 1, 0
        while True:
            _, _, il, ih = meta(j)
            red = ((j + par) & 1) == 0
            ozm, ozp = shl(*oc), shr(*oc)
            oym, oyp = rows(oc[0])
            upd = (h2 * fc + ((((ozm + ozp) + om) + op[0]) + (oym + oyp))) * sixth
            hn = np.where(redrow & red & has(il, ih, k), upd, oc[0]).astype(np.float32)
            if j - 1 >= a:
                ul, uh, il1, ih1 = meta(j - 1)
                ez = np.zeros((NW, 32), np.float32)
                hzm, hzp = shl(hc, ez), shr(hc, ez)
                hym, hyp = rows(hc)
                upd = (h2 * fm + ((((hzm + hzp) + hm) + hn) + (hym + hyp))) * sixth
                val = np.where(red & has(il1, ih1, k), upd, hc).astype(np.float32)
                st = owner & own & has(ul, uh, k) & np.ones((NW, C, 32), bool)
                wi, ci, li = np.nonzero(st)
                rr, kk = (r0 - 2 + wi), (k0 + li + 32 * ci)
                out[j - 1, rr, kk] = val[wi, ci, li]
                written[j - 1, rr, kk] += 1
            om, oc, op = oc[0], op, uq[s]
            hm, hc = hc, hn
            fm, fc = fc, fq[s]
            if j + 5 <= b + 1:
                uq[s] = ld_u(j + 5)
            if j + 4 <= b:
                fq[s] = ld_f(j + 4)
            j, s = j + 1, (s + 1) % 3
            if j > b:
                break
    return out, written


def _problem(n):
    T = oracle.Oracle(inputs.torus().phi_grid(n), 9).types(0).astype(np.int64)
    rng = np.random.default_rng(0)
    u = np.where(T > 0, rng.standard_normal(T.shape), 0).astype(np.float32)
    f = np.where(T == 1, rng.standard_normal(T.shape), 0).astype(np.float32)
    return u, f, T, (2.0 / (n - 1)) ** 2


@pytest.mark.parametrize("kernel,n", [("stream3d", 33), ("stream3d", 65), ("zmarch", 65),
                                      ("span3d-2", 65), ("span3d-3", 65), ("span3d-5", 33)])
def test_sweep_kernel_emulation_equals_red_black_in_place(kernel, n):
    u, f, T, h2 = _problem(n)
    if kernel.startswith("span3d"):
        out, written = emulate_span3d(u, f, T, h2, int(kernel[-1]))
    else:
        emulate = emulate_stream3d if kernel == "stream3d" else emulate_zmarch
        out, written = emulate(u, f, T, h2)
    ref = red_black_in_place(u, f, T, h2)
    unk = T > 0
    assert (written[unk] == 1).all() and written.max() <= 1
    assert np.array_equal(out[unk], ref[unk])


def test_span3d_emulation_with_several_windows_a_row():
    """At 257^3 a row's unknowns span 67 nodes: with 2 columns a lane (62
    owned nodes a window) the blocks need two windows side by side."""
    u, f, T, h2 = _problem(257)
    lo, hi, _, _, _ = row_spans(T)
    it = span_items(lo, hi, 2)
    assert len({(jb, a) for (jb, _, a, _) in it}) < len(it)   # some piece has two windows
    out, written = emulate_span3d(u, f, T, h2, 2)
    ref = red_black_in_place_fast(u, f, T, h2)
    unk = T > 0
    assert (written[unk] == 1).all() and written.max() <= 1
    assert np.array_equal(out[unk], ref[unk])


def row_segments(T):
    """Runs of consecutive inside nodes of every row (i, j), cut into
    segments of at most 64 nodes: (i * n + j, first, last)."""
    n = T.shape[0]
    ins = (T & 3) == 1
    out = []
    for r in np.nonzero(ins.reshape(n * n, n).any(-1))[0]:
        row = ins.reshape(n * n, n)[r]
        k = 0
        while k < n:
            if not row[k]:
                k += 1
                continue
            e = k
            while e + 1 < n and row[e + 1]:
                e += 1
            for k0 in range(k, e + 1, 64):
                out.append((r, k0, min(e, k0 + 63)))
            k = e + 1
    return out


def emulate_rows(u, f, T, h2):
    """k_rb_rows: the red launch then the black one, in place; per segment
    lane l updates the node of the colour at k_first + 2 l."""
    n = u.shape[0]
    u = u.copy().ravel()
    ff = f.ravel()
    s0 = n * n
    written = np.zeros(u.shape, int)
    segs = row_segments(T)
    lane = np.arange(32)
    for colour in (0, 1):
        for (r, k0, k1) in segs:
            i, j = divmod(r, n)
            k = k0 + ((i + j + k0 + colour) & 1) + 2 * lane
            k = k[k <= k1]
            p = r * n + k
            nb = (((u[p - 1] + u[p + 1]) + u[p - s0]) + u[p + s0]) + (u[p - n] + u[p + n])
            u[p] = (np.float32(h2) * ff[p] + nb) * np.float32(1 / 6)
            written[p] += 1
    return u.reshape(T.shape), written.reshape(T.shape)


@pytest.mark.parametrize("n,turn", [(33, False), (129, False), (65, True)])
def test_row_segment_sweep_emulation_equals_red_black_in_place(n, turn):
    """turn: the torus with its axis along axis 0, so that a row crosses the
    ring twice (two runs of inside nodes)."""
    u, f, T, h2 = _problem(n)
    if turn:
        u, f, T = (np.ascontiguousarray(x.transpose(2, 1, 0)) for x in (u, f, T))
        assert len(row_segments(T)) > len({r for (r, _, _) in row_segments(T)})
    out, written = emulate_rows(u, f, T, h2)
    ref = red_black_in_place_fast(u, f, T, h2)
    ins = (T & 3) == 1
    assert (written[ins] == 1).all() and (written[~ins] == 0).all()
    assert np.array_equal(out, ref)
