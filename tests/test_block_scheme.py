"""Host-side model of the blocking scheme of the cluster stepping kernels and
of the cluster band Cholesky, checked against dense triangular solves and
numpy's Cholesky (no GPU).

The model follows the kernels' arithmetic plan and index arithmetic:
* 64-row blocks, R = 64/CL own rows per CTA;
* the two-block lag (band products over blocks at least three away, the
  couplings C1, C2 / D1, D2 to the two nearest blocks);
* the deferred first backward block;
* the GEMV work items (4 lanes per forward item, H chunks per row, TB
  columns per backward warp);
* the rank-order sum of the CTAs' shares;
* the per-column mbarrier byte counts of the band Cholesky.

Arrays are bounds-checked and NaN-initialised, so a read outside the data or
of a value not yet formed fails the test.  This is a model for checking the
scheme, not the oracle (which factors with LAPACK), and shares no code with
either side.
"""
import numpy as np
import pytest
import scipy.linalg as sla

KB = 64                                   # rows per block
GW_OF = {1: 8, 2: 4, 4: 4, 8: 2}          # GEMV warps per cluster size


class Checked:
    """1D array whose reads and writes are bounds-checked."""

    def __init__(self, a, name):
        self.a, self.name = a, name

    def __getitem__(self, i):
        assert 0 <= i < len(self.a), (self.name, i)
        return self.a[i]

    def __setitem__(self, i, v):
        assert 0 <= i < len(self.a), (self.name, i)
        self.a[i] = v


def banded_spd(n, bw, rng):
    a = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - bw), i):
            if rng.random() < 0.7:
                a[i, j] = a[j, i] = rng.normal() * 0.1
    return a + np.eye(n) * (np.abs(a).sum(1).max() + 1.0)


def unit_band(a, bw):
    """Unit lower factor L~ = D^-1 L and its band storage LB[i (bw+1) + c - i + bw]."""
    n = a.shape[0]
    l = np.linalg.cholesky(a)
    lt = l / np.diag(l)[:, None]
    w = bw + 1
    lb = np.zeros(n * w)
    for i in range(n):
        for c in range(max(0, i - bw), i + 1):
            lb[i * w + (c - i + bw)] = lt[i, c]
    return lt, lb


def block_arrays(lb, n, bw):
    """B_b = inverse of the diagonal block (identity rows past n), C1, C2
    ([b][r][t]) and D1^T, D2^T ([b][t][r]), from the band alone."""
    nblk, w = (n + KB - 1) // KB, bw + 1

    def blk(bi, bj):
        o = np.zeros((KB, KB))
        if bi < 0 or bi >= nblk or bj < 0:
            return o
        for m in range(KB):
            for c in range(KB):
                i, col = bi * KB + m, bj * KB + c
                if i < n and col <= i and i - col <= bw:
                    o[m, c] = lb[i * w + (col - i + bw)]
        return o

    out = {k: np.zeros(nblk * KB * KB) for k in ("B", "C1", "C2", "D1", "D2")}
    for b in range(nblk):
        d = blk(b, b)
        for r in range(KB):
            if b * KB + r >= n:
                d[r, :] = 0.0
                d[r, r] = 1.0
        inv = np.linalg.inv(d)
        sl = slice(b * KB * KB, (b + 1) * KB * KB)
        out["B"][sl] = inv.ravel()
        out["C1"][sl] = (inv @ blk(b, b - 1)).ravel()
        out["C2"][sl] = (inv @ blk(b, b - 2)).ravel()
        out["D1"][sl] = (blk(b + 1, b) @ inv).ravel()
        out["D2"][sl] = (blk(b + 2, b) @ inv).ravel()
    return out


def ring_rows_of(bw):
    """Rows of the kernels' solved-row ring: a power of two >= bw + 256."""
    r = 256
    while r < bw + 4 * 64:
        r *= 2
    return r


def substitute(lb, arr, n, bw, w_in, cl, ring_rows=None, late_gemv=False):
    """Forward and backward substitution on a cluster of `cl` CTAs, as the
    kernels do it.  Returns every CTA's copy of the solution.

    ring_rows: each CTA keeps only its own rows of the work vector plus a ring
    of the last ring_rows solved rows (row r in slot r % ring_rows, tagged with
    r so that reading a row that is not, or no longer, there fails); the
    returned copies are assembled from the CTAs' own rows.  late_gemv: the band
    products of round j run as late as the warp hand-offs allow (after block
    j - 1 is stored), instead of as early (after block j - 3)."""
    r_own = KB // cl
    gw = GW_OF[cl]
    h = 8 * gw // r_own                   # forward chunks per own row
    tb = r_own // gw                      # backward own columns per GEMV warp
    kg = 32 // tb                         # backward row groups per column
    assert r_own * h == 8 * gw and tb * gw == r_own
    w_, nblk = bw + 1, (n + KB - 1) // KB
    g_end = 2 * nblk
    lbc = Checked(lb, "LB")
    B, C1, C2, D1, D2 = (Checked(arr[k], k) for k in ("B", "C1", "C2", "D1", "D2"))
    copies = [Checked(np.full(n, np.nan), f"w{q}") for q in range(cl)]
    shares = [np.full((2, cl, KB), np.nan) for _ in range(cl)]
    ring = [np.full((4, r_own), np.nan) for _ in range(cl)]
    pre = [np.full(KB, np.nan) for _ in range(cl)]
    own_rows = [Checked(np.full(nblk * r_own, np.nan), f"own{q}") for q in range(cl)]
    if ring_rows is not None:
        rvals = [np.full(ring_rows, np.nan) for _ in range(cl)]
        rtags = [np.full(ring_rows, -1) for _ in range(cl)]

    def put(q, row, v):                   # a solved row: ring (or copy) and own rows
        if ring_rows is None:
            copies[q][row] = v
            return
        rvals[q][row % ring_rows] = v
        rtags[q][row % ring_rows] = row
        t = row % KB - q * r_own
        if 0 <= t < r_own:
            own_rows[q][(row // KB) * r_own + t] = v

    def solved(q, row):                   # a solved row of any CTA (band products)
        if ring_rows is None:
            return copies[q][row]
        assert rtags[q][row % ring_rows] == row, ("ring", q, row, rtags[q][row % ring_rows])
        return rvals[q][row % ring_rows]

    def own_at(q, blk, t):                # own row t of block blk
        if ring_rows is None:
            return copies[q][blk * KB + q * r_own + t]
        v = own_rows[q][blk * r_own + t]
        assert np.isfinite(v), ("own row not formed", q, blk, t)
        return v

    for q in range(cl):                   # own rows of the right-hand side
        for idx in range(nblk * r_own):
            pi = (idx // r_own) * KB + q * r_own + idx % r_own
            if pi < n:
                if ring_rows is None:
                    copies[q][pi] = w_in[pi]
                else:
                    own_rows[q][idx] = w_in[pi]

    def block_of(g):
        return g if g < nblk else 2 * nblk - 1 - g

    def own(q, blk, t):
        row = blk * KB + q * r_own + t
        return own_at(q, blk, t) if row < n else 0.0

    def gemv(q, j):                       # s of round j over the blocks known after round j - 2
        acc = np.zeros(r_own)
        for warp in range(gw):
            for lane in range(32):
                if j < nblk:              # row i of block j, columns of blocks <= j - 3
                    item = warp * 8 + (lane >> 2)
                    t, hh, gl = item // h, item % h, lane & 3
                    i = j * KB + q * r_own + t
                    if i >= n:
                        continue
                    c, hi = max(0, i - bw) + 4 * hh + gl, (j - 2) * KB
                    while c < hi:
                        acc[t] += lbc[i * w_ + (c - i + bw)] * solved(q, c)
                        c += 4 * h
                else:                     # column c of block bt, rows of blocks >= bt + 3
                    bt = 2 * nblk - 1 - j
                    t, grp = warp * tb + lane % tb, lane // tb
                    c = bt * KB + q * r_own + t
                    if c >= n:
                        continue
                    k = (bt + 3) * KB + grp
                    while k <= min(n - 1, c + bw):
                        acc[t] += lbc[k * w_ + (c - k + bw)] * solved(q, k)
                        k += kg
        blk = block_of(j)
        for t in range(r_own):
            row = blk * KB + q * r_own + t
            ring[q][j & 3, t] = own_at(q, blk, t) - acc[t] if row < n else 0.0

    def pre_of(q, g1):                    # B s - C2 y_{b-2} (forward) or B^T s - D2^T u_{b+2}
        b1 = block_of(g1)
        for r in range(KB):
            v = 0.0
            for t in range(r_own):
                tc = q * r_own + t
                if g1 == nblk:            # first backward block: s = y_b, no couplings
                    v += B[b1 * KB * KB + tc * KB + r] * own(q, b1, t)
                elif g1 < nblk:
                    v += B[b1 * KB * KB + r * KB + tc] * ring[q][g1 & 3, t]
                    if b1 >= 2:
                        v -= C2[b1 * KB * KB + r * KB + tc] * own(q, b1 - 2, t)
                else:
                    v += B[b1 * KB * KB + tc * KB + r] * ring[q][g1 & 3, t]
                    if g1 >= nblk + 2:
                        v -= D2[b1 * KB * KB + tc * KB + r] * own(q, b1 + 2, t)
            assert np.isfinite(v), (g1, q, r)
            pre[q][r] = v

    for q in range(cl):                   # s of rounds 0 and 1: the right-hand side alone
        for j in (0, 1):
            if j < g_end and j != nblk:
                for t in range(r_own):
                    row = j * KB + q * r_own + t
                    ring[q][j & 3, t] = own_at(q, j, t) if row < n else 0.0
    for g in range(g_end + 1):
        if cl > 1 and g >= 1:             # gather the shares of round g - 1, rank order
            bp = block_of(g - 1)
            for q in range(cl):
                for r in range(KB):
                    v = shares[q][(g - 1) & 1, :, r]
                    assert np.all(np.isfinite(v))
                    if bp * KB + r < n:
                        put(q, bp * KB + r, v.sum())
        if g == g_end:
            break
        j = g if late_gemv else g + 2     # band products as late / as early as allowed
        if 2 <= j < g_end and j != nblk:
            for q in range(cl):
                gemv(q, j)
        for q in range(cl):
            pre_of(q, g)
        b, fwd = block_of(g), g < nblk
        new_shares = [x.copy() for x in shares]
        done_rows = []
        for q in range(cl):
            for r in range(KB):           # v = pre - C1 y_{b-1} or pre - D1^T u_{b+1}
                v = pre[q][r]
                for t in range(r_own):
                    tc = q * r_own + t
                    if fwd and b >= 1:
                        v -= C1[b * KB * KB + r * KB + tc] * own(q, b - 1, t)
                    if not fwd and g >= nblk + 1:
                        v -= D1[b * KB * KB + tc * KB + r] * own(q, b + 1, t)
                if cl == 1:
                    if b * KB + r < n:
                        done_rows.append((b * KB + r, v))
                else:
                    for p in range(cl):
                        new_shares[p][g & 1, q, r] = v
        shares = new_shares
        for i, v in done_rows:
            put(0, i, v)
    if ring_rows is None:
        return [c.a for c in copies]
    out = []                              # every CTA's own rows, gathered
    for q in range(cl):
        full = np.full(n, np.nan)
        for qq in range(cl):
            for idx in range(nblk * r_own):
                pi = (idx // r_own) * KB + qq * r_own + idx % r_own
                if pi < n:
                    full[pi] = own_rows[qq].a[idx]
        out.append(full)
    return out


@pytest.mark.parametrize("cl", [1, 2, 4, 8])
@pytest.mark.parametrize("n,bw", [(225, 15), (97, 31), (150, 70), (200, 130), (128, 127),
                                  (7, 3), (1, 0), (65, 64),
                                  # the annulus meshes' bandwidth: band products reach
                                  # blocks three away in both passes
                                  (450, 204), (400, 260)])
def test_cluster_substitution_scheme_solves_the_band_system(cl, n, bw):
    rng = np.random.default_rng(n * 1000 + bw * 10 + cl)
    lt, lb = unit_band(banded_spd(n, bw, rng), bw)
    arr = block_arrays(lb, n, bw)
    rhs = rng.normal(size=n)
    copies = substitute(lb, arr, n, bw, rhs, cl)
    y = sla.solve_triangular(lt, rhs, lower=True, unit_diagonal=True)
    u = sla.solve_triangular(lt.T, y, lower=False, unit_diagonal=True)
    for c in copies:
        assert np.allclose(c, u, rtol=1e-10, atol=1e-10)
    assert all(np.array_equal(copies[0], c) for c in copies)   # identical copies
    # own rows + ring of solved rows, band products as early and as late as
    # the hand-offs allow: the same values bit for bit
    for late in (False, True):
        dist = substitute(lb, arr, n, bw, rhs, cl, ring_rows=ring_rows_of(bw), late_gemv=late)
        assert all(np.array_equal(copies[0], c) for c in dist), late


@pytest.mark.parametrize("cl", [2, 8])
def test_ring_smaller_than_the_band_fails(cl):
    """A ring shorter than the rows the band products reach must be caught by
    the model (the check is not vacuous)."""
    n, bw = 450, 204
    rng = np.random.default_rng(5)
    lt, lb = unit_band(banded_spd(n, bw, rng), bw)
    arr = block_arrays(lb, n, bw)
    with pytest.raises(AssertionError):
        substitute(lb, arr, n, bw, rng.normal(size=n), cl, ring_rows=128, late_gemv=True)


def count_mod(a, b, r, nc):
    """#{i in [a, b] : i mod nc == r}"""
    if b < a:
        return 0
    first = a + ((r - a) % nc)
    return 0 if first > b else (b - first) // nc + 1


def cluster_cholesky(a, bw, nc):
    """Band Cholesky on `nc` CTAs as k_band_chol_cl does it: row i owned by
    CTA i mod nc and held in a ring of (bw + 1)/nc + 2 slots from the column
    where it enters the window until it is final, per column the scaled
    entries and the next pivot sent to every CTA; the products of the
    trailing updates summed in a separate ring of accumulators S (zeroed when a
    row enters) and subtracted once, when the row's entry is scaled; checks
    each CTA's received bytes against the count it arms its mbarrier with."""
    n = a.shape[0]
    w = bw + 1
    slots = (bw + 1 + nc - 1) // nc + 2
    g = np.zeros(n * w)                                    # the band of A in global memory
    for i in range(n):
        for c in range(max(0, i - bw), i + 1):
            g[i * w + (c - i + bw)] = a[i, c]
    out, done = np.full(n * w, np.nan), np.zeros(n, int)
    ring = [np.full((slots, w), np.nan) for _ in range(nc)]
    sring = [np.full((slots, w), np.nan) for _ in range(nc)]
    held = [[-1] * slots for _ in range(nc)]
    col = [np.full((2, max(bw, 1)), np.nan) for _ in range(nc)]
    piv = [np.full(2, np.nan) for _ in range(nc)]

    def load(rho, i):
        s = (i // nc) % slots
        assert held[rho][s] == -1 or done[held[rho][s]], ("slot still live", rho, i)
        ring[rho][s] = g[i * w:(i + 1) * w]
        sring[rho][s] = 0.0
        held[rho][s] = i

    def row(rho, i):
        s = (i // nc) % slots
        assert held[rho][s] == i, ("row not in the ring", rho, i)
        return ring[rho][s]

    def srow(rho, i):
        s = (i // nc) % slots
        assert held[rho][s] == i, ("row not in the ring", rho, i)
        return sring[rho][s]

    def store(rho, i):
        assert not done[i]
        out[i * w:(i + 1) * w] = row(rho, i)
        done[i] = 1

    for rho in range(nc):
        for i in range(rho, min(n, bw + 1), nc):
            load(rho, i)
    l00 = np.sqrt(g[bw])
    for rho in range(nc):
        piv[rho][0] = 1.0 / l00
    row(0, 0)[bw] = l00
    store(0, 0)
    for j in range(n):
        total = min(bw, n - 1 - j)
        got = [0] * nc
        for rho in range(nc):
            for i in range(j + 1, j + total + 1):
                if i % nc != rho:
                    continue
                ri, si = row(rho, i), srow(rho, i)
                l = (ri[j - i + bw] - si[j - i + bw]) * piv[rho][j & 1]
                ri[j - i + bw] = l
                for p in range(nc):
                    col[p][j & 1, i - j - 1] = l
                    got[p] += 8 * (p != rho)
                if i == j + 1:                             # the owner of row j + 1: its pivot
                    lj = np.sqrt(ri[bw] - (si[bw] + l * l))
                    ri[bw] = lj
                    for p in range(nc):
                        piv[p][(j + 1) & 1] = 1.0 / lj
                        got[p] += 8 * (p != rho)
        for rho in range(nc):
            own = count_mod(j + 1, j + total, rho, nc)
            pv = 1 if (j + 1 < n and (j + 1) % nc != rho) else 0
            assert got[rho] == 8 * (total - own + pv), (j, rho)
        for rho in range(nc):
            for i in range(j + 2, j + total + 1):
                if i % nc != rho:
                    continue
                si, li = srow(rho, i), col[rho][j & 1, i - j - 1]
                for c in range(j + 1, i + 1):
                    si[c - i + bw] += li * col[rho][j & 1, c - j - 1]
            if j + 1 < n and (j + 1) % nc == rho:
                store(rho, j + 1)
            if j + 1 + bw < n and (j + 1 + bw) % nc == rho:
                load(rho, j + 1 + bw)
    assert done.all()
    return out


@pytest.mark.parametrize("nc", [2, 8])
@pytest.mark.parametrize("n,bw", [(50, 7), (100, 40), (33, 32), (9, 3), (1, 0), (2, 1),
                                  (70, 69), (160, 100)])
def test_cluster_band_cholesky_scheme(nc, n, bw):
    a = banded_spd(n, bw, np.random.default_rng(7 * n + bw + nc))
    out = cluster_cholesky(a, bw, nc)
    l = np.linalg.cholesky(a)
    w = bw + 1
    for i in range(n):
        for c in range(max(0, i - bw), i + 1):
            assert abs(out[i * w + (c - i + bw)] - l[i, c]) < 1e-11, (i, c)
