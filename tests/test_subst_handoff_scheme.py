"""Host-side model of the warp hand-offs inside one block substitution of the
cluster stepping kernels (mqs_cluster.cu), and of the pre warps' skip of the
zero products of the triangular block inverses.

Each CTA of a cluster runs three warp roles per block round g (forward rounds
0 .. nblk-1, backward rounds nblk .. 2 nblk-1):
  * GEMV warps G(j): s of round j into the 4-slot ring s[j & 3], after the
    solved block of round j - 3 is in (wait ydone >= j - 2); release sdone = j.
  * pre warps, software pipelined: BS(j) forms B s of round j from s[j & 3]
    (wait sdone >= j; the first backward round waits ydone >= nblk instead);
    C2(g) adds the C2 term of round g (wait ydone >= g - 1 and until every
    exchange warp has its C1 product of round g - 1), writes pre[g & 1] and
    releases pdone = g, then BS(g + 1) follows.
  * exchange warps: A(g) gathers the shares of round g - 1 from V[(g-1) & 1]
    (sent by every CTA's C(g - 1)) and releases ydone = g; C(g) reads
    pre[g & 1] (wait pdone >= g) and sends its shares into every CTA's V[g & 1].
The model builds every operation of every CTA, adds an edge for program order
and for each wait, and checks on the transitive closure that every slot is
written only after the previous generation's reads and read only after its own
write -- for all interleavings the waits allow.
"""
import pytest

NX_OF = {1: 4, 2: 4, 4: 4, 8: 2}      # exchange warps per cluster size


class Model:
    def __init__(self, nblk, cl, s_slots=4, pre_slots=2, v_slots=2, ccount=True):
        self.nblk, self.cl, self.G = nblk, cl, 2 * nblk
        self.s_slots, self.pre_slots, self.v_slots = s_slots, pre_slots, v_slots
        self.ops, self.preds = [], []
        self.index = {}
        self.acc = []                  # (op, kind 'W'/'R', buffer, cta, slot, generation)
        G = self.G
        for q in range(cl):
            # GEMV warps
            prev = self.op(("Ginit", q))
            for j in (0, 1):
                if j < G and j != nblk:
                    self.acc.append((prev, "W", "s", q, j % s_slots, j))
            for j in range(2, G):
                o = self.op(("G", q, j), [prev])
                if j != nblk:
                    self.acc.append((o, "W", "s", q, j % s_slots, j))
                prev = o
            # pre warps
            prev = self.op(("BS", q, 0))
            if nblk != 0:
                self.acc.append((prev, "R", "s", q, 0, 0))
            for g in range(G):
                c2 = self.op(("C2", q, g), [prev])
                self.acc.append((c2, "W", "pre", q, g % pre_slots, g))
                prev = c2
                if g + 1 < G:
                    bs = self.op(("BS", q, g + 1), [prev])
                    if g + 1 != nblk:
                        self.acc.append((bs, "R", "s", q, (g + 1) % s_slots, g + 1))
                    prev = bs
            # exchange warps
            prev = None
            for g in range(G + 1):
                a = self.op(("A", q, g), [prev] if prev is not None else [])
                if cl > 1 and g >= 1:
                    self.acc.append((a, "R", "V", q, (g - 1) % v_slots, g - 1))
                prev = a
                if g == G:
                    break
                c = self.op(("C", q, g), [prev])
                self.acc.append((c, "R", "pre", q, g % pre_slots, g))
                if cl > 1:
                    for p in range(cl):
                        self.acc.append((c, "W", "V", p, g % v_slots, g))
                prev = c
        # waits
        for q in range(cl):
            for j in range(2, G):
                self.wait(("G", q, j), self.ydone(q, j - 2))
            for j in range(G):
                if j == nblk:
                    self.wait(("BS", q, j), self.ydone(q, nblk))
                else:
                    self.wait(("BS", q, j), self.sdone(q, j))
            for g in range(G):
                if g != nblk:
                    self.wait(("C2", q, g), self.ydone(q, g - 1))
                    if ccount and g >= 2:
                        self.wait(("C2", q, g), ("C", q, g - 1))
                self.wait(("C", q, g), ("C2", q, g))            # pdone >= g
            for g in range(1, G + 1):
                if cl > 1:
                    for p in range(cl):
                        self.wait(("A", q, g), ("C", p, g - 1))

    def op(self, key, preds=()):
        self.index[key] = len(self.ops)
        self.ops.append(key)
        self.preds.append([self.index[p] if isinstance(p, tuple) else p for p in preds])
        return self.index[key]

    def wait(self, key, on):
        if on is not None:
            self.preds[self.index[key]].append(self.index[on])

    def ydone(self, q, v):             # the release that first makes ydone >= v
        return None if v < 0 else ("A", q, v)

    def sdone(self, q, v):
        return ("Ginit", q) if v <= 1 else ("G", q, v)

    def closure(self):
        order, state = [], [0] * len(self.ops)

        def visit(u):
            stack = [(u, 0)]
            while stack:
                x, i = stack.pop()
                if i == 0:
                    if state[x] == 2:
                        continue
                    assert state[x] != 1, "cycle: the waits deadlock"
                    state[x] = 1
                if i < len(self.preds[x]):
                    stack.append((x, i + 1))
                    y = self.preds[x][i]
                    if state[y] != 2:
                        assert state[y] != 1, "cycle: the waits deadlock"
                        stack.append((y, 0))
                else:
                    state[x] = 2
                    order.append(x)

        for u in range(len(self.ops)):
            if state[u] == 0:
                visit(u)
        before = [0] * len(self.ops)   # bitset of ops that happen before
        for x in order:
            b = 0
            for y in self.preds[x]:
                b |= before[y] | (1 << y)
            before[x] = b
        return before

    def check(self):
        before = self.closure()
        hb = lambda a, b: bool(before[b] >> a & 1)
        by_slot = {}
        for o, kind, buf, cta, slot, gen in self.acc:
            by_slot.setdefault((buf, cta, slot), []).append((gen, kind, o))
        for key, accs in by_slot.items():
            writes = {}
            for gen, kind, o in accs:
                if kind == "W":
                    writes.setdefault(gen, []).append(o)
            gens = sorted(writes)
            for gen, kind, o in accs:
                if kind != "R":
                    continue
                for w in writes.get(gen, []):           # read after its write
                    assert hb(w, o), ("read before write", key, gen, self.ops[o])
                later = [g2 for g2 in gens if g2 > gen]
                if later:                               # next write after this read
                    for w in writes[later[0]]:
                        assert hb(o, w), ("overwritten before read", key, gen,
                                          self.ops[o], self.ops[w])


@pytest.mark.parametrize("cl", [1, 2, 4, 8])
@pytest.mark.parametrize("nblk", [1, 2, 3, 6])
def test_substitution_handoffs_keep_every_slot(cl, nblk):
    """The kernels' waits order every write of the s ring, the pre slots and
    the share buffers after the previous generation's reads, and every read
    after its write, and they do not deadlock."""
    Model(nblk, cl).check()


@pytest.mark.parametrize("cl", [2, 8])
def test_substitution_handoffs_without_the_priority_wait(cl):
    """The C2 term's wait for the exchange warps' C1 products orders work on
    the FP64 pipe; the slots stay safe without it."""
    Model(6, cl, ccount=False).check()


@pytest.mark.parametrize("cl,kw", [(2, {"s_slots": 2}), (2, {"pre_slots": 1}),
                                   (8, {"v_slots": 1}), (1, {"s_slots": 2}),
                                   (8, {"pre_slots": 1})])
def test_substitution_handoff_model_catches_short_buffers(cl, kw):
    """Too few slots must fail the model (the checks are not vacuous): with
    two s slots GEMV overwrites s of round j before the early B s reads it
    (three would do; the kernels keep four), C(g) and C2(g + 1) overlap on
    pre, and a CTA can send round g + 1's shares while another still reads
    round g's."""
    with pytest.raises(AssertionError):
        Model(6, cl, **kw).check()


# ---------------------------------------------------------------- triangular skip
def split(cl):
    """Pre-warp geometry of the kernels' role split: own rows R per block,
    pre warps NP with RWP rows each and LPRP lanes per row, TPP columns per lane
    (columns t = p_g + LPRP k of the CTA's R own columns)."""
    r = 64 // cl
    nx = NX_OF[cl]
    np_ = 8 if cl == 2 else nx
    rwp = 64 // np_
    lprp = 32 // rwp
    return r, np_, rwp, lprp, r // lprp


def skip_bounds(cl, q, w, forward):
    """The kernel's group bounds for pre warp w of rank q: groups k in
    [k_begin, k_end) are formed."""
    r, _, rwp, lprp, tpp = split(cl)
    r0, r1, c0 = w * rwp, w * rwp + rwp - 1, q * r
    if forward:
        return 0, (0 if r1 - c0 < 0 else (r1 - c0) // lprp + 1)
    x = r0 - c0 - lprp + 1
    return (0 if x <= 0 else (x + lprp - 1) // lprp), tpp


@pytest.mark.parametrize("cl", [1, 2, 4, 8])
def test_triangular_skip_drops_only_zero_products(cl):
    """B_b is lower triangular: the forward pre part B s touches column tc of
    row r only for tc <= r, the backward part B^T s only for tc >= r.  Every
    group a warp skips is zero for all of its lanes' rows and columns, and
    the skip removes at least the groups wholly outside the triangle."""
    r, np_, rwp, lprp, tpp = split(cl)
    kept = total = 0
    for q in range(cl):
        for w in range(np_):
            rows = range(w * rwp, w * rwp + rwp)
            for forward in (True, False):
                kb, ke = skip_bounds(cl, q, w, forward)
                for k in range(tpp):
                    cols = [q * r + pg + lprp * k for pg in range(lprp)]
                    nonzero = any((c <= row) if forward else (c >= row)
                                  for row in rows for c in cols)
                    formed = kb <= k < ke
                    assert formed or not nonzero, (cl, q, w, forward, k)
                    assert formed == nonzero, (cl, q, w, forward, k)
                    kept += formed
                    total += 1
    assert kept < total


def test_triangular_skip_bound_off_by_one_is_caught():
    """A forward bound one group too short drops nonzero products."""
    cl = 2
    r, np_, rwp, lprp, tpp = split(cl)
    caught = False
    for q in range(cl):
        for w in range(np_):
            kb, ke = skip_bounds(cl, q, w, True)
            k = ke - 1
            if 0 <= k < tpp:
                cols = [q * r + pg + lprp * k for pg in range(lprp)]
                rows = range(w * rwp, w * rwp + rwp)
                caught |= any(c <= row for row in rows for c in cols)
    assert caught
