"""Host-side model of the pipelined Parareal schedule (Sec. II-C, Eq. 12).

The banded Parareal driver overlaps iteration k's coarse sweep with the fine
propagation of iteration k + 1: the slices are cut into chunks, each fine
chunk runs on a stream of its own behind an event of the sweep chunk it
needs, and the sweep chunks run on the main stream behind the events of the
fine chunks they consume.  Slice starts U, fine ends E and the per-slice QoI
partials Q are double-buffered by iteration parity, and one iteration is
enqueued ahead of the host's stopping decision, then cancelled.

This model enqueues the same operations, streams and event waits as the
driver (run_parareal_pipelined), builds the happens-before graph that CUDA
stream and event semantics give them, and checks
  * no two operations that may run at the same time touch a buffer element
    that one of them writes, and
  * in an execution order the graph allows, every read sees the value the
    serial Parareal iteration defines (the version of U, E, G or Q of the
    right iteration and slice), including the final state and the per-slice
    QoI partials read after the cancelled iteration has run.
"""
import itertools

import pytest


class Graph:
    def __init__(self):
        self.ops = []          # (name, reads, writes)
        self.preds = []        # direct predecessors (op indices)
        self.last_on = {}      # stream -> last op index
        self.event_src = {}    # event -> op index recorded after (or None)

    def op(self, stream, name, steps=(), waits=()):
        """steps: [(reads, writes)] in the order one launch performs them."""
        i = len(self.ops)
        pre = set()
        if stream in self.last_on:
            pre.add(self.last_on[stream])
        for ev in waits:
            src = self.event_src.get(ev)
            if src is not None:
                pre.add(src)
        self.ops.append((name, [(list(r), list(w)) for r, w in steps]))
        self.preds.append(pre)
        self.last_on[stream] = i
        return i

    def record(self, ev, stream):
        self.event_src[ev] = self.last_on.get(stream)

    def reach(self):
        """reach[i] = bitset of ops that happen before op i."""
        r = []
        for i, pre in enumerate(self.preds):
            b = 0
            for p in pre:
                b |= r[p] | (1 << p)
            r.append(b)
        return r


def build_schedule(M, K, max_iters):
    """Enqueue the driver's operations for M slices when iteration K meets the
    stopping rule; returns the graph and the iterations enqueued."""
    cs = max(1, M // 16)
    J = (M + cs - 1) // cs
    g = Graph()
    g.op("main", "setup", [([], [("U", p, s) for p in (0, 1) for s in range(M)]
                            + [("Q", p, s) for p in (0, 1) for s in range(M)])])
    g.record("fork", "main")
    for j in range(J):
        g.op(("fine", j), "fork-wait", waits=["fork"])

    def sweep(k):
        pk = k & 1
        s_first = 0 if k == 0 else k - 1
        for j in range(J):
            lo, hi = max(j * cs, s_first), min((j + 1) * cs, M - 1)
            steps = []
            for s in range(lo, hi):
                reads = [("U", pk ^ 1 if s == s_first else pk, s, "start", k),
                         ("U", pk ^ 1, s + 1, "prev", k)]
                if k > 0:
                    reads += [("E", pk, s, "fine", k), ("G", s, "old", k)]
                steps.append((reads, [("U", pk, s + 1), ("G", s), ("J", k, s + 1),
                                      ("N", k, s + 1)]))
            waits = [("ev_fine", pk, j)] if k > 0 else []
            g.op("main", ("sweep", k, j), steps, waits)
            g.record(("ev_sweep", pk, j), "main")

    def fine(k):
        pk = k & 1
        for j in range(J):
            lo, hi = max(j * cs, k - 1), min((j + 1) * cs, M)
            steps = [([("U", pk ^ 1, s, "fstart", k)], [("E", pk, s), ("Q", pk, s)])
                     for s in range(lo, hi)]
            g.op(("fine", j), ("fine", k, j), steps, [("ev_sweep", pk ^ 1, j)])
            g.record(("ev_fine", pk, j), ("fine", j))

    sweep(0)
    fine(1)
    sweep(1)
    enq = 1
    for k in range(1, max_iters + 1):
        if k + 1 <= max_iters and k < M:
            fine(k + 1)
            sweep(k + 1)
            enq = k + 1
        if k == K:
            break
    for j in range(J):                                   # join the fine streams
        g.record(("fjoin", j), ("fine", j))
    g.op("main", "final",
         [([("E", K & 1, M - 1, "final", K)]
           + [("Q", min(K, s + 1) & 1, s, "qfinal", K) for s in range(M)], [])],
         waits=[("fjoin", j) for j in range(J)])
    return g, enq


def _loc(a):
    return a[:3] if a[0] in ("U", "E", "Q", "J", "N") else a[:2]


def expected(read, M):
    """The version the serial iteration defines for a read."""
    kind = read[0]
    if kind == "U":
        _, _, s, why, k = read
        if why == "start":          # U^k[s] of the sweep of iteration k
            it = k
        elif why == "prev":         # U^{k-1}[s] (jump), zero before iteration 0
            it = k - 1
        else:                       # "fstart": the fine start U^{k-1}[s]
            it = k - 1
        if it < 0 or s == 0:
            return ("zero",)
        return ("U", min(it, s), s)  # U[s] is last written in iteration min(it, s)
    if kind == "E":
        _, _, s, why, k = read
        return ("E", k, s)
    if kind == "G":
        _, s, _, k = read
        return ("G", k - 1, s)
    if kind == "Q":
        _, _, s, _, K = read
        return ("Q", min(K, s + 1), s)
    raise AssertionError(read)


def run_checks(M, K, max_iters):
    g, enq = build_schedule(M, K, max_iters)
    reach = g.reach()
    n = len(g.ops)
    # (1) operations without a happens-before edge may overlap: no conflicts
    touched = {}
    for i, (_, steps) in enumerate(g.ops):
        for reads, writes in steps:
            for w in writes:
                touched.setdefault(_loc(w), []).append((i, True))
            for r in reads:
                touched.setdefault(_loc(r), []).append((i, False))
    for loc, acc in touched.items():
        ws = [i for i, w in acc if w]
        for i in ws:
            for j, _ in acc:
                if i == j:
                    continue
                ordered = (reach[i] >> j) & 1 or (reach[j] >> i) & 1
                assert ordered, (loc, g.ops[i][0], g.ops[j][0])
    # (2) one execution order the graph allows (all orders agree by (1)):
    # iterations beyond K were cancelled and write invalid values
    mem = {}
    for i in range(n):
        name, steps = g.ops[i]
        cancelled = isinstance(name, tuple) and name[1] > K
        for reads, writes in steps:
            for r in reads:   # a cancelled operation's results are discarded
                got = mem.get(_loc(r), ("zero",))
                assert cancelled or got == expected(r, M), (name, r, got)
            for w in writes:
                if name == "setup":
                    mem[_loc(w)] = ("zero",)
                elif cancelled:
                    mem[_loc(w)] = ("cancelled",)
                elif w[0] == "G":
                    mem[_loc(w)] = ("G", name[1], w[1])
                else:
                    mem[_loc(w)] = (w[0], name[1], w[2])
    return enq


@pytest.mark.parametrize("M", [2, 3, 8, 16, 20, 64])
def test_pipelined_schedule_is_race_free_and_matches_the_serial_iteration(M):
    for K in sorted({1, 2, 3, M // 2, M - 1, M} - {0}):
        if K > M:
            continue
        enq = run_checks(M, K, M)
        assert enq == min(K + 1, M)   # one iteration enqueued ahead, then cancelled


def test_iteration_limit_below_the_slice_count():
    for M, mx in itertools.product([8, 64], [1, 2, 5]):
        for K in range(1, mx + 1):
            assert run_checks(M, K, mx) == min(K + 1, mx)


def test_model_detects_a_missing_wait():
    """The same model with the fine chunks' wait on the sweep event removed
    must report a conflict (the check is not vacuous)."""
    orig = Graph.op

    def no_fine_wait(self, stream, name, steps=(), waits=()):
        if isinstance(name, tuple) and name[0] == "fine":
            waits = ()
        return orig(self, stream, name, steps, waits)

    Graph.op = no_fine_wait
    try:
        with pytest.raises(AssertionError):
            run_checks(16, 3, 16)
    finally:
        Graph.op = orig


def test_model_detects_single_buffered_fine_ends():
    """Fine ends written to one buffer for every iteration (no parity): the
    speculative iteration overwrites the values the final read needs, or a
    fine chunk races a sweep chunk; the model must report it."""
    orig = Graph.op

    def one_buffer(self, stream, name, steps=(), waits=()):
        fix = lambda a: (a[0], 0) + tuple(a[2:]) if a[0] == "E" else a
        steps = [([fix(r) for r in rd], [fix(w) for w in wr]) for rd, wr in steps]
        return orig(self, stream, name, steps, waits)

    Graph.op = one_buffer
    try:
        with pytest.raises(AssertionError):
            run_checks(16, 3, 16)
    finally:
        Graph.op = orig
