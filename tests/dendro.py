"""Vectorised structure checks for large dendrograms (no linkage arithmetic).

A merge record t joins the clusters named by cids a < b in round r; the
cluster named b retires and the union keeps the name a.  A cluster merges at
most once per round, so the merges in which one cid takes part have strictly
increasing rounds, and the child of merge t on the side of cid c is the
previous merge in which c took part (none while c is still the singleton
point c).  These checks state the same invariants as the oracle's
`check_tree`, but as sorts and array comparisons, so that dendrograms of 10^7
merges are checked in seconds.
"""
import numpy as np


def children(d):
    """(child_a, child_b): for every merge, the merge index that produced each
    side, or -1 for a singleton, plus a list of problems with the round
    structure."""
    a = np.asarray(d["a"], np.int64)
    b = np.asarray(d["b"], np.int64)
    r = np.asarray(d["round"], np.int64)
    m = len(a)
    cid = np.concatenate([a, b])
    rnd = np.concatenate([r, r])
    t = np.concatenate([np.arange(m), np.arange(m)])
    order = np.lexsort((rnd, cid))  # by cid, then round
    cs, rs, ts = cid[order], rnd[order], t[order]
    same = cs[1:] == cs[:-1]
    probs = []
    bad = np.flatnonzero(same & (rs[1:] <= rs[:-1]))
    if len(bad):
        probs.append(f"cid {cs[bad[0]]} merges twice in round {rs[bad[0]]} or out of order")
    # a retired cid (side b) takes part in nothing later
    retired = order >= m
    after_b = np.flatnonzero(retired[:-1] & same)
    if len(after_b):
        probs.append(f"cid {cs[after_b[0]]} used after it retired")
    prev = np.full(2 * m, -1, np.int64)
    prev[1:][same] = ts[:-1][same]
    child = np.empty(2 * m, np.int64)
    child[order] = prev
    return child[:m], child[m:], probs


def check(d, n, rtol=1e-12):
    """Problems with a dendrogram of n points (empty when it is a valid tree
    whose heights do not decrease from child to parent beyond rtol)."""
    a = np.asarray(d["a"], np.int64)
    b = np.asarray(d["b"], np.int64)
    size = np.asarray(d["size"], np.int64)
    h = np.asarray(d["h"], np.float64)
    m = len(a)
    if m != n - 1:
        return [f"{m} merges for n={n}"]
    probs = []
    if m == 0:
        return probs
    if not (np.all(a >= 0) and np.all(a < b) and np.all(b < n)):
        probs.append("ids out of order or range")
        return probs
    ca, cb, p = children(d)
    probs += p
    if probs:
        return probs
    sa = np.where(ca >= 0, size[np.maximum(ca, 0)], 1)
    sb = np.where(cb >= 0, size[np.maximum(cb, 0)], 1)
    bad = np.flatnonzero(sa + sb != size)
    if len(bad):
        probs.append(f"merge {bad[0]}: sizes {sa[bad[0]]}+{sb[bad[0]]} != {size[bad[0]]}")
    if size.max() != n:
        probs.append(f"largest cluster has {size.max()} points, not {n}")
    for c in (ca, cb):
        k = c >= 0
        low = np.flatnonzero(h[k] < h[c[k]] * (1 - rtol) - 1e-300)
        if len(low):
            t = np.flatnonzero(k)[low[0]]
            probs.append(f"merge {t}: height {h[t]} below child height {h[c[t]]}")
    return probs


def members(d, t, ca, cb):
    """Point indices of the cluster made by merge t."""
    out, stack = [], [t]
    a, b = d["a"], d["b"]
    while stack:
        u = stack.pop()
        for cid, ch in ((a[u], ca[u]), (b[u], cb[u])):
            if ch >= 0:
                stack.append(int(ch))
            else:
                out.append(int(cid))
    return out


def sample_small(d, k, cap=64, seed=0):
    """Up to k merges whose cluster has at most cap points, with the point
    sets of their two sides: [(t, side_a, side_b)]."""
    ca, cb, probs = children(d)
    assert not probs, probs
    size = np.asarray(d["size"])
    small = np.flatnonzero(size <= cap)
    rng = np.random.default_rng(seed)
    pick = rng.choice(small, size=min(k, len(small)), replace=False)
    out = []
    for t in pick:
        sa = members(d, ca[t], ca, cb) if ca[t] >= 0 else [int(d["a"][t])]
        sb = members(d, cb[t], ca, cb) if cb[t] >= 0 else [int(d["b"][t])]
        out.append((int(t), sa, sb))
    return out


def sample_big(d, k, max_pairs):
    """The k merges with the most point pairs |A| x |B| among those with at
    most max_pairs, with the point sets of their two sides:
    [(t, side_a, side_b)]."""
    ca, cb, probs = children(d)
    assert not probs, probs
    size = np.asarray(d["size"], np.int64)
    sa = np.where(ca >= 0, size[np.maximum(ca, 0)], 1)
    sb = np.where(cb >= 0, size[np.maximum(cb, 0)], 1)
    pairs = sa * sb
    ok = np.flatnonzero(pairs <= max_pairs)
    pick = ok[np.argsort(pairs[ok], kind="stable")][-k:]
    out = []
    for t in pick:
        A = members(d, ca[t], ca, cb) if ca[t] >= 0 else [int(d["a"][t])]
        B = members(d, cb[t], ca, cb) if cb[t] >= 0 else [int(d["b"][t])]
        out.append((int(t), A, B))
    return out


def pick_merges(d, k_small, cap=32, k_big=0, big_cap=2048, every_size=False, seed=0):
    """Merges to check: k_small random ones whose cluster has at most cap
    points (any size with every_size), plus the k_big largest whose smaller
    side has at most big_cap points (every_size: the k_big last merges)."""
    size = np.asarray(d["size"])
    rng = np.random.default_rng(seed)
    pool = np.arange(len(size)) if every_size else np.flatnonzero(size <= cap)
    out = list(rng.choice(pool, size=min(k_small, len(pool)), replace=False))
    if k_big:
        ca, cb, _ = children(d)
        sa = np.where(ca >= 0, size[np.maximum(ca, 0)], 1)
        sb = np.where(cb >= 0, size[np.maximum(cb, 0)], 1)
        ok = np.ones(len(size), bool) if every_size else np.minimum(sa, sb) <= big_cap
        big = np.flatnonzero(ok)
        big = big[np.argsort(size[big], kind="stable")][-k_big:]
        out += [int(t) for t in big if t not in out]
    return [int(t) for t in out]


def rnn_check(d, X, linkage, picks, dist_to_all, rtol=1e-9, side_cap=None):
    """For every picked merge t (cids a < b, round r): among the clusters
    active when round r starts, b is a nearest neighbour of a (and a of b),
    every distance taken from the points by `dist_to_all` (the oracle's).
    Only sides of at most side_cap points are queried (None: both).

    Returns (problems, near_ties, values): a cluster closer than the partner
    by more than rtol is a problem; one within rtol and with a smaller cid is
    a near tie (its order is not decidable at this precision); values maps t
    to the partner distance seen from the first queried side."""
    a = np.asarray(d["a"], np.int64)
    b = np.asarray(d["b"], np.int64)
    r = np.asarray(d["round"], np.int64)
    n = len(X)
    order = np.argsort(r, kind="stable")
    rs = r[order]
    label = np.arange(n, dtype=np.int64)
    mp = np.arange(n, dtype=np.int64)
    cur = 0  # label holds the clusters at the start of round `cur`
    problems, ties, values = [], 0, {}
    for t in sorted(picks, key=lambda t: r[t]):
        while cur < r[t]:
            lo, hi = np.searchsorted(rs, cur), np.searchsorted(rs, cur, side="right")
            ta = a[order[lo:hi]]
            tb = b[order[lo:hi]]
            mp[tb] = ta
            label = mp[label]
            mp[tb] = tb
            cur += 1
        for q, other in ((a[t], b[t]), (b[t], a[t])):
            nq = int(np.count_nonzero(label == q))
            if nq == 0 or np.count_nonzero(label == other) == 0:
                problems.append(f"merge {t}: cid {q} or {other} not active in round {r[t]}")
                break
            if side_cap is not None and nq > side_cap:
                continue
            D = dist_to_all(linkage, X, label, q)
            dqo = D[other]
            values.setdefault(t, dqo)
            idx = np.arange(len(D))
            with np.errstate(invalid="ignore"):
                closer = np.flatnonzero((D < dqo * (1 - rtol)) & (idx != other))
                near = np.flatnonzero((np.abs(D - dqo) <= rtol * dqo) & (idx < other))
            if len(closer):
                c = int(closer[np.argmin(D[closer])])
                problems.append(f"merge {t} (round {r[t]}): cluster {c} at {D[c]!r} is closer "
                                f"to {q} than its partner {other} at {dqo!r}")
            ties += len(near)
    return problems, ties, values
