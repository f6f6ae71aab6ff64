"""Pins of the oracle's per-level statistics.

The GPU path is compared with the oracle's level statistics bit for bit, so
these statistics need a pin of their own.  Here a short recursion written
directly from the method's steps recomputes them on small inputs:

* Sec. 2.2 / Alg. 5: sample (counter-based SplitMix64 positions, with
  replacement), sort the sample, count duplicates, choose the RMI or the
  splitter tree, the sample imbalance test;
* Sec. 2.2: homogeneity check before any sample, base case for n <= T,
  stable partition into buckets, recursion with the same model
  (REFINE_GLOBAL) or a new sample (RETRAIN);
* Sec. 2.4: splitter tree, equality buckets (final, never recursed), the
  no-progress guard (a child holding all of its parent's keys is redone with
  equality buckets; below a REFINE_GLOBAL model, where no bucket resamples,
  such a child and one past the FP64 refinement limit take a radix split of
  the bits in which its keys differ instead).

The recursion uses the oracle only for the RMI fit and its bucket function,
which have their own pins (closed form, numpy.polyfit); sampling, splitter
trees, partitioning and every count are its own.  Each level's counts must
equal the oracle's exactly, and every key must end in exactly one terminal
state (base case, depth-limit fallback, equality bucket, homogeneous item,
or a bucket of one key).
"""
import math

import numpy as np
import pytest

import datagen
import oracle

GOLD = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1
REFINE_LIMIT = 2 ** 50
FIELDS = ["items", "learned", "splitter", "splitter_eq", "homogeneous", "noprogress", "base_items", "base_keys",
          "fallback_items", "fallback_keys", "keys", "max_child", "sumsq_child", "eq_keys", "radix"]


def splitmix64(z: int) -> int:
    """Vigna's SplitMix64 output function (pinned by the published vector)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def seed_item(seed: int, segment: int, level: int, gidx: int) -> int:
    tag = ((segment << 40) + (level << 32) + (gidx & 0xFFFFFFFF)) & M64
    return splitmix64(seed ^ tag)


def np_ord(keys: np.ndarray) -> np.ndarray:
    if keys.dtype == np.uint64:
        return keys.copy()
    b = keys.view(np.uint64)
    neg = (b >> np.uint64(63)).astype(bool)
    return np.where(neg, ~b, b | np.uint64(1 << 63))


def sample_size(n: int, p) -> int:
    want = math.ceil(p.sample_rate * float(n))
    if not want < n:
        S = n
    elif want < 1:
        S = 0
    else:
        S = int(want)
    return min(max(S, p.min_sample), n)


class Model:
    """Level statistics by a direct recursion over one key array."""

    def __init__(self, p, nlevels=48):
        self.p = p
        self.lv = [dict.fromkeys(FIELDS, 0) for _ in range(nlevels)]
        self.terminal = 0  # keys that reached a final state

    def splitters(self, s_ord: np.ndarray, bs_max: int, force_eq: bool):
        S = s_ord.size
        bs = 1
        while bs * 2 <= bs_max and bs * 2 <= S and bs * 2 <= 4096:
            bs *= 2
        bs = max(bs, 2)
        t = np.array([s_ord[((k + 1) * S) // bs] for k in range(bs - 1)], dtype=np.uint64)
        if force_eq or np.any(t[1:] == t[:-1]):
            return np.unique(t), True
        return t, False

    @staticmethod
    def splitter_ids(t: np.ndarray, eq: bool, u: np.ndarray) -> np.ndarray:
        k = np.searchsorted(t, u, side="left")  # splitters strictly below u
        if not eq:
            return k.astype(np.int64)
        hit = (k < t.size) & (t[np.minimum(k, t.size - 1)] == u)
        return (2 * k + hit).astype(np.int64)

    def item(self, keys, lo, hi, level, gidx, kind, model, mk, mg):
        p = self.p
        n = hi - lo
        L = self.lv[min(level, len(self.lv) - 1)]
        x = keys[lo:hi]
        if n <= 1:
            self.terminal += n
            return
        if n <= p.basecase_threshold:
            L["base_items"] += 1
            L["base_keys"] += n
            self.terminal += n
            keys[lo:hi] = x[np.argsort(np_ord(x), kind="stable")]
            return
        if level > p.max_depth:
            L["fallback_items"] += 1
            L["fallback_keys"] += n
            self.terminal += n
            keys[lo:hi] = x[np.argsort(np_ord(x), kind="stable")]
            return
        u = np_ord(x)
        if u.min() == u.max():
            L["homogeneous"] += 1
            self.terminal += n
            return
        # the highest bit in which two keys differ, from min and max (an
        # independent route to the oracle's OR of differences)
        top = int(u.max() ^ u.min()).bit_length()
        B = p.fanout
        fresh = True
        if kind == "radix":
            fresh = False
            decision = "radix"
            s = max(mk - 10, 0)
            rnb = 1 << (mk - s) if mk > s else 2
        if kind == "refine" and B ** (mk + 1) <= REFINE_LIMIT:
            fresh = False
            decision = "learned"
        if fresh:
            S = sample_size(n, p)
            if S >= n:
                samp = x.copy()
            else:
                h = seed_item(p.seed, 0, level, gidx)
                pos = [(splitmix64((h + (j + 1) * GOLD) & M64) * n) >> 64 for j in range(S)]
                samp = x[np.array(pos, dtype=np.int64)]
            samp = samp[np.argsort(np_ord(samp), kind="stable")]
            s_ord = np_ord(samp)
            dups = int(np.sum(s_ord[1:] == s_ord[:-1]))
            model, mk, mg = None, 0, 0
            if kind == "force_splitter":
                t, eq = self.splitters(s_ord, p.splitter_fanout, True)
                decision = "splitter"
            else:
                if p.partitioner == oracle.PART_LEARNED:
                    want = True
                elif p.partitioner == oracle.PART_AUTO:
                    want = n >= p.min_learned_n and dups / S <= p.dup_frac
                else:
                    want = False
                learned = False
                if want:
                    m, ok = oracle.fit(samp, B)
                    if ok and p.partitioner == oracle.PART_AUTO:
                        sid, _ = oracle.classify(m, samp, B)
                        imb = int(np.bincount(sid.astype(np.int64), minlength=B).max())
                        ok = imb <= max(p.imbalance_tau * S / B, 16.0)
                    if ok:
                        learned, model = True, m
                if learned:
                    decision = "learned"
                else:
                    bs = p.splitter_fanout
                    if p.partitioner == oracle.PART_AUTO:
                        bs = min(bs, p.auto_splitter_fanout)
                    t, eq = self.splitters(s_ord, bs, False)
                    decision = "splitter"
        if decision == "radix":
            ids = ((u >> np.uint64(s)) & np.uint64(rnb - 1)).astype(np.int64)
            nb, eq = rnb, False
        elif decision == "learned":
            ids, _ = oracle.classify(model, x, B, mk, mg)
            ids = ids.astype(np.int64)
            nb, eq = B, False
        else:
            ids = self.splitter_ids(t, eq, u)
            nb = 2 * t.size + 1 if eq else t.size + 1
        cnt = np.bincount(ids, minlength=nb)
        assert cnt.size == nb
        order = np.argsort(ids, kind="stable")  # stable partition (Sec. 2.2)
        keys[lo:hi] = x[order]
        L["items"] += 1
        L["keys"] += n
        if decision == "learned":
            L["learned"] += 1
        elif decision == "radix":
            L["radix"] += 1
        elif eq:
            L["splitter_eq"] += 1
        else:
            L["splitter"] += 1
        L["max_child"] = max(L["max_child"], int(cnt.max()))
        L["sumsq_child"] += int(np.sum(cnt.astype(object) ** 2))
        full = np.nonzero(cnt == n)[0]
        if full.size and not (eq and full[0] % 2 == 1):
            L["noprogress"] += 1
        start = np.concatenate([[0], np.cumsum(cnt)])
        for b in range(nb):
            sz = int(cnt[b])
            if eq and b % 2 == 1:
                L["eq_keys"] += sz
                self.terminal += sz
                continue
            if sz <= 1:
                self.terminal += sz
                continue
            clo = lo + int(start[b])
            refine = decision == "learned" and p.recurse_model == oracle.RECURSE_REFINE_GLOBAL
            if decision == "radix":
                self.item(keys, clo, clo + sz, level + 1, gidx * nb + b, "radix", None, s, 0)
            elif refine and (sz == n or B ** (mk + 2) > REFINE_LIMIT):
                # no sample below a REFINE_GLOBAL model: radix split instead
                self.item(keys, clo, clo + sz, level + 1, gidx * nb + b, "radix", None, top, 0)
            elif sz == n:
                self.item(keys, clo, clo + sz, level + 1, gidx * nb + b, "force_splitter", None, 0, 0)
            elif refine:
                self.item(keys, clo, clo + sz, level + 1, gidx * nb + b, "refine", model, mk + 1, mg * B + b)
            else:
                self.item(keys, clo, clo + sz, level + 1, gidx * nb + b, "fresh", None, 0, 0)

    def run(self, x):
        keys = x.copy()
        self.item(keys, 0, x.size, 0, 0, "fresh", None, 0, 0)
        used = 0
        for i, L in enumerate(self.lv):
            if L["items"] or L["base_items"] or L["homogeneous"] or L["fallback_items"]:
                used = i + 1
        return keys, self.lv[:used]


def _inputs():
    rng = np.random.default_rng(2024)
    out = []
    dists = ["uniform01", "normal", "lognormal", "mix_gauss", "exponential", "zipf", "root_dups", "two_dups",
             "skewed_u64"]
    for i in range(240):
        n = int(rng.choice([0, 1, 2, 17, 100, 333, 1000, 2500, 5000]))
        kind = i % 12
        if kind < 9:
            x = datagen.generate(dists[kind], max(n, 1), 100 + i)[:n]
        elif kind == 9:  # a few distinct values: equality buckets, homogeneous children
            x = rng.integers(0, int(rng.choice([1, 2, 3, 7])), n).astype(np.float64)
        elif kind == 10:  # u64 with long runs of equal keys and outliers
            x = np.repeat(rng.integers(0, 2**64 - 1, max(n // 50, 1), dtype=np.uint64), 50)[:n]
            rng.shuffle(x)
        else:  # tight cluster plus far outliers (clamped model inputs)
            x = np.concatenate([1.0 + rng.random(max(n - 3, 0)) * 1e-9, [-1e300, 1e300, 0.0][:min(n, 3)]])
            rng.shuffle(x)
        p = oracle.params(
            fanout=int(rng.choice([2, 3, 16, 100, 1000])),
            splitter_fanout=int(rng.choice([2, 4, 64, 1024])),
            basecase_threshold=int(rng.choice([1, 2, 16, 64])),
            partitioner=int(rng.integers(0, 3)),
            recurse_model=int(rng.integers(0, 2)),
            sample_rate=float(rng.choice([0.01, 0.1, 1.0])),
            min_sample=int(rng.choice([2, 16, 256])),
            min_learned_n=int(rng.choice([100, 1000, 100_000])),
            max_depth=int(rng.choice([1, 2, 16])),
            seed=int(rng.integers(0, 2**63)))
        if p.fanout == 2 and p.basecase_threshold < 16:
            x = x[:600]
        out.append((i, x, p))
    return out


CASES = _inputs()


@pytest.mark.parametrize("case", range(0, len(CASES), 20))
def test_level_statistics_match_direct_recursion(case):
    for i, x, p in CASES[case:case + 20]:
        out, rc, tr, _, _ = oracle.sort(x, p)
        assert rc == 0
        m = Model(p)
        ref_keys, ref_levels = m.run(x)
        # the recursion's own output is sorted, so its partition is a permutation
        assert np.array_equal(np.sort(np_ord(ref_keys)), np_ord(ref_keys))
        assert np.array_equal(out.view(np.uint64), ref_keys.view(np.uint64)), i
        # exact key conservation: every key ends in one terminal state
        assert m.terminal == x.size, (i, m.terminal, x.size)
        assert tr.levels() == ref_levels, (i, tr.levels(), ref_levels)
        if x.size > p.basecase_threshold and ref_levels and ref_levels[0]["items"]:
            assert ref_levels[0]["keys"] == x.size and ref_levels[0]["items"] == 1


def test_level_statistics_of_a_planted_example():
    """A hand-checked case: 8 keys, T = 2, splitter tree B_s = 4 on the full
    sample.  Splitters are the sorted keys at positions 2, 4, 6 = (2, 4, 6)
    of 0..7, so the buckets are {0,1,2}, {3,4}, {5,6}, {7}: three children of
    n > T = 2 partitioned further, one child of 2 keys to the base case, one
    of 1 key final."""
    x = np.array([7.0, 3.0, 5.0, 1.0, 0.0, 6.0, 2.0, 4.0])
    p = oracle.params(partitioner=oracle.PART_SPLITTER, splitter_fanout=4, basecase_threshold=2, sample_rate=1.0,
                      min_sample=2)
    out, rc, tr, _, _ = oracle.sort(x, p)
    assert rc == 0 and np.array_equal(out, np.arange(8.0))
    lv = tr.levels()
    assert lv[0]["items"] == 1 and lv[0]["keys"] == 8 and lv[0]["splitter"] == 1
    assert lv[0]["max_child"] == 3 and lv[0]["sumsq_child"] == 9 + 4 + 4 + 1
    # level 1: {0,1,2} (3 keys) is split again; {3,4} and {5,6} are base cases
    assert lv[1]["items"] == 1 and lv[1]["keys"] == 3
    assert lv[1]["base_items"] == 2 and lv[1]["base_keys"] == 4
    assert Model(p).run(x)[1] == lv


def test_flat_model_region_takes_the_radix_split():
    """Keys the model cannot tell apart (two distinct values far beyond the
    sample range share F, the model's input being clamped to the sample's
    range) make no progress under REFINE_GLOBAL; the bucket is then split on
    the bits in which its keys differ, with no new sample, and the split
    separates the two values."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=3000), np.full(50, 1e300), np.full(50, np.nextafter(1e300, np.inf))])
    rng.shuffle(x)
    p = oracle.params(fanout=1000, basecase_threshold=4, partitioner=oracle.PART_LEARNED, sample_rate=0.1,
                      min_sample=16)
    out, rc, tr, _, _ = oracle.sort(x, p)
    assert rc == 0
    lv = tr.levels()
    assert sum(l["radix"] for l in lv) >= 1
    assert all(l["splitter"] == 0 and l["splitter_eq"] == 0 for l in lv)  # no sample below the root
    m = Model(p)
    ref, ref_levels = m.run(x)
    assert ref_levels == lv and m.terminal == x.size
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
