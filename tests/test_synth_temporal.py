"""The array-based temporal preferential-attachment stream (the full-size
temporal workload's generator) against a step-by-step simulation of the same
model on the same random choices, plus its structural invariants."""
import numpy as np

import synth


def sequential(n, steps, p_repeat, seed, vertex_weight=None):
    """The model one step at a time, with the urn as an explicit list."""
    src_direct, repeat, s_rep, r, arrived, delta = synth._temporal_draws(n, steps, p_repeat, seed, vertex_weight)
    src = np.zeros(steps, np.int64)
    dst = np.zeros(steps, np.int64)
    for t in range(steps):
        if repeat[t]:
            src[t], dst[t] = src[s_rep[t]], dst[s_rep[t]]
            continue
        src[t] = src_direct[t]
        x = int(r[t])
        if x < delta * arrived[t]:
            dst[t] = x // delta
        else:
            e = x - delta * int(arrived[t])        # endpoint e % 2 of step e // 2
            dst[t] = src[e // 2] if e % 2 == 0 else dst[e // 2]
    return src, dst


def test_matches_step_by_step_model():
    for n, steps, p, seed, vw in [(300, 6000, 0.3, 1, None), (50, 4000, 0.5, 2, 1), (1000, 3000, 0.0, 3, 7)]:
        s, d = synth.temporal_pa_stream_vec(n, steps, p, seed, vw)
        rs, rd = sequential(n, steps, p, seed, vw)
        assert np.array_equal(s, rs) and np.array_equal(d, rd)


def test_invariants():
    n, steps = 2000, 60000
    s, d = synth.temporal_pa_stream_vec(n, steps, 0.3, 9)
    s2, d2 = synth.temporal_pa_stream_vec(n, steps, 0.3, 9)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)          # seeded
    assert s.max() < n and d.max() < n
    gap = steps // n
    first = np.full(n, steps)
    np.minimum.at(first, s, np.arange(steps))
    np.minimum.at(first, d, np.arange(steps))
    assert np.all(first >= np.maximum(0, np.arange(n) - 1) * gap)   # nobody before arrival
    assert np.all(first < steps)                                     # everyone interacts
    key = (np.minimum(s, d).astype(np.uint64) << np.uint64(32)) | np.maximum(s, d)
    repeated = 1 - np.unique(key).size / steps
    assert 0.25 < repeated < 0.45                                    # ~30% repeats plus collisions
    deg = np.bincount(np.concatenate([s, d]).astype(np.int64), minlength=n)
    assert deg.max() > 20 * deg.mean() and deg.max() < 0.05 * 2 * steps  # heavy tail, no condensation


def test_window_batches_keep_the_window_graph():
    """Applying a window batch to the graph of interactions [start, end)
    gives the graph of [start + size, end + size): every deletion removes
    weight that is present."""
    n, steps = 500, 20000
    s, d = synth.temporal_pa_stream_vec(n, steps, 0.3, 4)
    start, end = 0, 15000

    def as_dict(g):
        return {(int(u), int(v)): int(w) for u, v, w in zip(g.u, g.v, g.w)}

    cur = as_dict(synth.temporal_edges(s[start:end], d[start:end], n))
    for size in (30, 300, 1000):
        dels, ins = synth.window_batch(s, d, start, end, size)
        for u, v, w in dels:
            key = (min(u, v), max(u, v))
            assert cur.get(key, 0) >= w
            cur[key] -= int(w)
            if cur[key] == 0:
                del cur[key]
        for u, v, w in ins:
            key = (int(min(u, v)), int(max(u, v)))
            cur[key] = cur.get(key, 0) + int(w)
        start += size
        end += size
        assert cur == as_dict(synth.temporal_edges(s[start:end], d[start:end], n))
