"""The run-start rules of the stamped copy-count scan (the stateless
redistribute calls), restated on the host and checked against Algorithm 5
itself (the oracle's stable repeat of index rows).

The stateless calls do not clear their run-start array.  After the block
sums and their prefixes, block b of 4096 counts owns the output
window [w0, w0 + total) (windows are disjoint and tile [0, N)).  A window of
at most 8192 rows is written whole (-1, then the block's run starts); a
larger one writes -1 over its part of its two edge copy tiles and of every
copy tile where it puts a run start, then its run starts.  Every copy tile of
2048 rows that receives a run start is stamped.  (A window of up to 2^17
rows is set to -1 whole; the tile rule is also checked with that threshold
at 0 and a small tile queue, so both branches are exercised.)  The copy
kernel reads the run starts of stamped tiles only (an unstamped tile means -1 throughout),
max-scans them from the source of the tile's first row, and so must find
only run starts of this call in every slice it reads -- whatever the array
held before (here: stale garbage)."""
import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs

QTILE, RTILE, WIN = 4096, 2048, 8192


def stamped_sources(nc, rng, fill_all=1 << 17, max_tiles=128):
    n = len(nc)
    nb = (n + QTILE - 1) // QTILE
    nt = (n + RTILE - 1) // RTILE
    rs = rng.integers(-5, n + 5, size=n)  # stale contents from earlier calls
    stamps = np.zeros(nt, dtype=bool)
    tile_src = rng.integers(-5, n + 5, size=nt)
    sums = [int(nc[b * QTILE:(b + 1) * QTILE].sum()) for b in range(nb)]
    prefix = np.concatenate([[0], np.cumsum(sums)[:-1]])
    for b in rng.permutation(nb):  # blocks run in any order
        w0, tot = int(prefix[b]), sums[b]
        wend = min(w0 + tot, n)
        items = range(b * QTILE, min((b + 1) * QTILE, n))
        offs, o = [], w0
        for i in items:
            offs.append(o)
            o += int(nc[i])
        fill = {w0 // RTILE, (wend - 1) // RTILE} | {off // RTILE for i, off in zip(items, offs) if nc[i] > 0}
        if tot <= fill_all or len(fill) > max_tiles:
            rs[w0:wend] = -1
        else:
            for t in fill:
                rs[max(w0, t * RTILE):min(wend, (t + 1) * RTILE)] = -1
        for i, off in zip(items, offs):
            if nc[i] > 0:
                rs[off] = i
                stamps[off // RTILE] = True
                for kb in range(-(-off // RTILE) * RTILE, min(off + int(nc[i]), n), RTILE):
                    tile_src[kb // RTILE] = i
    src = np.empty(n, dtype=np.int64)
    for t in range(nt):
        k0, k1 = t * RTILE, min((t + 1) * RTILE, n)
        sl = rs[k0:k1] if stamps[t] else np.full(k1 - k0, -1)
        mark = sl.copy()
        mark[0] = max(mark[0], tile_src[t])
        src[k0:k1] = np.clip(np.maximum.accumulate(mark), 0, n - 1)
    return src


@pytest.mark.parametrize("n", [1, 4097, 12289, 70001])
@pytest.mark.parametrize("kind", ["multinomial", "skewed", "one_hot", "ones"])
@pytest.mark.parametrize("fill_all,max_tiles", [(1 << 17, 128), (0, 128), (0, 3)])
def test_stamped_sources_equal_algorithm_5(orc, n, kind, fill_all, max_tiles):
    nc = inputs.composition(n, seed=n + 3, kind=kind)
    want = orc.redistribute(nc, np.arange(n, dtype=np.int64).reshape(n, 1)).ravel()
    got = stamped_sources(nc, np.random.default_rng(n), fill_all=fill_all, max_tiles=max_tiles)
    assert np.array_equal(got, want)


def test_stamped_sources_long_runs(orc):
    """Few survivors with runs of thousands of copies: large windows whose
    edge tiles meet other large windows."""
    n = 90001
    rng = np.random.default_rng(5)
    w = np.exp(rng.normal(0.0, 25.0, n))
    nc = rng.multinomial(n, w / w.sum()).astype(np.int32)
    assert np.count_nonzero(nc) < 60
    want = orc.redistribute(nc, np.arange(n, dtype=np.int64).reshape(n, 1)).ravel()
    for fill_all in (1 << 17, 0):
        assert np.array_equal(stamped_sources(nc, rng, fill_all=fill_all), want)
