"""The source-resolution procedure of the gathering move (a sampler created
with SMC_FLAG_DEFER_REDISTRIBUTE), restated on the host and checked against
Algorithm 5 itself (the oracle's stable repeat of index rows).

Row k of the resampled set is row src(k), the last survivor whose run of
copies starts at or before k.  The scan leaves rs[off_i] = i for every
survivor (-1 elsewhere) and, for every 2048-row copy tile, the source of its
first row.  A move tile of 256 rows takes that copy-tile source, raises it to
the last run start between the copy tile's first row and its own (searched
backwards 32 rows at a time), then max-scans its own run starts 32 rows at a
time.  This is the argument the GPU kernel relies on; tests/test_gpu_defer.py
checks the kernel's results bit for bit."""
import numpy as np
import pytest

from paper_1905_10252_gb300 import inputs

COPY_TILE, MOVE_TILE, CHUNK = 2048, 256, 32


def resolve_sources(nc):
    n = len(nc)
    off = np.concatenate([[0], np.cumsum(nc)[:-1]])
    surv = np.nonzero(nc)[0]
    rs = np.full(n, -1, np.int64)
    rs[off[surv]] = surv
    # the scan's copy-tile sources: for every survivor, the copy tiles whose
    # first row falls in its run [off_i, off_i + nc_i)
    tile_src = np.full((n + COPY_TILE - 1) // COPY_TILE, -1, np.int64)
    for i in surv:
        first = -(-off[i] // COPY_TILE) * COPY_TILE
        for kb in range(first, min(off[i] + nc[i], n), COPY_TILE):
            tile_src[kb // COPY_TILE] = i
    src = np.empty(n, np.int64)
    for j in range((n + MOVE_TILE - 1) // MOVE_TILE):
        k0 = j * MOVE_TILE
        t0 = (k0 // COPY_TILE) * COPY_TILE
        carry = tile_src[k0 // COPY_TILE]
        q = k0 - CHUNK
        while q >= t0:
            m = rs[q:q + CHUNK].max()
            if m >= 0:
                carry = max(carry, m)
                break
            q -= CHUNK
        for r in range(MOVE_TILE // CHUNK):
            ks = np.arange(k0 + r * CHUNK, k0 + (r + 1) * CHUNK)
            v = np.where(ks < n, rs[np.minimum(ks, n - 1)], -1)
            s = np.clip(np.maximum(np.maximum.accumulate(v), carry), 0, n - 1)
            src[ks[ks < n]] = s[ks < n]
            carry = s[-1]
    return src


@pytest.mark.parametrize("n", [1, 255, 4097, 8193, 65537, 100003])
@pytest.mark.parametrize("kind", ["multinomial", "skewed", "one_hot", "ones"])
def test_sources_equal_algorithm_5(orc, n, kind):
    nc = inputs.composition(n, seed=n + 1, kind=kind)
    want = orc.redistribute(nc, np.arange(n, dtype=np.int64).reshape(n, 1)).ravel()
    assert np.array_equal(resolve_sources(nc), want)


def test_sources_long_runs(orc):
    """A handful of survivors, runs of thousands of copies spanning copy
    tiles: most move tiles start from the copy-tile source after a long
    backward search."""
    n = 60001
    rng = np.random.default_rng(4)
    w = np.exp(rng.normal(0.0, 25.0, n))
    nc = rng.multinomial(n, w / w.sum()).astype(np.int32)
    assert np.count_nonzero(nc) < 50
    want = orc.redistribute(nc, np.arange(n, dtype=np.int64).reshape(n, 1)).ravel()
    assert np.array_equal(resolve_sources(nc), want)
