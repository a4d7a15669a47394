"""The largest N the boundary accepts (2^31 - 1 particles, a ragged last tile
in every kernel): systematic resampling, redistribute and S-NS, checked in
full against their definitions (the oracle itself would take minutes at this
size).

  * eq. (9): the copy counts are non-negative and sum to N exactly;
  * Algorithm 5: the redistributed rows are the stable repeat of the input
    rows by the copy counts (rows hold their own index: the output must be
    non-decreasing and hold index i exactly ncopies_i times);
  * Algorithm 8: zero keys keep their order at the left end, positive keys
    appear in reverse order at the right end.

About 90 GB of device memory; skipped on smaller devices.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu

N_MAX = 2 ** 31 - 1


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10252_gb300 import build, native

    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    if torch.cuda.get_device_properties(0).total_memory < 150 * 2 ** 30:
        pytest.skip("needs ~90 GB of device memory")
    native.lib()
    return native


def test_resample_redistribute_nearly_sort_at_max_n(nat):
    n = N_MAX
    g = torch.Generator(device="cuda").manual_seed(5)
    logw = torch.randn(n, dtype=torch.float64, device="cuda", generator=g).mul_(2.0)
    ws = torch.empty(nat.smc_redistribute_ws_bytes(n), dtype=torch.uint8, device="cuda")
    nc, stats = nat.smc_resample_raw(logw, seed=3, t=1, mode=nat.RESAMPLE_ALWAYS, ws=ws)
    assert nat.smc_ws_status(ws) == nat.SMC_OK
    del logw
    torch.cuda.empty_cache()
    assert int(nc.min()) >= 0
    assert int(nc.sum(dtype=torch.int64)) == n
    survivors = int((nc > 0).sum())
    assert 0 < survivors < n
    rec = nat.decode_stats(stats)
    assert rec["resampled"] == 1 and rec["t"] == 1

    # Algorithm 5 on rows that carry their own index: the output is the
    # stable repeat iff it is non-decreasing and index i occurs nc[i] times
    rows = torch.arange(n, dtype=torch.int32, device="cuda").view(n, 1)
    out = nat.smc_redistribute_raw(nc, rows, ws=ws).view(-1)
    assert nat.smc_ws_status(ws) == nat.SMC_OK
    del ws
    assert bool((out[1:] >= out[:-1]).all())
    counts = torch.bincount(out.long(), minlength=n)
    assert torch.equal(counts, nc.long())
    del out, counts
    torch.cuda.empty_cache()

    # Algorithm 8 on the same keys and rows: the left part is a strictly
    # increasing run of the zero-key indices (there are n - m of them, so it
    # is all of them in order), the right part a strictly decreasing run of
    # the positive-key indices
    keys, srows = nat.smc_nearly_sort_raw(nc, rows)
    srows = srows.view(-1)
    m = survivors
    assert bool((keys[: n - m] == 0).all()) and bool((keys[n - m:] > 0).all())
    left, right = srows[: n - m], srows[n - m:]
    assert bool((left[1:] > left[:-1]).all()) and bool((nc[left.long()] == 0).all())
    assert bool((right[1:] < right[:-1]).all())
    assert torch.equal(keys[n - m:], nc[right.long()])


def test_sampler_iteration_at_max_n(nat):
    """A whole iteration of an FP32 sampler (D = 1, Gaussian target) at
    N = 2^31 - 1: eq. (9)'s copies land every particle somewhere, the
    log-weights are reset to -log N, and the estimate of eq. (7) is finite
    and near the target mean."""
    import math

    n = N_MAX
    s = nat.Sampler(n, 1, dtype=torch.float32, seed=4, mu=[0.7], sigma=[[1.5]], step=0.5, init_scale=2.0,
                    resample_mode=nat.RESAMPLE_ALWAYS)
    r = s.step(2, trace=True)
    s.sync()
    tr = nat.trace_dicts(r["trace"])
    assert [t["t"] for t in tr] == [1, 2] and all(t["resampled"] == 1 for t in tr)
    assert 0 < tr[-1]["survivors"] < n
    lw0 = float(s.logw[0])
    assert abs(lw0 + math.log(n)) < 1e-12 * math.log(n)
    assert bool((s.logw == lw0).all())
    x, lp = s.current()
    assert bool(torch.isfinite(x).all()) and bool(torch.isfinite(lp).all())
    assert abs(float(r["mean"][0]) - 0.7) < 0.05
    s.close()
