"""The benchmark's own paths at its full size (N = 2^24, D = 16 FP32 rows),
checked on every row against the FP64 CPU oracle.

* The stateless resample + redistribute call: copy counts from the oracle's
  systematic resampling (Algorithm 4, line 1, exact integer CDF) of seeded
  log-weights, rows from the oracle's S-R (Algorithm 5) -- all 2^24 rows.
* The gathered copy of a sampler created with SMC_FLAG_DEFER_REDISTRIBUTE
  (the benchmark's iteration).  A resampling iteration leaves its copy
  pending: the rows it moved and the log-weights it quantised stay in the
  caller's buffers.  The oracle resamples those log-weights and repeats those
  rows (Algorithm 4, then Algorithm 5); the copy the GPU then makes must equal
  that on all 2^24 rows, whether smc_materialize completes it or the next
  move gathers it.  The rows and weights are the GPU's own (its FP32
  Box-Muller move cannot be reproduced bit for bit on the CPU); what is
  checked is the copy stage, a deterministic function of them.
* To check the gathering move's source resolution exactly on every row, a
  sampler with proposal step 0 (the move leaves every coordinate unchanged:
  x + 0 z = x) gathers the pending copy: its moved rows are then exactly the
  oracle's repeated rows.  With the benchmark's step 0.5, rows at every
  256-particle tile boundary (where the sources are resolved) and a random
  sample are checked against the oracle's move of their oracle-given source
  row, within the FP32 tolerance.
"""
import numpy as np
import pytest
import torch

from paper_1905_10252_gb300 import inputs

pytestmark = pytest.mark.gpu

N, D = 1 << 24, 16


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10252_gb300 import build, native

    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    native.lib()
    return native


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("case", ["s2", "onehot"])
def test_full_size_redistribute_raw_all_rows(nat, orc, case):
    lw = inputs.one_hot_log_weights(N, 0) if case == "onehot" else inputs.log_weights(N, 2.0, seed=0)
    nc = orc.resample(lw, 0, 1, orc.RESAMPLE_ALWAYS)["ncopies"]
    assert int(nc.sum()) == N
    x = inputs.particles(N, D, seed=1)
    ws = torch.empty(nat.smc_redistribute_ws_bytes(N), dtype=torch.uint8, device="cuda")
    out = nat.smc_redistribute_raw(torch.as_tensor(nc, device="cuda"), torch.as_tensor(x, device="cuda"), ws=ws)
    torch.cuda.synchronize()
    assert nat.smc_ws_status(ws) == nat.SMC_OK
    assert np.array_equal(host(out), orc.redistribute(nc, x))


def _deferred(nat, seed, step):
    mu, Sigma = inputs.gaussian_target(D, seed=16)
    return nat.Sampler(N, D, dtype=torch.float32, seed=seed, mu=mu, sigma=Sigma, step=step,
                       resample_mode=nat.RESAMPLE_ALWAYS, flags=nat.FLAG_DEFER_REDISTRIBUTE)


def _pending_state(S, cur):
    """The rows, log pi and log-weights of a sampler whose copy is pending
    (read from the buffers directly: smc_current would complete the copy)."""
    x = S.x if cur == 0 else S.x_alt
    lp = S.logpi if cur == 0 else S.logpi_alt
    torch.cuda.synchronize()
    return host(x).copy(), host(lp).copy(), host(S.logw).copy()


def test_full_size_deferred_copy_materialized(nat, orc):
    seed = 4
    S = _deferred(nat, seed, 0.5)
    cur0 = 0 if S.current()[0].data_ptr() == S.x.data_ptr() else 1
    S.step(1)
    x1, lp1, lw1 = _pending_state(S, cur0)
    r = orc.resample(lw1, seed, 1, orc.RESAMPLE_ALWAYS)
    S.materialize()
    x, lp = S.current()
    S.sync()
    assert np.array_equal(host(x), orc.redistribute(r["ncopies"], x1))
    assert np.array_equal(host(lp), orc.redistribute(r["ncopies"], lp1))
    assert np.all(host(S.logw) == orc.reset_logw(N))
    assert S.stats()["survivors"] == int(np.count_nonzero(r["ncopies"]))
    S.close()


def test_full_size_gathering_move_sources_exact(nat, orc):
    # step 0: the second iteration's move writes row k = row src(k) of the
    # first iteration's (pending) rows, unchanged; its log pi is the source's
    seed = 4
    S = _deferred(nat, seed, 0.0)
    cur0 = 0 if S.current()[0].data_ptr() == S.x.data_ptr() else 1
    S.step(1)
    x1, lp1, lw1 = _pending_state(S, cur0)
    nc = orc.resample(lw1, seed, 1, orc.RESAMPLE_ALWAYS)["ncopies"]
    assert 0 < np.count_nonzero(nc) < N  # a real resampling (the initial weights differ)
    S.step(1)  # gathers; its own copy is pending again, in the other buffer
    x2, lp2, lw2 = _pending_state(S, 1 - cur0)
    assert np.array_equal(x2, orc.redistribute(nc, x1))
    assert np.array_equal(lp2, orc.redistribute(nc, lp1))
    # every particle started from -log N and kept its log pi: equal weights
    assert np.all(lw2 == orc.reset_logw(N))
    S.close()


def test_full_size_gathering_move_tile_rows(nat, orc):
    # the benchmark's step: the rows where each 256-particle tile resolves its
    # sources, plus a random sample, against the oracle's move of the source
    # row the oracle's Algorithm 5 gives them
    seed, step = 4, 0.5
    S = _deferred(nat, seed, step)
    cur0 = 0 if S.current()[0].data_ptr() == S.x.data_ptr() else 1
    S.step(1)
    x1, _, lw1 = _pending_state(S, cur0)
    nc = orc.resample(lw1, seed, 1, orc.RESAMPLE_ALWAYS)["ncopies"]
    S.step(1)
    x2, _, _ = _pending_state(S, 1 - cur0)
    src = orc.redistribute(nc, np.arange(N, dtype=np.int64).reshape(N, 1)).ravel()
    tiles = np.arange(0, N, 256)
    ks = np.unique(np.concatenate([tiles, tiles + 1, tiles + 255, np.random.default_rng(3).integers(0, N, 50000)]))
    ks = ks[ks < N]
    ref = np.empty((ks.size, D))
    for j, k in enumerate(ks):
        ref[j] = x1[src[k]].astype(np.float64) + step * orc.normals(seed, 2, orc.ORC_MOVE, int(k), D, 24)
    x0 = x1[src[ks]].astype(np.float64)
    assert np.all(np.abs(x2[ks] - ref) <= 4e-6 * (1 + np.abs(x0)))
    S.close()
