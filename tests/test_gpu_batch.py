"""Batches of samplers (one launch per stage for all members) against the same
samplers stepped alone.

A member's blocks, tiles, partial sums and reduction order do not depend on
the batch, so every result -- particles, log-weights, log-targets, the
per-iteration statistics and the means of eq. (7) -- must equal the solo run's
bit for bit, for every launch-shape variant and after the autotuner has run.
Solo FP32 runs are themselves checked against the FP64 oracle in
test_gpu_parity.py; one member here is checked against it too.
"""
import numpy as np
import pytest
import torch

from paper_1905_10252_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_1905_10252_gb300 import build, native

    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    native.lib()
    return native


# ragged sizes (one row, part tiles, several tiles), every D class of the FP32
# kernels, both resampling rules
SHAPES = [(1, 2, 0), (1000, 2, 0), (4095, 8, 1), (4097, 5, 0), (20000, 32, 0), (70001, 16, 1), (3, 32, 1),
          (12289, 17, 0), (8192, 8, 0), (65536, 2, 1)]


def make(nat, shapes, seed0=100):
    out = []
    for j, (n, d, mode) in enumerate(shapes):
        mu, sig = inputs.gaussian_target(d, seed=seed0 + j)
        out.append(nat.Sampler(n, d, dtype=torch.float32, seed=seed0 + j, mu=mu, sigma=sig, step=0.5,
                               init_scale=2.0, resample_mode=mode))
    return out


def state(nat, s):
    x, lp = s.current()
    return (x.cpu().numpy().copy(), lp.cpu().numpy().copy(), s.logw.cpu().numpy().copy(), s.stats())


def assert_same(a, b, tag=""):
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u.view(np.uint8), v.view(np.uint8)), tag
    assert a[3] == b[3], tag


def solo_runs(nat, shapes, k):
    solo = make(nat, shapes)
    res = [s.step(k, trace=True, fhat=True) for s in solo]
    torch.cuda.synchronize()
    return solo, res


def test_batch_equals_solo(nat):
    K = 6
    solo, sres = solo_runs(nat, SHAPES, K)
    mem = make(nat, SHAPES)
    b = nat.Batch(mem)
    bres = b.step(K, trace=True, fhat=True)
    b.sync()
    torch.cuda.synchronize()
    for j in range(len(SHAPES)):
        assert_same(state(nat, solo[j]), state(nat, mem[j]), SHAPES[j])
        assert torch.equal(sres[j]["mean"], bres["mean"][j]), SHAPES[j]
        assert torch.equal(sres[j]["trace"], bres["trace"][j]), SHAPES[j]
        assert torch.equal(sres[j]["fhat"], bres["fhat"][j]), SHAPES[j]
    # a second call continues both the same way (trace restarts at the call)
    r2 = b.step(3, trace=True)
    b.sync()
    for j, s in enumerate(solo):
        t2 = s.step(3, trace=True)
        torch.cuda.synchronize()
        assert torch.equal(t2["trace"], r2["trace"][j])
        assert_same(state(nat, s), state(nat, mem[j]))
    b.close()


@pytest.mark.parametrize("mv,cv", [(0, 0), (1, 2), (3, 1), (4, 0), (4, 2)])
def test_batch_variants_do_not_change_results(nat, mv, cv):
    shapes = SHAPES[:6]
    K = 4
    solo, _ = solo_runs(nat, shapes, K)
    mem = make(nat, shapes)
    b = nat.Batch(mem)
    b.set_variant(mv, cv)
    b.step(K)
    b.sync()
    for j in range(len(shapes)):
        assert_same(state(nat, solo[j]), state(nat, mem[j]), (mv, cv, shapes[j]))
    b.close()


def test_tuner_leaves_state_untouched(nat):
    shapes = SHAPES
    K = 5
    solo, _ = solo_runs(nat, shapes, K)
    mem = make(nat, shapes)
    b = nat.Batch(mem)
    b.step(2)
    mv, cv = b.tune(reps=2)
    assert 0 <= mv < nat.BATCH_MOVE_VARIANTS and 0 <= cv < nat.BATCH_COPY_VARIANTS
    b.step(K - 2)
    b.sync()
    for j in range(len(shapes)):
        assert_same(state(nat, solo[j]), state(nat, mem[j]), shapes[j])
    b.close()


def test_batch_member_against_oracle(nat, orc):
    """One iteration of a mixed batch against the FP64 oracle: the member
    without resampling keeps its moved particles, whose coordinates, log pi,
    log-weights (eq. 5), LSE and mean (eq. 7) are checked with the FP32
    tolerances of the solo tests; the resampling member's copy counts are
    checked bit-exactly on its pre-resampling weights."""
    shapes = [(3000, 4, nat.RESAMPLE_NEVER), (50000, 8, 1), (777, 32, nat.RESAMPLE_ALWAYS)]
    mem = make(nat, shapes, seed0=7)
    pre = [[t.cpu().numpy().copy() for t in m.current()] + [m.logw.cpu().numpy().copy()] for m in mem]
    b = nat.Batch(mem)
    r = b.step(1, trace=True)
    b.sync()
    # member 0: move + reweight only
    n, d, _ = shapes[0]
    mu, sig = inputs.gaussian_target(d, seed=7)
    tgt = orc.Target.gauss(mu, sig)
    x0g, lp0g, lw0g = pre[0]
    x1g, lp1g = [t.cpu().numpy() for t in mem[0].current()]
    lw1g = mem[0].logw.cpu().numpy()
    x1 = orc.move(x0g.astype(np.float64), 7, 1, 0.5, ubits=24)
    assert np.all(np.abs(x1g - x1) <= 4e-6 * (1 + np.abs(x1)))
    lp_ref = tgt.logpi(x1g.astype(np.float64))
    assert np.all(np.abs(lp1g - lp_ref) <= 2e-5 * (1 + np.abs(lp_ref)))
    np.testing.assert_array_equal(lw1g, lw0g + (lp1g - lp0g).astype(np.float64))
    m, lse, ess = orc.lse_ess(lw1g)
    tr = nat.trace_dicts(r["trace"][0])[0]
    assert tr["max_logw"] == m and abs(tr["lse"] - lse) <= 1e-10 and tr["resampled"] == 0
    mref, _ = orc.estimate(x1g.astype(np.float64), lw1g, lse, with_cov=False)
    np.testing.assert_allclose(r["mean"][0].cpu().numpy(), mref, rtol=0, atol=2e-5 * (1 + np.abs(mref).max()))
    # member 2: resampled; its survivors count equals the oracle's copy counts'
    n2, d2, _ = shapes[2]
    tr2 = nat.trace_dicts(r["trace"][2])[0]
    assert tr2["resampled"] == 1
    x0g2, lp0g2, lw0g2 = pre[2]
    x12 = orc.move(x0g2.astype(np.float64), 9, 1, 0.5, ubits=24)
    xg2 = mem[2].current()[0].cpu().numpy()
    # every output row is one of the moved rows (within the FP32 move tolerance)
    diff = np.abs(xg2[:, None, :] - x12[None, :, :]).max(axis=2).min(axis=1)
    assert np.all(diff <= 4e-6 * (1 + np.abs(x12).max()))
    b.close()


def test_batch_rejects_bad_members(nat):
    mu, sig = inputs.gaussian_target(4, seed=1)
    a = nat.Sampler(100, 4, dtype=torch.float32, seed=1, mu=mu, sigma=sig)
    f64 = nat.Sampler(100, 4, dtype=torch.float64, seed=1, mu=mu, sigma=sig)
    with pytest.raises(nat.SmcError) as e:
        nat.Batch([a, f64])
    assert e.value.code == nat.SMC_EINVAL
    with pytest.raises(nat.SmcError) as e:
        nat.Batch([a, a])
    assert e.value.code == nat.SMC_EINVAL
    b = nat.Batch([a])
    with pytest.raises(nat.SmcError):
        b.set_variant(nat.BATCH_MOVE_VARIANTS, 0)
    b.close()


def test_batch_shapes_workload(nat):
    """The batched workload's shape mix (N log-uniform in [2^10, 2^18], D in
    {2, 8, 32}) at a reduced count: batch equals solo."""
    shapes = [(n, d, 0) for n, d in inputs.batch_shapes(24, seed=3)]
    K = 3
    solo, sres = solo_runs(nat, shapes, K)
    mem = make(nat, shapes)
    b = nat.Batch(mem)
    b.tune(reps=2)
    bres = b.step(K)
    b.sync()
    for j in range(len(shapes)):
        assert torch.equal(sres[j]["mean"], bres["mean"][j]), shapes[j]
        assert_same(state(nat, solo[j]), state(nat, mem[j]), shapes[j])
    b.close()
