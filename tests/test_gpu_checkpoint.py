"""Checkpoint / resume: a sampler saved after K1 iterations and restored into
a fresh handle continues bit for bit as the uninterrupted run.

The random numbers of Algorithm 2 are Philox draws keyed by (seed, t,
particle), so the whole future of a run is a function of the particles, log
pi, log w and the device state block (t, LSE_{t-1}, the recycling sums of
eq. (6)) -- exactly what a checkpoint holds.  Every target and both
precisions; the tensor-core logistic likelihood included.
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


def gauss(d, seed):
    mu, sig = inputs.gaussian_target(d, seed=seed)
    return dict(target="gauss", mu=mu, sigma=sig)


X_LG, Y_LG, _ = inputs.logistic_data(1000, 8, seed=5)

CASES = {
    "gauss-f32-d16": (50000, 16, torch.float32, gauss(16, 1)),
    "gauss-f64-d4": (3000, 4, torch.float64, gauss(4, 2)),
    "gauss-f32-d32-ragged": (4097, 32, torch.float32, gauss(32, 3)),
    "student-f64": (5000, 1, torch.float64, dict(target="student_t", mu=[0.5], nu=5.0)),
    "logistic-f32-tc": (4096, 8, torch.float32, dict(target="logistic", X=X_LG, y=Y_LG, prior_var=4.0)),
    "logistic-f64": (1024, 8, torch.float64, dict(target="logistic", X=X_LG, y=Y_LG, prior_var=4.0)),
}


def make(nat, case, seed=11):
    n, d, dtype, kw = CASES[case]
    return nat.Sampler(n, d, dtype=dtype, seed=seed, step=0.5, init_scale=2.0, **kw)


def bits(t):
    return t.detach().cpu().contiguous().view(torch.uint8).numpy()


def snapshot(s, r):
    x, lp = s.current()
    out = {"x": bits(x), "logpi": bits(lp), "logw": bits(s.logw)}
    for k in ("mean", "trace", "fhat"):
        out[k] = bits(r[k])
    return out


def assert_same(a, b, tag):
    for k in a:
        assert np.array_equal(a[k], b[k]), (tag, k)


@pytest.mark.parametrize("case", list(CASES))
def test_restore_continues_bit_for_bit(nat, case):
    K1, K2 = 4, 5
    # uninterrupted run
    ref = make(nat, case)
    ref.step(K1)
    r_ref = ref.step(K2, trace=True, fhat=True)
    ref.sync()
    want = snapshot(ref, r_ref)
    # run, save, continue in the same handle
    a = make(nat, case)
    a.step(K1)
    blob = a.checkpoint()
    r_a = a.step(K2, trace=True, fhat=True)
    a.sync()
    assert_same(want, snapshot(a, r_a), case + " saved and continued")
    # a fresh handle (its own buffers, its own init) restored from the blob
    b = make(nat, case)
    b.step(2)  # state that the restore must overwrite completely
    b.restore(blob)
    r_b = b.step(K2, trace=True, fhat=True)
    b.sync()
    assert_same(want, snapshot(b, r_b), case + " restored")
    assert int(nat.trace_dicts(r_b["trace"])[0]["t"]) == K1 + 1


def test_checkpoint_size_and_header(nat):
    s = make(nat, "gauss-f32-d16")
    blob = s.checkpoint()
    n, d = CASES["gauss-f32-d16"][:2]
    assert blob[:8] == b"SMCCKPT1"
    assert len(blob) > n * (4 * d + 4 + 8)
    # the particle block right after the header and state block is x itself
    x, _ = s.current()
    xb = bits(x).tobytes()
    assert xb in blob


def test_restore_refuses_other_configurations(nat):
    blob = make(nat, "gauss-f32-d16").checkpoint()
    n, d, dtype, kw = CASES["gauss-f32-d16"]
    others = [
        nat.Sampler(n, d, dtype=dtype, seed=12, **kw),  # another seed
        nat.Sampler(n + 1, d, dtype=dtype, seed=11, **kw),  # another N
        nat.Sampler(n, d, dtype=torch.float64, seed=11, **kw),  # another dtype
    ]
    for o in others:
        o.step(2)
        o.sync()
        with pytest.raises(nat.SmcError) as e:
            o.restore(blob)
        assert e.value.code == nat.SMC_EINVAL
        # untouched and still usable
        o.step(1)
        o.sync()
    s = make(nat, "gauss-f32-d16")
    with pytest.raises(nat.SmcError):
        s.restore(b"\0" * len(blob))  # no magic
    with pytest.raises(nat.SmcError):
        s.restore(blob[: len(blob) // 2])  # truncated
    s.step(1)
    s.sync()


def test_restored_sampler_joins_a_batch(nat):
    """A restored sampler is an ordinary handle: batched with others it gives
    the same bits as stepped alone."""
    K1, K2 = 3, 4
    a = make(nat, "gauss-f32-d16")
    a.step(K1)
    blob = a.checkpoint()
    solo = a.step(K2, trace=True)
    a.sync()
    b = make(nat, "gauss-f32-d16")
    b.restore(blob)
    other = nat.Sampler(2000, 4, dtype=torch.float32, seed=3, **gauss(4, 9))
    bt = nat.Batch([b, other])
    r = bt.step(K2, trace=True)
    bt.sync()
    assert torch.equal(solo["trace"], r["trace"][0])
    assert torch.equal(solo["mean"], r["mean"][0])
    xa, _ = a.current()
    xb, _ = b.current()
    assert np.array_equal(bits(xa), bits(xb))
    bt.close()
