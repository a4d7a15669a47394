"""Race detection by repetition: every kernel of the path is deterministic by
construction (fixed reduction trees, integer prefix sums, counter-based
random numbers, covariance partials summed in block order), so identical
samplers -- run one after another, or at the same time on two streams so that
their blocks interleave differently -- must produce the same bits.  A
missing barrier, a read of a partial sum before its producer finished, or an
order-dependent floating-point atomic shows up here as a difference.  Sizes span many blocks and tiles of every kernel.
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


def bits(t):
    return t.detach().cpu().contiguous().view(torch.uint8).numpy()


def result(s, r):
    x, lp = s.current()
    return [bits(x), bits(lp), bits(s.logw), bits(r["mean"]), bits(r["trace"]), bits(r["fhat"]), bits(r["cov"])]


def same(a, b):
    return all(np.array_equal(u, v) for u, v in zip(a, b))


X_LG, Y_LG, _ = inputs.logistic_data(4096, 32, seed=21)
MU16, SIG16 = inputs.gaussian_target(16, seed=4)

CASES = {
    # 2^20 particles: 256 move blocks, 256 quantise tiles, 512 copy tiles
    "gauss-f32-d16-n2p20": lambda nat, st: nat.Sampler(1 << 20, 16, dtype=torch.float32, seed=5, mu=MU16,
                                                        sigma=SIG16, stream=st, resample_mode=nat.RESAMPLE_ALWAYS),
    "gauss-f64-d16": lambda nat, st: nat.Sampler(100003, 16, dtype=torch.float64, seed=5, mu=MU16, sigma=SIG16,
                                                 stream=st),
    # 2^15 particles x 4096 rows: 256 particle tiles on the tensor cores
    "logistic-f32-tc": lambda nat, st: nat.Sampler(1 << 15, 32, dtype=torch.float32, seed=5, target="logistic",
                                                   X=X_LG, y=Y_LG, prior_var=4.0, stream=st),
}


@pytest.mark.parametrize("case", list(CASES))
def test_repeats_and_concurrent_runs_agree(nat, case):
    K = 6
    ref = CASES[case](nat, None)
    r = ref.step(K, cov=True, trace=True, fhat=True)
    ref.sync()
    want = result(ref, r)
    del ref
    # two more, launched together on two streams
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a, b = CASES[case](nat, s1), CASES[case](nat, s2)
    ra, rb = [], []
    for _ in range(K):  # interleave the launches of the two samplers
        ra.append(a.step(1, cov=True, trace=True, fhat=True))
        rb.append(b.step(1, cov=True, trace=True, fhat=True))
    a.sync()
    b.sync()
    for s, rr in ((a, ra), (b, rb)):
        got = result(s, rr[-1])
        assert same(want[:4], got[:4]), case
        assert np.array_equal(want[4][-1], got[4][-1]), case  # the last iteration's record
        assert same(want[5:], got[5:]), case


def test_batch_repeats_agree(nat):
    shapes = inputs.batch_shapes(48, seed=3, n_min=1000, n_max=200000, dims=(2, 8, 16, 32))

    def run():
        mem = []
        for j, (n, d) in enumerate(shapes):
            mu, sig = inputs.gaussian_target(d, seed=j)
            mem.append(nat.Sampler(n, d, dtype=torch.float32, seed=j, mu=mu, sigma=sig))
        b = nat.Batch(mem)
        r = b.step(5, trace=True, fhat=True)
        b.sync()
        out = [bits(t) for t in r["mean"]] + [bits(t) for t in r["trace"]] + [bits(t) for t in r["fhat"]]
        for s in mem:
            x, _ = s.current()
            out.append(bits(x))
            out.append(bits(s.logw))
        b.close()
        return out

    first = run()
    for _ in range(2):
        assert same(first, run())
