"""The Bayesian logistic-regression target on the GPU against the FP64 oracle.

FP64 samplers evaluate log pi in the oracle's order with explicitly rounded
operations; only exp and log1p come from a different library, so each term
differs by at most a few ulp:  |d log pi| <= 1e-12 (1 + |log pi|).  The moved
particles are bit-identical (same Philox draws, same FMAs).
FP32 samplers on the CUDA cores: FP32 z and softplus, FP64 row sums:
|d log pi| <= 2e-5 (1 + |log pi|), the reduced-precision bound used for the
Gaussian FP32 path.  The tensor-core likelihood (BF16 hi / lo split, FP32
accumulation) is checked in test_gpu_logistic_tc.py.
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


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("N,D,M", [(1000, 5, 300), (257, 32, 1000), (1024, 8, 257), (33, 1, 64)])
def test_logistic_fp64_stages(nat, orc, N, D, M):
    X, y, _ = inputs.logistic_data(M, D, seed=M)
    Xd, yd = X.astype(np.float64), y.astype(np.float64)
    tgt = orc.Target.logistic(Xd, yd, 4.0)
    seed, step = 11, 0.3
    S = nat.Sampler(N, D, dtype=torch.float64, seed=seed, target="logistic", X=X, y=y, prior_var=4.0,
                    step=step, resample_mode=nat.RESAMPLE_ALWAYS)
    x0g, lp0g = [host(t).copy() for t in S.current()]
    lw0g = host(S.logw).copy()
    x0, lw0, lp0 = orc.init(tgt, N, seed, 2.0)
    assert np.array_equal(x0g, x0)
    assert np.all(np.abs(lp0g - lp0) <= 1e-12 * (1 + np.abs(lp0)))
    assert np.all(np.abs(lw0g - lw0) <= 1e-12 * (1 + np.abs(lw0)))
    S.move()
    S.reweight()
    x1g, lp1g = [host(t).copy() for t in S.current()]
    lw1g = host(S.logw).copy()
    x1 = orc.move(x0g, seed, 1, step)
    assert np.array_equal(x1g, x1)
    lp1 = tgt.logpi(x1g)
    assert np.all(np.abs(lp1g - lp1) <= 1e-12 * (1 + np.abs(lp1)))
    assert np.all(np.abs(lw1g - (lw0g + (lp1 - lp0g))) <= 1e-12 * (1 + np.abs(lw1g)))
    nc, did = S.resample()
    r = orc.resample(lw1g, seed, 1, orc.RESAMPLE_ALWAYS)
    assert np.array_equal(host(nc), r["ncopies"])
    S.sync()


@pytest.mark.parametrize("N,D,M", [(2000, 5, 300), (513, 32, 700), (1024, 16, 8192)])
def test_logistic_fp32_cuda_cores(nat, orc, N, D, M):
    X, y, _ = inputs.logistic_data(M, D, seed=M + 1)
    tgt = orc.Target.logistic(X.astype(np.float64), y.astype(np.float64), 4.0)
    S = nat.Sampler(N, D, dtype=torch.float32, seed=3, target="logistic", X=X, y=y, prior_var=4.0, step=0.2,
                    flags=nat.FLAG_LOGISTIC_CUDA_CORES, resample_mode=nat.RESAMPLE_NEVER)
    x0g, lp0g = [host(t).copy() for t in S.current()]
    ref0 = tgt.logpi(x0g.astype(np.float64))
    assert np.all(np.abs(lp0g - ref0) <= 2e-5 * (1 + np.abs(ref0)))
    S.move()
    S.reweight()
    x1g, lp1g = [host(t).copy() for t in S.current()]
    ref1 = tgt.logpi(x1g.astype(np.float64))
    assert np.all(np.abs(lp1g - ref1) <= 2e-5 * (1 + np.abs(ref1)))
    S.sync()


def test_logistic_fp64_run_matches_oracle(nat, orc):
    """K = 4 iterations with resampling by N_eff: the copy counts of every
    iteration (from the quantised weights) and the final particles agree with
    the oracle's run; log-weights within the FP64 tolerance."""
    N, D, M, K = 500, 4, 200, 4
    X, y, _ = inputs.logistic_data(M, D, seed=9)
    tgt = orc.Target.logistic(X.astype(np.float64), y.astype(np.float64), 4.0)
    S = nat.Sampler(N, D, dtype=torch.float64, seed=5, target="logistic", X=X, y=y, prior_var=4.0, step=0.3,
                    init_scale=1.0)
    r = S.step(K, trace=True)
    ref = orc.run(tgt, N, 5, K, init_scale=1.0, step=0.3)
    S.sync()
    tr = nat.trace_dicts(r["trace"])
    for k in range(K):
        assert tr[k]["resampled"] == int(ref["trace"][k][4])
        assert abs(tr[k]["lse"] - ref["trace"][k][0]) <= 1e-9 * (1 + abs(ref["trace"][k][0]))
    xg = host(S.current()[0])
    assert np.array_equal(xg, ref["x"])
