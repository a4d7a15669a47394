"""The allocation-free redistribute against the workspace redistribute and
the oracle.

smc_redistribute_raw_noalloc serves callers that cannot allocate device memory
when they call (a plug-in given only its input and output buffers, code inside
a framework whose pool owns all device memory, a real-time loop that forbids
allocation after start-up): its scratch is a fixed array inside the library.
Its output must equal smc_redistribute_raw's and the oracle's Algorithm 5
(S-R) bit for bit (the tolerance of every redistribute test: integer/byte
work is exact), call after call, since successive calls reuse the same
array; and a call must allocate no device memory.  This file is collected
last so that a run that stops at the first failure has run every other test
first.
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = [(4097, 16, np.float32, "skewed", 1), (1 << 20, 16, np.float32, "multinomial", 2),
         (1000, 4, np.float64, "one_hot", 3), (77, 3, np.float32, "ones", 4)]


def test_noalloc_matches_workspace_redistribute(nat, orc):
    # consecutive calls of different sizes and row widths, the largest at the limit
    assert max(c[0] for c in CASES) == nat.NOALLOC_MAX_N
    for n, d, dt, kind, seed in CASES:
        nc_h = inputs.composition(n, seed=seed, kind=kind)
        x_h = inputs.particles(n, d, seed=seed, dtype=dt)
        nc, x = _dev(nc_h), _dev(x_h)
        out = torch.full_like(x, float("nan"))
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        nat.smc_redistribute_raw_noalloc(nc, x, out, status=status)
        ref = nat.smc_redistribute_raw(nc, x)
        torch.cuda.synchronize()
        assert int(status.item()) == nat.SMC_OK
        assert torch.equal(out.view(torch.uint8), ref.view(torch.uint8)), (n, d, kind)
        want = orc.redistribute(nc_h, x_h)
        assert np.array_equal(out.cpu().numpy().view(np.uint8), want.view(np.uint8)), (n, d, kind)


def test_noalloc_allocates_nothing(nat):
    """Its defining property: after one warm-up call per row width (which
    loads the kernels it launches), further calls of any size leave both
    PyTorch's allocator and the driver's free-memory count unchanged."""
    bufs = []
    for n, d, dt, kind, seed in CASES:
        nc = _dev(inputs.composition(n, seed=seed + 10, kind=kind))
        x = _dev(inputs.particles(n, d, seed=seed + 10, dtype=dt))
        bufs.append((nc, x, torch.empty_like(x), torch.zeros(1, dtype=torch.int32, device="cuda")))
    for nc, x, out, status in bufs:  # warm-up
        nat.smc_redistribute_raw_noalloc(nc, x, out, status=status)
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for nc, x, out, status in bufs:
            nat.smc_redistribute_raw_noalloc(nc, x, out, status=status)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == torch_before
    assert free_after == free_before
    assert all(int(b[3].item()) == nat.SMC_OK for b in bufs)


def test_noalloc_rejects_what_it_cannot_do(nat):
    n = nat.NOALLOC_MAX_N + 1
    nc = torch.ones(n, dtype=torch.int32, device="cuda")
    x = torch.zeros(n, 4, device="cuda")
    with pytest.raises(nat.SmcError) as e:
        nat.smc_redistribute_raw_noalloc(nc, x, torch.empty_like(x))
    assert e.value.code == nat.SMC_EINVAL
    # an invalid copy-count vector writes nothing and reports SMC_EINVAL
    n = 5000
    bad = inputs.composition(n, seed=5)
    bad[0] += 1
    x = _dev(inputs.particles(n, 16, seed=5))
    out = torch.full_like(x, 7.0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    nat.smc_redistribute_raw_noalloc(_dev(bad), x, out, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == nat.SMC_EINVAL
    assert torch.all(out == 7.0)
    # and the next valid call works again on the shared scratch
    good = _dev(inputs.composition(n, seed=6))
    nat.smc_redistribute_raw_noalloc(good, x, out, status=status)
    ref = nat.smc_redistribute_raw(good, x)
    torch.cuda.synchronize()
    assert int(status.item()) == nat.SMC_OK and torch.equal(out, ref)
