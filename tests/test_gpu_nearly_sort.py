"""Sequential Nearly Sort (Algorithm 8) on the GPU against the oracle's
two-cursor loop, bit for bit: keys and rows, ragged sizes spanning several
tiles, every row width class, every key pattern the resampler produces (and
non-positive keys, which Algorithm 8 sends left), at full size too.  The N-R
local step (S-NS, then S-R on the nearly-sorted keys) matches the oracle's
composition and gives the same rows as the gather design, survivors in
reverse order."""
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


def keys(kind, n, seed=0):
    g = np.random.default_rng(seed)
    if kind == "multinomial":
        return inputs.composition(n, seed=seed)
    if kind == "one_hot":
        nc = np.zeros(n, dtype=np.int32)
        nc[g.integers(0, n)] = n
        return nc
    if kind == "ones":
        return np.ones(n, dtype=np.int32)
    if kind == "zeros":
        return np.zeros(n, dtype=np.int32)
    if kind == "signed":
        return g.integers(-3, 4, size=n).astype(np.int32)
    raise ValueError(kind)


@pytest.mark.parametrize("N", [1, 2, 7, 4095, 4096, 4097, 12289, 100003])
@pytest.mark.parametrize("kind", ["multinomial", "one_hot", "ones", "zeros", "signed"])
def test_nearly_sort_bit_exact(nat, orc, N, kind):
    nc = keys(kind, N, seed=N)
    x = np.random.default_rng(N + 1).standard_normal((N, 16)).astype(np.float32)
    k_ref, x_ref = orc.nearly_sort(nc, x)
    k, xo = nat.smc_nearly_sort_raw(torch.as_tensor(nc, device="cuda"), torch.as_tensor(x, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(k.cpu().numpy(), k_ref)
    assert np.array_equal(xo.cpu().numpy().view(np.uint32), x_ref.view(np.uint32))


@pytest.mark.parametrize("width_words", [1, 2, 3, 4, 5, 8, 32])
def test_nearly_sort_row_widths(nat, orc, width_words):
    """4-, 8- and 16-byte word paths, and row sizes that are not a multiple of
    the vector width."""
    N = 9000
    nc = keys("multinomial", N, seed=width_words)
    x = np.random.default_rng(width_words).integers(0, 2 ** 32, size=(N, width_words), dtype=np.uint32)
    k_ref, x_ref = orc.nearly_sort(nc, x)
    xi = torch.as_tensor(x.view(np.int32), device="cuda")
    k, xo = nat.smc_nearly_sort_raw(torch.as_tensor(nc, device="cuda"), xi)
    torch.cuda.synchronize()
    assert np.array_equal(k.cpu().numpy(), k_ref)
    assert np.array_equal(xo.cpu().numpy().view(np.uint32), x_ref)


@pytest.mark.parametrize("N", [5, 4097, 65553])
def test_nr_local_step(nat, orc, N):
    nc = keys("multinomial", N, seed=3)
    x = np.random.default_rng(7).standard_normal((N, 16)).astype(np.float32)
    k_ref, x_ref = orc.nearly_sort(nc, x)
    want = orc.redistribute(k_ref, x_ref)
    ncd, xd = torch.as_tensor(nc, device="cuda"), torch.as_tensor(x, device="cuda")
    k, xs = nat.smc_nearly_sort_raw(ncd, xd)
    got = nat.smc_redistribute_raw(k, xs)
    gather = nat.smc_redistribute_raw(ncd, xd)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # the same rows as the gather design, survivors in reverse index order
    pos = np.nonzero(nc)[0][::-1]
    assert np.array_equal(got, np.repeat(x[pos], nc[pos], axis=0))
    assert np.array_equal(np.sort(got, axis=0), np.sort(gather.cpu().numpy(), axis=0))


def test_nearly_sort_full_size(nat, orc):
    """N = 2^24 rows of 64 bytes (the redistribute benchmark's shape), whole
    output against the oracle, and repeatable."""
    N = 1 << 24
    nc = inputs.composition(N, seed=11)
    x = np.random.default_rng(12).standard_normal((N, 16)).astype(np.float32)
    k_ref, x_ref = orc.nearly_sort(nc, x)
    ncd, xd = torch.as_tensor(nc, device="cuda"), torch.as_tensor(x, device="cuda")
    k1, x1 = nat.smc_nearly_sort_raw(ncd, xd)
    k2, x2 = nat.smc_nearly_sort_raw(ncd, xd)
    torch.cuda.synchronize()
    assert np.array_equal(k1.cpu().numpy(), k_ref)
    assert np.array_equal(x1.cpu().numpy().view(np.uint32), x_ref.view(np.uint32))
    assert torch.equal(k1, k2) and torch.equal(x1.view(torch.int32), x2.view(torch.int32))


def test_nearly_sort_rejects_bad_arguments(nat):
    N = 100
    nc = torch.zeros(N + 4, dtype=torch.int32, device="cuda")
    x = torch.zeros(N, 4, device="cuda")
    with pytest.raises(nat.SmcError) as e:
        nat.smc_nearly_sort_raw(nc[1:N + 1], x)  # keys not 16-byte aligned
    assert e.value.code == nat.SMC_EINVAL
    L = nat.lib()
    ws = torch.empty(nat.smc_nearly_sort_ws_bytes(N), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(x)
    ko = torch.empty(N, dtype=torch.int32, device="cuda")
    assert L.smc_nearly_sort_raw(N, 6, nc.data_ptr(), x.data_ptr(), ko.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                 None) == nat.SMC_EINVAL  # row_bytes not a multiple of 4
    assert L.smc_nearly_sort_raw(0, 16, nc.data_ptr(), x.data_ptr(), ko.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                 None) == nat.SMC_EINVAL
