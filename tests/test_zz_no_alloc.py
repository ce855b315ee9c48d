"""tn_dot_noalloc: a split-K-shaped reduction with its scratch in a fixed device array,
for callers that must not allocate device memory on this path (a process whose device
memory another allocator already owns, or a latency-critical loop that cannot afford
cudaMalloc's possible device synchronization).

Checked against the existing entry point (tn_contract on the same two-tensor network,
whose split-K step keeps its partials in the plan's workspace), within the tolerance the
other GPU tests use, on two calls in a row: the second call must not depend on what the
first left in the shared array. Also checked: repeated calls leave the device's free
memory unchanged (nothing is allocated after the first call's address lookup), and
oversize or overflowing sizes are rejected before any launch. Collected last on purpose.
"""
import numpy as np
import pytest
import torch

from tests._lib import ensure_built

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def two_tensor_network(m_dims, n_dims, k_dims, seed):
    from tn_inputs.network import Network, Path
    rng = np.random.default_rng(seed)
    ext, lab = {}, 0
    M, N, K = [], [], []
    for grp, dims in ((M, m_dims), (N, n_dims), (K, k_dims)):
        for d in dims:
            ext[lab] = d
            grp.append(lab)
            lab += 1
    am, bm = tuple(M + K), tuple(N + K)
    shp = lambda ms: tuple(ext[x] for x in ms)
    A = (rng.standard_normal(shp(am)) + 1j * rng.standard_normal(shp(am))).astype(np.complex64)
    B = (rng.standard_normal(shp(bm)) + 1j * rng.standard_normal(shp(bm))).astype(np.complex64)
    return Network([A, B], [am, bm], ext, tuple(M + N)), Path([(0, 1)])


def rel_err(got, want):
    return float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


@pytest.mark.parametrize("m_dims,n_dims,k_dims", [((), (), (2,) * 16), ((2,), (2,), (5, 7, 500)),
                                                  ((4,), (2, 2), (2,) * 14)])
def test_dot_noalloc_matches_contract(tn, m_dims, n_dims, k_dims):
    m, n, k = int(np.prod(m_dims)), int(np.prod(n_dims)), int(np.prod(k_dims))
    results = []
    for call, seed in enumerate((31, 32)):
        net, path = two_tensor_network(m_dims, n_dims, k_dims, seed)
        plan = tn.Plan(net, path)
        assert plan.step(0)["cls"] == tn.TN_CLASS_SPLITK
        ins = [torch.tensor(t, device="cuda") for t in net.tensors]
        ref = torch.zeros(tuple(m_dims) + tuple(n_dims), dtype=torch.complex128, device="cuda")
        plan.contract(ins, ref)
        a = ins[0].reshape(1, m, k).contiguous()
        b = ins[1].reshape(1, n, k).contiguous()
        out = torch.full((1, m, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        tn.binding.dot_noalloc(a, b, 1, m, n, k, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(m, n)
        want = ref.cpu().numpy().reshape(m, n)
        assert rel_err(got, want) < REL, (call, got, want)
        results.append(got)
        plan.destroy()
    assert not np.allclose(results[0], results[1])  # two different inputs, two answers


def test_dot_noalloc_batched_two_calls(tn):
    """A batch of independent dot products, twice in a row with different data."""
    rng = np.random.default_rng(5)
    batch, m, n, k = 3, 2, 2, 3 * 4096 + 17
    for _ in range(2):
        a = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))).astype(np.complex64)
        b = (rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k))).astype(np.complex64)
        da, db = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
        out = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
        tn.binding.dot_noalloc(da, db, batch, m, n, k, out)
        torch.cuda.synchronize()
        want = np.einsum("bik,bjk->bij", a.astype(np.complex128), b.astype(np.complex128))
        assert rel_err(out.cpu().numpy(), want) < REL


def test_dot_noalloc_rejects_oversize(tn):
    with pytest.raises(tn.TnError) as e:
        tn.binding.dot_noalloc(1, 1, 1, 4, 8, 4096, 1)        # 32 outputs > 16
    assert e.value.status == tn.TN_ERR_INVALID and "exceeds" in str(e.value)
    with pytest.raises(tn.TnError) as e:
        tn.binding.dot_noalloc(1, 1, 65535, 4, 4, 1 << 20, 1)  # partials beyond the scratch
    assert e.value.status == tn.TN_ERR_INVALID and "scratch" in str(e.value)
    with pytest.raises(tn.TnError) as e:
        tn.binding.dot_noalloc(1, 1, 1, 1 << 32, 1 << 32, 4096, 1)  # m*n wraps to 0 in int64
    assert e.value.status == tn.TN_ERR_INVALID and "exceeds" in str(e.value)
    with pytest.raises(tn.TnError) as e:
        tn.binding.dot_noalloc(1, 1, 1, 1, 1, 1 << 62, 1)  # ceil(k/4096) beyond the scratch
    assert e.value.status == tn.TN_ERR_INVALID and "scratch" in str(e.value)


def test_dot_noalloc_allocates_nothing(tn):
    """After the first call (the address lookup), repeated calls leave the device's free
    memory exactly as it was: the partials go to the fixed array, not to new memory."""
    rng = np.random.default_rng(9)
    batch, m, n, k = 4, 2, 4, 2 * 4096 + 5
    a = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))).astype(np.complex64)
    b = (rng.standard_normal((batch, n, k)) + 1j * rng.standard_normal((batch, n, k))).astype(np.complex64)
    da, db = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    out = torch.zeros((batch, m, n), dtype=torch.complex128, device="cuda")
    tn.binding.dot_noalloc(da, db, batch, m, n, k, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        tn.binding.dot_noalloc(da, db, batch, m, n, k, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    want = np.einsum("bik,bjk->bij", a.astype(np.complex128), b.astype(np.complex128))
    assert rel_err(out.cpu().numpy(), want) < REL
