"""The allocation-free cell index (amb_cell_index_noalloc) against the
allocating one (amb_cell_index), through the C ABI, on two calls in a row.

The allocation-free entry point is for callers that cannot allocate device
memory while they run (their device memory is handed out up front by another
allocator, or they must not risk the device-wide synchronisation that
cudaMalloc / cudaFree can cause); its scratch is a static device array that
every call reuses, so the second call checks that the leftovers of the first
do not leak into the result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2601_16292_gb300 import amb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _index(fn, x, y, L, n):
    start = torch.empty(L * L + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    fn(x, y, L, start, ids[:n])
    return start.cpu().numpy(), ids[:n].cpu().numpy()


def _sorted_within_cells(start, ids):
    out = ids.copy()
    for c in np.nonzero(np.diff(start) > 1)[0]:
        out[start[c]:start[c + 1]] = np.sort(out[start[c]:start[c + 1]])
    return out


def test_noalloc_index_equals_allocating_index_twice():
    # the second call uses a smaller grid and fewer agents, so stale counts
    # or cursors left by the first call would show
    for call, (n, L) in enumerate([(300_000, 1000), (20_011, 77)]):
        rng = np.random.default_rng(40 + call)
        x = torch.from_numpy(rng.integers(0, L, n).astype(np.int32)).cuda()
        y = torch.from_numpy(rng.integers(0, L, n).astype(np.int32)).cuda()
        s_ref, i_ref = _index(amb.amb_cell_index, x, y, L, n)
        s_new, i_new = _index(amb.amb_cell_index_noalloc, x, y, L, n)
        assert np.array_equal(s_new, s_ref)
        assert s_new[-1] == n
        assert np.array_equal(_sorted_within_cells(s_new, i_new), _sorted_within_cells(s_ref, i_ref))


def test_noalloc_index_rejects_grids_beyond_its_scratch():
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    start = torch.empty(1025 * 1025 + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(amb.AmbError) as e:
        amb.amb_cell_index_noalloc(x, x, 1025, start, ids)
    assert e.value.status == amb.AMB_EINVAL


def _random_xy(n, L, seed):
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(rng.integers(0, L, n).astype(np.int32)).cuda()
    y = torch.from_numpy(rng.integers(0, L, n).astype(np.int32)).cuda()
    return x, y


@pytest.mark.parametrize("n,L", [(0, 5), (0, 1), (1, 1), (37, 1), (1000, 2)])
def test_noalloc_index_small_and_empty_cases(n, L):
    x, y = _random_xy(n, L, 7 + n + L)
    s_ref, i_ref = _index(amb.amb_cell_index, x, y, L, n)
    s_new, i_new = _index(amb.amb_cell_index_noalloc, x, y, L, n)
    assert np.array_equal(s_new, s_ref)
    assert s_new[-1] == n
    assert np.array_equal(_sorted_within_cells(s_new, i_new), _sorted_within_cells(s_ref, i_ref))


def test_noalloc_index_reports_coordinates_outside_the_grid_and_recovers():
    L, n = 40, 5000
    x, y = _random_xy(n, L, 11)
    x[17] = L  # one agent outside [0, L)
    start = torch.empty(L * L + 1, dtype=torch.int32, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(amb.AmbError) as e:
        amb.amb_cell_index_noalloc(x, y, L, start, ids)
    assert e.value.status == amb.AMB_EINVAL
    assert int(start[-1]) == n - 1  # the agent is left out, as amb_cell_index does
    # the next call starts from a clean error word
    x[17] = 0
    s_ref, i_ref = _index(amb.amb_cell_index, x, y, L, n)
    s_new, i_new = _index(amb.amb_cell_index_noalloc, x, y, L, n)
    assert np.array_equal(s_new, s_ref)
    assert np.array_equal(_sorted_within_cells(s_new, i_new), _sorted_within_cells(s_ref, i_ref))


def test_noalloc_index_rejects_a_misaligned_start_buffer():
    L, n = 8, 10
    x, y = _random_xy(n, L, 3)
    buf = torch.empty(L * L + 2, dtype=torch.int32, device="cuda")
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(amb.AmbError) as e:
        amb.amb_cell_index_noalloc(x, y, L, buf[1:], ids)  # 4 bytes past a 16-byte boundary
    assert e.value.status == amb.AMB_EINVAL


def test_noalloc_index_asynchronous_on_a_side_stream():
    # sync = 0 on a non-default stream: the call only queues the work; after
    # the stream is synchronised the result equals the allocating index
    L, n = 300, 120_000
    x, y = _random_xy(n, L, 19)
    s_ref, i_ref = _index(amb.amb_cell_index, x, y, L, n)
    side = torch.cuda.Stream()
    start = torch.full((L * L + 1,), -1, dtype=torch.int32, device="cuda")
    ids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):  # twice in a row on the same stream
        amb.amb_cell_index_noalloc(x, y, L, start, ids, stream=side, sync=False)
    side.synchronize()
    s_new, i_new = start.cpu().numpy(), ids.cpu().numpy()
    assert np.array_equal(s_new, s_ref)
    assert np.array_equal(_sorted_within_cells(s_new, i_new), _sorted_within_cells(s_ref, i_ref))
