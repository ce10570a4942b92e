"""The block hash on its own: insert-or-find and lookup against the plain
definition (equal keys share one pool index, distinct keys get distinct
indices 0..n_distinct-1 in allocation order, block coordinates stored at
their index), with duplicates, repeated batches, a table at load factor
0.85, pool exhaustion and out-of-range keys."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check_partition(coords, pool, n_blocks, stored):
    """equal keys <-> equal pools; the pools are exactly 0..n_distinct-1;
    stored[pool] == key"""
    u, inv = np.unique(coords, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    assert n_blocks == len(u)
    first = np.full(len(u), -1)
    first[inv[::-1]] = pool[::-1]                          # any member's pool
    assert np.array_equal(pool, first[inv])                # equal keys share a pool
    assert np.array_equal(np.sort(first), np.arange(len(u)))   # a permutation of 0..n-1
    assert np.array_equal(stored[pool], coords)


def _insert(h, coords):
    import torch
    from paper_2410_21149_gb300 import _capi
    c = torch.from_numpy(np.ascontiguousarray(coords, np.int32)).cuda()
    p = torch.empty(len(coords), dtype=torch.int32, device="cuda")
    _capi.cvx_block_hash_insert(h, c, p)
    return p.cpu().numpy()


def _find(h, coords):
    import torch
    from paper_2410_21149_gb300 import _capi
    c = torch.from_numpy(np.ascontiguousarray(coords, np.int32)).cuda()
    p = torch.empty(len(coords), dtype=torch.int32, device="cuda")
    _capi.cvx_block_hash_find(h, c, p)
    return p.cpu().numpy()


def test_insert_find_with_duplicates_and_repeats():
    from paper_2410_21149_gb300 import _capi
    rng = np.random.default_rng(0)
    distinct = np.unique(rng.integers(-3000, 3000, (60000, 3)), axis=0)
    coords = distinct[rng.integers(0, len(distinct), 250000)]
    h = _capi.cvx_block_hash_create(1 << 18, 1 << 17)
    pool = _insert(h, coords)
    st, nb, stored = _capi.cvx_block_hash_info(h, with_keys=True)
    assert st == 0
    _check_partition(coords, pool, nb, stored)
    assert np.array_equal(_find(h, coords), pool)
    assert np.array_equal(_insert(h, coords[::-1]), pool[::-1])   # a repeated batch finds every key
    assert _capi.cvx_block_hash_info(h)[1] == nb
    absent = np.array([[5000, 0, 0], [-1048576, 7, 7], [0, 0, 4000]], np.int32)
    assert (_find(h, absent) == -1).all()
    _capi.cvx_block_hash_destroy(h)


def test_load_factor_085():
    from paper_2410_21149_gb300 import _capi
    rng = np.random.default_rng(1)
    slots = 1 << 16
    keys = np.unique(rng.integers(-(1 << 19), 1 << 19, (int(0.9 * slots), 3)), axis=0)[: int(0.85 * slots)]
    keys = keys[rng.permutation(len(keys))]
    h = _capi.cvx_block_hash_create(slots, len(keys))
    pool = _insert(h, keys)
    st, nb, stored = _capi.cvx_block_hash_info(h, with_keys=True)
    assert st == 0
    _check_partition(keys, pool, nb, stored)
    assert np.array_equal(_find(h, keys), pool)
    _capi.cvx_block_hash_destroy(h)


def test_pool_exhaustion_and_key_range():
    from paper_2410_21149_gb300 import _capi
    rng = np.random.default_rng(2)
    keys = np.unique(rng.integers(-500, 500, (3000, 3)), axis=0)
    h = _capi.cvx_block_hash_create(1 << 13, 1000)
    pool = _insert(h, keys)
    st, nb, stored = _capi.cvx_block_hash_info(h, with_keys=True)
    assert st == _capi.CVX_ERR_CAPACITY and nb == 1000
    ok = pool >= 0
    assert ok.sum() == 1000 and np.array_equal(np.sort(pool[ok]), np.arange(1000))
    assert np.array_equal(stored[pool[ok]], keys[ok])
    h2 = _capi.cvx_block_hash_create(1 << 8, 16)
    p2 = _insert(h2, np.array([[0, 0, 0], [1 << 20, 0, 0], [0, -(1 << 20) - 1, 0]], np.int32))
    assert p2[0] == 0 and (p2[1:] == -1).all()
    assert _capi.cvx_block_hash_info(h2)[0] == _capi.CVX_ERR_KEY_RANGE
    _capi.cvx_block_hash_destroy(h)
    _capi.cvx_block_hash_destroy(h2)
