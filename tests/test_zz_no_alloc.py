"""hcc_sort_noalloc: the sort for callers that cannot allocate device memory.

Such callers (a program whose device memory is all reserved by its own
allocator, or a latency-bound loop that cannot take the synchronisation a
cudaMalloc may imply) call hcc_sort_noalloc, which uses a fixed scratch array
owned by the library.  Its result must equal hcc_sort's and the oracle's
stable sort, bit for bit, on two calls in a row (the second call reuses the
array the first one left behind), including the largest size at 64-bit keys
(the layout that sizes the array) and a call without an error word.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import build, hcc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _reference_perm(ctx, keys_t, k, n):
    perm = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    hcc.hcc_sort(ctx, keys_t, k, n, perm)
    hcc.hcc_sync(ctx)
    return perm


@pytest.mark.parametrize("n,k", [(300_001, 32), (hcc.HCC_SORT_NOALLOC_MAX_N, 48),
                                 (hcc.HCC_SORT_NOALLOC_MAX_N, 64)])
def test_noalloc_sort_matches_hcc_sort_and_oracle_on_two_calls(n, k):
    build()
    ctx = hcc.hcc_create(0)
    try:
        rng = np.random.default_rng(2024 + k)
        dt = np.uint32 if k <= 32 else np.uint64
        keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
        keys = (keys & np.uint64((1 << k) - 1 if k < 64 else 0xFFFFFFFFFFFFFFFF)).astype(dt)
        keys[::7] = keys[0]  # plenty of equal keys: stability matters
        keys_t = torch.from_numpy(keys.view(np.int32 if dt == np.uint32 else np.int64)).to(DEV)
        ref = _reference_perm(ctx, keys_t, k, n)
        expect = oracle.stable_sort(keys.astype(np.uint64))
        assert np.array_equal(ref.cpu().numpy().view(np.uint32), expect)
        for call in range(2):  # two calls in a row on the same static scratch
            perm = torch.full((n,), -1, dtype=torch.int32, device=DEV)
            err = torch.zeros(1, dtype=torch.int32, device=DEV)
            hcc.hcc_sort_noalloc(keys_t, k, n, perm, err_word=err if call == 0 else None)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            assert torch.equal(perm, ref), (n, k, call)
            assert np.array_equal(perm.cpu().numpy().view(np.uint32), expect), (n, k, call)
    finally:
        hcc.hcc_destroy(ctx)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    build()
    n = hcc.HCC_SORT_NOALLOC_MAX_N + 1
    keys = torch.zeros(n, dtype=torch.int32, device=DEV)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    with pytest.raises(hcc.HccError) as ei:
        hcc.hcc_sort_noalloc(keys, 32, n, perm)
    assert ei.value.status == 1
    with pytest.raises(hcc.HccError):
        hcc.hcc_sort_noalloc(keys, 0, 16, perm)
