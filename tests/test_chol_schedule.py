"""Host logic of the single-launch factorization (no GPU): the worker task
list the library hands to the kernel (hs_chol_task_list).  It must hold every
tile task of the blocked factorization exactly once (with and without the
inverse factor), and list each task after the worker tasks it reads, which is
what makes the kernel's bounded waits free of deadlock: a task waits only on
earlier list entries or on the diagonal chain.

Tasks of step k (tile size 32, T tiles): C(i,k) L_ik = A_ik L_kk^{-T} for
i >= k+2 (the chain forms L_{k+1,k}); UA(i,j,k) A_ij -= L_ik L_jk^T for
k < j <= i except (k+1, k+1) (the chain applies that one); with the inverse
factor also X(k,j) = L_kk^{-1} B_kj for j < k and UB(i,j,k) B_ij -= L_ik X_kj
for i > k, j <= k.  In the single launch's list each C(i,k) also applies
UA(i,k+1,k) (code j = k + 1), which the list then leaves out.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1608_04329_gb300 import _build
    import paper_1608_04329_gb300 as pkg
    _build.build()
    return pkg.load_library()


def _tasks(T, inv):
    out = set()
    for k in range(T):
        out |= {(0, i, k, k) for i in range(k + 2, T)}
        out |= {(2, i, j, k) for j in range(k + 1, T) for i in range(j, T) if not (i == j == k + 1)}
        if inv:
            out |= {(1, k, j, k) for j in range(k)}
            out |= {(3, i, j, k) for i in range(k + 1, T) for j in range(k + 1)}
    return out


def _deps(task):
    kind, i, j, k = task
    d = []
    if kind == 0:
        if k >= 1:
            d.append((2, i, k, k - 1))
    elif kind == 1:
        if k >= 1:
            d.append((3, k, j, k - 1))
    elif kind == 2:
        if i >= k + 2:
            d.append((0, i, k, k))
        if j >= k + 2 and j != i:
            d.append((0, j, k, k))
        if k >= 1:
            d.append((2, i, j, k - 1))
    else:
        if i >= k + 2:
            d.append((0, i, k, k))
        if j < k:
            d.append((1, k, j, k))
        if k > j:
            d.append((3, i, j, k - 1))
    return d


def _merged(task):
    """The list entry that performs a task: UA(i,k+1,k) (i >= k+2) is done by C(i,k)."""
    kind, i, j, k = task
    if kind == 2 and j == k + 1 and i >= k + 2:
        return (0, i, k, k)
    return task


@pytest.mark.parametrize("inv", [0, 1])
@pytest.mark.parametrize("T", [1, 2, 3, 4, 7, 16, 32, 40])
@pytest.mark.parametrize("workers", [1, 7, 300])
def test_task_list_is_complete_and_topological(lib, T, inv, workers):
    n = lib.hs_chol_task_list(T, workers, inv, None, 0)
    every = _tasks(T, inv)
    want = {t for t in every if _merged(t) == t}
    assert n == len(want)
    codes = np.zeros(max(n, 1), dtype=np.int32)
    assert lib.hs_chol_task_list(T, workers, inv, codes.ctypes.data, n) == n
    got = []
    for c in codes[:n].tolist():
        kind, k, i, j = c & 3, (c >> 2) & 0xFF, (c >> 10) & 0xFF, (c >> 18) & 0xFF
        if kind == 0:
            assert j == k + 1, "a C entry of the single launch carries its merged update"
            got.append((0, i, k, k))
        else:
            got.append((kind, i, j, k))
    assert len(set(got)) == n and set(got) == want
    pos = {t: p for p, t in enumerate(got)}
    # every task of the blocked factorization, merged or not, runs after the
    # entries it reads (a merged update reads its own C task's output in place)
    for t in every:
        mt = _merged(t)
        for d in _deps(t):
            md = _merged(d)
            if md == mt:
                assert mt != t and d == mt, (t, d)  # the merged update reads its own C task
            else:
                assert pos[md] < pos[mt], (t, d)


def test_task_list_rejects_bad_arguments(lib):
    assert lib.hs_chol_task_list(0, 4, 1, None, 0) == -1
    assert lib.hs_chol_task_list(257, 4, 1, None, 0) == -1
    assert lib.hs_chol_task_list(8, 0, 1, None, 0) == -1
    assert lib.hs_chol_task_list(8, 4, 2, None, 0) == -1
    assert lib.hs_chol_task_list(8, 4, 1, None, 5) == -1


def _block_tasks(T, k0, k1):
    out = set()
    for k in range(k0, k1):
        out |= {(0, i, k, k) for i in range(k + 2, T)}
        out |= {(2, i, j, k) for j in range(k + 1, k1) for i in range(j, T) if not (i == j == k + 1)}
    return out


@pytest.mark.parametrize("workers", [1, 17, 500])
@pytest.mark.parametrize("T", [1, 2, 3, 5, 7, 8, 17, 32, 125])
def test_block_column_task_lists(lib, T, workers):
    """The tensor-core schedule's block-column launches (tile columns
    [4b, 4b + 4), list-scheduled for a number of task slots): each list holds
    the panel tiles C(i, k) and the updates
    UA(i, j, k) of the block column's later tile columns exactly once, every
    task after the tasks of the same launch it reads (the updates of earlier
    block columns come from the tensor-core launches between them)."""
    for k0 in range(0, T, 4):
        k1 = min(k0 + 4, T)
        n = lib.hs_chol_block_task_list(T, k0, k1, workers, None, 0)
        want = _block_tasks(T, k0, k1)
        assert n == len(want)
        codes = np.zeros(max(n, 1), dtype=np.int32)
        assert lib.hs_chol_block_task_list(T, k0, k1, workers, codes.ctypes.data, n) == n
        got = []
        for c in codes[:n].tolist():
            kind, k, i, j = c & 3, (c >> 2) & 0xFF, (c >> 10) & 0xFF, (c >> 18) & 0xFF
            got.append((kind, i, j, k) if kind == 2 else (kind, i, k, k))
        assert len(set(got)) == n and set(got) == want
        pos = {t: p for p, t in enumerate(got)}
        for t in got:
            for d in _deps(t):
                if d[3] >= k0:  # tasks of this launch
                    assert d in pos, (t, d)
                    assert pos[d] < pos[t], (t, d)
    assert lib.hs_chol_block_task_list(8, 4, 4, 4, None, 0) == -1
    assert lib.hs_chol_block_task_list(8, 0, 9, 4, None, 0) == -1
    assert lib.hs_chol_block_task_list(8, 0, 4, 0, None, 0) == -1
