"""The library's host clustering (the regrid's Berger-Rigoutsos step, through
tsu_cluster_flags; no GPU) against the oracle's independent implementation:
identical box lists on hand-drawn masks, on random blob masks large enough
for the threaded prefix-sum build, with and without a nesting constraint,
and with patch splitting."""
import numpy as np
import pytest

import oracle
from paper_1901_06798_gb300 import binding


def _blobs(rng, ny, nx, n, rmax):
    yy, xx = np.mgrid[0:ny, 0:nx]
    m = np.zeros((ny, nx), dtype=np.uint8)
    for _ in range(n):
        cy, cx = rng.uniform(0, ny), rng.uniform(0, nx)
        ry, rx = rng.uniform(2, rmax), rng.uniform(2, rmax)
        m |= (((yy - cy) / ry) ** 2 + ((xx - cx) / rx) ** 2 <= 1).astype(np.uint8)
    return m


def _same(f, nest=None, eff=0.7, ratio=1, patch_max=1 << 30):
    a = oracle.cluster(f, nest, eff=eff, ratio=ratio, patch_max=patch_max)
    b = binding.cluster_flags(f, nest, eff=eff, ratio=ratio, patch_max=patch_max)
    assert a.shape == b.shape and np.array_equal(a, b), (a[:5], b[:5])
    return b


def test_hand_drawn_masks():
    m = np.zeros((12, 16), dtype=np.uint8)
    assert _same(m).shape == (0, 4)
    m[3:7, 4:10] = 1
    assert _same(m).tolist() == [[4, 3, 6, 4]]
    m[9:11, 1:3] = 1
    m[2:5, 13:15] = 1
    _same(m)
    L = np.zeros((20, 20), dtype=np.uint8)
    L[2:18, 2:6] = 1
    L[14:18, 2:18] = 1
    _same(L)
    _same(L, eff=0.95)


def test_cut_rules_worked_by_hand():
    """The masks whose boxes the oracle pins derive by hand from the
    clustering reading (acceptance at equality, nearest hole, left part first,
    strongest inflection): the host clustering gives those boxes too."""
    f = np.array([[1, 1, 0, 0, 0, 0, 1, 1]], np.uint8)
    assert binding.cluster_flags(f, None, eff=0.5, ratio=1, patch_max=1 << 30).tolist() == [[0, 0, 8, 1]]
    f = np.array([[1, 0, 1, 1, 0, 1, 1, 1, 1, 1, 1]], np.uint8)
    assert binding.cluster_flags(f, None, eff=0.85, ratio=1, patch_max=1 << 30).tolist() == \
        [[0, 0, 1, 1], [2, 0, 2, 1], [5, 0, 6, 1]]
    f = np.zeros((10, 20), np.uint8)
    f[2:6, 12:16] = 1
    f[2:6, 1:5] = 1
    assert binding.cluster_flags(f, None, eff=0.7, ratio=1, patch_max=1 << 30).tolist() == [[1, 2, 4, 4], [12, 2, 4, 4]]
    f = np.array([[1, 1, 1, 1, 1, 1], [0, 0, 1, 0, 1, 0], [0, 0, 0, 0, 0, 0]], np.uint8)
    assert binding.cluster_flags(f, None, eff=0.7, ratio=1, patch_max=1 << 30).tolist() == \
        [[0, 0, 1, 1], [1, 0, 2, 2], [3, 0, 1, 1], [4, 0, 2, 2]]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_blobs_large(seed):
    rng = np.random.default_rng(seed)
    ny, nx = 700 + 37 * seed, 900 - 41 * seed
    f = _blobs(rng, ny, nx, 40, 60)
    boxes = _same(f)
    cov = np.zeros_like(f, dtype=bool)
    for i0, j0, w, h in boxes:
        cov[j0:j0 + h, i0:i0 + w] = True
    assert np.all(cov[f > 0])
    nest = np.ones_like(f)
    nest[:, : nx // 3] = 0
    f2 = f.copy()
    f2[:, : nx // 3] = 0
    _same(f2, nest | f2)
    _same(f, ratio=4, patch_max=60)
    _same(f, eff=0.5, ratio=2, patch_max=64)


def test_flags_touching_the_mask_edges():
    rng = np.random.default_rng(7)
    f = _blobs(rng, 300, 500, 25, 40)
    f[0, :] = 1
    f[:, -1] = 1
    _same(f)
    g = np.zeros((1, 1), dtype=np.uint8)
    g[0, 0] = 1
    assert _same(g).tolist() == [[0, 0, 1, 1]]


def test_clustering_in_a_forked_child():
    """The host pool behind the clustering survives a fork: a child forked
    after the pool started gets a pool of its own and returns the parent's
    boxes (a pool without its worker threads would wait forever)."""
    import os
    import warnings
    from paper_1901_06798_gb300 import binding
    F = np.zeros((900, 1100), np.uint8)
    F[300:500, 200:700] = 1
    F[620:700, 100:160] = 1
    N = np.ones_like(F)
    a = binding.cluster_flags(F, N, 0.7, 4, 60)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", DeprecationWarning)
        pid = os.fork()
    if pid == 0:
        b = binding.cluster_flags(F, N, 0.7, 4, 60)
        os._exit(0 if np.array_equal(a, b) else 3)
    _, status = os.waitpid(pid, 0)
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0


def test_clustering_from_concurrent_threads():
    """Several host threads clustering at once share one worker pool (its
    loops run one at a time): every call returns the boxes of a serial call."""
    import threading
    from paper_1901_06798_gb300 import binding
    rng = np.random.default_rng(11)
    masks = []
    for k in range(6):
        F = (rng.random((700, 900)) < 0.01).astype(np.uint8)
        F[100 + 40 * k:300 + 40 * k, 150:600] = 1
        masks.append(F)
    N = np.ones_like(masks[0])
    ref = [binding.cluster_flags(F, N, 0.7, 4, 60) for F in masks]
    out = [None] * len(masks)

    def work(k):
        for _ in range(3):
            out[k] = binding.cluster_flags(masks[k], N, 0.7, 4, 60)

    th = [threading.Thread(target=work, args=(k,)) for k in range(len(masks))]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in th)
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)
