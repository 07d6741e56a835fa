"""Pins of the codebook reference (oracle/codebook.py): the nearest-entry assignment against
scipy's vector quantiser, one Lloyd step against scipy's k-means with the same starting entries,
and the features and decoding on hand-built records."""
import numpy as np
import pytest

from oracle import codebook as cb
from paper_2406_09733_gb300 import scenes


def test_assignment_matches_scipy_vq():
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(5)
    X = np.zeros((3000, cb.NFEAT))
    X[:, 13:29] = rng.random((3000, 16))
    book = np.zeros((cb.K, cb.NFEAT))
    book[:, 13:29] = rng.random((cb.K, 16))
    codes, d1, _ = cb.assign(X, book, "material")
    ref, dist = vq.vq(X[:, 13:29], book[:, 13:29])
    assert np.array_equal(codes, ref)
    np.testing.assert_allclose(np.sqrt(d1), dist, rtol=1e-12)


def test_lloyd_step_matches_scipy_kmeans2():
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(6)
    X = np.zeros((20000, cb.NFEAT))
    X[:, 0:3] = rng.normal(size=(20000, 3))
    book = cb.initial_book(X)
    codes, _, _ = cb.assign(X, book, "scale")
    new = cb.lloyd_step(X, book, codes, "scale")
    ref, _ = vq.kmeans2(X[:, 0:3], book[:, 0:3], iter=1, minit="matrix", missing="warn")
    np.testing.assert_allclose(new[:, 0:3], ref, rtol=1e-12, atol=1e-12)


def test_features_and_decode_by_hand():
    s = scenes.tiny_scene(n=8, seed=2)
    s.quat[3] *= -1.0                          # q and -q are the same rotation
    X = cb.features(s)
    assert np.all(X[:, 3] >= 0)
    np.testing.assert_allclose(np.exp(X[:, 0:3]), s.scale, rtol=1e-7)
    np.testing.assert_allclose(np.linalg.norm(X[:, 3:7], axis=1), 1.0, rtol=1e-12)
    # a record by hand: codes (5, 7, 9, 11), type 2
    book = np.arange(cb.K * cb.NFEAT, dtype=np.float64).reshape(cb.K, cb.NFEAT) * 1e-4
    rec = np.zeros((1, 24), np.uint8)
    rec[0, :16] = np.array([1.5, -2.0, 3.25, 0.75], np.float32).view(np.uint8)
    rec[0, 16:24] = np.array([5, 7, 9, 11 | (2 << 12)], np.uint16).view(np.uint8)
    d = cb.decode(rec, book)
    assert d["mtype"][0] == 2 and list(d["codes"][0]) == [5, 7, 9, 11]
    np.testing.assert_array_equal(d["mean"][0], [1.5, -2.0, 3.25])
    assert d["magnitude"][0] == 0.75
    np.testing.assert_allclose(d["scale"][0], np.exp(book[5, 0:3]))
    np.testing.assert_allclose(d["sggx"][0], book[9, 7:13])
    np.testing.assert_allclose(d["disney"][0], book[11, 20:29])
