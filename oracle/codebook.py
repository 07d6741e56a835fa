"""FP64 reference of the codebook-quantised primitive records (the per-attribute codebook
compression with random-access decoding that the paper combines with level of detail).

TEST INFRASTRUCTURE ONLY: plain numpy, imported by tests alone.  It states the definitions
the GPU encoder and decoder follow:

* features: per primitive the log scales (3), the unit quaternion with w >= 0 (4), the SGGX
  matrix (6) and the material vector (albedo 3, roughness, emission 3, Disney 9: 16);
* assignment: the nearest codebook entry of each group by squared Euclidean distance, ties to
  the lower index;
* one Lloyd step: every entry that has points moves to their mean, the others stay;
* the initial entries are the points of index floor(k n / K);
* decoding: a table lookup per record (scale = exp, quaternion normalised).
"""
from __future__ import annotations

import numpy as np

K = 4096
GROUPS = {"scale": (0, 3), "rotation": (3, 4), "sggx": (7, 6), "material": (13, 16)}
ORDER = ("scale", "rotation", "sggx", "material")
NFEAT = 29


def features(scene) -> np.ndarray:
    n = scene.n
    X = np.zeros((n, NFEAT))
    X[:, 0:3] = np.log(np.asarray(scene.scale, np.float64))
    q = np.asarray(scene.quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    X[:, 3:7] = q
    X[:, 7:13] = scene.sggx
    X[:, 13:16] = scene.albedo
    X[:, 16] = scene.roughness
    X[:, 17:20] = scene.emission
    if getattr(scene, "disney", None) is not None:
        X[:, 20:29] = scene.disney
    return X


def initial_book(X: np.ndarray) -> np.ndarray:
    n = X.shape[0]
    return X[(np.arange(K, dtype=np.int64) * n) // K].copy()


def assign(X: np.ndarray, book: np.ndarray, group: str, chunk: int = 2048):
    """(codes, squared distance to the chosen entry, to the runner-up) of every point."""
    o, d = GROUPS[group]
    B = np.asarray(book, np.float64)[:, o:o + d]
    codes = np.zeros(X.shape[0], np.int64)
    d1 = np.zeros(X.shape[0])
    d2 = np.zeros(X.shape[0])
    for s in range(0, X.shape[0], chunk):
        x = X[s:s + chunk, o:o + d]
        dist = ((x[:, None, :] - B[None, :, :]) ** 2).sum(-1)
        idx = np.argmin(dist, axis=1)              # the first minimum: ties to the lower index
        codes[s:s + chunk] = idx
        d1[s:s + chunk] = dist[np.arange(len(idx)), idx]
        dist[np.arange(len(idx)), idx] = np.inf
        d2[s:s + chunk] = dist.min(axis=1)
    return codes, d1, d2


def lloyd_step(X: np.ndarray, book: np.ndarray, codes: np.ndarray, group: str) -> np.ndarray:
    """Entries of `group` moved to the mean of their points (entries without points stay)."""
    o, d = GROUPS[group]
    new = np.asarray(book, np.float64).copy()
    cnt = np.bincount(codes, minlength=K)
    for j in range(d):
        s = np.bincount(codes, weights=X[:, o + j], minlength=K)
        has = cnt > 0
        new[has, o + j] = s[has] / cnt[has]
    return new


def decode(records: np.ndarray, book: np.ndarray) -> dict:
    r = np.ascontiguousarray(records, np.uint8)
    n = r.shape[0]
    f = r[:, :16].copy().view(np.float32).reshape(n, 4)
    w = r[:, 16:24].copy().view(np.uint16).reshape(n, 4).astype(np.int64)
    cs, cr, cg, cm = w[:, 0], w[:, 1], w[:, 2], w[:, 3] & 0xFFF
    B = np.asarray(book, np.float64)
    q = B[cr, 3:7]
    return dict(mean=f[:, :3].astype(np.float64), magnitude=f[:, 3].astype(np.float64),
                mtype=(w[:, 3] >> 12).astype(np.uint8), scale=np.exp(B[cs, 0:3]),
                quat=q / np.linalg.norm(q, axis=1, keepdims=True), sggx=B[cg, 7:13],
                albedo=B[cm, 13:16], roughness=B[cm, 16], emission=B[cm, 17:20], disney=B[cm, 20:29],
                codes=np.stack([cs, cr, cg, cm], 1))
