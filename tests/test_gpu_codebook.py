"""Codebook-quantised records on the GPU (ugp_codebook_encode / ugp_codebook_decode) against the
FP64 reference of oracle/codebook.py, on a room scene with Disney materials.

* After one Lloyd iteration the GPU's codebook equals the reference's step from the same
  starting entries (the points of index floor(k n / 4096)), entry by entry.
* The final codes are the nearest entries of the GPU's codebook, except where the two nearest
  are within float32 rounding of each other.
* Decoding is the table lookup of the reference, record by record; means, magnitudes and types
  pass through exactly; a record is 24 bytes.
"""
import numpy as np
import pytest

from paper_2406_09733_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09733_gb300 import build, ugp
    build.build()
    ugp.lib()
    return torch


def _encode(torch, s, iters):
    from paper_2406_09733_gb300 import ugp
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mats = ugp.Materials(t(s.sggx), t(s.mtype), t(s.albedo), t(s.roughness), t(s.emission), t(s.disney))
    book, rec = ugp.codebook_encode(t(s.mean), t(s.quat), t(s.scale), t(s.magnitude), mats, iters=iters)
    torch.cuda.synchronize()
    return book, rec


def test_codebook_encode_decode_matches_reference(gpu):
    from oracle import codebook as cb
    from paper_2406_09733_gb300 import ugp
    torch = gpu
    s = scenes.with_disney(scenes.room_scene(30_000, seed=7, n_clusters=9), 0.3, seed=1)
    X = cb.features(s)
    # one Lloyd iteration from the same starting entries, group by group
    book1, _ = _encode(torch, s, iters=1)
    B1 = book1.double().cpu().numpy()
    init = cb.initial_book(X)
    for g in cb.ORDER:
        o, d = cb.GROUPS[g]
        codes0, e1, e2 = cb.assign(X, init, g)
        ref = cb.lloyd_step(X, init, codes0, g)
        err = np.abs(B1[:, o:o + d] - ref[:, o:o + d]).max(1) / (np.abs(ref[:, o:o + d]).max(1) + 1e-6)
        # points within float32 rounding of a tie may sit in either entry: entries that hold such
        # a point are compared by their counts only
        tie = np.abs(e2 - e1) <= 1e-5 * (e1 + 1e-12) + 1e-10
        loose = np.zeros(cb.K, bool)
        loose[codes0[tie]] = True
        print(f"{g}: max rel entry error {err[~loose].max():.2e}, {loose.sum()} entries with a near-tie point")
        # the GPU forms its features in float32 (log, normalisation): a point whose two nearest
        # entries are within about 1e-5 of each other may land in the other one and move a mean by
        # a fraction of their distance
        assert err[~loose].max() <= 1e-4 and np.quantile(err[~loose], 0.99) <= 1e-6, g
    # the final fit: codes are nearest entries of the returned codebook
    book, rec = _encode(torch, s, iters=6)
    B = book.double().cpu().numpy()
    R = rec.cpu().numpy()
    assert R.shape == (s.n, 24)
    dec = cb.decode(R, B)
    for gi, g in enumerate(cb.ORDER):
        codes, e1, e2 = cb.assign(X, B, g)
        got = dec["codes"][:, gi]
        bad = got != codes
        o, d = cb.GROUPS[g]
        dg = ((X[:, o:o + d] - B[got, o:o + d]) ** 2).sum(1)
        ok_tie = np.abs(dg - e1) <= 1e-5 * (e1 + 1e-12) + 1e-9
        print(f"{g}: {bad.sum()} codes differ from the FP64 nearest entry, all within rounding: {ok_tie[bad].all()}")
        assert bad.mean() < 1e-3 and ok_tie[bad].all(), g
    assert np.array_equal(dec["mtype"], s.mtype)
    np.testing.assert_array_equal(dec["mean"], s.mean.astype(np.float64))
    np.testing.assert_array_equal(dec["magnitude"], s.magnitude.astype(np.float64))
    # the GPU's decoder is the same lookup
    out = ugp.codebook_decode(rec, book)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["mtype"].cpu().numpy(), dec["mtype"])
    np.testing.assert_array_equal(out["mean"].cpu().numpy(), s.mean)
    for k in ("scale", "quat", "sggx", "albedo", "roughness", "emission", "disney"):
        np.testing.assert_allclose(out[k].double().cpu().numpy(), dec[k], rtol=2e-6, atol=1e-7, err_msg=k)
    # quantisation error of the fit: small against the spread of each group
    for g in cb.ORDER:
        o, d = cb.GROUPS[g]
        q = ((X[:, o:o + d] - B[dec["codes"][:, cb.ORDER.index(g)], o:o + d]) ** 2).sum(1).mean()
        v = X[:, o:o + d].var(0).sum()
        print(f"{g}: mean squared quantisation error {q:.3g} of variance {v:.3g}")
        assert q < 0.05 * v + 1e-12, g
