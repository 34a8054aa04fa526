"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each value comes from a worked
example in the paper (Fig. 7), a hand computation (tests/golden/), a closed
form, an invariant, or an independent library routine (numpy sort, numpy IEEE
float32 division, torch's bfloat16 / float8 casts, scikit-learn's SVM decision
function).  Every function of oracle/rgbd_oracle.c is covered by at least one.
"""
import os

import numpy as np
import pytest

from paper_1504_01883_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rotl8(c, k):
    return ((c << k) | (c >> (8 - k))) & 0xFF


# ---------------------------------------------------------------------------------------------
# S3: LBP codes (Eq. 2, Fig. 7)
# ---------------------------------------------------------------------------------------------

def test_fig7_worked_example(orc):
    """Fig. 7: pattern 11110001 (bits 0,4,5,6,7 set, read from p7 down to p0) gives 241."""
    # centre 50; p0, p4, p5, p6, p7 brighter; p1, p2, p3 darker.
    #   p0 p1 p2      60 40 40
    #   p7  c p3  ->  60 50 40
    #   p6 p5 p4      60 60 60
    g = np.array([[60, 40, 40], [60, 50, 40], [60, 60, 60]], np.uint8)
    v = np.ones((3, 3), np.uint8)
    assert orc.lbp_code(g, v, 1, 1) == 241
    assert 241 == 0b11110001 == 1 + 16 + 32 + 64 + 128


def _read_lbp_golden():
    lines = [ln.split("#")[0].strip() for ln in open(os.path.join(GOLDEN, "lbp_4x4.txt"))]
    lines = [ln for ln in lines if ln]
    gi = lines.index("grey")
    vi = lines.index("valid")
    g = np.array([[int(t) for t in lines[gi + 1 + r].split()] for r in range(4)], np.uint8)
    v = np.array([[int(t) for t in lines[vi + 1 + r].split()] for r in range(4)], np.uint8)
    cases = [tuple(int(t) for t in ln.split()) for ln in lines[vi + 5:]]
    return g, v, cases


def test_lbp_hand_computed_4x4(orc):
    g, v, cases = _read_lbp_golden()
    assert len(cases) >= 10
    for i, j, flags, code in cases:
        assert orc.lbp_code(g, v, i, j, flags) == code, (i, j, flags)
    # an invalid centre produces no code at all
    codes = orc.lbp_codes(g, v)
    assert codes[1, 2] == -1 and (codes >= 0).sum() == 15


def test_constant_patch(orc):
    g = np.full((16, 16), 77, np.uint8)
    v = np.ones((16, 16), np.uint8)
    assert (orc.lbp_codes(g, v) == 0).all()                 # strict > : no bit set
    assert (orc.lbp_codes(g, v, orc.LBP_GE) == 255).all()   # >= would set all eight


def test_rotation_bit_rotates_codes_and_permutes_cells(orc):
    """Rotating grey and depth 90 degrees clockwise maps every code c to rotl8(c, 2)
    and moves cell (cy, cx) to (cx, G-1-cy).  Holds only for a circular ring order."""
    g, d = synth.crops(77, 1, 64)
    g, d = g[0], d[0]
    gr, dr = np.rot90(g, -1).copy(), np.rot90(d, -1).copy()
    m = orc.median_nonzero(d)
    assert orc.median_nonzero(dr) == m
    v, vr = orc.valid_mask(d, m), orc.valid_mask(dr, m)
    c, cr = orc.lbp_codes(g, v), orc.lbp_codes(gr, vr)
    S = 64
    ii, jj = np.nonzero(c >= 0)
    assert ii.size > 1000
    assert (cr[jj, S - 1 - ii] == _rotl8(c[ii, jj], 2)).all()
    # histograms: cell permutation plus the bin permutation U(c) -> U(rotl8(c, 2))
    lut = orc.uniform_table()
    h = orc.histograms(g, v).reshape(8, 8, 59)
    hr = orc.histograms(gr, vr).reshape(8, 8, 59)
    perm = np.arange(59)
    for code in range(256):
        if lut[code] < 58:
            perm[lut[code]] = lut[_rotl8(code, 2)]
    for cy in range(8):
        for cx in range(8):
            moved = np.zeros(59, np.int64)
            moved[perm] = h[cy, cx]
            assert (hr[cx, 7 - cy] == moved).all()


def test_cell_histogram_sums_to_valid_count(orc):
    g, d = synth.crops(5, 1, 64)
    m = orc.median_nonzero(d[0])
    v = orc.valid_mask(d[0], m)
    h = orc.histograms(g[0], v).reshape(8, 8, 59)
    vc = v.reshape(8, 8, 8, 8).transpose(0, 2, 1, 3).sum(axis=(2, 3))
    assert (h.sum(axis=2) == vc).all()
    assert vc.sum() > 0.5 * 64 * 64  # face covers more than half of the crop
    # the paper's own 0-255 histogram (Section 3) keeps the same count
    h256 = orc.histograms(g[0], v, nbins=256).reshape(8, 8, 256)
    assert (h256.sum(axis=2) == vc).all()


def test_paper_range_histogram_bins_are_raw_codes(orc):
    """Section 3's 0-255 histogram: one 3x3 cell, the Fig. 7 centre lands in bin 241."""
    g = np.array([[60, 40, 40], [60, 50, 40], [60, 60, 60]], np.uint8)
    v = np.ones((3, 3), np.uint8)
    h = orc.histograms(g, v, cell=3, nbins=256)
    assert h.shape == (256,) and h.sum() == 9 and h[241] >= 1


# ---------------------------------------------------------------------------------------------
# S4: the uniform-pattern map
# ---------------------------------------------------------------------------------------------

def test_uniform_table_closed_form(orc):
    lut = orc.uniform_table()
    P = 8
    uniform = [c for c in range(256) if lut[c] < 58]
    assert len(uniform) == P * (P - 1) + 2 == 58
    # independent description: 0, 255 and every rotation of a run of k ones (k = 1..7)
    runs = {0, 255}
    for k in range(1, 8):
        base = (1 << k) - 1
        for r in range(8):
            runs.add(_rotl8(base, r))
    assert set(uniform) == runs
    assert lut[0] == 0 and lut[255] == 57
    assert list(lut[uniform]) == list(range(58))  # ranked in ascending code order
    assert (lut[[c for c in range(256) if c not in runs]] == 58).all()


# ---------------------------------------------------------------------------------------------
# S2: median and mask
# ---------------------------------------------------------------------------------------------

def test_median_matches_sort(orc):
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 4, 5, 64, 255, 4096]:
        for hi in [3, 50, 65535]:
            d = rng.integers(0, hi + 1, n).astype(np.uint16)
            nz = np.sort(d[d != 0])
            want = int(nz[(nz.size - 1) // 2]) if nz.size else -1
            assert orc.median_nonzero(d) == want
    assert orc.median_nonzero(np.zeros(10, np.uint16)) == -1
    assert orc.median_nonzero(np.array([0, 9, 0], np.uint16)) == 9
    assert orc.median_nonzero(np.array([4, 8], np.uint16)) == 4  # lower median


def test_mask_strict_window(orc):
    d = np.array([1000, 1149, 1150, 851, 850, 0, 65535], np.uint16)
    assert list(orc.valid_mask(d, 1000, 150)) == [1, 1, 0, 1, 0, 0, 0]
    assert list(orc.valid_mask(d, -1, 150)) == [0] * 7


def test_all_hole_crop_gives_zero_features(orc):
    g, _ = synth.crops(9, 1, 64)
    d = np.zeros((1, 64, 64), np.uint16)
    f, med = orc.features_batch(g, d, None, 64, return_medians=True)
    assert med[0] == -1 and not f.any()


def test_background_only_median(orc):
    # a crop with no face: the mask keeps the depth band around the median
    rng = np.random.default_rng(0)
    d = rng.integers(2500, 4001, (64, 64)).astype(np.uint16)
    m = orc.median_nonzero(d)
    v = orc.valid_mask(d, m)
    assert v.sum() == ((np.abs(d.astype(int) - m) < 150)).sum()


# ---------------------------------------------------------------------------------------------
# S1: resample
# ---------------------------------------------------------------------------------------------

def _read_resample_golden():
    cases = []
    lines = [ln.split("#")[0].strip() for ln in open(os.path.join(GOLDEN, "resample_small.txt"))]
    lines = [ln for ln in lines if ln]
    i = 0
    while i < len(lines):
        t = lines[i].split()
        assert t[0] == "case"
        H, W, x, y, w, h, oh, ow = map(int, t[2:])
        i += 1
        blocks = {}
        for name, rows in [("grey_in", H), ("depth_in", H), ("grey_out", oh), ("depth_out", oh)]:
            assert lines[i] == name
            blocks[name] = np.array([[int(v) for v in lines[i + 1 + r].split()] for r in range(rows)])
            i += 1 + rows
        cases.append(((x, y, w, h), oh, ow, blocks))
    return cases


def test_resample_hand_computed(orc):
    cases = _read_resample_golden()
    assert len(cases) == 3
    for rect, oh, ow, b in cases:
        og, od = orc.crop(b["grey_in"].astype(np.uint8), b["depth_in"].astype(np.uint16), rect, oh, ow)
        assert (og == b["grey_out"]).all(), rect
        assert (od == b["depth_out"]).all(), rect


def test_resample_identity_and_translation(orc):
    g, d = synth.crops(11, 1, 64)
    og, od = orc.crop(g[0], d[0], (0, 0, 64, 64), 64, 64)
    assert (og == g[0]).all() and (od == d[0]).all()
    assert orc.rect_coord_q16(0, 64, 64, 5) == 5 * 65536
    # integer translation through the general affine form (Eq. 1 with unit basis vectors)
    aff = np.array([65536, 0, 7 * 65536, 0, 65536, 3 * 65536], np.int32)
    big_g = np.pad(g[0], 16, mode="edge")
    big_d = np.pad(d[0], 16, mode="edge")
    ag, ad = orc.crop(big_g, big_d, (0, 0, 1, 1), 32, 32, affine=aff)
    assert (ag == big_g[3:35, 7:39]).all() and (ad == big_d[3:35, 7:39]).all()


def test_resample_constant_image_is_exact(orc):
    # the Q8 weights sum to 2^16, so any rect over a constant image returns the constant
    g = np.full((40, 50), 173, np.uint8)
    d = np.full((40, 50), 1234, np.uint16)
    for rect in [(3, 4, 17, 29), (-10, -10, 90, 70), (45, 35, 30, 30)]:
        og, od = orc.crop(g, d, rect, 13, 11)
        assert (og == 173).all() and (od == 1234).all()


# ---------------------------------------------------------------------------------------------
# S5: normalisation, quantisation and the SVM decision function
# ---------------------------------------------------------------------------------------------

def test_normalize_matches_ieee_division(orc):
    rng = np.random.default_rng(1)
    f = rng.integers(0, 5, (3, 4 * 59)).astype(np.uint16)
    f[0, :59] = 0  # an empty cell
    x32 = orc.normalize_f32(f)
    tot = f.reshape(3, 4, 59).sum(axis=2, keepdims=True).astype(np.float32)
    with np.errstate(invalid="ignore", divide="ignore"):
        want = np.where(tot > 0, f.reshape(3, 4, 59).astype(np.float32) / tot, 0).astype(np.float32)
    assert (x32.reshape(3, 4, 59).view(np.uint32) == want.view(np.uint32)).all()
    x64 = orc.normalize_f64(f).reshape(3, 4, 59)
    s = x64.sum(axis=2)
    assert np.allclose(s[tot[..., 0] > 0], 1.0) and (s[tot[..., 0] == 0] == 0).all()
    # every quotient h / n of two counts n <= 64 rounds as numpy's IEEE float32 division
    for n in range(1, 65):
        for hv in range(0, n + 1):
            row = np.zeros((1, 59), np.uint16)
            row[0, 0], row[0, 1] = hv, n - hv
            got = orc.normalize_f32(row)[0, 0]
            assert got.view(np.uint32) == (np.float32(hv) / np.float32(n)).view(np.uint32)


def test_bf16_and_e4m3_match_torch():
    torch = pytest.importorskip("torch")
    import oracle
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.random(2000).astype(np.float32),
                        rng.random(500).astype(np.float32) * 448.0,
                        np.array([0.0, 1.0 / 64, 1.0 / 59, 2.0 ** -9, 2.0 ** -10, 447.9, 448.0],
                                 np.float32)])
    bf = oracle.f32_to_bf16(x)
    tb = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert (bf == tb).all()
    if hasattr(torch, "float8_e4m3fn"):
        e = oracle.f32_to_e4m3(x)
        te = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
        assert (e == te).all()
        back = oracle.e4m3_to_f64(e)
        tb2 = torch.from_numpy(te).view(torch.float8_e4m3fn).to(torch.float64).numpy()
        assert (back == tb2).all()


def test_rbf_matches_sklearn_decision_function(orc):
    sklearn = pytest.importorskip("sklearn")
    from sklearn.svm import SVC
    rng = np.random.default_rng(4)
    X = rng.random((60, 12))
    y = (X[:, 0] + 0.3 * X[:, 3] > 0.7).astype(int)
    gamma = 1.0 / 12
    clf = SVC(kernel="rbf", gamma=gamma, C=3.0).fit(X, y)
    Xt = rng.random((25, 12))
    s = orc.svm_rbf(Xt, clf.support_vectors_, clf.dual_coef_, clf.intercept_, gamma)
    assert np.allclose(s[:, 0], clf.decision_function(Xt), rtol=1e-12, atol=1e-12)


def test_linear_matches_sklearn_and_identity(orc):
    pytest.importorskip("sklearn")
    from sklearn.svm import LinearSVC
    rng = np.random.default_rng(5)
    X = rng.random((80, 9))
    y = rng.integers(0, 3, 80)
    clf = LinearSVC(C=1.0, max_iter=20000).fit(X, y)
    Xt = rng.random((10, 9))
    s = orc.svm_linear(Xt, clf.coef_, clf.intercept_)
    assert np.allclose(s, clf.decision_function(Xt), rtol=1e-12, atol=1e-12)
    # W = I, b: the score is x + b
    b = np.array([0.5, -1.0, 2.0])
    x = rng.random((4, 3))
    assert np.allclose(orc.svm_linear(x, np.eye(3), b), x + b, rtol=0, atol=1e-15)


def test_rbf_special_cases(orc):
    x = np.array([[0.25, 0.5, 0.125]])
    # one support vector equal to x: K = 1 exactly
    s = orc.svm_rbf(x, x.copy(), np.array([[2.5]]), np.array([-1.0]), 0.7)
    assert s[0, 0] == 1.5
    # far support vector: K underflows to 0, score = bias
    s = orc.svm_rbf(x, x + 1e3, np.array([[2.5]]), np.array([-1.0]), 0.7)
    assert s[0, 0] == -1.0


def test_argmax_lowest_index_on_ties(orc):
    s = np.array([[1.0, 3.0, 3.0], [2.0, 2.0, 2.0], [-1.0, -5.0, 0.0]])
    assert list(orc.argmax(s)) == [1, 0, 2]


# ---------------------------------------------------------------------------------------------
# Composition of S1..S4 on a frame
# ---------------------------------------------------------------------------------------------

def test_features_batch_composes_steps(orc):
    g, d, r = synth.frames_with_rects(21, 1, 3, 40, 90, H=120, W=160)
    feats, meds = orc.features_batch(g, d, r, out_h=64, return_medians=True)
    for k in range(3):
        rr = r[k]
        cg, cd = orc.crop(g[0], d[0], (rr["x"], rr["y"], rr["w"], rr["h"]), 64, 64)
        m = orc.median_nonzero(cd)
        assert m == meds[k]
        v = orc.valid_mask(cd, m)
        assert (orc.histograms(cg, v) == feats[k]).all()
    # an invalid descriptor gives a zero row
    bad = r.copy()
    bad[1]["frame"] = 5
    f2 = orc.features_batch(g, d, bad, out_h=64)
    assert not f2[1].any() and (f2[0] == feats[0]).all()


# ---------------------------------------------------------------------------------------------
# Section 2.3: nearest-centre tracking
# ---------------------------------------------------------------------------------------------

def test_track_nearest_hand_cases(orc):
    R = orc.RECT_DTYPE
    # stream 0: A at centre (50, 50); the next frame has faces at centres (60, 50), (45, 58), (200, 10)
    prev = np.array([(0, 40, 40, 20, 20), (1, 0, 0, 10, 10), (0, 190, 0, 20, 20)], R)
    cur = np.array([(0, 50, 40, 20, 20), (0, 35, 48, 20, 20), (0, 190, 0, 20, 20), (2, 0, 0, 4, 4)], R)
    m = orc.track_nearest(prev, cur)
    # A: distances 10 and sqrt(25 + 64) = 9.43 -> index 1; stream 1 has no current face -> -1;
    # the third face sits exactly on cur[2] -> 2
    assert list(m) == [1, -1, 2]
    # a tie (both at distance 5) keeps the lower index
    cur2 = np.array([(0, 45, 40, 20, 20), (0, 35, 40, 20, 20)], R)
    assert list(orc.track_nearest(prev[:1], cur2)) == [0]
    # brute force with numpy on random layouts
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = np.zeros(7, R)
        c = np.zeros(9, R)
        for arr in (p, c):
            arr["frame"] = rng.integers(0, 3, len(arr))
            arr["x"] = rng.integers(-50, 600, len(arr))
            arr["y"] = rng.integers(-50, 450, len(arr))
            arr["w"] = rng.integers(10, 200, len(arr))
            arr["h"] = arr["w"]
        got = orc.track_nearest(p, c)
        for i in range(len(p)):
            same = np.nonzero(c["frame"] == p[i]["frame"])[0]
            if same.size == 0:
                assert got[i] == -1
                continue
            d = np.hypot((c["x"][same] + c["w"][same] / 2) - (p["x"][i] + p["w"][i] / 2),
                         (c["y"][same] + c["h"][same] / 2) - (p["y"][i] + p["h"][i] / 2))
            assert got[i] == same[np.argmin(d)]


def _track_state(orc, S, M):
    return {"rects": np.zeros((S, M), orc.RECT_DTYPE), "ids": np.full((S, M), -1, np.int32),
            "count": np.zeros(S, np.int32)}


def test_track_streams_hand_cases(orc):
    """Section 2.3: identities follow the nearest centre from frame to frame, per stream."""
    R = orc.RECT_DTYPE
    st = _track_state(orc, 3, 4)
    # batch 1: stream 0 sees A (centre 50,50) and B (centre 200,100); stream 2 sees C
    ids = orc.track_streams(st, [0, 2], [0, 2, 3],
                            np.array([(0, 40, 40, 20, 20), (0, 190, 90, 20, 20), (0, 300, 300, 40, 40)], R),
                            [7, 3, 5])
    assert list(ids) == [7, 3, 5]                      # empty state: the classifier's labels
    assert list(st["count"]) == [2, 0, 1]
    # batch 2: stream 0's faces moved a little and come in the other order, plus a new face D;
    # the classifier now calls B "1" (a misclassification tracking corrects); stream 1 starts
    ids = orc.track_streams(st, [0, 1], [0, 3, 4],
                            np.array([(0, 195, 95, 20, 20), (0, 45, 42, 20, 20), (0, 500, 10, 30, 30),
                                      (0, 10, 10, 10, 10)], R),
                            [1, 1, 9, 4])
    assert list(ids) == [3, 7, 9, 4]
    assert list(st["count"]) == [3, 1, 1] and list(st["ids"][0][:3]) == [3, 7, 9]
    # batch 3: two frames of stream 0.  First only A remains (B and D also pick it as their
    # nearest current face, but A's previous face is the nearest of the three); then A and a
    # face where B was
    ids = orc.track_streams(st, [0, 0], [0, 1, 3],
                            np.array([(0, 47, 44, 20, 20), (0, 48, 44, 20, 20), (0, 196, 96, 20, 20)], R),
                            [2, 2, 8])
    assert list(ids) == [7, 7, 8]
    assert list(st["count"]) == [2, 1, 1] and list(st["ids"][0][:2]) == [7, 8]
    # stream id out of range: labels pass through, no state changes
    before = {k: v.copy() for k, v in st.items()}
    ids = orc.track_streams(st, [5], [0, 1], np.array([(0, 0, 0, 9, 9)], R), [6])
    assert list(ids) == [6] and all((st[k] == before[k]).all() for k in st)
    # more faces than the state holds: all get identities, the first max_faces are kept
    st2 = _track_state(orc, 1, 2)
    ids = orc.track_streams(st2, [0], [0, 3], np.array([(0, i * 50, 0, 10, 10) for i in range(3)], R), [1, 2, 3])
    assert list(ids) == [1, 2, 3] and st2["count"][0] == 2


def test_track_streams_brute_force(orc):
    """Random batches against a direct numpy restatement of the three steps."""
    R = orc.RECT_DTYPE
    rng = np.random.default_rng(11)
    S, M = 4, 5
    st = _track_state(orc, S, M)
    ref = {s: ([], []) for s in range(S)}  # stream -> (rect rows, ids)
    for _ in range(12):
        nfr = int(rng.integers(1, 6))
        fs = rng.integers(0, S, nfr)
        counts = rng.integers(0, 8, nfr)
        start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        n = int(start[-1])
        rects = np.zeros(n, R)
        rects["x"] = rng.integers(0, 600, n)
        rects["y"] = rng.integers(0, 440, n)
        rects["w"] = rng.integers(10, 100, n)
        rects["h"] = rects["w"]
        labels = rng.integers(0, 20, n).astype(np.int32)
        got = orc.track_streams(st, fs, start, rects, labels)
        want = labels.copy()
        for f in range(nfr):
            s, k0, k1 = int(fs[f]), int(start[f]), int(start[f + 1])
            prev, pid = ref[s]
            cx = rects["x"][k0:k1] + rects["w"][k0:k1] / 2
            cy = rects["y"][k0:k1] + rects["h"][k0:k1] / 2
            chosen = {}
            for j, (px, py) in enumerate(prev):
                if k1 == k0:
                    break
                d = np.hypot(cx - px, cy - py)
                k = int(np.argmin(d))  # first minimum = lowest index
                if k not in chosen or d[k] < chosen[k][0]:
                    chosen[k] = (d[k], j)
            for k, (_, j) in chosen.items():
                want[k0 + k] = pid[j]
            keep = min(k1 - k0, M)
            ref[s] = ([(cx[i], cy[i]) for i in range(keep)], [int(want[k0 + i]) for i in range(keep)])
        assert (got == want).all()


def _calib(orc, a, parallax=0, d_min=1, d_max=65535, cw=640, ch=480):
    c = np.zeros((), orc.CALIB_DTYPE)
    c["a"] = a
    c["parallax"], c["d_min"], c["d_max"], c["colour_w"], c["colour_h"] = parallax, d_min, d_max, cw, ch
    return c


def test_face_roi_hand_cases(orc):
    """Section 2.1: the depth pixels that map into the colour rect, and their bounding rect."""
    R = orc.RECT_DTYPE
    ident = [65536, 0, 0, 0, 65536, 0]
    d = np.full((6, 8), 1000, np.uint16)
    d[2, 1] = 0          # hole inside the rect
    d[4, 4] = 0
    # identity mapping: colour rect x 1..4, y 2..4 -> the same depth pixels; holes at the rect's
    # corners do not shrink it while other pixels of that row / column remain
    out = orc.face_roi(d, _calib(orc, ident, cw=8, ch=6), np.array([(0, 1, 2, 4, 3)], R))
    assert tuple(out[0]) == (0, 1, 2, 4, 3)
    # remove the whole column x = 1 of the rect: the box starts at x = 2
    d2 = d.copy()
    d2[2:5, 1] = 0
    out = orc.face_roi(d2, _calib(orc, ident, cw=8, ch=6), np.array([(0, 1, 2, 4, 3)], R))
    assert tuple(out[0]) == (0, 2, 2, 3, 3)
    # parallax: 20 px at 1000 mm (20 * 1000 * 256 in 1/256 px mm) shifts colour x by +20, so the
    # colour rect x 30..39 is depth x 10..19
    d3 = np.full((20, 40), 1000, np.uint16)
    c = _calib(orc, ident, parallax=20 * 1000 * 256)
    out = orc.face_roi(d3, c, np.array([(0, 30, 5, 10, 4)], R))
    assert tuple(out[0]) == (0, 10, 5, 10, 4)
    # at 2000 mm the shift halves: colour 30..39 is depth 20..29 (clipped to the 40-wide frame)
    d4 = np.full((20, 40), 2000, np.uint16)
    out = orc.face_roi(d4, c, np.array([(0, 30, 5, 10, 4)], R))
    assert tuple(out[0]) == (0, 20, 5, 10, 4)
    # depth range: pixels nearer than d_min do not map
    c2 = _calib(orc, ident, parallax=20 * 1000 * 256, d_min=1500)
    out = orc.face_roi(d3, c2, np.array([(0, 30, 5, 10, 4)], R))
    assert tuple(out[0]) == (0, 0, 0, 0, 0)
    # a colour image at twice the resolution: colour x = 2j, so colour 10..20 is depth 5..10
    c3 = _calib(orc, [131072, 0, 0, 0, 131072, 0])
    out = orc.face_roi(d3, c3, np.array([(0, 10, 4, 11, 6)], R))
    assert tuple(out[0]) == (0, 5, 2, 6, 3)
    # floor, not truncation: an offset of -0.5 px sends depth column 0 to colour x = -1 (outside)
    c4 = _calib(orc, [65536, 0, -32768, 0, 65536, 0])
    out = orc.face_roi(d3, c4, np.array([(0, 0, 0, 3, 3)], R))
    assert tuple(out[0]) == (0, 1, 0, 3, 3)   # colour x 0..2 <- depth j 1..3
    # bad descriptors and a rect outside the colour image
    out = orc.face_roi(d3, c, np.array([(1, 0, 0, 5, 5), (0, 0, 0, 0, 5), (0, 900, 0, 5, 5)], R))
    assert [tuple(o) for o in out] == [(1, 0, 0, 0, 0), (0, 0, 0, 0, 0), (0, 0, 0, 0, 0)]


def test_face_roi_brute_force(orc):
    """Random frames and calibrations (shear, scale, offset, parallax) against a vectorised
    numpy restatement of the mapping."""
    R = orc.RECT_DTYPE
    rng = np.random.default_rng(31)
    for it in range(10):
        F, H, W = 2, int(rng.integers(10, 40)), int(rng.integers(10, 50))
        d = rng.integers(300, 5000, (F, H, W)).astype(np.uint16)
        d[rng.random((F, H, W)) < 0.1] = 0
        a = [int(rng.integers(40000, 90000)), int(rng.integers(-9000, 9000)), int(rng.integers(-300000, 300000)),
             int(rng.integers(-9000, 9000)), int(rng.integers(40000, 90000)), int(rng.integers(-300000, 300000))]
        c = _calib(orc, a, parallax=int(rng.integers(0, 30 * 1000 * 256)), d_min=400, d_max=4500,
                   cw=int(rng.integers(20, 60)), ch=int(rng.integers(15, 45)))
        rects = np.zeros(6, R)
        rects["frame"] = rng.integers(0, F, 6)
        rects["x"] = rng.integers(-5, 50, 6)
        rects["y"] = rng.integers(-5, 40, 6)
        rects["w"] = rng.integers(1, 30, 6)
        rects["h"] = rng.integers(1, 30, 6)
        got = orc.face_roi(d, c, rects)
        ii, jj = np.meshgrid(np.arange(H, dtype=np.int64), np.arange(W, dtype=np.int64), indexing="ij")
        for k, r in enumerate(rects):
            dd = d[r["frame"]].astype(np.int64)
            ok = (dd >= 400) & (dd <= 4500)
            par = np.where(ok, c["parallax"] // np.maximum(dd, 1), 0) * 256
            X = a[0] * jj + a[1] * ii + a[2] + par
            Y = a[3] * jj + a[4] * ii + a[5]
            x, y = np.floor_divide(X, 65536), np.floor_divide(Y, 65536)
            m = ok & (x >= 0) & (x < c["colour_w"]) & (y >= 0) & (y < c["colour_h"])
            m &= (x >= r["x"]) & (x < r["x"] + r["w"]) & (y >= r["y"]) & (y < r["y"] + r["h"])
            if not m.any():
                assert tuple(got[k])[1:] == (0, 0, 0, 0)
                continue
            ys, xs = np.nonzero(m)
            assert tuple(got[k]) == (r["frame"], xs.min(), ys.min(), xs.max() - xs.min() + 1,
                                     ys.max() - ys.min() + 1), it


def test_svm_train_two_points_closed_form(orc):
    """Two points of opposite classes: alpha = 1 / (1 - k) with k = K(x0, x1) (one SMO step),
    b = 0 by symmetry, and the decision function is +1 / -1 on the two points."""
    x = np.array([[0.2, 0.8, 0.0], [0.5, 0.1, 0.4]])
    gamma = 1.3
    k = np.exp(-gamma * ((x[0] - x[1]) ** 2).sum())
    a, b, it = orc.svm_train_rbf(x, np.array([0, 1], np.int32), 1, gamma, cost=100.0, eps=1e-9)
    assert it[0] == 1
    assert abs(a[0, 0] - 1.0 / (1.0 - k)) < 1e-12 and abs(a[0, 1] + 1.0 / (1.0 - k)) < 1e-12
    assert abs(b[0]) < 1e-12
    # a box that binds: alpha stops at cost, the point is not free, b from the bounds
    a, b, it = orc.svm_train_rbf(x, np.array([0, 1], np.int32), 1, gamma, cost=0.5, eps=1e-9)
    assert list(a[0]) == [0.5, -0.5]
    f0 = a[0, 0] + a[0, 1] * k + b[0]
    assert f0 < 1.0  # the margin is not reached with a binding box


def _svm_data(seed, n, dim, C):
    rng = np.random.default_rng(seed)
    protos = rng.uniform(0.5, 1.5, (C, dim))
    lab = rng.integers(0, C, n).astype(np.int32)
    X = rng.poisson(3.0 * protos[lab]).astype(np.float64)
    X /= np.maximum(X.sum(1, keepdims=True), 1.0)
    Xt = rng.poisson(3.0 * protos[rng.integers(0, C, 40)]).astype(np.float64)
    Xt /= np.maximum(Xt.sum(1, keepdims=True), 1.0)
    return X, lab, Xt


def test_svm_train_matches_libsvm_and_kkt(orc):
    """One-vs-rest training against scikit-learn's SVC (libsvm: the same dual, the same working
    set rule) on decision values, and the KKT conditions at the solution."""
    sk = pytest.importorskip("sklearn.svm")
    X, lab, Xt = _svm_data(3, 90, 40, 3)
    gamma, cost, eps = 5.0, 2.0, 1e-6
    a, b, it = orc.svm_train_rbf(X, lab, 3, gamma, cost, eps=eps)
    K = lambda A, B: np.exp(-gamma * ((A[:, None, :] - B[None, :, :]) ** 2).sum(-1))
    f = K(Xt, X) @ a.T + b
    ftr = K(X, X) @ a.T + b
    for c in range(3):
        y = np.where(lab == c, 1, -1)
        m = sk.SVC(kernel="rbf", gamma=gamma, C=cost, tol=eps).fit(X, y)
        assert np.abs(m.decision_function(Xt) - f[:, c]).max() < 1e-5
        alpha = a[c] * y
        assert (alpha >= 0).all() and (alpha <= cost).all() and abs((y * alpha).sum()) < 1e-9
        yf = y * ftr[:, c]
        free = (alpha > 1e-9) & (alpha < cost - 1e-9)
        assert (yf[alpha <= 1e-9] >= 1 - 1e-4).all()
        assert (yf[alpha >= cost - 1e-9] <= 1 + 1e-4).all()
        assert np.abs(yf[free] - 1).max() < 1e-4
    # a class with no member: every alpha stays 0 and f = b = -1 (all rows are "rest")
    a2, b2, it2 = orc.svm_train_rbf(X, lab, 4, gamma, cost, eps=eps)
    assert (a2[3] == 0).all() and b2[3] == -1.0 and it2[3] == 0


# ---- centring of the SVM rows -----------------------------------------------------------------

def test_sv_centre_hand_example(orc):
    """Column means of three hand-made rows (a row mean or a wrong count would differ)."""
    x = np.array([[0.25, 1.0, 0.0], [0.75, 0.0, 0.0], [0.5, 0.5, 0.3]], np.float32)
    mu = orc.sv_centre(x)
    assert mu.dtype == np.float32
    assert mu.tolist() == [0.5, 0.5, np.float32(0.1)]
    c = orc.centre_rows(x, mu)
    assert c.tolist()[0] == [-0.25, 0.5, -np.float32(0.1)]


def test_centred_columns_sum_to_zero_and_rbf_scores_are_unchanged(orc):
    """Centred columns sum to zero within fp32 rounding, and the fp64 RBF scores of centred
    rows equal those of the raw rows (the kernel depends only on x - sv)."""
    rng = np.random.default_rng(5)
    sv32 = orc.normalize_f32(rng.poisson(3.0, (40, 6 * 59)).astype(np.uint16))
    x32 = orc.normalize_f32(rng.poisson(3.0, (7, 6 * 59)).astype(np.uint16))
    mu = orc.sv_centre(sv32)
    c = orc.centre_rows(sv32, mu).astype(np.float64)
    assert np.abs(c.sum(0)).max() <= 40 * 2.0 ** -24
    a = rng.normal(0.0, 1.0, (3, 40))
    b = rng.normal(0.0, 1.0, 3)
    g = 1.0 / (6 * 59)
    raw = orc.svm_rbf(x32.astype(np.float64), sv32.astype(np.float64), a, b, g)
    cen = orc.svm_rbf(x32.astype(np.float64) - mu, sv32.astype(np.float64) - mu, a, b, g)
    assert np.abs(raw - cen).max() < 1e-12
