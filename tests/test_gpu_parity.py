"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Integer outputs (crops, LBP histograms) and the IEEE-division fp32 / bf16 / FP8 normalised
rows must match bit for bit.  fp32 scores must agree with the fp64 oracle within 1e-5 of
sum_i |a_ci| K_i + |b_c| (the oracle's score can be near zero when sum_i a_ci = 0).
"""
import numpy as np
import pytest

from paper_1504_01883_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1504_01883_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


from gpu_util import dev_f32, dev_u16, dev_u8, host_bits32, host_u16, rbf_error_scale, rel_score_error  # noqa: E402


# ---------------------------------------------------------------------------------------------
# A1-A5 on the three crop layouts
# ---------------------------------------------------------------------------------------------

def test_plain_64_crop_features_and_linear_svm(B, ctx, orc):
    wl = synth.plain_crop()
    want = orc.features_batch(wl.grey, wl.depth, None, 64)
    f, x, q = B.lbp_fused_features(ctx, dev_u8(wl.grey), dev_u16(wl.depth), None, crop=64, x_dtype="f32")
    torch.cuda.synchronize()
    assert (host_u16(f) == want).all()
    x32 = orc.normalize_f32(want)
    xh = x.cpu().numpy()
    assert (xh[:, :3776].view(np.uint32) == x32.view(np.uint32)).all()
    assert (xh[:, 3776:] == 0).all() and xh.shape[1] == 3840
    assert np.allclose(q.cpu().numpy(), (x32.astype(np.float64) ** 2).sum(1), rtol=1e-6)
    model = B.svm_train_data_pack(ctx, None, dev_f32(wl.coef), dev_f32(wl.bias), kernel=B.KERNEL_LINEAR, dim=3776)
    s, lab = B.svm_score(ctx, model, x, q)
    x64 = orc.normalize_f64(want)
    ref = orc.svm_linear(x64, wl.coef, wl.bias)
    scale = np.abs(x64) @ np.abs(wl.coef.astype(np.float64)).T + np.abs(wl.bias)[None, :]
    assert np.all(np.abs(s.cpu().numpy() - ref) <= 1e-5 * scale)
    assert (lab.cpu().numpy() == orc.argmax(ref)).all()
    assert ctx.status() == 0


def test_single_frame_crops_features_and_rbf_f32(B, ctx, orc):
    wl = synth.single_frame()
    g, d, r = dev_u8(wl.grey), dev_u16(wl.depth), B.rects_tensor(wl.rects)
    cg, cd = B.rgbd_crop_affine(ctx, g, d, r, 128, 128)
    for k, rr in enumerate(wl.rects):
        og, od = orc.crop(wl.grey[rr["frame"]], wl.depth[rr["frame"]], (rr["x"], rr["y"], rr["w"], rr["h"]), 128, 128)
        assert (cg[k].cpu().numpy() == og).all()
        assert (host_u16(cd[k]) == od).all()
    want = orc.features_batch(wl.grey, wl.depth, wl.rects, 128)
    f, x, q = B.lbp_fused_features(ctx, g, d, r, crop=128, x_dtype="f32")
    assert (host_u16(f) == want).all()
    sv = dev_u16(wl.sv_counts)
    model = B.svm_train_data_pack(ctx, sv, dev_f32(wl.coef), dev_f32(wl.bias), gamma=wl.gamma, dtype="f32")
    s, lab = B.svm_score(ctx, model, x, q)
    x64, sv64 = orc.normalize_f64(want), orc.normalize_f64(wl.sv_counts)
    ref = orc.svm_rbf(x64, sv64, wl.coef, wl.bias, wl.gamma)
    err = rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, wl.coef, wl.bias, wl.gamma))
    assert err <= 1e-5, err
    assert (lab.cpu().numpy() == orc.argmax(ref)).all()


def _edge_frames():
    """Ragged rect sizes (4..300 px, partly outside the frame), an all-hole frame, a rect on
    background only, and two invalid descriptors."""
    g, d, r = synth.frames_with_rects(99, 4, [5, 3, 6, 4], 4, 300, H=240, W=320)
    d[2][:] = 0  # every rect of frame 2 is all holes
    extra = np.zeros(4, synth.RECT_DTYPE)
    extra[0] = (1, 250, 10, 60, 60)   # background-only region (may overlap nothing)
    extra[1] = (0, -50, -40, 30, 30)  # entirely outside the frame: clamped edge pixels
    extra[2] = (7, 10, 10, 50, 50)    # frame index out of range
    extra[3] = (1, 10, 10, 0, 40)     # zero width
    return g, d, np.concatenate([r, extra])


@pytest.mark.parametrize("crop", [32, 64, 96, 128])
def test_ragged_batch_and_edge_cases(B, ctx, orc, crop):
    g, d, r = _edge_frames()
    want = orc.features_batch(g, d, r, crop)
    ctx.status(clear=True)
    f, x, q = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop, x_dtype="f32")
    got = host_u16(f)
    assert (got == want).all(), np.nonzero((got != want).any(1))
    assert not got[-2:].any()
    assert ctx.status() & B.STATUS_BAD_RECT
    x32 = orc.normalize_f32(want)
    dim = want.shape[1]
    assert (x.cpu().numpy()[:, :dim].view(np.uint32) == x32.view(np.uint32)).all()


@pytest.mark.parametrize("W", [322, 318])
def test_frame_width_not_a_multiple_of_4(B, ctx, orc, W):
    """Frame rows that are not word-aligned take the byte-gather resample (the 8-byte grey
    windows need 4-byte aligned rows); rects reach the right edge."""
    g, d, r = synth.frames_with_rects(57, 2, 6, 20, 200, H=200, W=W)
    r = np.concatenate([r, np.array([(0, W - 30, 5, 30, 60), (1, W - 200, 100, 200, 100)], synth.RECT_DTYPE)])
    for crop in (64, 128):
        want = orc.features_batch(g, d, r, crop)
        f, _, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop)
        assert (host_u16(f) == want).all(), crop


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_lbp_option_flags(B, ctx, orc, flags):
    g, d, r = synth.frames_with_rects(5, 2, 4, 40, 200, H=240, W=320)
    want = orc.features_batch(g, d, r, 64, flags=flags)
    f, _, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=64, flags=flags)
    assert (host_u16(f) == want).all()


@pytest.mark.parametrize("crop", [64, 128])
@pytest.mark.parametrize("flags", [0, 1, 2])
def test_tile_shapes_bit_exact(B, ctx, orc, crop, flags):
    """Every tile shape of the fused kernel (one thread per cell, per half cell, per quarter
    cell), one and two CTAs per SM: features bit-exact with the oracle, and the same normalised
    rows and norms."""
    g, d, r = synth.frames_with_rects(70 + crop + flags, 3, 7, 40, 256, H=240, W=320)
    want = orc.features_batch(g, d, r, crop, flags=flags)
    rows = {}
    try:
        for shape in (1, 2, 3):
            for ctas in (1, 2):
                ctx.set_tuning(B.TUNE_LBP_SHAPE, shape)
                ctx.set_tuning(B.TUNE_LBP_CTAS_PER_SM, ctas)
                f, x, q = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop, flags=flags,
                                               x_dtype="bf16")
                assert (host_u16(f) == want).all(), (shape, ctas)
                rows[(shape, ctas)] = (x.view(torch.int16).cpu().numpy(), q.cpu().numpy())
    finally:
        ctx.set_tuning(B.TUNE_LBP_SHAPE, 0)
        ctx.set_tuning(B.TUNE_LBP_CTAS_PER_SM, 0)
    x0, q0 = rows[(2, 2)]
    for k, (x, q) in rows.items():
        assert (x == x0).all(), k
        assert np.allclose(q, q0, rtol=1e-6), k
    assert ctx.status() == 0


@pytest.mark.parametrize("crop", [64, 128])
@pytest.mark.parametrize("shape", [1, 2, 3])
def test_tile_shapes_on_edge_cases_precut_crops_and_affine(B, ctx, orc, crop, shape):
    """Each tile shape (one thread per cell, per half cell, per quarter cell) on the edge frames
    (all-hole faces, off-frame and bad rects), on pre-cut crops (no rects) and through the general
    affine path: bit-exact with the oracle."""
    ctx.set_tuning(B.TUNE_LBP_SHAPE, shape)
    try:
        g, d, r = _edge_frames()
        want = orc.features_batch(g, d, r, crop)
        ctx.status(clear=True)
        f, _, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop)
        assert (host_u16(f) == want).all()
        assert ctx.status() & B.STATUS_BAD_RECT
        gc, dc = synth.crops(21, 5, crop)
        f, _, _ = B.lbp_fused_features(ctx, dev_u8(gc), dev_u16(dc), None, crop=crop)
        assert (host_u16(f) == orc.features_batch(gc, dc, None, crop)).all()
        g, d, r = synth.frames_with_rects(23, 2, 3, 60, 160, H=240, W=320)
        n = r.shape[0]
        aff = np.zeros((n, 6), np.int32)
        for k in range(n):
            sc = r[k]["w"] / float(crop)
            aff[k] = [int(0.9 * sc * 65536), int(-0.3 * sc * 65536), int(r[k]["x"] * 65536),
                      int(0.3 * sc * 65536), int(0.9 * sc * 65536), int(r[k]["y"] * 65536)]
        f, _, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop,
                                       affine=torch.from_numpy(aff).cuda())
        assert (host_u16(f) == orc.features_batch(g, d, r, crop, affine=aff)).all()
    finally:
        ctx.set_tuning(B.TUNE_LBP_SHAPE, 0)


def test_general_affine_q16(B, ctx, orc):
    g, d, r = synth.frames_with_rects(8, 2, 3, 60, 160, H=240, W=320)
    n = r.shape[0]
    rng = np.random.default_rng(1)
    aff = np.zeros((n, 6), np.int32)
    for k in range(n):
        th = rng.uniform(-0.4, 0.4)
        s = r[k]["w"] / 96.0
        c, sn = np.cos(th) * s, np.sin(th) * s
        aff[k] = [int(c * 65536), int(-sn * 65536), int(r[k]["x"] * 65536),
                  int(sn * 65536), int(c * 65536), int(r[k]["y"] * 65536)]
    want = orc.features_batch(g, d, r, 96, affine=aff)
    f, _, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=96,
                                   affine=torch.from_numpy(aff).cuda())
    assert (host_u16(f) == want).all()
    cg, cd = B.rgbd_crop_affine(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), 96, 96, affine=torch.from_numpy(aff).cuda())
    for k in range(n):
        og, od = orc.crop(g[r[k]["frame"]], d[r[k]["frame"]], (0, 0, 1, 1), 96, 96, affine=aff[k])
        assert (cg[k].cpu().numpy() == og).all() and (host_u16(cd[k]) == od).all()


def test_quantised_rows_bit_exact(B, ctx, orc):
    g, d, r = synth.frames_with_rects(12, 2, 5, 48, 256)
    want = orc.features_batch(g, d, r, 128)
    x32 = orc.normalize_f32(want)
    dim = want.shape[1]
    _, xb, qb = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=128, feats=False,
                                     x_dtype="bf16")
    assert (xb.view(torch.int16).cpu().numpy().view(np.uint16)[:, :dim] == orc.f32_to_bf16(x32)).all()
    scale = np.float32(448.0)
    _, x8, q8 = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=128, feats=False,
                                     x_dtype="fp8", x_scale=float(scale))
    codes = orc.f32_to_e4m3((x32 * scale).astype(np.float32))
    assert (x8.cpu().numpy()[:, :dim] == codes).all()
    back = orc.e4m3_to_f64(codes) / float(scale)
    assert np.allclose(q8.cpu().numpy(), (back ** 2).sum(1), rtol=1e-5)
    # the same rows from stored counts (lbp_normalize_features)
    xn, _ = B.lbp_normalize_features(ctx, dev_u16(want), "bf16")
    assert (xn.view(torch.int16).cpu().numpy().view(np.uint16)[:, :dim] == orc.f32_to_bf16(x32)).all()
    # split bf16: hi = bf16(x), lo = bf16(x - hi) in fp32
    hi = orc.f32_to_bf16(x32)
    hi_f = (hi.astype(np.uint32) << 16).view(np.float32)
    lo = orc.f32_to_bf16((x32 - hi_f).astype(np.float32))
    for xs in [B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=128, feats=False,
                                    x_dtype="bf16x3")[1],
               B.lbp_normalize_features(ctx, dev_u16(want), "bf16x3")[0]]:
        planes = xs.view(torch.int16).cpu().numpy().view(np.uint16)
        assert planes.shape[0] == 2
        assert (planes[0][:, :dim] == hi).all() and (planes[1][:, :dim] == lo).all()


def test_normalize_poisson_counts(B, ctx, orc):
    rng = synth.rng_for(3)
    cnt = synth.poisson_counts(rng, 37, 16 * 16 * 59)
    cnt[3, :59 * 4] = 0  # empty cells
    x, q = B.lbp_normalize_features(ctx, dev_u16(cnt), "f32")
    x32 = orc.normalize_f32(cnt)
    assert (x.cpu().numpy()[:, :cnt.shape[1]].view(np.uint32) == x32.view(np.uint32)).all()


def test_alone_equals_in_mix(B, ctx, orc):
    g, d, r = synth.frames_with_rects(31, 4, 10, 48, 256)
    rt = B.rects_tensor(r)
    f_all, x_all, q_all = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), rt, x_dtype="bf16")
    for k in [0, 7, 19, 39]:
        f1, x1, q1 = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), rt[k:k + 1].contiguous(), x_dtype="bf16")
        assert torch.equal(f1[0], f_all[k]) and torch.equal(x1[0], x_all[k]) and torch.equal(q1[0], q_all[k])


# ---------------------------------------------------------------------------------------------
# A6-A7: scoring paths against the fp64 oracle
# ---------------------------------------------------------------------------------------------

def _scoring_problem(seed, n, n_sv, C, cells=16):
    rng = synth.rng_for(seed)
    dim = cells * 59
    X = synth.poisson_counts(rng, n, dim)
    SV = synth.poisson_counts(rng, n_sv, dim)
    a, b = synth.rbf_coefficients(rng, C, n_sv)
    b = rng.normal(0, 0.01, C).astype(np.float32)
    return X, SV, a, b, 1.0 / dim


@pytest.mark.parametrize("n,n_sv,C", [(3, 300, 10), (8, 1000, 64), (300, 700, 10), (100, 3000, 64)])
def test_rbf_f32_paths(B, ctx, orc, n, n_sv, C):
    X, SV, a, b, gamma = _scoring_problem(n * 7 + n_sv, n, n_sv, C)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype="f32")
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), "f32")
    s, lab = B.svm_score(ctx, model, x, q)
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, a, b, gamma))
    assert err <= 1e-5, err
    agree = (lab.cpu().numpy() == orc.argmax(ref)).mean()
    assert agree >= 0.99, agree


@pytest.mark.parametrize("dt", ["bf16", "tf32", "fp8", "bf16x3"])
@pytest.mark.parametrize("n,n_sv,C", [(300, 700, 10), (100, 3000, 64), (5, 256, 16)])
def test_rbf_tensor_core_paths(B, ctx, orc, dt, n, n_sv, C):
    X, SV, a, b, gamma = _scoring_problem(n * 11 + n_sv, n, n_sv, C)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype=dt)
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), dt, x_scale=448.0)
    s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
    assert ctx.status() == 0
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, a, b, gamma))
    bound = {"tf32": 2e-5, "bf16": 5e-5, "fp8": 1e-3, "bf16x3": 1e-8}[dt]
    print(f"{dt} n={n} n_sv={n_sv} C={C}: rel err {err:.3e}")
    assert err <= bound, err


def test_centred_model_and_rows_bit_exact(B, ctx, orc):
    """A model packed with centring: its centre equals the oracle's column means of the fp32 SV
    rows (fp64 sums in row order) bit for bit, and rows centred at it -- from stored counts and
    from the fused kernel -- equal the oracle's fp32 differences after each conversion."""
    rng = synth.rng_for(61)
    dim = 16 * 16 * 59
    SV = synth.poisson_counts(rng, 700, dim)
    a, b = synth.rbf_coefficients(rng, 12, 700)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=1.0 / dim, dtype="bf16",
                                  centred=True)
    assert model.centred
    mu = model.centre().cpu().numpy()
    want_mu = orc.sv_centre(orc.normalize_f32(SV))
    assert (mu[:dim].view(np.uint32) == want_mu.view(np.uint32)).all()
    assert (mu[dim:] == 0).all()
    g, d, r = synth.frames_with_rects(62, 2, 6, 48, 256)
    counts = orc.features_batch(g, d, r, 128)
    xc = orc.centre_rows(orc.normalize_f32(counts), mu[:dim])
    hi = orc.f32_to_bf16(xc)
    for dt in ["bf16", "f32", "fp8", "bf16x3"]:
        fused = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=128, feats=False,
                                     x_dtype=dt, x_centre=model)[1]
        stored = B.lbp_normalize_features(ctx, dev_u16(counts), dt, x_centre=model)[0]
        for xs in (fused, stored):
            if dt == "bf16":
                assert (host_u16(xs.view(torch.int16))[:, :dim] == hi).all()
            elif dt == "f32":
                assert (xs.cpu().numpy()[:, :dim].view(np.uint32) == xc.view(np.uint32)).all()
                assert (xs.cpu().numpy()[:, dim:] == 0).all()
            elif dt == "fp8":
                assert (xs.cpu().numpy()[:, :dim] == orc.f32_to_e4m3((xc * np.float32(448.0)).astype(np.float32))).all()
            else:
                planes = host_u16(xs.view(torch.int16))
                hi_f = (hi.astype(np.uint32) << 16).view(np.float32)
                assert (planes[0][:, :dim] == hi).all()
                assert (planes[1][:, :dim] == orc.f32_to_bf16((xc - hi_f).astype(np.float32))).all()


@pytest.mark.parametrize("dt", ["bf16", "fp8", "f32", "bf16x3"])
def test_centred_scores_against_the_oracle(B, ctx, orc, dt):
    """Scores of a centred model on centred rows against the fp64 oracle of the uncentred
    problem (centring leaves the RBF kernel unchanged): within each type's bound, and for bf16
    and FP8 tighter than the same problem scored without centring."""
    X, SV, a, b, gamma = _scoring_problem(63, 300, 1500, 32)
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    scale = rbf_error_scale(x64, sv64, a, b, gamma)
    errs = {}
    for centred in (False, True):
        model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype=dt,
                                      centred=centred)
        x, q = B.lbp_normalize_features(ctx, dev_u16(X), dt, x_scale=448.0, x_centre=model if centred else None)
        s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
        assert ctx.status() == 0
        errs[centred] = rel_score_error(s.cpu().numpy(), ref, scale)
    bound = {"f32": 1e-5, "bf16": 5e-5, "fp8": 1e-3, "bf16x3": 1e-8}[dt]
    print(f"{dt}: rel err raw {errs[False]:.3e}, centred {errs[True]:.3e}")
    assert errs[True] <= bound, errs
    if dt in ("bf16", "fp8"):
        assert errs[True] < errs[False], errs


def test_epilogue_expm1_accuracy(B):
    """The epilogue's e^z - 1 (Taylor polynomial near 0, expm1f beyond 2^-5) against fp64 and
    against CUDA's expm1f (torch.expm1): within 2 ulp of the exact value (3 of expm1f) everywhere, across the
    switch point and at the extremes of the scoring arguments."""
    rng = np.random.default_rng(5)
    z = np.concatenate([rng.uniform(-0.04, 0.04, 200000), rng.uniform(-1e-3, 1e-3, 100000),
                        rng.normal(0, 1e-6, 10000), np.linspace(-0.0313, -0.0312, 1001),
                        np.linspace(0.0312, 0.0313, 1001), rng.uniform(-20, 5, 10000),
                        [0.0, -0.0, 0.03125, -0.03125, 1e-30, -1e-30]]).astype(np.float32)
    zt = torch.from_numpy(z).cuda()
    ours = B.rgbd_debug_expm1(zt).cpu().numpy().astype(np.float64)
    cuda = torch.expm1(zt).cpu().numpy().astype(np.float64)
    exact = np.expm1(z.astype(np.float64))
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    ulp = np.maximum(ulp, np.float64(np.finfo(np.float32).tiny))
    assert np.max(np.abs(ours - exact) / ulp) <= 2.0
    assert np.max(np.abs(ours - cuda) / ulp) <= 3.0


def test_bounded_wait_gives_up_and_context_survives(B, ctx, orc):
    """Failure path of the tensor-core kernel's waits: a barrier phase that nothing completes makes
    the bounded wait give up after its limit (2 ms here), flag RGBD_STATUS_WAIT_TIMEOUT and return
    instead of hanging; the same context then scores correctly."""
    ctx.status(clear=True)
    res = B.rgbd_debug_wait_timeout(ctx, 2_000_000)
    torch.cuda.synchronize()
    assert res.item() == 1
    assert ctx.status(clear=True) & B.STATUS_WAIT_TIMEOUT
    X, SV, a, b, gamma = _scoring_problem(9, 20, 300, 10)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype="bf16")
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), "bf16")
    s, _ = B.svm_score(ctx, model, x, q)
    assert ctx.status() == 0
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    assert rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, a, b, gamma)) <= 5e-5


@pytest.mark.parametrize("mc", [3, 2])
@pytest.mark.parametrize("dt", ["bf16", "fp8", "tf32", "bf16x3"])
def test_tensor_core_pairing_modes(B, ctx, orc, dt, mc):
    """Each CTA pairing of the tensor-core kernel (2-CTA MMA pairs, single CTAs)
    against the fp64 oracle: 3 row blocks (so one padded CTA in a pair), 600 SVs (a ragged third
    SV tile), 100 classes (112 padded, 56 per CTA of a pair)."""
    X, SV, a, b, gamma = _scoring_problem(77 + mc, 300, 600, 100)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype=dt)
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), dt, x_scale=448.0)
    ctx.set_tuning(B.TUNE_TC_PAIRING, mc)
    try:
        s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
        assert ctx.status() == 0
    finally:
        ctx.set_tuning(B.TUNE_TC_PAIRING, 0)
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, a, b, gamma))
    bound = {"tf32": 2e-5, "bf16": 5e-5, "fp8": 1e-3, "bf16x3": 1e-8}[dt]
    print(f"{dt} pairing {mc}: rel err {err:.3e}")
    assert err <= bound, err


@pytest.mark.parametrize("splits", [1, 3])
def test_fp8_odd_k_block_count_in_pairs(B, ctx, orc, splits):
    """2-CTA pairs fill and release ring stages two at a time; an FP8 row of 3 x 3 cells
    (531 values, k_pad 640 = 5 k-blocks of 128 bytes) with 3 SV tiles per split ends a split on
    a half group (15 k-blocks), which the FULL/EMPTY bookkeeping must close."""
    X, SV, a, b, gamma = _scoring_problem(91 + splits, 300, 700, 12, cells=9)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype="fp8")
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), "fp8", x_scale=448.0)
    ctx.set_tuning(B.TUNE_TC_SPLITS, splits)
    ctx.set_tuning(B.TUNE_TC_PAIRING, 3)
    try:
        s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
        assert ctx.status() == 0
    finally:
        ctx.set_tuning(B.TUNE_TC_SPLITS, 0)
        ctx.set_tuning(B.TUNE_TC_PAIRING, 0)
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy(), ref, rbf_error_scale(x64, sv64, a, b, gamma))
    assert err <= 1e-3, err


@pytest.mark.parametrize("splits,mc", [(1, 2), (3, 2), (8, 2), (2, 3), (8, 3)])
def test_tuning_changes_layout_not_results(B, ctx, orc, splits, mc):
    """Forced SV splits / CTA pairing (the autotuner's knobs) keep the scores within tolerance."""
    X, SV, a, b, gamma = _scoring_problem(5, 300, 2000, 16)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype="bf16")
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), "bf16")
    s0, _ = B.svm_score(ctx, model, x, q)
    ctx.set_tuning(B.TUNE_TC_SPLITS, splits)
    ctx.set_tuning(B.TUNE_TC_PAIRING, mc)
    try:
        s1, _ = B.svm_score(ctx, model, x, q)
    finally:
        ctx.set_tuning(B.TUNE_TC_SPLITS, 0)
        ctx.set_tuning(B.TUNE_TC_PAIRING, 0)
    scale = rbf_error_scale(orc.normalize_f64(X), orc.normalize_f64(SV), a, b, gamma)
    assert rel_score_error(s1.cpu().numpy(), s0.cpu().numpy().astype(np.float64), scale) <= 1e-5


@pytest.mark.parametrize("dt,n,kz,n_sv,C,centred", [
    ("bf16", 1, 0, 2000, 24, False), ("bf16", 6, 0, 2000, 24, False), ("bf16", 100, 0, 2000, 24, False),
    ("bf16", 128, 0, 2000, 24, False), ("bf16", 37, 3, 2000, 24, False), ("bf16", 5, 59, 2000, 24, False),
    ("fp8", 12, 0, 2000, 24, False), ("tf32", 9, 5, 2000, 24, False), ("bf16x3", 17, 4, 2000, 24, False),
    ("bf16", 3, 0, 100, 3, False), ("bf16", 20, 0, 300, 128, False), ("bf16", 6, 0, 2000, 24, True),
    ("fp8", 12, 0, 2000, 24, True)])
def test_small_batch_split_k(B, ctx, orc, dt, n, kz, n_sv, C, centred):
    """Batches of one 128-row block split the K extent of every SV tile over several CTAs
    (automatically when the tiles alone fill few SMs; kz forces that many ranges): scores
    within the path's tolerance of the fp64 oracle, labels equal where the margin allows, and
    the same scores as the tile kernel within rounding."""
    # 2000 SVs: 8 SV tiles, the last ragged (100: one partial tile; 300 with 128 classes: the
    # widest coefficient rows); 64 cells: 30 FP8 k-blocks, so even FP8 has 3 K ranges
    X, SV, a, b, gamma = _scoring_problem(300 + n + kz, n, n_sv, C, cells=64)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype=dt, centred=centred)
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), dt, x_scale=448.0, x_centre=model if centred else None)
    ctx.set_tuning(B.TUNE_TC_SPLITK, kz)
    try:
        s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
        assert ctx.status() == 0
        ctx.set_tuning(B.TUNE_TC_SPLITK, 1)  # the tile kernel, for comparison
        s_tile, _ = B.svm_score(ctx, model, x, q, x_scale=448.0)
    finally:
        ctx.set_tuning(B.TUNE_TC_SPLITK, 0)
    x64, sv64 = orc.normalize_f64(X), orc.normalize_f64(SV)
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    scale = rbf_error_scale(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy(), ref, scale)
    bound = {"tf32": 2e-5, "bf16": 5e-5, "fp8": 1e-3, "bf16x3": 1e-8}[dt]
    print(f"{dt}{' centred' if centred else ''} n {n} kz {kz}: rel err {err:.3e}")
    assert err <= bound, err
    assert rel_score_error(s.cpu().numpy(), s_tile.cpu().numpy().astype(np.float64), scale) <= 2 * bound
    srt = np.sort(ref, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 4 * bound * scale.max()
    assert (lab.cpu().numpy()[clear] == orc.argmax(ref)[clear]).all()


# ---------------------------------------------------------------------------------------------
# Section 3's 0-255 face histogram and Section 2.3's nearest-centre tracking
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("crop", [200, 57, 255])
def test_face_histogram_256(B, ctx, orc, crop):
    g, d, r = synth.frames_with_rects(17, 2, 3, 40, 260, H=240, W=320)
    want = orc.features_batch(g, d, r, crop, cell=crop, nbins=256)
    f, x, q = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=crop,
                                   flags=B.LBP_FACE_HIST256, x_dtype="f32")
    assert (host_u16(f) == want).all()
    x32 = orc.normalize_f32(want, nbins=256)
    assert (x.cpu().numpy()[:, :256].view(np.uint32) == x32.view(np.uint32)).all()
    # pre-cut 200x200 crops, the paper's face size
    gc, dc = synth.crops(4, 2, 200)
    want2 = orc.features_batch(gc, dc, None, 200, cell=200, nbins=256)
    f2, _, _ = B.lbp_fused_features(ctx, dev_u8(gc), dev_u16(dc), None, crop=200, flags=B.LBP_FACE_HIST256)
    assert (host_u16(f2) == want2).all()


def test_face_histogram_256_centred_rows(B, ctx, orc):
    """Section 3's 0-255 face histogram with rows centred at a given vector: fp32 differences of
    the oracle's IEEE quotients, bit for bit; a centre that is not 16-byte aligned is rejected."""
    g, d, r = synth.frames_with_rects(19, 2, 3, 40, 260, H=240, W=320)
    want = orc.features_batch(g, d, r, 200, cell=200, nbins=256)
    rng = np.random.default_rng(3)
    mu = np.zeros(256 + 4, np.float32)
    mu[:256] = rng.uniform(0.0, 0.02, 256).astype(np.float32)
    mu_dev = dev_f32(mu)
    _, x, _ = B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=200,
                                   flags=B.LBP_FACE_HIST256, x_dtype="f32", x_centre=mu_dev[:256])
    xc = orc.centre_rows(orc.normalize_f32(want, nbins=256), mu[:256])
    assert (x.cpu().numpy()[:, :256].view(np.uint32) == xc.view(np.uint32)).all()
    with pytest.raises(B.RgbdError, match="aligned"):
        B.lbp_fused_features(ctx, dev_u8(g), dev_u16(d), B.rects_tensor(r), crop=200, flags=B.LBP_FACE_HIST256,
                             x_dtype="f32", x_centre=mu_dev[1:257])


def test_track_nearest(B, ctx, orc):
    rng = np.random.default_rng(5)
    R = synth.RECT_DTYPE
    prev = np.zeros(300, R)
    cur = np.zeros(280, R)
    for arr in (prev, cur):
        arr["frame"] = rng.integers(0, 32, len(arr))
        arr["x"] = rng.integers(-50, 600, len(arr))
        arr["y"] = rng.integers(-50, 450, len(arr))
        arr["w"] = rng.integers(48, 257, len(arr))
        arr["h"] = arr["w"]
    m = B.rgbd_track_nearest(ctx, B.rects_tensor(prev), B.rects_tensor(cur))
    assert (m.cpu().numpy() == orc.track_nearest(prev, cur)).all()


def test_track_streams_against_oracle(B, ctx, orc):
    """Per-stream identities over a sequence of batches: ids and the device-resident state equal
    the oracle's, including streams that skip batches, empty frames, repeated streams within a
    batch, more faces than the state holds and an out-of-range stream id."""
    R = orc.RECT_DTYPE
    rng = np.random.default_rng(23)
    S, M = 6, 5
    state = B.TrackState(S, M)
    ref = {"rects": np.zeros((S, M), R), "ids": np.full((S, M), -1, np.int32), "count": np.zeros(S, np.int32)}
    for it in range(25):
        nfr = int(rng.integers(1, 9))
        fs = rng.integers(0, S, nfr).astype(np.int32)
        if it == 7:
            fs[0] = S + 3  # out of range: labels pass through
        counts = rng.integers(0, 9, nfr)
        start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        n = int(start[-1])
        rects = np.zeros(n, R)
        rects["frame"] = 99
        rects["x"] = rng.integers(-20, 620, n)
        rects["y"] = rng.integers(-20, 460, n)
        rects["w"] = rng.integers(8, 120, n)
        rects["h"] = rng.integers(8, 120, n)
        labels = rng.integers(0, 30, n).astype(np.int32)
        want = orc.track_streams(ref, fs, start, rects, labels)
        got = B.rgbd_track_streams(ctx, state, torch.from_numpy(fs).cuda(), torch.from_numpy(start).cuda(),
                                   B.rects_tensor(rects), torch.from_numpy(labels).cuda())
        assert (got.cpu().numpy() == want).all(), it
        ctx.status(clear=True)
    assert (state.count.cpu().numpy() == ref["count"]).all()
    for s in range(S):
        c = int(ref["count"][s])
        assert (state.ids.cpu().numpy()[s, :c] == ref["ids"][s, :c]).all()
        got_r = state.rects.cpu().numpy()[s, :c]
        for k, f in enumerate(["frame", "x", "y", "w", "h"]):
            assert (got_r[:, k] == ref["rects"][f][s, :c]).all()


# ---------------------------------------------------------------------------------------------
# Section 2.1: depth-space region of a colour-detected face
# ---------------------------------------------------------------------------------------------

def test_face_roi_against_oracle(B, ctx, orc):
    """Synthetic frames, calibrations and colour boxes (plus rects outside the colour image,
    partly outside, tiny, with a bad frame index and a degenerate calibration): the depth rects
    equal the oracle's full-frame scan exactly."""
    rng = synth.rng_for(41)
    grey, depth, rects = synth.frames_with_rects(41, 3, 5, 48, 256)
    boxes = synth.colour_boxes(rng, rects)
    extra = np.array([(0, 700, 10, 40, 40), (1, -30, -30, 50, 50), (2, 300, 200, 1, 1), (5, 10, 10, 20, 20),
                      (0, 10, 10, 0, 20)], orc.RECT_DTYPE)
    boxes = np.concatenate([boxes, extra])
    d_dev = torch.from_numpy(depth.view(np.int16)).cuda()
    for k in range(4):
        cal = synth.calibration(rng)
        if k == 3:  # a mapping that collapses the y axis: the kernel scans the whole frame
            cal["a"][3], cal["a"][4] = 0, 0
        want = orc.face_roi(depth, cal, boxes)
        got = B.rgbd_face_roi(ctx, d_dev, B.Calib.from_record(cal), B.rects_tensor(boxes)).cpu().numpy()
        for i, f in enumerate(["frame", "x", "y", "w", "h"]):
            assert (got[:, i] == want[f]).all(), (k, f)
        if k == 0:
            assert (want["w"][:15] > 0).all()  # the synthetic faces are found
        ctx.status(clear=True)


# ---------------------------------------------------------------------------------------------
# Section 2.5: one-vs-rest RBF SVM training (SMO) on the GPU
# ---------------------------------------------------------------------------------------------

def _class_counts(seed, n, cells, C):
    rng = synth.rng_for(seed)
    dim = cells * 59
    protos = rng.uniform(0.5, 1.5, (C, dim))
    lab = rng.integers(0, C, n).astype(np.int32)
    counts = rng.poisson(3.0 * protos[lab]).astype(np.uint16)
    test = rng.poisson(3.0 * protos[rng.integers(0, C, 64)]).astype(np.uint16)
    return counts, lab, test


def test_svm_train_against_oracle_and_scoring(B, ctx, orc):
    """GPU SMO (fp32 kernel matrix and gradient) against the fp64 oracle on decision values of
    unseen rows, then the trained coefficients packed and scored through svm_score."""
    C, gamma, cost, eps = 4, 5.0, 1.0, 1e-4
    counts, lab, test = _class_counts(61, 300, 16, C)
    x, q = B.lbp_normalize_features(ctx, dev_u16(counts), "f32")
    coef, bias, iters = B.svm_train_rbf(ctx, x, q, torch.from_numpy(lab).cuda(), C, gamma, cost, eps)
    assert ctx.status() == 0
    a, b, it = orc.svm_train_rbf(orc.normalize_f64(counts), lab, C, gamma, cost, eps=eps)
    x64, t64 = orc.normalize_f64(counts), orc.normalize_f64(test)
    Kt = np.exp(-gamma * ((t64[:, None, :] - x64[None, :, :]) ** 2).sum(-1))
    f_gpu = Kt @ coef.cpu().numpy().astype(np.float64).T + bias.cpu().numpy()
    f_orc = Kt @ a.T + b
    assert np.abs(f_gpu - f_orc).max() < 2e-3, np.abs(f_gpu - f_orc).max()
    assert (iters.cpu().numpy() > 0).all() and (iters.cpu().numpy() < 200000).all()
    # box and equality constraints hold on the GPU solution
    y = np.where(lab[None, :] == np.arange(C)[:, None], 1, -1)
    alpha = coef.cpu().numpy() * y
    assert (alpha >= 0).all() and (alpha <= cost * (1 + 1e-6)).all()
    assert np.abs((coef.cpu().numpy()).sum(1)).max() < 1e-3
    # train -> pack -> score: the library's scoring of the trained model equals its definition
    model = B.svm_train_data_pack(ctx, dev_u16(counts), coef, bias, gamma=gamma, dtype="f32")
    xt, qt = B.lbp_normalize_features(ctx, dev_u16(test), "f32")
    s, labels = B.svm_score(ctx, model, xt, qt)
    assert np.abs(s.cpu().numpy() - f_gpu).max() < 1e-4
    srt = np.sort(f_orc, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 5e-3
    assert (labels.cpu().numpy()[clear] == np.argmax(f_orc, axis=1)[clear]).all()


# ---------------------------------------------------------------------------------------------
# The batch workload at full size, and empty inputs
# ---------------------------------------------------------------------------------------------

def test_full_batch_workload_sampled(B, ctx, orc):
    """The headline batch at its full size (256 frames 640x480, 4096 faces of side 48-256, 4096
    SVs x 64 classes, bf16 scoring) in the default launch layout: every face's feature row is
    bit-exact with the oracle; 32 sampled faces' scores are within the bf16 bound of the fp64
    oracle, and their labels agree wherever the fp64 margin is clear of that bound."""
    wl = synth.batching()
    model = B.svm_train_data_pack(ctx, dev_u16(wl.sv_counts), dev_f32(wl.coef), dev_f32(wl.bias), gamma=wl.gamma,
                                  dtype="bf16")
    f, x, q = B.lbp_fused_features(ctx, dev_u8(wl.grey), dev_u16(wl.depth), B.rects_tensor(wl.rects), crop=128,
                                   x_dtype="bf16")
    s, lab = B.svm_score(ctx, model, x, q)
    assert ctx.status() == 0
    want_all = orc.features_batch(wl.grey, wl.depth, wl.rects, 128)
    got_all = host_u16(f)
    bad = np.flatnonzero((got_all != want_all).any(axis=1))
    assert bad.size == 0, f"{bad.size} of {wl.n_crops} feature rows differ, first {bad[:8]}"
    idx = np.linspace(0, wl.n_crops - 1, 32).astype(int)
    want = want_all[idx]
    x64, sv64 = orc.normalize_f64(want), orc.normalize_f64(wl.sv_counts)
    ref = orc.svm_rbf(x64, sv64, wl.coef, wl.bias, wl.gamma)
    scale = rbf_error_scale(x64, sv64, wl.coef, wl.bias, wl.gamma)
    assert rel_score_error(s.cpu().numpy()[idx], ref, scale) <= 5e-5
    srt = np.sort(ref, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 2 * 5e-5 * scale.max()
    assert (lab.cpu().numpy()[idx][clear] == orc.argmax(ref)[clear]).all()


@pytest.mark.parametrize("dt,centred,bound", [("bf16", False, 5e-5), ("bf16", True, 5e-5), ("fp8", False, 1e-3)])
def test_precision_workload_full_size_sampled(B, ctx, orc, dt, centred, bound):
    """The precision workload at its full size (65536 rows x 16384 SVs x 15104 dims, 128
    classes) in the default launch layout: 12 sampled rows' scores within the type's bound of the
    fp64 oracle, labels equal wherever the fp64 margin clears twice that bound."""
    dim, n_rows, n_sv, C = 16 * 16 * 59, 65536, 16384, 128
    X = synth.poisson_counts_device(1507, n_rows, dim, "cuda")
    SV = synth.poisson_counts_device(1508, n_sv, dim, "cuda")
    a, b = synth.rbf_coefficients(synth.rng_for(1509), C, n_sv)
    gamma = 1.0 / dim
    model = B.svm_train_data_pack(ctx, SV, dev_f32(a), dev_f32(b), gamma=gamma, dtype=dt, centred=centred)
    x, q = B.lbp_normalize_features(ctx, X, dt, x_scale=448.0, x_centre=model if centred else None)
    s, lab = B.svm_score(ctx, model, x, q, x_scale=448.0)
    assert ctx.status() == 0
    idx = np.linspace(0, n_rows - 1, 12).astype(int)
    xs = X[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint16)
    x64, sv64 = orc.normalize_f64(xs), orc.normalize_f64(SV.cpu().numpy().view(np.uint16))
    ref = orc.svm_rbf(x64, sv64, a, b, gamma)
    scale = rbf_error_scale(x64, sv64, a, b, gamma)
    err = rel_score_error(s.cpu().numpy()[idx], ref, scale)
    print(f"{dt} centred={centred}: rel err {err:.3e}")
    assert err <= bound, err
    srt = np.sort(ref, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 2 * bound * scale.max()
    assert (lab.cpu().numpy()[idx][clear] == orc.argmax(ref)[clear]).all()
    model.free()


def test_empty_inputs(B, ctx, orc):
    """Every batch entry point accepts zero items: nothing is launched, nothing is flagged."""
    g, d, _ = synth.frames_with_rects(3, 1, 1, 48, 64, H=64, W=64)
    gd, dd = dev_u8(g), dev_u16(d)
    none = torch.zeros((0, 5), dtype=torch.int32, device="cuda")
    og, od = B.rgbd_crop_affine(ctx, gd, dd, none, 32, 32)
    assert og.shape == (0, 32, 32)
    f, x, q = B.lbp_fused_features(ctx, gd, dd, none, crop=64, x_dtype="bf16")
    assert f.shape[0] == 0 and x.shape[0] == 0
    x0, q0 = B.lbp_normalize_features(ctx, torch.zeros((0, 3776), dtype=torch.int16, device="cuda"), "f32")
    rng = synth.rng_for(4)
    sv = synth.poisson_counts(rng, 300, 16 * 59)
    a, b = synth.rbf_coefficients(rng, 10, 300)
    for dt in ("f32", "bf16"):
        model = B.svm_train_data_pack(ctx, dev_u16(sv), dev_f32(a), dev_f32(b), gamma=1.0 / (16 * 59), dtype=dt)
        xe = torch.zeros(B.x_shape(B._dt(dt), 0, model.k_pad), dtype=B.x_torch_dtype(B._dt(dt)), device="cuda")
        qe = torch.zeros((0,), dtype=torch.float32, device="cuda")
        s, lab = B.svm_score(ctx, model, xe, qe)
        assert s.shape == (0, 10)
        if dt == "bf16":
            s, lab = B.svm_score_noalloc(ctx, model, xe, qe)
            assert s.shape == (0, 10)
    assert B.rgbd_track_nearest(ctx, none, none).shape == (0,)
    st = B.TrackState(2, 4)
    ids = B.rgbd_track_streams(ctx, st, torch.zeros((0,), dtype=torch.int32, device="cuda"),
                               torch.zeros((1,), dtype=torch.int32, device="cuda"), none,
                               torch.zeros((0,), dtype=torch.int32, device="cuda"))
    assert ids.shape == (0,)
    cal = synth.calibration(rng, 64, 64)
    assert B.rgbd_face_roi(ctx, dd, B.Calib.from_record(cal), none).shape == (0, 5)
    torch.cuda.synchronize()
    assert ctx.status() == 0
