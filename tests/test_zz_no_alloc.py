"""svm_score_noalloc: tensor-core RBF scoring that allocates no device memory.

Some callers cannot let a library call cudaMalloc: real-time loops that cannot take the
device-wide synchronisation of cudaMalloc / cudaFree in the middle of a frame, and processes
whose device memory another allocator already owns.  For them svm_score_noalloc keeps its
partial sums in a fixed 16 MiB array that the library holds on each GPU.  This file is
collected last (tests/test_zz_*), so a run that stops at its first failure has run every other
test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1504_01883_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from gpu_util import dev_f32, dev_u16, rbf_error_scale, rel_score_error  # noqa: E402


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


def _problem(B, ctx, seed, n, n_sv, C, dt):
    rng = synth.rng_for(seed)
    dim = 16 * 59
    X = synth.poisson_counts(rng, n, dim)
    SV = synth.poisson_counts(rng, n_sv, dim)
    a, b = synth.rbf_coefficients(rng, C, n_sv)
    model = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=1.0 / dim, dtype=dt)
    x, q = B.lbp_normalize_features(ctx, dev_u16(X), dt, x_scale=448.0)
    return X, SV, a, b, 1.0 / dim, model, x, q


def test_noalloc_matches_svm_score_on_two_calls_in_a_row(B, ctx, orc):
    """Three different problems back to back through the C ABI: each result must equal the
    existing svm_score's within the fp32 score tolerance of the parity tests (1e-5 of
    sum_i |a_ci| K_i + |b_c|), with identical labels, although the second call finds the
    first call's partial sums still in the shared scratch."""
    probs = [_problem(B, ctx, 41, 300, 700, 10, "bf16"), _problem(B, ctx, 42, 100, 3000, 64, "tf32"),
             _problem(B, ctx, 44, 200, 900, 20, "bf16x3")]
    for X, SV, a, b, gamma, model, x, q in probs:
        s_ref, l_ref = B.svm_score(ctx, model, x, q, x_scale=448.0)
        s_na, l_na = B.svm_score_noalloc(ctx, model, x, q, x_scale=448.0)
        torch.cuda.synchronize()
        scale = rbf_error_scale(orc.normalize_f64(X), orc.normalize_f64(SV), a, b, gamma)
        err = rel_score_error(s_na.cpu().numpy(), s_ref.cpu().numpy().astype(np.float64), scale)
        assert err <= 1e-5, err
        assert torch.equal(l_na, l_ref)
    assert ctx.status() == 0


def test_noalloc_rejects_sizes_above_its_scratch(B, ctx):
    X, SV, a, b, gamma, model, x, q = _problem(B, ctx, 43, 8, 256, 128, "bf16")
    # 40000 rows x 128 classes of fp32 partial sums exceed the 16 MiB array
    big = torch.zeros((40000, x.shape[1]), dtype=x.dtype, device=x.device)
    bq = torch.zeros((40000,), dtype=torch.float32, device=x.device)
    with pytest.raises(B.RgbdError, match="scratch"):
        B.svm_score_noalloc(ctx, model, big, bq, x_scale=448.0)
    f32 = B.svm_train_data_pack(ctx, dev_u16(SV), dev_f32(a), dev_f32(b), gamma=gamma, dtype="f32")
    with pytest.raises(B.RgbdError):
        B.svm_score_noalloc(ctx, f32, x.float(), q)


def test_noalloc_call_takes_no_device_memory(B, ctx, orc):
    """A call on a fresh context leaves the device's free memory unchanged.  Outputs are passed
    in, and a call on another context has already looked the scratch array up and loaded the
    kernels, so any change would come from the call itself (svm_score, on the same fresh
    context, would have to grow the empty workspace with cudaMalloc)."""
    X, SV, a, b, gamma, model, x, q = _problem(B, ctx, 45, 600, 1200, 32, "bf16")
    s_out = torch.empty((600, 32), dtype=torch.float32, device=x.device)
    l_out = torch.empty((600,), dtype=torch.int32, device=x.device)
    B.svm_score_noalloc(ctx, model, x, q, scores=s_out, labels=l_out)  # another context's call
    c = B.Context(0)
    try:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        B.svm_score_noalloc(c, model, x, q, scores=s_out, labels=l_out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        s_ref, l_ref = B.svm_score(c, model, x, q)
        torch.cuda.synchronize()
        scale = rbf_error_scale(orc.normalize_f64(X), orc.normalize_f64(SV), a, b, gamma)
        err = rel_score_error(s_out.cpu().numpy(), s_ref.cpu().numpy().astype(np.float64), scale)
        assert err <= 1e-5, err
        assert torch.equal(l_out, l_ref)
        assert c.status() == 0
    finally:
        c.close()
