"""The continuous-batching request loop: admission by memory (host logic, CPU) and, on the GPU,
every frame's scores are the same when served alone as in the mix of a busy run."""
import numpy as np
import pytest

from paper_1504_01883_gb300 import synth


def test_admission_waits_for_memory_and_slots():
    torch = pytest.importorskip("torch")  # noqa: F841 (serve imports torch)
    from paper_1504_01883_gb300.serve import MemoryAdmission
    free = {"bytes": 1 << 30}
    adm = MemoryAdmission(2, reserve_bytes=512 << 20, mem_get_info=lambda: (free["bytes"], 1 << 34))
    a, b = adm.try_admit(), adm.try_admit()
    assert {a, b} == {0, 1}
    assert adm.try_admit() == -1           # no slot
    adm.release(a)
    free["bytes"] = 100 << 20              # the device is short of memory (a fake mem_get_info)
    assert adm.try_admit() == -1 and adm.rejections == 1
    free["bytes"] = 1 << 30
    assert adm.try_admit() == a


def test_admission_charges_each_frames_bytes_against_the_budget():
    pytest.importorskip("torch")
    from paper_1504_01883_gb300.serve import MemoryAdmission
    adm = MemoryAdmission(4, reserve_bytes=0, mem_get_info=lambda: (1 << 40, 1 << 40), budget_bytes=1000)
    a = adm.try_admit(600)
    assert a >= 0 and adm.used == 600
    assert adm.try_admit(500) == -1 and adm.rejections == 1   # a slot is free, the bytes are not
    b = adm.try_admit(400)
    assert b >= 0 and adm.used == 1000
    adm.release(a)
    assert adm.used == 400
    assert adm.try_admit(500) >= 0 and adm.used == 900


def test_arrivals_are_seeded_and_ordered():
    ev = synth.serving_arrivals(seed=3, n_streams=4, seconds=1.0)
    assert ev == sorted(ev)
    assert ev == synth.serving_arrivals(seed=3, n_streams=4, seconds=1.0)
    assert all(1 <= k <= 12 for _, _, k in ev)
    assert 60 < len(ev) < 200  # about 4 x 30 per second


@pytest.mark.gpu
def test_each_frame_is_the_same_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1504_01883_gb300 import _build, serve
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(99)
    sv = synth.poisson_counts(rng, 1024, dim)
    a, b = synth.rbf_coefficients(rng, 16, 1024)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).cuda(), torch.from_numpy(a).cuda(),
                                  torch.from_numpy(b).cuda(), gamma=1.0 / dim, dtype="bf16")
    streams = serve.make_streams(seed=7, n_streams=6, frames_per_stream=2)
    events = synth.serving_arrivals(seed=7, n_streams=6, seconds=0.3)
    srv = serve.BatchServer(ctx, model, streams, n_slots=24, max_faces=512)
    rep, reqs = srv.run(events, keep_results=True, realtime=False)  # everything at once: big mixed batches
    assert rep.frames == len(events) and rep.batches < len(events)
    alone = serve.BatchServer(ctx, model, streams, n_slots=2, max_faces=16)
    scale = np.abs(a).sum(1)[None, :] + np.abs(b)[None, :]
    for req in reqs[:: max(1, len(reqs) // 12)]:
        one = alone.serve_one(req.stream, req.index)
        assert one.n_faces == req.n_faces
        assert np.max(np.abs(one.scores - req.scores) / scale) <= 5e-5
        # labels are unique where the top two classes are further apart than the tolerance
        srt = np.sort(req.scores, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > 5e-5 * scale.max()
        assert (one.labels[clear] == req.labels[clear]).all()
    assert ctx.status() == 0


@pytest.mark.gpu
def test_served_identities_follow_the_tracking_rule():
    """The batched loop's per-stream device state gives every served face the identity the
    oracle's Section 2.3 tracking gives when the same frames and labels are replayed in
    arrival order."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle as orc
    from paper_1504_01883_gb300 import _build, serve
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(98)
    sv = synth.poisson_counts(rng, 512, dim)
    a, b = synth.rbf_coefficients(rng, 8, 512)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).cuda(), torch.from_numpy(a).cuda(),
                                  torch.from_numpy(b).cuda(), gamma=1.0 / dim, dtype="bf16")
    streams = serve.make_streams(seed=8, n_streams=5, frames_per_stream=3)
    events = synth.serving_arrivals(seed=8, n_streams=5, seconds=0.4)
    srv = serve.BatchServer(ctx, model, streams, n_slots=12, max_faces=256)
    rep, reqs = srv.run(events, keep_results=True, realtime=False)
    assert rep.frames == len(reqs)
    state = {"rects": np.zeros((5, 16), orc.RECT_DTYPE), "ids": np.full((5, 16), -1, np.int32),
             "count": np.zeros(5, np.int32)}
    order = sorted(range(len(reqs)), key=lambda i: (reqs[i].t_arrival, i))
    for i in order:
        req = reqs[i]
        rects = streams[req.stream].rects[req.index % len(streams[req.stream].rects)]
        want = orc.track_streams(state, [req.stream], [0, len(rects)], rects, req.labels)
        assert (req.ids == want).all()
    assert ctx.status() == 0


@pytest.mark.gpu
def test_native_request_loop_matches_the_oracle_and_the_python_loop():
    """The library's own request loop (rgbd_server): every frame's scores equal its scores served
    alone and the Python loop's within the bf16 tolerance, labels agree where the top two classes
    are clear of it, and the identities follow the oracle's Section 2.3 tracking replayed in
    submission order.  A stream id out of range is rejected at submission."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle as orc
    from paper_1504_01883_gb300 import _build, serve
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(97)
    sv = synth.poisson_counts(rng, 1024, dim)
    a, b = synth.rbf_coefficients(rng, 16, 1024)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).cuda(), torch.from_numpy(a).cuda(),
                                  torch.from_numpy(b).cuda(), gamma=1.0 / dim, dtype="bf16")
    streams = serve.make_streams(seed=9, n_streams=6, frames_per_stream=3)
    events = synth.serving_arrivals(seed=9, n_streams=6, seconds=0.3)
    nat = serve.NativeBatchServer(ctx, model, streams, n_slots=24, max_faces=512)
    try:
        rep, reqs = nat.run(events, keep_results=True, realtime=False)  # all at once: mixed batches
        assert rep.frames == len(events) and rep.batches < len(events)
        py = serve.BatchServer(ctx, model, streams, n_slots=24, max_faces=512)
        _, preqs = py.run(events, keep_results=True, realtime=False)
        scale = np.abs(a).sum(1)[None, :] + np.abs(b)[None, :]
        for req, pr in zip(reqs, preqs):
            assert np.max(np.abs(req.scores - pr.scores) / scale) <= 5e-5
        for req in reqs[:: max(1, len(reqs) // 8)]:
            one = nat.serve_one(req.stream, req.index)
            assert np.max(np.abs(one.scores - req.scores) / scale) <= 5e-5
            srt = np.sort(req.scores, axis=1)
            clear = (srt[:, -1] - srt[:, -2]) > 5e-5 * scale.max()
            assert (one.labels[clear] == req.labels[clear]).all()
        # identities of the mixed run against the oracle's tracking in submission order (the
        # alone calls above came after it and do not change these results)
        state = {"rects": np.zeros((6, 16), orc.RECT_DTYPE), "ids": np.full((6, 16), -1, np.int32),
                 "count": np.zeros(6, np.int32)}
        for req in reqs:
            rects = streams[req.stream].rects[req.index % len(streams[req.stream].rects)]
            want = orc.track_streams(state, [req.stream], [0, len(rects)], rects, req.labels)
            assert (req.ids == want).all()
        g = torch.zeros((8, 8), dtype=torch.uint8)
        with pytest.raises(B.RgbdError, match="stream"):
            nat.srv.submit(99, g, g.view(torch.int16), torch.zeros((0, 5), dtype=torch.int32),
                           torch.zeros((0, 16)), torch.zeros((0,), dtype=torch.int32))
    finally:
        nat.close()
    assert ctx.status() == 0


@pytest.mark.gpu
def test_native_loop_edge_cases():
    """Frames without faces pass through, a frame with more faces than a batch holds is
    rejected, and destroying the server with requests still queued (more than its frame slots)
    serves them first: every copy of the same frame gets the same scores."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1504_01883_gb300 import _build, serve
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(96)
    sv = synth.poisson_counts(rng, 256, dim)
    a, b = synth.rbf_coefficients(rng, 8, 256)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).cuda(), torch.from_numpy(a).cuda(),
                                  torch.from_numpy(b).cuda(), gamma=1.0 / dim, dtype="bf16")
    streams = serve.make_streams(seed=11, n_streams=2, frames_per_stream=2)
    H, W = streams[0].grey.shape[1:]
    srv = B.NativeServer(model, H, W, n_streams=2, n_slots=4, max_batch_faces=16)
    g = torch.from_numpy(streams[0].grey[0]).pin_memory()
    d = torch.from_numpy(streams[0].depth[0].view(np.int16)).pin_memory()
    rects = torch.from_numpy(np.ascontiguousarray(streams[0].rects[0]).view(np.int32).reshape(-1, 5))
    n = rects.shape[0]
    none = torch.zeros((0, 5), dtype=torch.int32)
    ids = []
    outs = []
    for k in range(12):  # more than the slots: the queue drains through them
        r = rects if k % 3 else none
        sc = torch.empty((r.shape[0], 8))
        lb = torch.empty((r.shape[0],), dtype=torch.int32)
        outs.append((r.shape[0], sc, lb))
        ids.append(srv.submit(k % 2, g, d, r, sc, lb))
    big = torch.zeros((17, 5), dtype=torch.int32)
    with pytest.raises(B.RgbdError, match="faces"):
        srv.submit(0, g, d, big, torch.empty((17, 8)), torch.empty((17,), dtype=torch.int32))
    # a rect of zero width: the face gets zero features and its batch reports the flag
    bad = rects[:1].clone()
    bad[0, 3] = 0
    bad_id = srv.submit(0, g, d, bad, torch.empty((1, 8)), torch.empty((1,), dtype=torch.int32))
    flags = None
    for _ in range(200):
        for c in srv.poll(wait_us=50000):
            if c[0] == bad_id:
                flags = c[5]
        if flags is not None:
            break
    assert flags is not None and flags & B.STATUS_BAD_RECT
    for k in range(12):  # queue more than the slots again, then stop with them pending
        r = rects if k % 3 else none
        sc = torch.empty((r.shape[0], 8))
        lb = torch.empty((r.shape[0],), dtype=torch.int32)
        outs.append((r.shape[0], sc, lb))
        srv.submit(k % 2, g, d, r, sc, lb)
    srv.close()  # serves the queued requests before it stops
    ref = None
    for nf, sc, lb in outs:
        if nf:
            ref = sc if ref is None else ref
            assert torch.allclose(sc, ref, rtol=0, atol=5e-5 * float(np.abs(a).sum(1).max()))
    assert ref is not None and n > 0
    assert ctx.status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("dt,centred", [("fp8", False), ("bf16", True), ("f32", False)])
def test_native_loop_model_types(dt, centred):
    """The request loop scores with the model's own type (FP8 rows at the configured scale,
    centred rows for a centred model, exact fp32): each frame's scores equal those of the C-ABI
    calls made by hand on the same frame, within that type's parity tolerance."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1504_01883_gb300 import _build, serve
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(95)
    sv = synth.poisson_counts(rng, 300, dim)
    a, b = synth.rbf_coefficients(rng, 10, 300)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).cuda(), torch.from_numpy(a).cuda(),
                                  torch.from_numpy(b).cuda(), gamma=1.0 / dim, dtype=dt, centred=centred)
    streams = serve.make_streams(seed=12, n_streams=3, frames_per_stream=2)
    H, W = streams[0].grey.shape[1:]
    srv = B.NativeServer(model, H, W, n_streams=3, n_slots=4, max_batch_faces=64, x_scale=448.0)
    scale = np.abs(a).sum(1)[None, :] + np.abs(b)[None, :]
    bound = {"fp8": 1e-3, "bf16": 5e-5, "f32": 1e-5}[dt]
    try:
        for s_id, st in enumerate(streams):
            for k in range(2):
                g = torch.from_numpy(st.grey[k]).pin_memory()
                d = torch.from_numpy(st.depth[k].view(np.int16)).pin_memory()
                rr = np.ascontiguousarray(st.rects[k])
                rects = torch.from_numpy(rr.view(np.int32).reshape(-1, 5))
                sc = torch.empty((rects.shape[0], 10))
                lb = torch.empty((rects.shape[0],), dtype=torch.int32)
                rid = srv.submit(s_id, g, d, rects, sc, lb)
                got = []
                for _ in range(200):
                    got += [c for c in srv.poll(wait_us=50000) if c[0] == rid]
                    if got:
                        break
                assert got and got[0][1] == 0
                _, x, q = B.lbp_fused_features(ctx, g.cuda()[None], d.cuda()[None], B.rects_tensor(rr), crop=128,
                                               feats=False, x_dtype=dt, x_scale=448.0,
                                               x_centre=model if centred else None)
                want, _ = B.svm_score(ctx, model, x, q, x_scale=448.0)
                assert np.max(np.abs(sc.numpy() - want.cpu().numpy()) / scale) <= bound
    finally:
        srv.close()
    assert ctx.status() == 0
