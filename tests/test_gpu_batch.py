"""The batched form (one persistent score launch over many scenes, replayed
as a CUDA graph) gives bit-identical scores, masks, thresholds and
compacted scenes to the per-scene entry points, on every replay."""
import numpy as np
import pytest

from paper_2606_09074_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09074_gb300 import binding as rb
    ctx = rb.Context(0)
    yield torch, rb, ctx
    ctx.close()


def upload(torch, rb, w):
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(w.scene.pos).to(dev)
    if w.scene.dtype == "bf16":
        attr = torch.from_numpy(w.scene.attr.view(np.int16)).to(dev).view(torch.bfloat16)
    elif w.scene.dtype == "bf16s":
        attr = rb.MixedRows.from_float(w.scene.attr, device=dev)
    else:
        attr = torch.from_numpy(w.scene.attr).to(dev)
    return pos, attr, rb.cameras_to_device(w.cams, dev)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_equals_single(env, dtype):
    torch, rb, ctx = env
    # the last scene is large enough for the single-scene compaction's segment form
    specs = [(11, 3000, 7), (12, 40_000, 50), (13, 257, 3), (14, 123_457, 120), (15, 1, 1), (16, 70_001, 300),
             (17, 1_900_003, 6)]
    ws = []
    for seed, n, v in specs:
        w = synth.random_scene(seed=seed, n=n, v=v, means="core_shell")
        if dtype == "bf16":
            w.scene = w.scene.to_bf16()
        ws.append(w)
    ratios = [0.5, 0.66, 0.9, 0.0, 0.5, 0.3, 0.5]
    up = [upload(torch, rb, w) for w in ws]
    jobs = [{"pos": p, "attr": a, "cams": c, "ratio": r} for (p, a, c), r in zip(up, ratios)]
    batch = rb.Batch(ctx, jobs)
    for rep in range(2):
        batch.run()
        assert batch.launches() >= 6 * len(jobs)  # recorded on the first run
        nk_b, thr_b = batch.results()
        for k, ((p, a, c), r) in enumerate(zip(up, ratios)):
            s = ctx.score(p, a, c)
            m, thr, nk = ctx.select(s, r)
            op, oa, idx = ctx.compact(p, a, m, nk)
            out = batch.outputs[k]
            assert torch.equal(out["scores"], s), (rep, k)
            n = p.shape[1]
            assert torch.equal(out["mask"][: (n + 31) // 32], m[: (n + 31) // 32])
            assert nk_b[k] == nk and thr_b[k] == thr
            assert torch.equal(out["idx"][:nk], idx)
            assert torch.equal(out["out_pos"][:, :nk], op)
            assert torch.equal(out["out_attr"][:, :nk], oa)
    ctx.check()
    batch.close()


def test_batch_rejects_bad_jobs(env):
    torch, rb, ctx = env
    w1 = synth.random_scene(seed=1, n=100, v=4)
    p1, a1, c1 = upload(torch, rb, w1)
    with pytest.raises(rb.RefineError):
        rb.Batch(ctx, [{"pos": p1, "attr": a1, "cams": c1, "ratio": 1.0}])
    with pytest.raises(rb.RefineError):
        rb.Batch(ctx, [{"pos": p1[:, :0], "attr": a1[:, :0], "cams": c1, "ratio": 0.5}])  # an empty scene


def test_batch_mixed_storage_and_flags(env):
    """Scenes of all three storage types share one batched launch; each
    equals its own per-scene run (scores, and the compacted rows of the
    mixed-layout scene), for every projection mode."""
    torch, rb, ctx = env
    ws = []
    for k, (seed, n, v) in enumerate([(41, 5000, 9), (42, 33_333, 40), (43, 700, 3), (44, 20_011, 17)]):
        w = synth.random_scene(seed=seed, n=n, v=v, means="core_shell")
        if k == 1:
            w.scene = w.scene.to_bf16()
        elif k == 3:
            w.scene = w.scene.to_bf16s()
        ws.append(w)
    up = [upload(torch, rb, w) for w in ws]
    jobs = [{"pos": p, "attr": a, "cams": c, "ratio": 0.5} for (p, a, c) in up]
    for flags in (rb.FLAG_NORM_ATTR, rb.FLAG_NORM_ATTR | rb.FLAG_NO_PROJ, rb.FLAG_NORM_ATTR | rb.FLAG_FULL_JACOBIAN):
        prm = rb.default_params(flags=flags)
        batch = rb.Batch(ctx, jobs, params=prm)
        batch.run()
        nk_b, thr_b = batch.results()
        for k, (p, a, c) in enumerate(up):
            s = ctx.score(p, a, c, params=prm)
            m, thr, nk = ctx.select(s, 0.5)
            assert torch.equal(batch.outputs[k]["scores"], s), (flags, k)
            assert nk_b[k] == nk and thr_b[k] == thr
            if isinstance(a, rb.MixedRows):
                op, oa, idx = ctx.compact(p, a, m, nk)
                assert torch.equal(batch.outputs[k]["idx"][:nk], idx)
                assert torch.equal(batch.outputs[k]["out_attr"][:, :nk].float(), oa.float())
        batch.close()


def test_every_shape_gives_the_same_scores(env):
    """The work-item shape (tile 32/64, CTA 128/256 threads, CTAs per SM)
    changes speed only: plain and batched scores are bit-identical for every
    shape, and the autotuner reports every candidate and keeps the fastest."""
    torch, rb, ctx = env
    ws = [synth.random_scene(seed=51, n=20_000, v=30, means="core_shell"),
          synth.random_scene(seed=52, n=4_097, v=5, means="core_shell")]
    ws[1].scene = ws[1].scene.to_bf16()
    up = [upload(torch, rb, w) for w in ws]
    jobs = [{"pos": p, "attr": a, "cams": c, "ratio": 0.5} for (p, a, c) in up]
    default = ctx.get_shape()
    ref = [ctx.score(p, a, c) for (p, a, c) in up]
    try:
        for tile in (32, 64):
            for cta in (128, 256):
                for cap in (0, 2):
                    ctx.set_shape(tile, cta, cap)
                    for k, (p, a, c) in enumerate(up):
                        assert torch.equal(ctx.score(p, a, c), ref[k]), (tile, cta, cap, k)
                    batch = rb.Batch(ctx, jobs, compact=False)
                    batch.run()
                    batch.results()
                    for k in range(len(up)):
                        assert torch.equal(batch.outputs[k]["scores"], ref[k]), (tile, cta, cap, k)
                    batch.close()
        best, table = ctx.autotune(jobs, reps=1)
        # 30 views at most: every camera block splits the scenes alike, so one is tried
        assert len(table) == 8 and all(t["ms"] > 0 for t in table)
        assert best["ms"] == min(t["ms"] for t in table)
        got = ctx.get_shape()
        assert all(got[k] == best[k] for k in ("tile", "cta_threads", "ctas_per_sm", "camera_block"))
        for bad in ((48, 256, 0, 512), (64, 256, 0, 48), (64, 256, 0, 544), (64, 256, 0, 0)):
            with pytest.raises(rb.RefineError):
                ctx.set_shape(*bad)
    finally:
        ctx.set_shape(default["tile"], default["cta_threads"], default["ctas_per_sm"], default["camera_block"])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_matches_oracle(env, dtype):
    """The batched form's own outputs against the FP64 oracle, scene by scene
    (every scene of up to 150k primitives of the mixed batch above): scores
    within the float32 tolerance, keep masks agreeing with the oracle's
    selection outside the threshold band, and the compacted rows equal to the
    oracle's gather with the batch's mask."""
    import oracle
    from parity_helpers import assert_scores_only_parity, check_mask_vs_oracle_scores
    torch, rb, ctx = env
    specs = [(11, 3000, 7, 0.5), (12, 40_000, 50, 0.66), (13, 257, 3, 0.9), (14, 123_457, 120, 0.0),
             (15, 1, 1, 0.5), (16, 70_001, 300, 0.3)]
    ws = []
    for seed, n, v, _ in specs:
        w = synth.random_scene(seed=seed, n=n, v=v, means="core_shell")
        if dtype == "bf16":
            w.scene = w.scene.to_bf16()
        ws.append(w)
    up = [upload(torch, rb, w) for w in ws]
    jobs = [{"pos": p, "attr": a, "cams": c, "ratio": sp[3]} for (p, a, c), sp in zip(up, specs)]
    batch = rb.Batch(ctx, jobs)
    batch.run()
    nk_b, _ = batch.results()
    for k, (w, sp) in enumerate(zip(ws, specs)):
        ref = oracle.score(w.scene.params_f64(), w.cams)
        out = batch.outputs[k]
        n = w.scene.n
        assert_scores_only_parity(out["scores"].cpu().numpy(), ref)
        words = out["mask"][: (n + 31) // 32].cpu().numpy().view(np.uint32)
        assert check_mask_vs_oracle_scores(words, ref, sp[3], n) > 0.999
        nk = nk_b[k]
        kp, ki = oracle.compact(np.ascontiguousarray(w.scene.pos), words)
        ka, _ = oracle.compact(np.ascontiguousarray(w.scene.attr), words)
        assert nk == n - int(np.floor(sp[3] * n)) == ki.shape[0]
        assert np.array_equal(out["idx"][:nk].cpu().numpy(), ki)
        assert np.array_equal(out["out_pos"][:, :nk].cpu().numpy(), kp)
        got = out["out_attr"][:, :nk].contiguous().cpu()
        got = got.view(torch.int16).numpy().view(np.uint16) if dtype == "bf16" else got.numpy()
        assert np.array_equal(got, ka)
    ctx.check()
    batch.close()


def test_many_views_in_camera_blocks(env):
    """Scenes with more views than a camera block.  refine_score gives the
    same bits for camera blocks of 512, 256, 128 and 96 views (a primitive's
    running Kahan pair is carried from block to block); the batch, which
    scores block p of every scene in its p-th launch, and the request queue,
    which scores further blocks right after its batched launch, equal it bit
    for bit for every block size, and so do their masks."""
    torch, rb, ctx = env
    specs = [(71, 20_001, 1100, "f32"), (72, 5000, 40, "f32"), (73, 33_333, 600, "bf16")]
    ws = []
    for seed, n, v, st in specs:
        w = synth.random_scene(seed=seed, n=n, v=v, means="core_shell")
        if st == "bf16":
            w.scene = w.scene.to_bf16()
        ws.append(w)
    up = [upload(torch, rb, w) for w in ws]
    default = ctx.get_shape()
    ref = None
    try:
        for cb in (512, 256, 128, 96):
            ctx.set_shape(default["tile"], default["cta_threads"], default["ctas_per_sm"], cb)
            s = [ctx.score(p, a, c) for (p, a, c) in up]
            if ref is None:
                ref = s
                masks = [ctx.select(x, 0.5)[0] for x in ref]
            for k in range(len(up)):
                assert torch.equal(s[k], ref[k]), (cb, k)
            batch = rb.Batch(ctx, [{"pos": p, "attr": a, "cams": c, "ratio": 0.5} for (p, a, c) in up])
            batch.run()
            batch.results()
            for k, (p, _, _) in enumerate(up):
                n = p.shape[1]
                assert torch.equal(batch.outputs[k]["scores"], ref[k]), (cb, k)
                assert torch.equal(batch.outputs[k]["mask"][: (n + 31) // 32], masks[k][: (n + 31) // 32])
            batch.close()
            q = rb.Queue(ctx, budget_bytes=4 << 30, max_slots=4)
            try:
                tickets = [q.submit(w.scene.pos, w.scene.attr, w.cams, 0.5, scores=True) for w in ws]
                for k, t in enumerate(tickets):
                    res, out = q.poll(t, timeout_ms=120_000)
                    assert res["status"] == 0, (cb, k)
                    assert np.array_equal(np.asarray(out["scores"]).view(np.uint32),
                                          ref[k].cpu().numpy().view(np.uint32)), (cb, k)
            finally:
                q.close()
        ctx.check()
    finally:
        ctx.set_shape(default["tile"], default["cta_threads"], default["ctas_per_sm"], default["camera_block"])
