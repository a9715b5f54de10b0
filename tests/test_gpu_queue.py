"""The request queue (refine_queue_*): a request's scores, mask, threshold
and compacted scene are bit-identical to the per-scene entry points whether
it runs alone or in a mix of requests that share rounds of the batched
kernel; admission keeps the device bytes of admitted requests within the
budget; errors are reported on the request that caused them."""
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


SPECS = [  # seed, n, views, ratio, storage
    (21, 3000, 7, 0.5, "f32"),
    (22, 60_001, 50, 0.66, "bf16"),
    (23, 257, 3, 0.9, "f32"),
    (24, 150_000, 120, 0.5, "bf16"),
    (25, 1, 1, 0.5, "f32"),
    (26, 90_017, 300, 0.0, "f32"),
    (27, 45_001, 64, 0.66, "bf16s"),
]


def scenes():
    out = []
    for seed, n, v, r, st in SPECS:
        w = synth.random_scene(seed=seed, n=n, v=v, means="core_shell")
        if st == "bf16":
            w.scene = w.scene.to_bf16()
        elif st == "bf16s":
            w.scene = w.scene.to_bf16s()
        out.append((w, r))
    return out


def plain(torch, rb, ctx, w, ratio):
    """The per-scene entry points on device copies of the scene."""
    dev = torch.device("cuda", 0)
    pos = torch.from_numpy(w.scene.pos).to(dev)
    if w.scene.dtype == "bf16":
        attr = torch.from_numpy(w.scene.attr.view(np.int16)).to(dev).view(torch.bfloat16)
    elif w.scene.dtype == "bf16s":
        attr = rb.MixedRows.from_float(w.scene.attr, device=dev)
    else:
        attr = torch.from_numpy(w.scene.attr).to(dev)
    cams = rb.cameras_to_device(w.cams, dev)
    s = ctx.score(pos, attr, cams)
    m, thr, nk = ctx.select(s, ratio)
    op, oa, idx = ctx.compact(pos, attr, m, nk)
    n = pos.shape[1]
    if w.scene.dtype == "bf16":
        oa_h = oa.contiguous().cpu().view(torch.int16).numpy().view(np.uint16)
    elif w.scene.dtype == "bf16s":
        oa_h = oa.float().cpu().numpy()  # widened exactly
    else:
        oa_h = oa.cpu().numpy()
    return {"scores": s.cpu().numpy(), "mask": m[: (n + 31) // 32].cpu().numpy().view(np.uint32),
            "out_pos": op.cpu().numpy(), "out_attr": oa_h, "idx": idx.cpu().numpy(), "thr": thr, "nk": nk}


def check_same(ref, res, out, w):
    assert res["status"] == 0
    assert res["n_keep"] == ref["nk"]
    assert np.float32(res["threshold"]) == np.float32(ref["thr"]) or (
        np.isneginf(res["threshold"]) and np.isneginf(ref["thr"]))
    assert np.array_equal(np.asarray(out["scores"]).view(np.uint32), ref["scores"].view(np.uint32))
    assert np.array_equal(np.asarray(out["mask"]).view(np.uint32), ref["mask"])
    assert np.array_equal(np.asarray(out["idx"]), ref["idx"])
    assert np.array_equal(np.asarray(out["out_pos"]).view(np.uint32), ref["out_pos"].view(np.uint32))
    oa = host_attr_array(out["out_attr"])
    if w.scene.dtype == "bf16":
        assert np.array_equal(oa.view(np.uint16), ref["out_attr"])
    else:
        assert np.array_equal(oa.view(np.uint32), ref["out_attr"].view(np.uint32))


def host_attr_array(a):
    """A host attribute output as a numpy array (the mixed layout widened to
    float32, which is exact)."""
    from paper_2606_09074_gb300 import binding as rb
    return a.float().numpy() if isinstance(a, rb.MixedRows) else np.asarray(a)


def host_inputs(w, pin=False):
    from paper_2606_09074_gb300 import binding as rb
    if w.scene.dtype == "bf16s":
        return w.scene.pos, rb.MixedRows.from_float(w.scene.attr, pin_memory=pin), w.cams
    return w.scene.pos, w.scene.attr, w.cams


def dtype_code(rb, w):
    return {"f32": rb.REFINE_F32, "bf16": rb.REFINE_BF16, "bf16s": rb.REFINE_BF16S}[w.scene.dtype]


def test_alone_equals_mix_equals_plain(env):
    torch, rb, ctx = env
    sc = scenes()
    refs = [plain(torch, rb, ctx, w, r) for w, r in sc]
    q = rb.Queue(ctx, budget_bytes=8 << 30, max_slots=8)
    try:
        # alone: one request in the queue at a time
        for (w, r), ref in zip(sc, refs):
            t = q.submit(*host_inputs(w), r, scores=True)
            res, out = q.poll(t, timeout_ms=60_000)
            assert res["round_size"] == 1
            check_same(ref, res, out, w)
        # mix: everything submitted at once, several times over
        tickets = []
        for rep in range(3):
            for (w, r) in sc:
                tickets.append(q.submit(*host_inputs(w), r, scores=True))
        rounds = []
        for k, t in enumerate(tickets):
            res, out = q.poll(t, timeout_ms=60_000)
            w, _ = sc[k % len(sc)]
            check_same(refs[k % len(sc)], res, out, w)
            rounds.append(res["round_size"])
            assert res["submit_ms"] <= res["admit_ms"] <= res["done_ms"]
        st = q.stats()
        assert st["completed"] == len(sc) + len(tickets) and st["in_flight"] == 0 and st["pending"] == 0
        assert max(rounds) >= 2, "no round scored more than one request"
        assert st["bytes_in_use"] == 0
    finally:
        q.close()


def test_pinned_buffers_and_budget_admission(env):
    torch, rb, ctx = env
    sc = scenes()
    refs = [plain(torch, rb, ctx, w, r) for w, r in sc]
    big = max(rb.Queue.footprint(w.scene.n, dtype_code(rb, w), len(w.cams), r) for w, r in sc)
    budget = big + big // 2  # never two of the largest at once
    q = rb.Queue(ctx, budget_bytes=budget, max_slots=4)
    try:
        tickets = []
        for rep in range(2):
            for (w, r) in sc:
                pos = torch.from_numpy(w.scene.pos).pin_memory()
                if w.scene.dtype == "bf16s":
                    attr = host_inputs(w, pin=True)[1]
                else:
                    attr = (torch.from_numpy(w.scene.attr.view(np.int16)).view(torch.bfloat16)
                            if w.scene.dtype == "bf16" else torch.from_numpy(w.scene.attr)).pin_memory()
                tickets.append(q.submit(pos, attr, w.cams, r, scores=True, pin=True))
        for k, t in enumerate(tickets):
            res, out = q.poll(t, timeout_ms=60_000)
            w, _ = sc[k % len(sc)]
            outn = {key: (v if isinstance(v, rb.MixedRows) else
                          v.view(torch.int16).numpy().view(np.uint16) if v.dtype == torch.bfloat16 else v.numpy())
                    for key, v in out.items()}
            check_same(refs[k % len(sc)], res, outn, w)
        st = q.stats()
        assert st["peak_bytes"] <= budget
        assert st["completed"] == len(tickets)
    finally:
        q.close()


def test_errors_stay_with_their_request(env):
    torch, rb, ctx = env
    w_ok, r_ok = scenes()[1]
    ref = plain(torch, rb, ctx, w_ok, r_ok)
    w_bad = synth.random_scene(seed=31, n=5000, v=4, means="core_shell")
    cams_bad = w_bad.cams.copy()
    cams_bad["zfar"][2] = cams_bad["znear"][2] * 0.5  # zfar < znear: an invalid camera
    q = rb.Queue(ctx, budget_bytes=4 << 30, max_slots=4)
    try:
        t1 = q.submit(*host_inputs(w_ok), r_ok, scores=True)
        t2 = q.submit(w_bad.scene.pos, w_bad.scene.attr, cams_bad, 0.5)
        t3 = q.submit(*host_inputs(w_ok), r_ok, scores=True)
        res1, out1 = q.poll(t1, timeout_ms=60_000)
        res2, _ = q.poll(t2, timeout_ms=60_000)
        res3, out3 = q.poll(t3, timeout_ms=60_000)
        assert res2["status"] == rb.REFINE_EINVAL
        check_same(ref, res1, out1, w_ok)
        check_same(ref, res3, out3, w_ok)
        with pytest.raises(rb.RefineError):
            q.poll(t2, timeout_ms=0)  # already returned
        with pytest.raises(rb.RefineError):
            q.submit(*host_inputs(w_ok), 1.0)  # ratio out of range
        small = rb.Queue(ctx, budget_bytes=1 << 20, max_slots=1)
        try:
            with pytest.raises(rb.RefineError):
                small.submit(*host_inputs(w_ok), r_ok)  # footprint above the whole budget
        finally:
            small.close()
    finally:
        q.close()


def test_destroy_with_work_in_flight(env):
    torch, rb, ctx = env
    w, r = scenes()[3]
    q = rb.Queue(ctx, budget_bytes=2 << 30, max_slots=2)
    for _ in range(6):
        q.submit(*host_inputs(w), r)
    q.close()  # cancels what is pending, waits for what is admitted
    # the context still works afterwards
    ref = plain(torch, rb, ctx, w, r)
    assert ref["nk"] == w.scene.n - int(np.floor(r * w.scene.n))


def test_queue_matches_oracle(env):
    """Every request of a mixed round against the FP64 oracle on its own
    scene: scores within the float32 tolerance, the keep mask agreeing with
    the oracle's selection outside the threshold band, and the kept rows
    equal to the oracle's gather with the returned mask."""
    import oracle
    from parity_helpers import assert_scores_only_parity, check_mask_vs_oracle_scores
    torch, rb, ctx = env
    sc = scenes()
    q = rb.Queue(ctx, budget_bytes=8 << 30, max_slots=8)
    try:
        tickets = [q.submit(*host_inputs(w), r, scores=True) for (w, r) in sc]
        for (w, r), t in zip(sc, tickets):
            res, out = q.poll(t, timeout_ms=60_000)
            assert res["status"] == 0
            ref = oracle.score(w.scene.params_f64(), w.cams)
            n = w.scene.n
            assert_scores_only_parity(np.asarray(out["scores"]), ref)
            words = np.asarray(out["mask"]).view(np.uint32)[: (n + 31) // 32]
            assert check_mask_vs_oracle_scores(words, ref, r, n) > 0.999
            kp, ki = oracle.compact(np.ascontiguousarray(w.scene.pos), words)
            ka, _ = oracle.compact(np.ascontiguousarray(w.scene.attr), words)
            assert res["n_keep"] == ki.shape[0]
            assert np.array_equal(np.asarray(out["idx"]), ki)
            assert np.array_equal(np.asarray(out["out_pos"]).view(np.uint32), kp.view(np.uint32))
            oa = host_attr_array(out["out_attr"])
            assert np.array_equal(oa.view(np.uint16 if w.scene.dtype == "bf16" else np.uint32),
                                  ka.view(np.uint16 if w.scene.dtype == "bf16" else np.uint32))
    finally:
        q.close()


def test_errors_stay_with_their_request_while_the_round_ring_turns(env):
    """Two slots: a long request holds one while short requests go through
    the other, so the round ring (one entry per slot) is reused while the
    long request is still in flight.  An invalid camera fails only its own
    request; every other request, the long one included, succeeds and equals
    the per-scene path."""
    torch, rb, ctx = env
    long_w = synth.random_scene(seed=61, n=1_500_000, v=300, means="core_shell")
    short = [synth.random_scene(seed=62 + k, n=2000 + 37 * k, v=4 + k, means="core_shell") for k in range(8)]
    bad = 5
    cams_bad = short[bad].cams.copy()
    cams_bad["zfar"][1] = cams_bad["znear"][1] * 0.5  # zfar < znear: an invalid camera
    refs = [plain(torch, rb, ctx, w, 0.5) for w in short]
    ref_long = plain(torch, rb, ctx, long_w, 0.5)
    q = rb.Queue(ctx, budget_bytes=8 << 30, max_slots=2)
    try:
        t_long = q.submit(*host_inputs(long_w), 0.5, scores=True)
        tickets = [q.submit(w.scene.pos, w.scene.attr, cams_bad if k == bad else w.cams, 0.5, scores=True)
                   for k, w in enumerate(short)]
        for k, t in enumerate(tickets):
            res, out = q.poll(t, timeout_ms=120_000)
            if k == bad:
                assert res["status"] == rb.REFINE_EINVAL
            else:
                check_same(refs[k], res, out, short[k])
        res, out = q.poll(t_long, timeout_ms=120_000)
        check_same(ref_long, res, out, long_w)
        assert q.stats()["rounds"] > 2  # the two ring entries were reused
    finally:
        q.close()


def test_poll_any_returns_in_completion_order(env):
    """refine_queue_poll_any hands out every request exactly once, whichever
    finishes first, with the same results as polling by ticket; with nothing
    outstanding it reports ENOTFOUND."""
    torch, rb, ctx = env
    sc = scenes()
    refs = [plain(torch, rb, ctx, w, r) for w, r in sc]
    q = rb.Queue(ctx, budget_bytes=8 << 30, max_slots=4)
    try:
        tickets = {q.submit(*host_inputs(w), r, scores=True): k for k, (w, r) in enumerate(sc)}
        got = set()
        for _ in range(len(tickets)):
            t, res, out = q.poll_any(timeout_ms=60_000)
            assert t in tickets and t not in got
            got.add(t)
            k = tickets[t]
            check_same(refs[k], res, out, sc[k][0])
        assert got == set(tickets)
        with pytest.raises(rb.RefineError):
            q.poll_any(timeout_ms=0)
    finally:
        q.close()
