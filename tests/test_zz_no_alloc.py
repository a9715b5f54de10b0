"""refine_select_noalloc: the allocation-free selection entry point for
callers that cannot call cudaMalloc (engines that own all device memory,
fixed-memory real-time loops).  Its keep mask, threshold and kept count must
equal refine_select's on the same scores, on two calls in a row through the
C ABI (the fixed scratch array is reused and must be reset by each call),
also with nothing pruned and without the threshold read-back.  This file is
collected last so that a run stopping at the first failure has run every
other test."""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(rb, scores, ratio, mask, stream):
    thr = C.c_float()
    nk = C.c_int64()
    err = C.create_string_buffer(256)
    st = rb.refine_select_noalloc(C.c_void_p(scores.data_ptr()), scores.numel(), float(ratio),
                                  C.c_void_p(mask.data_ptr()), C.byref(thr), C.byref(nk), err,
                                  C.sizeof(err), C.c_void_p(stream.cuda_stream))
    return st, thr.value, nk.value, err.value.decode()


def test_noalloc_matches_select_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09074_gb300 import binding as rb
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = rb.Context(0)
    rng = np.random.default_rng(77)
    cases = [
        (np.where(rng.random(300_001) < 0.4, 0.0, rng.random(300_001)).astype(np.float32), 0.5),
        (rng.integers(0, 5, 123_457).astype(np.float32), 0.66),  # heavy ties, different size
    ]
    for s_np, ratio in cases:  # two calls in a row, reusing the fixed scratch
        s = torch.from_numpy(s_np).to(dev)
        n = s.numel()
        words = (n + 31) // 32
        mask_a = torch.full((words,), -1, dtype=torch.int32, device=dev)
        st, thr, nk, err = _noalloc(rb, s, ratio, mask_a, stream)
        assert st == rb.REFINE_OK, err
        mask_b, thr_b, nk_b = ctx.select(s, ratio)
        assert nk == nk_b == n - math.floor(ratio * n)
        assert thr == thr_b
        assert torch.equal(mask_a, mask_b[:words])
    # ratio 0: nothing pruned, every bit of the mask set; no threshold read-back
    s = torch.from_numpy(cases[0][0]).to(dev)
    n = s.numel()
    words = (n + 31) // 32
    mask_z = torch.zeros(words, dtype=torch.int32, device=dev)
    st, thr, nk, err = _noalloc(rb, s, 0.0, mask_z, stream)
    assert st == rb.REFINE_OK and nk == n and thr == -math.inf, err
    mask_r, _, _ = ctx.select(s, 0.0)
    assert torch.equal(mask_z, mask_r[:words])
    mask_n = torch.zeros(words, dtype=torch.int32, device=dev)
    nk_c = C.c_int64()
    err_b = C.create_string_buffer(256)
    st = rb.refine_select_noalloc(C.c_void_p(s.data_ptr()), n, 0.5, C.c_void_p(mask_n.data_ptr()), None,
                                  C.byref(nk_c), err_b, C.sizeof(err_b), C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize(dev)
    mask_h, _, _ = ctx.select(s, 0.5)
    assert st == rb.REFINE_OK and nk_c.value == n - n // 2 and torch.equal(mask_n, mask_h[:words])
    # sizes beyond the fixed scratch are refused with a message
    big = torch.empty(1, dtype=torch.float32, device=dev)
    thr = C.c_float()
    err = C.create_string_buffer(256)
    st = rb.refine_select_noalloc(C.c_void_p(big.data_ptr()), (1 << 26) + 1, 0.5, C.c_void_p(big.data_ptr()),
                                  C.byref(thr), None, err, C.sizeof(err), C.c_void_p(stream.cuda_stream))
    assert st == rb.REFINE_EINVAL and b"limit" in err.value
    ctx.close()
