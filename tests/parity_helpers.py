"""Checks shared by the GPU parity tests: scores against the FP64 oracle
within RTOL outside its float32 band, keep masks against the oracle's own
selection outside the threshold band."""
import numpy as np

import oracle

RTOL = 1e-5


def assert_score_parity(s_gpu, S_gpu, ref, rtol=RTOL):
    clean = ref["nborder"] == 0
    for name, got, want in (("S", S_gpu, ref["S"]), ("score", s_gpu, ref["scores"])):
        g = got.astype(np.float64)
        zero = clean & (want == 0)
        assert np.all(g[zero] == 0), f"{name}: nonzero where oracle is exactly 0"
        nz = clean & (want != 0)
        rel = np.abs(g[nz] - want[nz]) / np.abs(want[nz])
        if rel.size:
            worst = int(np.argmax(rel))
            assert rel.max() <= rtol, (f"{name}: max rel err {rel.max():.3e} at {np.nonzero(nz)[0][worst]}",
                                       g[nz][worst], want[nz][worst])
    ok = oracle.valid_alternative(S_gpu.astype(np.float64), ref, rtol)
    assert ok.all(), f"borderline primitives with no valid alternative: {np.nonzero(~ok)[0][:10]}"
    return clean


def unpack(mask_words, n):
    return np.unpackbits(np.asarray(mask_words, dtype=np.uint32).view(np.uint8), bitorder="little")[:n].astype(bool)


def check_mask_vs_oracle_scores(got_mask, ref, ratio, n):
    m_ref, thr_ref, nk_ref = oracle.select(ref["scores"], ratio)
    a, b = unpack(got_mask, n), unpack(m_ref, n)
    diff = np.nonzero(a != b)[0]
    band = (np.abs(ref["scores"] - thr_ref) <= RTOL * abs(thr_ref)) | (ref["nborder"] > 0)
    assert np.all(band[diff]), f"mask differs outside the threshold band at {diff[~band[diff]][:10]}"
    return 1.0 - diff.size / max(n, 1)


def assert_scores_only_parity(scores, ref, rtol=RTOL):
    """Scores alone (no view sums, as the batched and queued forms return
    them) against the oracle: every primitive outside the float32 band within
    rtol (exactly 0 where the oracle's is 0); a primitive with borderline
    pairs between the scores of its extreme alternatives, the oracle's score
    scaled by (S_sure, S_sure + all borderline terms) / S."""
    g = np.asarray(scores, dtype=np.float64)
    want = ref["scores"]
    clean = ref["nborder"] == 0
    zero = clean & (want == 0)
    assert np.all(g[zero] == 0), "nonzero where the oracle is exactly 0"
    nz = clean & (want != 0)
    rel = np.abs(g[nz] - want[nz]) / np.abs(want[nz])
    if rel.size:
        assert rel.max() <= rtol, f"max rel err {rel.max():.3e} at {np.nonzero(nz)[0][int(np.argmax(rel))]}"
    border = np.nonzero(~clean & (ref["S"] > 0))[0]
    scale = want[border] / ref["S"][border]
    lo = scale * ref["S_sure"][border]
    hi = scale * (ref["S_sure"][border] + ref["bterms"][border].sum(axis=1))
    many = ref["nborder"][border] > 4
    hi[many] = np.inf
    ok = (g[border] >= lo * (1 - rtol)) & (g[border] <= hi * (1 + rtol))
    assert ok.all(), f"borderline primitives outside their alternatives: {border[~ok][:10]}"
    return clean


