"""The C ABI library builds, loads without a GPU and exports every entry
point that include/refine.h declares; the binding's ctypes layouts match
the header's struct layouts (checked with a C compiler).  CPU only."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "refine.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(refine_[a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_09074_gb300 import build
    return ctypes.CDLL(build.build_library())


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2606_09074_gb300 import binding
    assert set(declared_functions()) <= set(binding._SIGNATURES)


def test_struct_layouts_match_header(tmp_path):
    from paper_2606_09074_gb300 import binding as b
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "refine.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(refine_camera), sizeof(refine_scene), sizeof(refine_params), sizeof(refine_scene_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(refine_camera, width), offsetof(refine_camera, zfar), offsetof(refine_scene, pos), offsetof(refine_scene, row_stride));
  printf("%zu %zu %zu %zu\\n", offsetof(refine_params, e_ln_gem), offsetof(refine_params, flags), offsetof(refine_scene_stats, mean_m), offsetof(refine_scene_stats, exact_warp_axes));
  printf("%zu %zu %zu\\n", sizeof(refine_request), sizeof(refine_result), sizeof(refine_queue_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(refine_request, ratio), offsetof(refine_request, kept_idx_host), offsetof(refine_result, threshold), offsetof(refine_result, done_ms));
  printf("%zu %zu %zu\\n", offsetof(refine_queue_stats, max_round), offsetof(refine_queue_stats, kernel_launches), offsetof(refine_queue_stats, retire_ms));
  printf("%zu %zu\\n", sizeof(refine_shape), offsetof(refine_shape, ms));
  return 0; }
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().split("\n") if l]
    C = ctypes
    assert got[0] == [C.sizeof(b.refine_camera), C.sizeof(b.refine_scene), C.sizeof(b.refine_params),
                      C.sizeof(b.refine_scene_stats)]
    assert got[1] == [b.refine_camera.width.offset, b.refine_camera.zfar.offset, b.refine_scene.pos.offset,
                      b.refine_scene.row_stride.offset]
    assert got[2] == [b.refine_params.e_ln_gem.offset, b.refine_params.flags.offset,
                      b.refine_scene_stats.mean_m.offset, b.refine_scene_stats.exact_warp_axes.offset]
    assert got[3] == [C.sizeof(b.refine_request), C.sizeof(b.refine_result), C.sizeof(b.refine_queue_stats)]
    assert got[4] == [b.refine_request.ratio.offset, b.refine_request.kept_idx_host.offset,
                      b.refine_result.threshold.offset, b.refine_result.done_ms.offset]
    assert got[5] == [b.refine_queue_stats.max_round.offset, b.refine_queue_stats.kernel_launches.offset,
                      b.refine_queue_stats.retire_ms.offset]
    assert got[6] == [C.sizeof(b.refine_shape), b.refine_shape.ms.offset]


def test_camera_dtype_matches_struct():
    from paper_2606_09074_gb300 import binding as b, synth
    assert synth.CAMERA_DTYPE.itemsize == ctypes.sizeof(b.refine_camera)
    assert synth.CAMERA_DTYPE.fields["width"][1] == b.refine_camera.width.offset
    assert synth.CAMERA_DTYPE.fields["zfar"][1] == b.refine_camera.zfar.offset


def test_params_default_and_errors_without_gpu(lib):
    from paper_2606_09074_gb300 import binding as b
    p = b.default_params()
    assert abs(p.eta - 0.05) < 1e-8 and p.flags == b.FLAG_NORM_ATTR
    assert b.refine_params_default(None) == b.REFINE_EINVAL
    # no context: every call must refuse cleanly rather than crash
    assert b.refine_score(None, None, None, 1, None, None, None) == b.REFINE_EINVAL
    assert b.refine_select(None, None, 0, 0.5, None, None, None, None) == b.REFINE_EINVAL
    assert b.refine_ctx_launch_count(None) == -1
    assert b.refine_queue_submit(None, None, None) == b.REFINE_EINVAL
    assert b.refine_queue_poll(None, 1, None, 0) == b.REFINE_EINVAL
    assert b.refine_queue_stats_get(None, None) == b.REFINE_EINVAL
    assert b.refine_autotune(None, None, 0, None, 1, None, None, 0, None) == b.REFINE_EINVAL
    assert b.refine_ctx_get_shape(None, None) == b.REFINE_EINVAL
    b.refine_queue_destroy(None)


def test_queue_footprint_host_only(lib):
    """The admission size is host arithmetic: it covers the scene copy, the
    outputs and the scratch, grows with n and rejects malformed requests."""
    from paper_2606_09074_gb300 import binding as b
    fp = b.Queue.footprint
    n = 1_000_000
    f32 = fp(n, b.REFINE_F32, 200, 0.5)
    bf16 = fp(n, b.REFINE_BF16, 200, 0.5)
    assert f32 > 236 * n + 120 * n          # scene copy + compacted half
    assert bf16 < f32 and bf16 > 124 * n
    bf16s = fp(n, b.REFINE_BF16S, 200, 0.5)   # 6 more bytes per primitive (and per kept one) than bf16
    assert bf16 < bf16s < f32 and bf16s - bf16 >= 6 * n
    assert fp(n, b.REFINE_F32, 200, 0.5, compact=False) < f32
    assert fp(2 * n, b.REFINE_F32, 200, 0.5) > f32
    assert fp(0, b.REFINE_F32, 200, 0.5) == 0 and fp(n, 7, 200, 0.5) == 0
    # sized for the smallest camera block (32 views): from 33 views on a scene may take several passes and
    # then holds a running (sum, compensation) pair per primitive
    assert fp(n, b.REFINE_F32, 33, 0.5) >= fp(n, b.REFINE_F32, 32, 0.5) + 8 * n
    assert fp(n, b.REFINE_F32, 1100, 0.5) > fp(n, b.REFINE_F32, 200, 0.5)
    assert fp(n, b.REFINE_F32, 65536, 0.5) == 0 and fp(n, b.REFINE_F32, 200, 1.0) == 0


def test_storage_type_codes_match_header():
    """The binding's storage-type codes are the header's enum values."""
    import re
    from paper_2606_09074_gb300 import binding as b
    hdr = open(os.path.join(ROOT, "include", "refine.h")).read()
    m = re.search(r"enum\s*\{\s*REFINE_F32\s*=\s*(\d+),\s*REFINE_BF16\s*=\s*(\d+),\s*REFINE_BF16S\s*=\s*(\d+)\s*\}", hdr)
    assert m, "storage-type enum not found in include/refine.h"
    assert (b.REFINE_F32, b.REFINE_BF16, b.REFINE_BF16S) == tuple(int(x) for x in m.groups())


def test_mixed_rows_container_host_only():
    """MixedRows (the REFINE_BF16S layout in one byte buffer): the float32
    block and the bfloat16 block sit where the header says (the bfloat16 rows
    at byte 12 * stride), column views keep the stride, the widened rows are
    exact, and the column bytes are 118."""
    torch = pytest.importorskip("torch")
    from paper_2606_09074_gb300 import binding as b
    rng = np.random.default_rng(3)
    n, stride = 37, 40
    a = rng.standard_normal((56, n)).astype(np.float32)
    want = a.copy()
    want[3:] = torch.from_numpy(a[3:]).to(torch.bfloat16).float().numpy()
    m = b.MixedRows.empty(n, stride=stride)
    m.f32_rows()[:, :n] = torch.from_numpy(a[:3])
    m.bf16_rows()[:, :n] = torch.from_numpy(a[3:]).to(torch.bfloat16)
    assert m.shape == (56, n) and m.stride(0) == stride and m.stride(1) == 1
    assert b.attr_col_bytes(m) == 118 and m.buf.numel() == 118 * stride
    raw = m.buf.numpy()
    assert np.array_equal(raw[: 12 * stride].view(np.float32).reshape(3, stride)[:, :n], a[:3])
    bf = raw[12 * stride: 118 * stride].view(np.uint16).reshape(53, stride)[:, :n]
    assert np.array_equal(bf, want[3:].view(np.uint32) >> 16)
    assert np.array_equal(m.float().numpy(), want)
    v = m[:, :10]
    assert v.shape == (56, 10) and v.stride(0) == stride and np.array_equal(v.float().numpy(), want[:, :10])
    f = b.MixedRows.from_float(a)
    assert f.row_stride == n and np.array_equal(f.float().numpy(), want)
    e = b.empty_attr_like(f, 5)
    assert isinstance(e, b.MixedRows) and e.shape == (56, 5)
    assert b.empty_attr_like(torch.zeros(56, 3, dtype=torch.bfloat16), 4).dtype == torch.bfloat16

