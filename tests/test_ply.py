"""Scene files (refine_write_ply / refine_read_ply): the 3DGS PLY layout,
written and read by the library's host code (no GPU)."""
import numpy as np
import pytest

from paper_2606_09074_gb300 import synth

PROPS = (["x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"] + [f"f_rest_{k}" for k in range(45)]
         + ["opacity", "scale_0", "scale_1", "scale_2", "rot_0", "rot_1", "rot_2", "rot_3"])


@pytest.fixture(scope="module")
def rb():
    pytest.importorskip("torch")
    from paper_2606_09074_gb300 import binding
    return binding


def parse(path):
    data = open(path, "rb").read()
    end = data.index(b"end_header\n") + len(b"end_header\n")
    head = data[:end].decode().splitlines()
    n = int([h for h in head if h.startswith("element vertex")][0].split()[2])
    props = [h.split()[2] for h in head if h.startswith("property")]
    return head, props, np.frombuffer(data[end:], dtype="<f4").reshape(n, len(props))


def test_write_layout_and_round_trip(rb, tmp_path):
    sc = synth.random_scene(seed=5, n=5000, v=1).scene
    path = str(tmp_path / "scene.ply")
    rb.write_ply(path, sc.pos, sc.attr)
    head, props, rows = parse(path)
    assert head[1] == "format binary_little_endian 1.0" and props == PROPS
    # column by column against the row mapping of refine_scene
    assert np.array_equal(rows[:, 0:3].T, sc.pos)
    assert np.all(rows[:, 3:6] == 0)
    assert np.array_equal(rows[:, 6:9].T, sc.attr[8:11])       # SH DC
    assert np.array_equal(rows[:, 9:54].T, sc.attr[11:56])     # SH rest, channel-major
    assert np.array_equal(rows[:, 54], sc.attr[7])             # opacity logit
    assert np.array_equal(rows[:, 55:58].T, sc.attr[0:3])      # log-scales
    assert np.array_equal(rows[:, 58:62].T, sc.attr[3:7])      # quaternion w x y z
    pos, attr = rb.read_ply(path)
    assert np.array_equal(pos, sc.pos) and np.array_equal(attr, sc.attr)


def test_bf16_is_widened_exactly(rb, tmp_path):
    sc = synth.random_scene(seed=6, n=777, v=1).scene.to_bf16()
    path = str(tmp_path / "bf16.ply")
    rb.write_ply(path, sc.pos, sc.attr)
    _, attr = rb.read_ply(path)
    assert np.array_equal(attr, synth.bf16_bits_to_f32(sc.attr))


def test_mixed_layout_is_widened_exactly(rb, tmp_path):
    """Host rows in the REFINE_BF16S layout (log-scales float32, the rest
    bfloat16) are written with every value widened exactly."""
    sc = synth.random_scene(seed=7, n=555, v=1).scene.to_bf16s()
    rows = rb.MixedRows.from_float(sc.attr)
    assert rows.row_stride == sc.n and np.array_equal(rows.float().numpy(), sc.attr)
    path = str(tmp_path / "bf16s.ply")
    rb.write_ply(path, sc.pos, rows)
    pos, attr = rb.read_ply(path)
    assert np.array_equal(pos, sc.pos) and np.array_equal(attr, sc.attr)


def test_reads_properties_by_name(rb, tmp_path):
    """A file with the properties in another order plus an extra one."""
    rng = np.random.default_rng(0)
    n = 300
    order = PROPS[::-1] + ["extra"]
    vals = rng.normal(size=(n, len(order))).astype("<f4")
    head = ["ply", "format binary_little_endian 1.0", "comment other writer", f"element vertex {n}"]
    head += [f"property float {p}" for p in order] + ["end_header"]
    path = tmp_path / "other.ply"
    path.write_bytes(("\n".join(head) + "\n").encode() + vals.tobytes())
    pos, attr = rb.read_ply(str(path))
    col = {p: vals[:, k] for k, p in enumerate(order)}
    assert np.array_equal(pos[0], col["x"]) and np.array_equal(pos[2], col["z"])
    assert np.array_equal(attr[0], col["scale_0"]) and np.array_equal(attr[3], col["rot_0"])
    assert np.array_equal(attr[7], col["opacity"]) and np.array_equal(attr[55], col["f_rest_44"])


def test_rejects_other_files(rb, tmp_path):
    bad = tmp_path / "ascii.ply"
    bad.write_text("ply\nformat ascii 1.0\nelement vertex 1\nproperty float x\nend_header\n0\n")
    with pytest.raises(rb.RefineError):
        rb.read_ply(str(bad))
    missing = tmp_path / "missing.ply"
    missing.write_bytes(b"ply\nformat binary_little_endian 1.0\nelement vertex 1\nproperty float x\nend_header\n"
                        + np.zeros(1, "<f4").tobytes())
    with pytest.raises(rb.RefineError):
        rb.read_ply(str(missing))
    with pytest.raises(rb.RefineError):
        rb.read_ply(str(tmp_path / "nope.ply"))
