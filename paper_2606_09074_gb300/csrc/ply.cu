// Scene files: the binary little-endian PLY layout of 3D Gaussian Splatting
// checkpoints (one float32 vertex per primitive: x y z nx ny nz f_dc_0-2
// f_rest_0-44 opacity scale_0-2 rot_0-3; scales are logs, the quaternion is
// (w, x, y, z), opacity a logit, f_rest channel-major), the format in which
// a pruned scene is saved (Sec. 4.2).  Host code only.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "refine.h"
#include "common.cuh"

namespace {

constexpr int kPlyProps = 62;

// Row of the scene for every PLY property (-1 = normal, written as 0):
// rows 0-2 of pos are the means, rows 0-55 of attr follow at 3.
std::vector<std::string> prop_names()
{
    std::vector<std::string> v = {"x", "y", "z", "nx", "ny", "nz", "f_dc_0", "f_dc_1", "f_dc_2"};
    for (int k = 0; k < 45; ++k) v.push_back("f_rest_" + std::to_string(k));
    v.push_back("opacity");
    for (int k = 0; k < 3; ++k) v.push_back("scale_" + std::to_string(k));
    for (int k = 0; k < 4; ++k) v.push_back("rot_" + std::to_string(k));
    return v;
}

// scene row (0-58, pos then attr) of PLY property p, or -1 for a normal
int scene_row(int p)
{
    if (p < 3) return p;                 // x y z
    if (p < 6) return -1;                // nx ny nz
    if (p < 9) return 3 + 8 + (p - 6);   // f_dc_*  = attr rows 8-10
    if (p < 54) return 3 + 11 + (p - 9); // f_rest_* = attr rows 11-55
    if (p == 54) return 3 + 7;           // opacity  = attr row 7
    if (p < 58) return 3 + (p - 55);     // scale_*  = attr rows 0-2
    return 3 + 3 + (p - 58);             // rot_*    = attr rows 3-6
}

// Attribute row r (0..55) of primitive i, widened to float: float32 rows
// first, then bfloat16 rows, each of row_stride elements.
float load(const void *attr, int dtype, int r, int64_t row_stride, int64_t i)
{
    const int nf = refine::attr_f32_rows(dtype);
    if (r < nf) return static_cast<const float *>(attr)[r * row_stride + i];
    const unsigned short *b =
        reinterpret_cast<const unsigned short *>(static_cast<const char *>(attr) + (size_t)nf * 4 * row_stride);
    unsigned int u = (unsigned int)b[(r - nf) * row_stride + i] << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

}  // namespace

extern "C" {

refine_status refine_write_ply(const char *path, int64_t n, int32_t dtype, const float *pos_host,
                               const void *attr_host, int64_t row_stride)
{
    if (!path || n < 0 || !refine::valid_dtype(dtype) || row_stride < n ||
        (n > 0 && (!pos_host || !attr_host)))
        return REFINE_EINVAL;
    FILE *f = fopen(path, "wb");
    if (!f) return REFINE_EINVAL;
    std::string hdr = "ply\nformat binary_little_endian 1.0\nelement vertex " + std::to_string((long long)n) + "\n";
    for (const std::string &name : prop_names()) hdr += "property float " + name + "\n";
    hdr += "end_header\n";
    bool ok = fwrite(hdr.data(), 1, hdr.size(), f) == hdr.size();
    const int64_t chunk = 4096;
    std::vector<float> buf((size_t)chunk * kPlyProps);
    for (int64_t i0 = 0; i0 < n && ok; i0 += chunk) {
        const int64_t m = n - i0 < chunk ? n - i0 : chunk;
        for (int64_t j = 0; j < m; ++j) {
            const int64_t i = i0 + j;
            float *row = &buf[(size_t)j * kPlyProps];
            for (int p = 0; p < kPlyProps; ++p) {
                const int r = scene_row(p);
                row[p] = r < 0 ? 0.f : (r < 3 ? pos_host[r * row_stride + i] : load(attr_host, dtype, r - 3, row_stride, i));
            }
        }
        // PLY binary_little_endian: the hosts this builds for are little-endian
        ok = fwrite(buf.data(), sizeof(float) * kPlyProps, (size_t)m, f) == (size_t)m;
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? REFINE_OK : REFINE_EINVAL;
}

refine_status refine_read_ply(const char *path, int64_t *n_out, float *pos_host, float *attr_host,
                              int64_t row_stride)
{
    if (!path || !n_out) return REFINE_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return REFINE_EINVAL;
    // header: binary_little_endian, one vertex element, float properties
    char line[512];
    long long nv = -1;
    bool le = false, in_vertex = false, bad = false;
    std::vector<std::string> props;
    if (!fgets(line, sizeof line, f) || strncmp(line, "ply", 3) != 0) bad = true;
    while (!bad && fgets(line, sizeof line, f)) {
        if (!strncmp(line, "end_header", 10)) break;
        char a[64], b[64], c[128];
        if (sscanf(line, "format %63s", a) == 1) {
            le = !strcmp(a, "binary_little_endian");
        } else if (sscanf(line, "element %63s %lld", a, &nv) == 2) {
            in_vertex = !strcmp(a, "vertex");
            if (!in_vertex) bad = true;  // only a vertex element is expected
        } else if (sscanf(line, "property %63s %127s", b, c) == 2) {
            if (!in_vertex || (strcmp(b, "float") && strcmp(b, "float32"))) bad = true;
            props.push_back(c);
        }
        (void)a;
    }
    if (bad || !le || nv < 0) {
        fclose(f);
        return REFINE_EINVAL;
    }
    // column of every needed property
    const std::vector<std::string> want = prop_names();
    std::vector<int> col(kPlyProps, -1);
    for (int p = 0; p < kPlyProps; ++p) {
        for (size_t k = 0; k < props.size(); ++k)
            if (props[k] == want[p]) col[p] = (int)k;
        if (col[p] < 0 && scene_row(p) >= 0) {
            fclose(f);
            return REFINE_EINVAL;
        }
    }
    *n_out = nv;
    if (!pos_host && !attr_host) {
        fclose(f);
        return REFINE_OK;
    }
    if (!pos_host || !attr_host || row_stride < nv) {
        fclose(f);
        return REFINE_EINVAL;
    }
    const size_t np = props.size();
    const int64_t chunk = 4096;
    std::vector<float> buf((size_t)chunk * np);
    bool ok = true;
    for (int64_t i0 = 0; i0 < nv && ok; i0 += chunk) {
        const int64_t m = nv - i0 < chunk ? nv - i0 : chunk;
        ok = fread(buf.data(), sizeof(float) * np, (size_t)m, f) == (size_t)m;
        for (int64_t j = 0; ok && j < m; ++j)
            for (int p = 0; p < kPlyProps; ++p) {
                const int r = scene_row(p);
                if (r < 0) continue;
                const float v = buf[(size_t)j * np + col[p]];
                if (r < 3) pos_host[r * row_stride + i0 + j] = v;
                else attr_host[(r - 3) * row_stride + i0 + j] = v;
            }
    }
    fclose(f);
    return ok ? REFINE_OK : REFINE_EINVAL;
}

}  // extern "C"
