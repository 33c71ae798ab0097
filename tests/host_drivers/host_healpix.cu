// CPU driver of the HEALPix resampling (healpix.cu): hp_pixel_xy, hp_bilinear,
// hp_row_in_belt, hp_cubic_coeffs and hp_cubic_eval -- the kernels' own
// host-callable code -- run for every segment-image pixel on the host, with the
// row path (k >= 6, equatorial belt) and the exact path split as the kernels do.
// usage: host_healpix dir   (dir holds hdr = [w, h, nside_seg, k, n_seg, has_flags], wcs (6 f64),
//                           segs (i64 [n_seg]), frame [h][w] f32, flags [h][w] u8; receives out, cov)
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "healpix.cu"

// library helpers the translation unit references (host driver only)
int argus_check_shape(const argus_shape&, size_t) { return 0; }
void argus_count_launch(int) {}
int argus_launch_status() { return 0; }

int main(int argc, char** argv) {
    const char* dir = argv[1];
    char path[512];
    auto rd = [&](const char* name, void* p, size_t bytes) {
        snprintf(path, sizeof path, "%s/%s", dir, name);
        FILE* f = fopen(path, "rb");
        if (!f || fread(p, 1, bytes, f) != bytes) { fprintf(stderr, "read %s\n", path); exit(1); }
        fclose(f); };
    auto wr = [&](const char* name, const void* p, size_t bytes) {
        snprintf(path, sizeof path, "%s/%s", dir, name);
        FILE* f = fopen(path, "wb");
        if (!f || fwrite(p, 1, bytes, f) != bytes) { fprintf(stderr, "write %s\n", path); exit(1); }
        fclose(f); };
    int hdr[6];
    rd("hdr.bin", hdr, sizeof hdr);
    const int w = hdr[0], h = hdr[1], nside_seg = hdr[2], k = hdr[3], n_seg = hdr[4];
    argus_wcs wcs;
    rd("wcs.bin", &wcs, sizeof wcs);
    std::vector<long long> segs(n_seg);
    rd("segs.bin", segs.data(), segs.size() * 8);
    std::vector<float> frame((size_t)w * h);
    std::vector<uint8_t> fl((size_t)w * h);
    rd("frame.bin", frame.data(), frame.size() * 4);
    rd("flags.bin", fl.data(), fl.size());
    const long m = 1L << k;
    std::vector<float> out((size_t)n_seg * m * m);
    std::vector<uint8_t> cov(out.size());
    HpArgs a;
    a.frame = frame.data(); a.flags = hdr[5] ? fl.data() : nullptr; a.pitch = w; a.w = w; a.h = h;
    a.segs = segs.data(); a.n_seg = n_seg; a.nside_seg = nside_seg; a.k = k; a.out = out.data(); a.cov = cov.data();
    hp_fill_wcs(a, wcs);
    auto exact = [&](long e, long long seg, int c, int r) {
        double x, y;
        float v = 0.0f;
        const bool ok = hp_pixel_xy(a, seg, c, r, x, y) && hp_bilinear(a, x, y, v);
        out[e] = ok ? v : 0.0f;
        cov[e] = ok ? 1 : 0;
    };
    for (int s = 0; s < n_seg; s++)
        for (int r = 0; r < m; r++) {
            const long base = ((long)s * m + r) * m;
            if (k < 6 || !hp_row_in_belt(a, segs[s], r)) {      // the exact path
                for (int c = 0; c < m; c++) exact(base + c, segs[s], c, r);
                continue;
            }
            for (int p = 0; p < m / HP_PIECE; p++) {            // the row path, piece by piece
                double fx[4], fy[4];
                bool all = true;
                for (int j = 0; j < 4; j++) all = hp_pixel_xy(a, segs[s], p * HP_PIECE + hp_node(j), r, fx[j], fy[j]) && all;
                double dx[4], dy[4];
                hp_cubic_coeffs(fx, dx);
                hp_cubic_coeffs(fy, dy);
                for (int t = 0; t < HP_PIECE; t++) {
                    const int c = p * HP_PIECE + t;
                    if (!all) {
                        exact(base + c, segs[s], c, r);
                        continue;
                    }
                    float v = 0.0f;
                    const bool ok = hp_bilinear(a, hp_cubic_eval(dx, (double)t), hp_cubic_eval(dy, (double)t), v);
                    out[base + c] = ok ? v : 0.0f;
                    cov[base + c] = ok ? 1 : 0;
                }
            }
        }
    wr("out.bin", out.data(), out.size() * 4);
    wr("cov.bin", cov.data(), cov.size());
    return 0;
}
