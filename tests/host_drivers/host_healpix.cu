// CPU driver of the HEALPix resampling (healpix.cu): hp_pixel_xy and
// hp_bilinear -- the kernel's own host-callable code -- run for every
// segment-image pixel on the host.
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
    for (long e = 0; e < (long)out.size(); e++) {
        const long s = e / (m * m), q = e - s * m * m;
        double x, y;
        float v = 0.0f;
        const bool ok = hp_pixel_xy(a, segs[s], (int)(q & (m - 1)), (int)(q >> k), x, y) && hp_bilinear(a, x, y, v);
        out[e] = ok ? v : 0.0f;
        cov[e] = ok ? 1 : 0;
    }
    wr("out.bin", out.data(), out.size() * 4);
    wr("cov.bin", cov.data(), cov.size());
    return 0;
}
