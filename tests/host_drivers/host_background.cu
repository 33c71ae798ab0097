// CPU driver of the background map (background.cu): box_load, box_hist,
// box_le_min, median_of_keys, filter_cell, axis_weight and bilinear -- the
// kernels' own host-callable code -- run thread by thread on the host; the
// cross-thread steps (histogram bin pick, sums, minima) and the mesh-fill
// selection restate the kernels' reductions serially.
// usage: host_background dir   (dir holds hdr = [w, h, box, filt, has_flags], frac (float),
//                               img [h][w] f32, flags [h][w] u8; receives raw, mesh (f64), map (f32))
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include "background.cu"

// library helpers the translation unit references (host driver only)
int argus_check_shape(const argus_shape&, size_t) { return 0; }
void argus_count_launch(int) {}
int argus_launch_status() { return 0; }
int argus_check_ptr16(const void*) { return 0; }

// bin holding the k-th element in bin order; k becomes the rank inside it
static int pick_serial(const int* hist, int& k) {
    int run = 0;
    for (int b = 0; b < 256; b++) {
        if (k < run + hist[b]) {
            k -= run;
            return b;
        }
        run += hist[b];
    }
    fprintf(stderr, "rank outside the histogram\n");
    exit(1);
}

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
    int hdr[5];
    float frac;
    rd("hdr.bin", hdr, sizeof hdr);
    rd("frac.bin", &frac, 4);
    const int w = hdr[0], h = hdr[1], box = hdr[2], filt = hdr[3];
    std::vector<float> img((size_t)w * h);
    std::vector<uint8_t> fl((size_t)w * h);
    rd("img.bin", img.data(), img.size() * 4);
    rd("flags.bin", fl.data(), fl.size());
    const int nx = (w + box - 1) / box, ny = (h + box - 1) / box;
    std::vector<double> raw((size_t)nx * ny), mesh((size_t)nx * ny);
    std::vector<float> map((size_t)w * h);
    double fill = 0.0;
    BgArgs a;
    a.img = img.data(); a.flags = hdr[4] ? fl.data() : nullptr; a.raw = raw.data(); a.mesh = mesh.data();
    a.fill = &fill; a.map = map.data(); a.pitch = w; a.w = w; a.h = h; a.box = box; a.filt = filt;
    a.nx = nx; a.ny = ny; a.min_frac = frac;
    // 1. box medians
    std::vector<unsigned> key(BM_THREADS * BM_MAX_PER);
    std::vector<char> okc(BM_THREADS * BM_MAX_PER);
    for (int by = 0; by < ny; by++)
        for (int bx = 0; bx < nx; bx++) {
            bool ok[BM_THREADS][BM_MAX_PER];
            int n = 0;
            for (int t = 0; t < BM_THREADS; t++) n += box_load(a, bx, by, t, &key[t * BM_MAX_PER], ok[t]);
            const int npx = std::min(box, w - bx * box) * std::min(box, h - by * box);
            double out = NAN;
            if (box_has_value(n, npx, frac)) {
                int k = (n - 1) / 2;
                unsigned prefix = 0, mask = 0;
                for (int shift = 24; shift >= 0; shift -= 8) {
                    int hist[256] = {0};
                    for (int t = 0; t < BM_THREADS; t++)
                        box_hist(&key[t * BM_MAX_PER], ok[t], mask, prefix, shift, [&](int b) { hist[b]++; });
                    const int b = pick_serial(hist, k);
                    prefix |= (unsigned)b << shift;
                    mask |= 255u << shift;
                }
                const unsigned k1 = prefix;
                unsigned k2 = k1;
                if ((n & 1) == 0) {
                    int nle = 0;
                    unsigned mm = 0xffffffffu;
                    for (int t = 0; t < BM_THREADS; t++) {
                        int le;
                        unsigned m;
                        box_le_min(&key[t * BM_MAX_PER], ok[t], k1, le, m);
                        nle += le;
                        mm = std::min(mm, m);
                    }
                    k2 = nle >= n / 2 + 1 ? k1 : mm;
                }
                out = median_of_keys(k1, k2);
            }
            raw[(size_t)by * nx + bx] = out;
        }
    // 2. fill: median of the box values (the mesh-fill kernel's selection, serially)
    {
        std::vector<unsigned long long> ks;
        for (double v : raw) if (!std::isnan(v)) ks.push_back(key64(v));
        const int n = (int)ks.size();
        if (n) {
            int k = (n - 1) / 2;
            unsigned long long prefix = 0, mask = 0;
            for (int shift = 56; shift >= 0; shift -= 8) {
                int hist[256] = {0};
                for (auto kk : ks) if ((kk & mask) == prefix) hist[(kk >> shift) & 255ull]++;
                const int b = pick_serial(hist, k);
                prefix |= (unsigned long long)b << shift;
                mask |= 255ull << shift;
            }
            const unsigned long long k1 = prefix;
            unsigned long long k2 = k1;
            if ((n & 1) == 0) {
                int le = 0;
                unsigned long long m = ~0ull;
                for (auto kk : ks) { if (kk <= k1) le++; else m = kk < m ? kk : m; }
                k2 = le >= n / 2 + 1 ? k1 : m;
            }
            fill = 0.5 * (unkey64(k1) + unkey64(k2));
        }
    }
    // 3. filter, 4. map
    for (int c = 0; c < nx * ny; c++) mesh[c] = filter_cell(raw.data(), nx, ny, c % nx, c / nx, filt, fill);
    for (int y = 0; y < h; y++) {
        int iy; float ty;
        axis_weight(y, h, box, ny, iy, ty);
        const int jy = ny > 1 ? nx : 0, jx = nx > 1 ? 1 : 0;
        for (int x = 0; x < w; x++) {
            int ix; float tx;
            axis_weight(x, w, box, nx, ix, tx);
            map[(size_t)y * w + x] = bilinear(mesh.data() + (long)iy * nx, ix, jx, jy, tx, ty);
        }
    }
    wr("raw.bin", raw.data(), raw.size() * 8);
    wr("mesh.bin", mesh.data(), mesh.size() * 8);
    wr("map.bin", map.data(), map.size() * 4);
    return 0;
}
