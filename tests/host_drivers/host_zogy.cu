// CPU driver of the ZOGY path (zogy.cu) on one T x T tile at the frame origin:
// PSF placement, the FFT passes and zogy_pair -- the kernels' own host-callable
// code -- run on the host; pack, unpack and sigma_S restate the kernels' element
// loops.  usage: host_zogy T dir   (dir holds hdr, tile, N, R, pn, pr; receives D, S, P, sig)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>
#include "proper.cu"
#include "host_pass.h"

// library helpers the translation unit references (host driver only)
int argus_check_shape(const argus_shape&, size_t) { return 0; }
void argus_count_launch(int) {}
int argus_launch_status() { return 0; }

template <int T>
void run(const char* dir) {
    char path[512];
    auto rd = [&](const char* name, void* p, size_t bytes) {
        snprintf(path, sizeof path, "%s/%s", dir, name);
        FILE* f = fopen(path, "rb");
        if (!f || fread(p, 1, bytes, f) != bytes) { fprintf(stderr, "read %s\n", path); exit(1); }
        fclose(f); };
    int hdr[2]; rd("hdr.bin", hdr, sizeof hdr);
    const int ps = hdr[0];
    argus_zogy_tile tp; rd("tile.bin", &tp, sizeof tp);
    std::vector<float> N(T * T), R(T * T), pn(ps * ps), pr(ps * ps);
    rd("N.bin", N.data(), N.size() * 4); rd("R.bin", R.data(), R.size() * 4);
    rd("pn.bin", pn.data(), pn.size() * 4); rd("pr.bin", pr.data(), pr.size() * 4);
    std::vector<float2> z1(T * T), z3(T * T);
    std::vector<double2> z2(T * T, make_double2(0, 0));
    for (int q = 0; q < T * T; q++) z1[q] = make_float2(N[q], R[q]);                  // tile at (0, 0) of a T x T frame
    const int hh = ps / 2;
    for (int v = 0; v < ps; v++)
        for (int u = 0; u < ps; u++) {
            const int yy = (v - hh + T) & (T - 1), xx = (u - hh + T) & (T - 1);
            z2[yy * T + xx] = make_double2(pn[v * ps + u], pr[v * ps + u]);
        }
    std::vector<float2> tw32(T); std::vector<double2> tw64(T);
    for (int m = 0; m < T; m++) {
        const double a = 6.283185307179586476925286766559 * m / T;
        tw64[m] = make_double2(cos(a), -sin(a)); tw32[m] = make_float2((float)tw64[m].x, (float)tw64[m].y);
    }
    host_pass<T, -1, false, float>(z1.data(), 1, tw32.data()); host_pass<T, -1, true, float>(z1.data(), 1, tw32.data());
    host_pass<T, -1, false, double>(z2.data(), 1, tw64.data()); host_pass<T, -1, true, double>(z2.data(), 1, tw64.data());
    double psd = 0;
    const double eps = 1e-8;
    for (int q = 0; q < T * T; q++) {
        const int ky = q / T, kx = q - ky * T;
        const int pq = ((T - ky) & (T - 1)) * T + ((T - kx) & (T - 1));
        if (pq < q) continue;
        float2 Wq, Wp, PD; double p2;
        zogy_pair(z1[q], z1[pq], z2[q], z2[pq], tp, eps * eps, Wq, Wp, PD, p2);
        z1[q] = Wq; if (pq != q) z1[pq] = Wp;
        z3[q] = PD; if (pq != q) z3[pq] = make_float2(PD.x, -PD.y);
        psd += p2 * (pq != q ? 2.0 : 1.0);
    }
    host_pass<T, 1, false, float>(z1.data(), 1, tw32.data()); host_pass<T, 1, true, float>(z1.data(), 1, tw32.data());
    host_pass<T, 1, false, float>(z3.data(), 1, tw32.data()); host_pass<T, 1, true, float>(z3.data(), 1, tw32.data());
    const float inv = 1.0f / ((float)T * (float)T);
    std::vector<float> D(T * T), S(T * T), P(T * T);
    for (int q = 0; q < T * T; q++) { D[q] = z1[q].x * inv; S[q] = z1[q].y * inv; P[q] = z3[q].x * inv; }
    const double FD = (double)tp.Fr * tp.Fn / sqrt((double)tp.sn * tp.sn * tp.Fr * tp.Fr + (double)tp.sr * tp.sr * tp.Fn * tp.Fn);
    const double sig = FD * sqrt(psd / ((double)T * T));
    auto wr = [&](const char* name, const void* p, size_t bytes) {
        snprintf(path, sizeof path, "%s/%s", dir, name);
        FILE* f = fopen(path, "wb");
        if (!f || fwrite(p, 1, bytes, f) != bytes) { fprintf(stderr, "write %s\n", path); exit(1); }
        fclose(f); };
    wr("D.bin", D.data(), D.size() * 4); wr("S.bin", S.data(), S.size() * 4); wr("P.bin", P.data(), P.size() * 4);
    wr("sig.bin", &sig, 8);
}

int main(int argc, char** argv) {
    if (argc == 2 && !strcmp(argv[1], "reuse")) {       // the PSF-reuse argument check, one line per case
        for (int held = -1; held <= 3; held++)
            for (int per = 0; per <= 1; per++)
                for (int n = 1; n <= 4; n++) printf("%d %d %d %d\n", held, per, n, (int)zogy_psf_reuse_ok(held, per, n));
        return 0;
    }
    const int T = atoi(argv[1]);
    if (T == 256) run<256>(argv[2]); else if (T == 512) run<512>(argv[2]); else run<1024>(argv[2]);
    return 0;
}
