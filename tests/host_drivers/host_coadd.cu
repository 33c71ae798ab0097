// CPU driver of the proper coadd (proper.cu) on one T x T tile at the frame
// origin: PSF placement, the FFT passes, coadd_accum_point and
// coadd_final_point -- the kernels' own host-callable code -- run on the host;
// pack, unpack and the norms restate the kernels' element loops.
// usage: host_coadd T dir   (dir holds hdr = [J, ps], M [J][T][T], P [J][ps][ps],
//                            F [J], sig [J]; receives S, R, PR, norms = [F_R, sigma_S])
#include <cstdio>
#include <cstdlib>
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
    auto wr = [&](const char* name, const void* p, size_t bytes) {
        snprintf(path, sizeof path, "%s/%s", dir, name);
        FILE* f = fopen(path, "wb");
        if (!f || fwrite(p, 1, bytes, f) != bytes) { fprintf(stderr, "write %s\n", path); exit(1); }
        fclose(f); };
    int hdr[2];
    rd("hdr.bin", hdr, sizeof hdr);
    const int J = hdr[0], ps = hdr[1], pp = ps * ps, hh = ps / 2;
    std::vector<float> M((size_t)J * T * T), P((size_t)J * pp), F(J), sig(J);
    rd("M.bin", M.data(), M.size() * 4); rd("P.bin", P.data(), P.size() * 4);
    rd("F.bin", F.data(), J * 4); rd("sig.bin", sig.data(), J * 4);
    std::vector<float2> tw32(T);
    std::vector<double2> tw64(T);
    for (int m = 0; m < T; m++) {
        const double a = 6.283185307179586476925286766559 * m / T;
        tw64[m] = make_double2(cos(a), -sin(a));
        tw32[m] = make_float2((float)tw64[m].x, (float)tw64[m].y);
    }
    std::vector<float2> z1(T * T), acc(T * T, make_float2(0, 0));
    std::vector<double2> z2(T * T), acc2(T * T, make_double2(0, 0));
    for (int j0 = 0; j0 < J; j0 += 2) {
        const bool two = j0 + 1 < J;
        for (int q = 0; q < T * T; q++)
            z1[q] = make_float2(M[(size_t)j0 * T * T + q], two ? M[(size_t)(j0 + 1) * T * T + q] : 0.0f);
        for (auto& v : z2) v = make_double2(0, 0);
        for (int i = 0; i < pp; i++) {
            const int v = i / ps, u = i - v * ps;
            const int yy = (v - hh + T) & (T - 1), xx = (u - hh + T) & (T - 1);
            z2[yy * T + xx] = make_double2(P[(size_t)j0 * pp + i], two ? P[(size_t)(j0 + 1) * pp + i] : 0.0);
        }
        host_pass<T, -1, false, float>(z1.data(), 1, tw32.data()); host_pass<T, -1, true, float>(z1.data(), 1, tw32.data());
        host_pass<T, -1, false, double>(z2.data(), 1, tw64.data()); host_pass<T, -1, true, double>(z2.data(), 1, tw64.data());
        float w0, w1;
        double a0, a1;
        frame_weights(F.data(), sig.data(), J, j0, w0, a0);
        frame_weights(F.data(), sig.data(), J, j0 + 1, w1, a1);
        for (int q = 0; q < T * T; q++) {
            const int ky = q / T, kx = q - ky * T;
            const int pq = ((T - ky) & (T - 1)) * T + ((T - kx) & (T - 1));
            coadd_accum_point(z1[q], z1[pq], z2[q], z2[pq], w0, w1, a0, a1, acc[q], acc2[q]);
        }
    }
    double fr2 = 0.0, v = 0.0;
    for (int j = 0; j < J; j++) {
        float w;
        double aj;
        frame_weights(F.data(), sig.data(), J, j, w, aj);
        double s2 = 0.0;
        for (int i = 0; i < pp; i++) s2 += (double)P[(size_t)j * pp + i] * P[(size_t)j * pp + i];
        v += aj * s2;
        fr2 += aj;
    }
    const double FR = sqrt(fr2);
    const double eps = 1e-8;
    std::vector<float2> z3(T * T);
    for (int q = 0; q < T * T; q++) coadd_final_point(acc[q], acc2[q], FR, eps * eps, z1[q], z3[q]);
    host_pass<T, 1, false, float>(z1.data(), 1, tw32.data()); host_pass<T, 1, true, float>(z1.data(), 1, tw32.data());
    host_pass<T, 1, false, float>(z3.data(), 1, tw32.data()); host_pass<T, 1, true, float>(z3.data(), 1, tw32.data());
    const float inv = 1.0f / ((float)T * (float)T);
    std::vector<float> S(T * T), R(T * T), PR(T * T);
    for (int q = 0; q < T * T; q++) { S[q] = z1[q].x * inv; R[q] = z1[q].y * inv; PR[q] = z3[q].x * inv; }
    const double norms[2] = {FR, sqrt(v)};
    wr("S.bin", S.data(), S.size() * 4); wr("R.bin", R.data(), R.size() * 4); wr("PR.bin", PR.data(), PR.size() * 4);
    wr("norms.bin", norms, sizeof norms);
}

int main(int argc, char** argv) {
    const int T = atoi(argv[1]);
    if (T == 256) run<256>(argv[2]); else if (T == 512) run<512>(argv[2]); else run<1024>(argv[2]);
    return 0;
}
