// CPU driver of the batched 2-D FFT (fft.cuh): reads n tiles of T x T complex
// values, transforms them (sign -1 forward, +1 inverse, unscaled) with the
// kernels' code run on the host, writes the result.
// usage: host_fft T is_double n sign in.bin out.bin
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include "host_pass.h"

template <int T, typename R>
void run(const char* in, const char* out, int n, int sign) {
    using C = typename Cx<R>::T;
    std::vector<C> d((size_t)n * T * T), tw(T);
    FILE* f = fopen(in, "rb");
    if (!f || fread(d.data(), sizeof(C), d.size(), f) != d.size()) { fprintf(stderr, "read %s\n", in); exit(1); }
    fclose(f);
    for (int m = 0; m < T; m++) { double a = 6.283185307179586476925286766559 * m / T; tw[m].x = (R)cos(a); tw[m].y = (R)-sin(a); }
    if (sign < 0) { host_pass<T, -1, false, R>(d.data(), n, tw.data()); host_pass<T, -1, true, R>(d.data(), n, tw.data()); }
    else { host_pass<T, 1, false, R>(d.data(), n, tw.data()); host_pass<T, 1, true, R>(d.data(), n, tw.data()); }
    f = fopen(out, "wb"); fwrite(d.data(), sizeof(C), d.size(), f); fclose(f);
}

int main(int argc, char** argv) {
    int T = atoi(argv[1]), dbl = atoi(argv[2]), n = atoi(argv[3]), sign = atoi(argv[4]);
    if (dbl) { if (T == 256) run<256, double>(argv[5], argv[6], n, sign); else if (T == 512) run<512, double>(argv[5], argv[6], n, sign); else run<1024, double>(argv[5], argv[6], n, sign); }
    else { if (T == 256) run<256, float>(argv[5], argv[6], n, sign); else if (T == 512) run<512, float>(argv[5], argv[6], n, sign); else run<1024, float>(argv[5], argv[6], n, sign); }
    return 0;
}
