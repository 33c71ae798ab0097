// CPU driver of the segment fit's FP16 range scale (segments_tc.cu): f16_range_scale, the
// kernels' own host-callable code, for every value of a file.
// usage: host_segscale in out   (in: f32 [n], out: f32 [n] scales)
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "segments_tc.cu"

// library helpers the translation unit references (host driver only)
void argus_count_launch(int) {}
int argus_launch_status() { return 0; }
int argus_cuda_fail(cudaError_t) { return ARGUS_ERR_CUDA; }

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 1;
    std::vector<float> v;
    float x;
    while (fread(&x, 4, 1, f) == 1) v.push_back(x);
    fclose(f);
    std::vector<float> out(v.size());
    for (size_t i = 0; i < v.size(); i++) out[i] = f16_range_scale(v[i]);
    FILE* g = fopen(argv[2], "wb");
    if (!g || fwrite(out.data(), 4, out.size(), g) != out.size()) return 1;
    fclose(g);
    return 0;
}
