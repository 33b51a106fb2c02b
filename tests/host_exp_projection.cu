// Host build of the CUDA path's exponential-cone projection (the same __host__ __device__
// source the kernels run), for CPU tests: reads n cones as (v[3], d[3]) doubles from the
// file argv[1] (an int32 count first), projects each onto D K_exp with exp_project_fast
// (no cached root, no network) and writes the n x 3 results to argv[2].
#include <cmath>
#include <cstdio>
#include <vector>

#include "../paper_2505_00311_gb300/csrc/cone_math.cuh"

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    int n = 0;
    if (std::fread(&n, sizeof(int), 1, f) != 1 || n < 0) return 4;
    std::vector<double> in(6 * (size_t)n);
    if (std::fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 5;
    std::fclose(f);
    std::vector<double> out(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double* a = &in[6 * (size_t)i];
        const double lg[3] = {std::log(a[3]), std::log(a[4]), std::log(a[5])};
        pdcs::exp_project_fast(a[0], a[1], a[2], a[3], a[4], a[5], lg, &out[3 * (size_t)i], nullptr);
    }
    FILE* g = std::fopen(argv[2], "wb");
    if (!g) return 6;
    if (std::fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 7;
    std::fclose(g);
    return 0;
}
