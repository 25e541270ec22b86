// Host instantiation of the SUM-AN kernels' corner function (gf_sum_an.cu,
// compiled into this translation unit) for a CPU test against the oracle:
// for each case, the field of the prism [lo, hi] (unit density, G = 1) as
// the signed sum of the corner function over its eight corners, all three
// components from an_corner and the vertical one again from an_corner_z.
//
//   usage: sum_an_corner_host in.bin out.bin
//   in.bin : doubles  n, then n records lo[3] hi[3] r[3]
//   out.bin: doubles  n records gx gy gz gz'
//
// and of the FMM form's near field (gf_sum_an.cuh: an_near_block) in FP32
// and FP64:
//   usage: sum_an_corner_host in.bin out.bin near
//   in.bin : doubles  nb, M, rho[nb^3] (x fastest), t[M][3] (voxel units)
//   out.bin: doubles  M records g32[3] g64[3]
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "gf_sum_an.cu"

// the library symbols gf_sum_an.cu refers to, unused here
namespace gf {
void set_error(const char *, ...) {}
void count_launch(int) {}
gf_status DeviceArena::alloc(void **p, size_t) {
    *p = nullptr;
    return GF_ERR_UNSUPPORTED;
}
}  // namespace gf

static int near_mode(const char *in, const char *outp) {
    FILE *fi = fopen(in, "rb");
    if (!fi) return 3;
    double hdr[2];
    if (fread(hdr, sizeof(double), 2, fi) != 2) return 4;
    const int nb = (int)hdr[0];
    const long M = (long)hdr[1];
    std::vector<double> rho((size_t)nb * nb * nb), t(3 * (size_t)M), out(6 * (size_t)M);
    if (fread(rho.data(), sizeof(double), rho.size(), fi) != rho.size()) return 5;
    if (fread(t.data(), sizeof(double), t.size(), fi) != t.size()) return 6;
    fclose(fi);
    std::vector<float> rf(rho.begin(), rho.end());
    for (long j = 0; j < M; ++j) {
        float g32[3];
        double g64[3];
        gf::an_near_block<float>(rf.data(), nb, (float)t[3 * j], (float)t[3 * j + 1], (float)t[3 * j + 2], g32);
        gf::an_near_block<double>(rho.data(), nb, t[3 * j], t[3 * j + 1], t[3 * j + 2], g64, 3);
        for (int a = 0; a < 3; ++a) {
            out[6 * j + a] = g32[a];
            out[6 * j + 3 + a] = g64[a];
        }
    }
    FILE *fo = fopen(outp, "wb");
    if (!fo) return 7;
    fwrite(out.data(), sizeof(double), out.size(), fo);
    fclose(fo);
    return 0;
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    if (argc > 3) return near_mode(argv[1], argv[2]);
    FILE *fi = fopen(argv[1], "rb");
    if (!fi) return 3;
    double nd;
    if (fread(&nd, sizeof(double), 1, fi) != 1) return 4;
    const long n = (long)nd;
    std::vector<double> in(9 * (size_t)n), out(4 * (size_t)n);
    if (fread(in.data(), sizeof(double), in.size(), fi) != in.size()) return 5;
    fclose(fi);
    for (long t = 0; t < n; ++t) {
        const double *lo = &in[9 * t], *hi = lo + 3, *r = lo + 6;
        double g[3] = {0, 0, 0}, gz2 = 0;
        for (int c = 0; c < 8; ++c) {
            const int a = c & 1, b = (c >> 1) & 1, e = c >> 2;
            const double s = ((a + b + e) & 1) ? 1.0 : -1.0;
            const double u = (a ? hi[0] : lo[0]) - r[0], v = (b ? hi[1] : lo[1]) - r[1],
                         w = (e ? hi[2] : lo[2]) - r[2];
            double fx, fy, fz;
            gf::an_corner<double>(u, v, w, fx, fy, fz);
            g[0] += s * fx;
            g[1] += s * fy;
            g[2] += s * fz;
            gz2 += s * gf::an_corner_z<double>(u, v, w);
        }
        out[4 * t + 0] = g[0];
        out[4 * t + 1] = g[1];
        out[4 * t + 2] = g[2];
        out[4 * t + 3] = gz2;
    }
    FILE *fo = fopen(argv[2], "wb");
    if (!fo) return 6;
    fwrite(out.data(), sizeof(double), out.size(), fo);
    fclose(fo);
    return 0;
}
