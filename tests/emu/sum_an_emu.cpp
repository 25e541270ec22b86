// Host model of a near field that integrates constant-density voxels in
// closed form (SUM-AN, Sec. 2.1), to fix its arithmetic before a GPU kernel:
// the sum over voxels is regrouped onto the voxel-corner lattice,
//
//   g(r) = G sum_corners D_c F(c - r),   D_c = sum over the (up to) eight
//          voxels v sharing corner c of s(v, c) rho_v,
//
// with F the corner function of the closed form (one vector per corner:
// three logarithms, three arctangents, one square root) and s(v, c) = +1
// when c is reached from v's lower corner by an odd number of upper limits,
// -1 otherwise.  The same voxels are also summed with n^3-point Gauss rules
// (n = 2, 3, 4), and with the midpoint rule plus the l = 4 (hexadecapole)
// term of a uniform cube, for comparison.  Each voxel is assigned to a shell by its
// Chebyshev distance, in voxels, from the voxel holding the observer, and
// every method is evaluated shell by shell so the caller can see where each
// is accurate enough.
//
//   usage: sum_an_emu in.bin out.bin
//   in.bin : doubles  nb, M, rho[nb^3] (x fastest), obs[M][3]; voxel
//            (i, j, k) spans [i, i+1) x [j, j+1) x [k, k+1) (h = 1), G = 1
//   out.bin: doubles  g[method][shell][M][3] for methods
//            0 lattice FP64, 1 lattice FP32, 2 Gauss 2^3 FP32,
//            3 Gauss 3^3 FP32, 4 Gauss 4^3 FP32, 5 midpoint + cube
//            hexadecapole FP32, and shells 0..kShells-1
//            (the last shell holds every voxel at distance >= kShells-1)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

static constexpr int kShells = 6;
static constexpr int kMethods = 6;

// ln(a + R) with R = sqrt(a^2 + q), q = the other two squares; the form
// without cancellation when a < 0
template <class T>
static inline T log_aR(T a, T q, T R) {
    return a >= T(0) ? std::log(a + R) : std::log(q / (R - a));
}

// corner function of the closed form (source corner minus observer = (u,v,w))
template <class T>
static inline void corner(T u, T v, T w, T *f) {
    const T u2 = u * u, v2 = v * v, w2 = w * w;
    const T R = std::sqrt(u2 + v2 + w2);
    f[0] = f[1] = f[2] = T(0);
    if (R == T(0)) return;
    // logarithms ln(a + R) for a = u, v, w (only where their coefficient
    // can be nonzero)
    const T Lu = (v2 + w2) > T(0) ? log_aR(u, v2 + w2, R) : T(0);
    const T Lv = (u2 + w2) > T(0) ? log_aR(v, u2 + w2, R) : T(0);
    const T Lw = (u2 + v2) > T(0) ? log_aR(w, u2 + v2, R) : T(0);
    // g_x: v ln(w+R) + w ln(v+R) - u atan(v w / (u R)), cyclically
    f[0] = v * Lw + w * Lv - (u != T(0) ? u * std::atan((v * w) / (u * R)) : T(0));
    f[1] = w * Lu + u * Lw - (v != T(0) ? v * std::atan((w * u) / (v * R)) : T(0));
    f[2] = u * Lv + v * Lu - (w != T(0) ? w * std::atan((u * v) / (w * R)) : T(0));
}

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    FILE *fi = fopen(argv[1], "rb");
    if (!fi) return 3;
    double hdr[2];
    if (fread(hdr, sizeof(double), 2, fi) != 2) return 4;
    const int nb = (int)hdr[0], M = (int)hdr[1];
    const int nv = nb * nb * nb;
    std::vector<double> rho(nv), obs(3 * (size_t)M);
    if (fread(rho.data(), sizeof(double), nv, fi) != (size_t)nv) return 5;
    if (fread(obs.data(), sizeof(double), 3 * (size_t)M, fi) != 3 * (size_t)M) return 6;
    fclose(fi);

    std::vector<double> out((size_t)kMethods * kShells * M * 3, 0.0);
    auto at = [&](int m, int s, int j) { return &out[(((size_t)m * kShells + s) * M + j) * 3]; };
    const int nc = nb + 1;

    for (int j = 0; j < M; ++j) {
        const double ox = obs[3 * j], oy = obs[3 * j + 1], oz = obs[3 * j + 2];
        const int vi = (int)std::floor(ox), vj = (int)std::floor(oy), vk = (int)std::floor(oz);
        auto shell = [&](int i, int jj, int k) {
            const int d = std::max(std::abs(i - vi), std::max(std::abs(jj - vj), std::abs(k - vk)));
            return std::min(d, kShells - 1);
        };
        for (int s = 0; s < kShells; ++s) {
            // corner weights of this shell's voxels
            std::vector<double> D((size_t)nc * nc * nc, 0.0);
            bool any = false;
            for (int k = 0; k < nb; ++k)
                for (int jj = 0; jj < nb; ++jj)
                    for (int i = 0; i < nb; ++i) {
                        if (shell(i, jj, k) != s) continue;
                        const double r = rho[((size_t)k * nb + jj) * nb + i];
                        any = true;
                        for (int c = 0; c < 8; ++c) {
                            const int a = c & 1, b = (c >> 1) & 1, e = c >> 2;
                            const double sg = ((a + b + e) & 1) ? 1.0 : -1.0;
                            D[((size_t)(k + e) * nc + (jj + b)) * nc + (i + a)] += sg * r;
                        }
                    }
            if (!any) continue;
            double *g64 = at(0, s, j), *g32 = at(1, s, j);
            for (int K = 0; K < nc; ++K)
                for (int J = 0; J < nc; ++J)
                    for (int I = 0; I < nc; ++I) {
                        const double d = D[((size_t)K * nc + J) * nc + I];
                        if (d == 0.0) continue;
                        double f[3];
                        corner<double>(I - ox, J - oy, K - oz, f);
                        for (int a = 0; a < 3; ++a) g64[a] += d * f[a];
                        float ff[3];
                        // FP32: the offset from the observer is formed in FP32 from
                        // the integer corner index and the FP32 observer position
                        const float fx = (float)ox, fy = (float)oy, fz = (float)oz;
                        corner<float>((float)I - fx, (float)J - fy, (float)K - fz, ff);
                        for (int a = 0; a < 3; ++a) g32[a] += (double)((float)d * ff[a]);
                    }
            // Gauss rules, FP32 arithmetic per point, FP64 sums
            for (int n = 2; n <= 4; ++n) {
                double x[4], w[4];
                if (n == 2) {
                    x[0] = -1.0 / std::sqrt(3.0); x[1] = -x[0]; w[0] = w[1] = 1.0;
                } else if (n == 3) {
                    x[0] = -std::sqrt(0.6); x[1] = 0.0; x[2] = -x[0];
                    w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
                } else {
                    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
                    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
                    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
                    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
                    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
                }
                double *gg = at(n, s, j);
                for (int k = 0; k < nb; ++k)
                    for (int jj = 0; jj < nb; ++jj)
                        for (int i = 0; i < nb; ++i) {
                            if (shell(i, jj, k) != s) continue;
                            const float m0 = (float)(rho[((size_t)k * nb + jj) * nb + i] / 8.0);
                            float acc[3] = {0.f, 0.f, 0.f};
                            for (int c = 0; c < n; ++c)
                                for (int b = 0; b < n; ++b)
                                    for (int a = 0; a < n; ++a) {
                                        const float dx = (float)ox - (float)(i + 0.5 + 0.5 * x[a]);
                                        const float dy = (float)oy - (float)(jj + 0.5 + 0.5 * x[b]);
                                        const float dz = (float)oz - (float)(k + 0.5 + 0.5 * x[c]);
                                        const float r2 = dx * dx + dy * dy + dz * dz;
                                        if (r2 == 0.f) continue;
                                        const float ri = 1.0f / std::sqrt(r2);
                                        const float m = m0 * (float)(w[a] * w[b] * w[c]) * ri * ri * ri;
                                        acc[0] += m * dx;
                                        acc[1] += m * dy;
                                        acc[2] += m * dz;
                                    }
                            for (int a = 0; a < 3; ++a) gg[a] += acc[a];
                        }
            }
            // midpoint + hexadecapole of the unit cube: with R = r - c,
            // Phi = G m [1/R - (7/192) (sum R_i^4 - 3/5 R^4) / R^9] up to
            // l = 6 (a cube has no quadrupole), g = -grad Phi
            double *gm = at(5, s, j);
            for (int k = 0; k < nb; ++k)
                for (int jj = 0; jj < nb; ++jj)
                    for (int i = 0; i < nb; ++i) {
                        if (shell(i, jj, k) != s) continue;
                        const float m = (float)rho[((size_t)k * nb + jj) * nb + i];
                        const float R[3] = {(float)ox - (float)(i + 0.5), (float)oy - (float)(jj + 0.5),
                                            (float)oz - (float)(k + 0.5)};
                        const float r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
                        if (r2 == 0.f) continue;
                        const float ri = 1.0f / std::sqrt(r2), ri2 = ri * ri;
                        const float ri3 = ri * ri2, ri9 = ri3 * ri3 * ri3, ri11 = ri9 * ri2;
                        const float S4 = R[0] * R[0] * R[0] * R[0] + R[1] * R[1] * R[1] * R[1] +
                                         R[2] * R[2] * R[2] * R[2];
                        const float q = 9.f * (S4 - 0.6f * r2 * r2) * ri11;
                        for (int a = 0; a < 3; ++a) {
                            const float t = (4.f * R[a] * R[a] - 2.4f * r2) * R[a] * ri9 - q * R[a];
                            gm[a] += (double)(m * (R[a] * ri3 + (7.f / 192.f) * t));
                        }
                    }
        }
    }
    FILE *fo = fopen(argv[2], "wb");
    if (!fo) return 7;
    fwrite(out.data(), sizeof(double), out.size(), fo);
    fclose(fo);
    return 0;
}
