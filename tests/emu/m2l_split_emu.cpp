// Host emulation of the mixed-precision M2L arithmetic for one observer box
// (parity class 0: its 189 interaction-list offsets, Sec. 2.3) and the far
// field it produces (L2P gradient at points of the box), to check the FP16
// operand scaling of the tensor-core M2L against FP64 and against 3xTF32.
//
//   usage: m2l_split_emu p mode     (mode 0: positive densities, 1: zero
//   mean, 2: box weights spread over four decades)
//   prints: trunc tf32 f16 f16_unit  -- relative L2 errors of the far field:
//   FP64 M2L vs the direct sum over the same sources (truncation), and the
//   3xTF32, scaled 3xFP16 and unit-scaled 3xFP16 M2L vs the FP64 M2L.
//
// The 3-product split keeps a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 sums
// per offset, offsets added in FP32 (the promotion of the kernel).  FP16
// subnormals are flushed to zero (the worst case for the split).  Scales:
// the inputs by 2^sh with the largest |input| in (2^14, 2^15]; output
// column n of the operators by 2^(14 - ceil(log2 max_{o,k} |T_o[n][k]|)).
// This program uses the library's harmonics and operator entries
// (fmm_math.cuh, host-compilable); the splits and scales are restated here.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "fmm_math.cuh"

using namespace gf;

static float tf32(float x) {   // nearest, ties away from zero, 10 mantissa bits
    uint32_t u;
    memcpy(&u, &x, 4);
    u = (u + 0x1000u) & ~0x1FFFu;
    float r;
    memcpy(&r, &u, 4);
    return r;
}
static float f16_ftz(float x) {
    const float r = (float)(_Float16)x;
    return std::fabs(r) < 6.103515625e-05f ? 0.f : r;
}
static int ceil_log2(double x) {   // exact for the powers of two
    int e;
    const double f = std::frexp(x, &e);   // x = f 2^e, f in [0.5, 1)
    return f == 0.5 ? e - 1 : e;
}

int main(int argc, char **argv) {
    const int p = argc > 1 ? atoi(argv[1]) : 12, mode = argc > 2 ? atoi(argv[2]) : 0;
    const int K = (p + 1) * (p + 1);
    double lf[kLogFactN];
    for (int i = 0; i < kLogFactN; ++i) lf[i] = std::lgamma(i + 1.0);
    std::mt19937_64 rng(7 + 31 * mode + p);
    std::normal_distribution<double> nd(0, 1);
    std::uniform_real_distribution<double> ud(-0.5, 0.5);
    std::vector<int> offs;   // class 0: [-2, 3]^3 without max-norm <= 1
    for (int dz = -2; dz <= 3; ++dz)
        for (int dy = -2; dy <= 3; ++dy)
            for (int dx = -2; dx <= 3; ++dx)
                if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) >= 2) offs.push_back((dz + 3) * 49 + (dy + 3) * 7 + dx + 3);
    const int no = (int)offs.size();
    auto ctr = [&](int op, double c[3]) {
        c[0] = op % 7 - 3;
        c[1] = (op / 7) % 7 - 3;
        c[2] = op / 49 - 3;
    };
    std::vector<double> T((size_t)no * K * K);   // T[o][out][in]
    {
        const int H = 2 * p, nt = (H + 1) * (H + 2) / 2;
        std::vector<double> re(nt), im(nt);
        for (int o = 0; o < no; ++o) {
            double d[3];
            ctr(offs[o], d);
            irregular_harmonics<double>(H, d[0], d[1], d[2], re.data(), im.data());
            for (int r = 0; r < K; ++r)
                for (int c = 0; c < K; ++c) T[((size_t)o * K + r) * K + c] = op_entry(OP_M2L, p, r, c, re.data(), im.data(), lf);
        }
    }
    std::vector<float> cs(K);
    for (int r = 0; r < K; ++r) {
        double mx = 0;
        for (int o = 0; o < no; ++o)
            for (int c = 0; c < K; ++c) mx = std::max(mx, std::fabs(T[((size_t)o * K + r) * K + c]));
        cs[r] = mx > 0 ? std::ldexp(1.0f, 14 - ceil_log2(mx)) : 1.f;
    }
    const int nr = (p + 1) * (p + 2) / 2;
    std::vector<double> rr(nr), ri(nr);
    double err2[4] = {0, 0, 0, 0}, ref2 = 0;
    for (int trial = 0; trial < 3; ++trial) {
        std::vector<double> ME((size_t)no * K, 0.0), pts;
        for (int o = 0; o < no; ++o) {
            double c[3];
            ctr(offs[o], c);
            const double bw = mode == 2 ? std::pow(10.0, 4.0 * (ud(rng) + 0.5)) : 1.0;
            for (int iz = 0; iz < 4; ++iz)
                for (int iy = 0; iy < 4; ++iy)
                    for (int ix = 0; ix < 4; ++ix) {
                        const double y[3] = {(ix + 0.5) / 4 - 0.5, (iy + 0.5) / 4 - 0.5, (iz + 0.5) / 4 - 0.5};
                        const double q = bw * 1e6 * (mode == 1 ? nd(rng) : 2000.0 + 150.0 * nd(rng));
                        regular_harmonics<double>(p, y[0], y[1], y[2], rr.data(), ri.data());
                        for (int n = 0; n <= p; ++n)
                            for (int m = 0; m <= n; ++m) {
                                if (m == 0) {
                                    ME[(size_t)o * K + n * n] += q * rr[tri(n, 0)];
                                } else {
                                    ME[(size_t)o * K + n * n + 2 * m - 1] += q * rr[tri(n, m)];
                                    ME[(size_t)o * K + n * n + 2 * m] -= q * ri[tri(n, m)];
                                }
                            }
                        pts.insert(pts.end(), {c[0] + y[0], c[1] + y[1], c[2] + y[2], q});
                    }
        }
        double mx = 0;
        for (double x : ME) mx = std::max(mx, std::fabs(x));
        const float sig = std::ldexp(1.0f, 15 - ceil_log2(mx)), sig_unit = std::ldexp(1.0f, -ceil_log2(mx));
        // LE[variant][k]: 0 FP64, 1 3xTF32, 2 scaled 3xFP16, 3 unit-scaled 3xFP16
        std::vector<std::vector<double>> LE(4, std::vector<double>(K, 0.0));
        std::vector<float> acc1(K, 0.f), acc2(K, 0.f), acc3(K, 0.f);
        for (int o = 0; o < no; ++o)
            for (int r = 0; r < K; ++r) {
                double s0 = 0;
                float d1 = 0.f, d2 = 0.f, d3 = 0.f;
                for (int c = 0; c < K; ++c) {
                    const double t = T[((size_t)o * K + r) * K + c], x = ME[(size_t)o * K + c];
                    s0 += t * x;
                    {
                        const float a = (float)x, b = (float)t;
                        const float ah = tf32(a), al = tf32(a - ah), bh = tf32(b), bl = tf32(b - bh);
                        d1 += ah * bh + (ah * bl + al * bh);
                    }
                    {
                        const float a = (float)x * sig, b = (float)t * cs[r];
                        const float ah = f16_ftz(a), al = f16_ftz(a - ah), bh = f16_ftz(b), bl = f16_ftz(b - bh);
                        d2 += ah * bh + (ah * bl + al * bh);
                    }
                    {
                        const float a = (float)x * sig_unit, b = (float)t;
                        const float ah = f16_ftz(a), al = f16_ftz(a - ah), bh = f16_ftz(b), bl = f16_ftz(b - bh);
                        d3 += ah * bh + (ah * bl + al * bh);
                    }
                }
                LE[0][r] += s0;
                acc1[r] += d1;
                acc2[r] += d2;
                acc3[r] += d3;
            }
        for (int r = 0; r < K; ++r) {
            LE[1][r] = acc1[r];
            LE[2][r] = (double)acc2[r] / cs[r] / sig;
            LE[3][r] = (double)acc3[r] / sig_unit;
        }
        const int KD = p * p;
        std::vector<double> Dx(KD), Dy(KD), Dz(KD);
        for (int pt = 0; pt < 32; ++pt) {
            const double X = ud(rng), Y = ud(rng), Z = ud(rng);
            double g[4][3], gd[3] = {0, 0, 0};
            for (int v = 0; v < 4; ++v) {
                for (int k = 0; k < KD; ++k) grad_coeff<double>(LE[v].data(), k, Dx[k], Dy[k], Dz[k]);
                l2p_sum<double>(p, Dx.data(), Dy.data(), Dz.data(), X, Y, Z, g[v][0], g[v][1], g[v][2]);
            }
            for (size_t i = 0; i < pts.size(); i += 4) {   // -grad of sum q / |x - y|
                const double dx = X - pts[i], dy = Y - pts[i + 1], dz = Z - pts[i + 2];
                const double r2 = dx * dx + dy * dy + dz * dz, ir3 = 1.0 / (r2 * std::sqrt(r2));
                gd[0] -= pts[i + 3] * dx * ir3;
                gd[1] -= pts[i + 3] * dy * ir3;
                gd[2] -= pts[i + 3] * dz * ir3;
            }
            for (int a = 0; a < 3; ++a) {
                ref2 += g[0][a] * g[0][a];
                err2[0] += (g[0][a] - gd[a]) * (g[0][a] - gd[a]);
                for (int v = 1; v < 4; ++v) err2[v] += (g[v][a] - g[0][a]) * (g[v][a] - g[0][a]);
            }
        }
    }
    printf("%.6e %.6e %.6e %.6e\n", std::sqrt(err2[0] / ref2), std::sqrt(err2[1] / ref2), std::sqrt(err2[2] / ref2),
           std::sqrt(err2[3] / ref2));
    return 0;
}
