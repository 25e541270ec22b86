// gf_m2l.cu -- M2L over the interaction list, as a batched dense contraction.
//
// Observer boxes of a level are grouped by parity class (their position in
// the parent), because the 189 interaction-list offsets depend only on that
// class.  A block takes up to 32 columns -- (box, batch member) pairs of one
// class -- and, offset by offset, multiplies the K x K operator T_o by the
// K x 32 matrix of gathered source expansions ME[t + o], accumulating the
// K x 32 result in registers.  Sources outside the source block contribute
// zero columns.  Each output is written once, so the result is deterministic.
#include <cuda_fp16.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "gf_m2l.cuh"

namespace gf {

__constant__ signed char c_il[8][189][3];

gf_status m2l_upload_offsets(const signed char h_il[8][189][3]) {
    GF_CUDA(cudaMemcpyToSymbol(c_il, h_il, sizeof(signed char) * 8 * 189 * 3));
    return GF_OK;
}

namespace {

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The same rounding (to nearest, ties away from zero, on the magnitude) with
// two integer operations: add half a TF32 ulp to the bits and clear the 13
// dropped bits.  Finite inputs only (the callers flag non-finite ones).
__device__ __forceinline__ uint32_t to_tf32_int(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

// Byte offset of element (row, k), k < 16, in a [rows][16] FP32 tile stored
// K-major with the 64-byte swizzle: 8-row atoms of 512 bytes, the 16-byte
// chunk index XOR-ed with bits 1-2 of the row inside the atom.
__host__ __device__ __forceinline__ uint32_t swz64(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((((k >> 2) ^ (row >> 1)) & 3) << 4) + (k & 3) * 4);
}

// Byte offset of FP16 element (row, k), k < 32, in a [rows][32] tile in the
// same swizzled layout (the swizzle acts on 16-byte chunks, 8 halves each).
__host__ __device__ __forceinline__ uint32_t swz64h(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((((k >> 3) ^ (row >> 1)) & 3) << 4) + (k & 7) * 2);
}

// Column scales of an M2L operator set (one block per output component n <
// Npad): s_n = 2^(14 - ceil(log2 max |T_o[n][k]|)), the maximum over the
// used offset slots and every input k.  cs[n] = s_n, cs[Npad + n] = 1 / s_n
// (1 for empty columns and n >= K).
__global__ void m2l_colscale(const double *__restrict__ tab, int K, int Npad, float *__restrict__ cs) {
    __shared__ double red[256];
    const int n = blockIdx.x;
    double mx = 0.0;
    if (n < K)
        for (int e = threadIdx.x; e < 343 * K; e += blockDim.x) {
            const int off = e / K, kin = e - off * K;
            const int dx = off % 7 - 3, dy = (off / 7) % 7 - 3, dz = off / 49 - 3;
            if (max(abs(dx), max(abs(dy), abs(dz))) < 2) continue;
            mx = fmax(mx, fabs(tab[(size_t)off * K * K + (size_t)kin * K + n]));
        }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int sh = 0;
        if (red[0] > 0.0) {
            int e;
            const double f = frexp(red[0], &e);   // red = f 2^e, f in [0.5, 1)
            sh = 14 - (f == 0.5 ? e - 1 : e);
        }
        cs[n] = ldexpf(1.f, sh);
        cs[Npad + n] = ldexpf(1.f, -sh);
    }
}

// FP16 operator images of the tensor-core M2L: img[off][c][part][Npad][32],
// part 0 = FP16(T s), part 1 = FP16(T s - part 0), T = T_off[k_out][k_in]
// for the 32 inputs of chunk c, s = the column scale of k_out.
__global__ void build_h16_images(const double *__restrict__ tab, int K, int Npad, int nck,
                                 const float *__restrict__ cs, __half *__restrict__ img) {
    const int off = blockIdx.x;
    const int dx = off % 7 - 3, dy = (off / 7) % 7 - 3, dz = off / 49 - 3;
    const bool used = max(abs(dx), max(abs(dy), abs(dz))) >= 2;
    const size_t tile = (size_t)Npad * 32;
    for (int c = 0; c < nck; ++c) {
        __half *hi = img + ((size_t)off * nck + c) * 2 * tile;
        __half *lo = hi + tile;
        for (int e = threadIdx.x; e < Npad * 32; e += blockDim.x) {
            const int n = e / 32, kk = e % 32, kin = 32 * c + kk;
            const double v = (used && n < K && kin < K) ? tab[(size_t)off * K * K + (size_t)kin * K + n] * cs[n] : 0.0;
            const float f = (float)v;
            const __half h = __float2half_rn(f);
            const uint32_t o = swz64h(n, kk) / 2;
            hi[o] = h;
            lo[o] = __float2half_rn(f - __half2float(h));
        }
    }
}

// Operator images for the tensor-core M2M / L2L / P2M: img[off][c][part][Npad*16],
// part 0 = TF32(T), part 1 = TF32(T - TF32(T)), T = T_off[k_out][k_in] for
// the 16 inputs k_in of chunk c.
// With all_used (M2M / L2L: 8 octant operators) every slot is filled; for the
// M2L's 343 slots only offsets of max-norm >= 2 are.
__global__ void build_tc_images(const double *__restrict__ m2l_d, int K, int Npad, int nck,
                                float *__restrict__ img, int all_used = 0, int Kin = 0) {
    if (Kin == 0) Kin = K;   // operators [slot][Kin][K], input-component major
    const int off = blockIdx.x;
    const int dx = off % 7 - 3, dy = (off / 7) % 7 - 3, dz = off / 49 - 3;
    const bool used = all_used || max(abs(dx), max(abs(dy), abs(dz))) >= 2;
    const size_t tile = (size_t)Npad * 16;
    for (int c = 0; c < nck; ++c) {
        float *hi = img + ((size_t)off * nck + c) * 2 * tile;
        float *lo = hi + tile;
        for (int e = threadIdx.x; e < Npad * 16; e += blockDim.x) {
            const int n = e / 16, kk = e % 16, kin = 16 * c + kk;
            const double v = (used && n < K && kin < Kin) ? m2l_d[(size_t)off * Kin * K + (size_t)kin * K + n] : 0.0;
            const float f = (float)v;
            const float h = __uint_as_float(to_tf32(f));
            const float l = __uint_as_float(to_tf32(f - h));
            const uint32_t o = swz64(n, kk) / 4;
            hi[o] = h;
            lo[o] = l;
        }
    }
}

}  // namespace

gf_status build_p2m_tc_image(const double *pd, int K, int npad, int b3, float *img, cudaStream_t st) {
    build_tc_images<<<1, 256, 0, st>>>(pd, K, npad, b3 / 16, img, 1, b3);
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status build_p2m_up_tc_image(const double *q, int K, int npad, int b3, float *img, cudaStream_t st) {
    build_tc_images<<<8, 256, 0, st>>>(q, K, npad, b3 / 16, img, 1, b3);
    GF_KERNEL_DONE();
    return GF_OK;
}

gf_status m2l_prepare_tables(Tables *T, cudaStream_t st) {
    const int npad = (T->K + 15) & ~15;
    if (npad > 256) return GF_OK;  // beyond one MMA's N: SIMT only
    T->tc_npad = npad;
    T->tc_nck = (T->K + 15) / 16;
    T->tc_nck_h = (T->K + 31) / 32;
    const size_t n = (size_t)343 * T->tc_nck_h * 2 * npad * 32;
    for (int adj = 0; adj < 2; ++adj) {
        const double *tab = adj ? T->am2l_d : T->m2l_d;
        void *&img = adj ? T->am2l_tc : T->m2l_tc;
        float *&cs = adj ? T->am2l_cs : T->m2l_cs;
        GF_CUDA(cudaMalloc(&cs, 2 * npad * sizeof(float)));
        m2l_colscale<<<npad, 256, 0, st>>>(tab, T->K, npad, cs);
        GF_KERNEL_DONE();
        GF_CUDA(cudaMalloc(&img, n * sizeof(__half)));
        build_h16_images<<<343, 256, 0, st>>>(tab, T->K, npad, T->tc_nck_h, cs, (__half *)img);
        GF_KERNEL_DONE();
    }
    const size_t n8 = (size_t)8 * T->tc_nck * 2 * npad * 16;
    GF_CUDA(cudaMalloc(&T->m2m_tc, n8 * sizeof(float)));
    build_tc_images<<<8, 256, 0, st>>>(T->m2m_d, T->K, npad, T->tc_nck, T->m2m_tc, 1);
    GF_KERNEL_DONE();
    GF_CUDA(cudaMalloc(&T->l2l_tc, n8 * sizeof(float)));
    build_tc_images<<<8, 256, 0, st>>>(T->l2l_d, T->K, npad, T->tc_nck, T->l2l_tc, 1);
    GF_KERNEL_DONE();
    return GF_OK;
}

namespace {

struct M2LArgs {
    const void *me;    // input rows (forward: ME_l; adjoint: LE_l duals)
    void *le;          // output rows (forward: LE_l; adjoint: ME_l duals)
    int K, ldk, B, nbox;
    const int32_t *order;
    int64_t cls_off[9];
    const uint64_t *tkey;
    int64_t blo[3], bn[3];   // source block of the level
    const void *tab;   // [343][K][K], input component major
    int adj;           // adjoint: columns are source boxes, inputs via imap
    const int32_t *imap;
    int64_t mlo[3], mn[3];
    int shift;                   // level - 2
    uint32_t part_lo, part_hi;   // source partition (forward)
};

constexpr int kCK = 32;  // input components per shared-memory chunk

template <class T>
struct XStride {
    static constexpr int v = 36;
};
template <>
struct XStride<double> {
    static constexpr int v = 34;
};

__device__ __forceinline__ int64_t dm(uint64_t k, int s) {
    int64_t c = 0;
    for (int bit = 0; bit < 21; ++bit) c |= (int64_t)((k >> (3 * bit + s)) & 1) << bit;
    return c;
}

// Boxes of a dense block [lo, lo + n) whose coordinates have the parities of
// class `cls` (bit a = parity on axis a): per-axis first offset and count.
__host__ __device__ __forceinline__ void class_lattice(int cls, const int64_t *lo, const int64_t *n, int64_t *i0,
                                                       int64_t *cnt) {
    for (int a = 0; a < 3; ++a) {
        const int64_t par = (cls >> a) & 1;
        i0[a] = (par - (lo[a] & 1) + 2) & 1;
        cnt[a] = n[a] > i0[a] ? (n[a] - i0[a] + 1) / 2 : 0;
    }
}

// j-th box of class `cls` in a dense block: coordinates relative to lo.
__device__ __forceinline__ void class_box(int cls, const int64_t *lo, const int64_t *n, int64_t j, int64_t &x,
                                          int64_t &y, int64_t &z) {
    int64_t i0[3], c[3];
    class_lattice(cls, lo, n, i0, c);
    x = i0[0] + 2 * (j % c[0]);
    y = i0[1] + 2 * ((j / c[0]) % c[1]);
    z = i0[2] + 2 * (j / (c[0] * c[1]));
}

template <class T, int RPT>
__global__ void __launch_bounds__(256)
m2l_simt(M2LArgs a) {
    constexpr int S = XStride<T>::v;
    constexpr int KP = 32 * RPT;
    extern __shared__ unsigned char shraw[];
    T *Xs = reinterpret_cast<T *>(shraw);  // [kCK][S]
    T *Ts = Xs + kCK * S;                  // [kCK][KP]
    __shared__ int64_t tbox[32];
    __shared__ int tc[32][3];
    __shared__ int64_t srow[32];
    const int cls = blockIdx.y;
    const int64_t cbeg = a.cls_off[cls], ccnt = a.cls_off[cls + 1] - cbeg;
    const int64_t tile0 = (int64_t)blockIdx.x * a.nbox;
    if (tile0 >= ccnt) return;
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int K = a.K, B = a.B;
    const T *me = reinterpret_cast<const T *>(a.me);
    const T *tab = reinterpret_cast<const T *>(a.tab);
    if (tid < 32) {
        const int64_t s = tile0 + tid;
        if (tid < a.nbox && s < ccnt) {
            if (!a.adj) {
                const int64_t t = a.order[cbeg + s];
                tbox[tid] = t;
                const uint64_t key = a.tkey[t];
                tc[tid][0] = (int)(dm(key, 0) - a.blo[0]);
                tc[tid][1] = (int)(dm(key, 1) - a.blo[1]);
                tc[tid][2] = (int)(dm(key, 2) - a.blo[2]);
            } else {
                int64_t x, y, z;
                class_box(cls, a.blo, a.bn, s, x, y, z);
                tbox[tid] = (z * a.bn[1] + y) * a.bn[0] + x;
                tc[tid][0] = (int)x;
                tc[tid][1] = (int)y;
                tc[tid][2] = (int)z;
            }
        } else {
            tbox[tid] = -1;
        }
    }
    __syncthreads();
    T acc[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    for (int oi = 0; oi < 189; ++oi) {
        const int dx = c_il[cls][oi][0], dy = c_il[cls][oi][1], dz = c_il[cls][oi][2];
        int any = 0;
        if (tid < 32) {
            const int slot = tid / B, bb = tid - slot * B;
            int64_t row = -1;
            if (slot < a.nbox && tbox[slot] >= 0) {
                const int64_t sx = tc[slot][0] + dx, sy = tc[slot][1] + dy, sz = tc[slot][2] + dz;
                if (!a.adj) {
                    if (sx >= 0 && sy >= 0 && sz >= 0 && sx < a.bn[0] && sy < a.bn[1] && sz < a.bn[2] &&
                        in_source_part(sx + a.blo[0], sy + a.blo[1], sz + a.blo[2], a.shift, a.part_lo, a.part_hi))
                        row = (((sz * a.bn[1] + sy) * a.bn[0] + sx) * B + bb) * a.ldk;
                } else {
                    const int64_t wx = sx + a.blo[0] - a.mlo[0], wy = sy + a.blo[1] - a.mlo[1],
                                  wz = sz + a.blo[2] - a.mlo[2];
                    if (wx >= 0 && wy >= 0 && wz >= 0 && wx < a.mn[0] && wy < a.mn[1] && wz < a.mn[2]) {
                        const int32_t m = a.imap[(wz * a.mn[1] + wy) * a.mn[0] + wx];
                        if (m >= 0) row = ((int64_t)m * B + bb) * a.ldk;
                    }
                }
            }
            srow[tid] = row;
            any = row >= 0;
        }
        if (!__syncthreads_or(any)) continue;
        const T *tabo = tab + (size_t)((dz + 3) * 49 + (dy + 3) * 7 + (dx + 3)) * K * K;
        for (int c0 = 0; c0 < K; c0 += kCK) {
            for (int e = tid; e < kCK * 32; e += 256) {
                const int cc = e % kCK, j = e / kCK;
                const int64_t row = srow[j];
                const int c = c0 + cc;
                Xs[cc * S + j] = (row >= 0 && c < K) ? me[row + c] : T(0);
            }
            for (int e = tid; e < kCK * KP; e += 256) {
                const int cc = e / KP, k = e - cc * KP;
                const int c = c0 + cc;
                Ts[e] = (c < K && k < K) ? tabo[(size_t)c * K + k] : T(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int cc = 0; cc < kCK; ++cc) {
                T xv[4], tv[RPT];
#pragma unroll
                for (int c = 0; c < 4; ++c) xv[c] = Xs[cc * S + tx * 4 + c];
#pragma unroll
                for (int r = 0; r < RPT; ++r) tv[r] = Ts[cc * KP + ty * RPT + r];
#pragma unroll
                for (int r = 0; r < RPT; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += tv[r] * xv[c];
            }
            __syncthreads();
        }
    }
    T *le = reinterpret_cast<T *>(a.le);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = tx * 4 + c;
        const int slot = j / B, bb = j - slot * B;
        if (slot >= a.nbox || tbox[slot] < 0) continue;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = ty * RPT + r;
            if (k < K) le[(tbox[slot] * B + bb) * a.ldk + k] = acc[r][c];
        }
    }
}

// Batched M2M / L2L translations with the same SIMT tiling: a block takes
// 32 columns (box, batch member), gathers the K inputs of each column for
// every translation step into shared memory and multiplies them by the
// step's K x K operator (streamed in 32-row chunks), accumulating in Tc.
//   M2M: columns = parent boxes of the dense source block of level l, steps
//        = the 8 child positions; out = sum_oct T_oct ME_{l+1}[child] (store)
//   L2L: columns = observer boxes of level l of one parity class (the child
//        position), one step; out = LE_l + T_class LE_{l-1}[parent] (update)
struct XArgs {
    const void *in;
    void *out;
    int K, ldk, B, nbox, kind;      // 0 M2M, 1 L2L, 2 M2M^T, 3 L2L^T
    int64_t nout;                   // M2M: parents; L2L^T: observer boxes
    int64_t plo[3], pn[3];          // M2M, M2M^T: parent block
    int64_t clo[3], cn[3];          // M2M, M2M^T: child block
    const int32_t *order;           // L2L: class-grouped observer boxes
    int64_t cls_off[9];             // L2L: observer classes; M2M^T: source classes
    const int32_t *tparent;         // L2L
    const int32_t *child;           // L2L^T: [nout][8] child box or -1
    const void *tab;                // [8][K][K] input-major
};

template <class Ts, class Tc, int RPT>
__global__ void __launch_bounds__(256)
xlate_simt(XArgs a) {
    constexpr int S = XStride<Tc>::v;
    constexpr int KP = 32 * RPT;
    extern __shared__ unsigned char shraw[];
    Tc *Xs = reinterpret_cast<Tc *>(shraw);
    Tc *Ts_ = Xs + kCK * S;
    __shared__ int64_t obox[32];
    __shared__ int64_t srow[32];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int K = a.K, B = a.B;
    int cls = 0;
    int64_t cbeg = 0, ccnt = a.nout;
    if (a.kind == 1 || a.kind == 2) {
        cls = blockIdx.y;
        cbeg = a.cls_off[cls];
        ccnt = a.cls_off[cls + 1] - cbeg;
    }
    const int64_t tile0 = (int64_t)blockIdx.x * a.nbox;
    if (tile0 >= ccnt) return;
    const Ts *in = reinterpret_cast<const Ts *>(a.in);
    const Tc *tab = reinterpret_cast<const Tc *>(a.tab);
    if (tid < 32) {
        const int64_t sidx = tile0 + tid;
        int64_t ob = -1;
        if (tid < a.nbox && sidx < ccnt) {
            if (a.kind == 1) {
                ob = a.order[cbeg + sidx];
            } else if (a.kind == 2) {
                int64_t x, y, z;
                class_box(cls, a.clo, a.cn, sidx, x, y, z);
                ob = (z * a.cn[1] + y) * a.cn[0] + x;
            } else {
                ob = sidx;
            }
        }
        obox[tid] = ob;
    }
    __syncthreads();
    Tc acc[RPT][4];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = Tc(0);
    const int nsteps = (a.kind == 0 || a.kind == 3) ? 8 : 1;
    for (int st = 0; st < nsteps; ++st) {
        const int op = (a.kind == 0 || a.kind == 3) ? st : cls;
        if (tid < 32) {
            const int slot = tid / B, bb = tid - slot * B;
            int64_t row = -1;
            if (slot < a.nbox && obox[slot] >= 0) {
                const int64_t ob = obox[slot];
                if (a.kind == 0) {
                    const int64_t px = a.plo[0] + ob % a.pn[0], py = a.plo[1] + (ob / a.pn[0]) % a.pn[1],
                                  pz = a.plo[2] + ob / (a.pn[0] * a.pn[1]);
                    const int64_t cx = 2 * px + (op & 1) - a.clo[0], cy = 2 * py + ((op >> 1) & 1) - a.clo[1],
                                  cz = 2 * pz + ((op >> 2) & 1) - a.clo[2];
                    if (cx >= 0 && cy >= 0 && cz >= 0 && cx < a.cn[0] && cy < a.cn[1] && cz < a.cn[2])
                        row = (((cz * a.cn[1] + cy) * a.cn[0] + cx) * B + bb) * a.ldk;
                } else if (a.kind == 1) {
                    row = ((int64_t)a.tparent[ob] * B + bb) * a.ldk;
                } else if (a.kind == 2) {
                    const int64_t x = a.clo[0] + ob % a.cn[0], y = a.clo[1] + (ob / a.cn[0]) % a.cn[1],
                                  z = a.clo[2] + ob / (a.cn[0] * a.cn[1]);
                    const int64_t px = (x >> 1) - a.plo[0], py = (y >> 1) - a.plo[1], pz = (z >> 1) - a.plo[2];
                    row = (((pz * a.pn[1] + py) * a.pn[0] + px) * B + bb) * a.ldk;
                } else {
                    const int32_t c = a.child[ob * 8 + st];
                    if (c >= 0) row = ((int64_t)c * B + bb) * a.ldk;
                }
            }
            srow[tid] = row;
        }
        __syncthreads();
        const Tc *tabo = tab + (size_t)op * K * K;
        for (int c0 = 0; c0 < K; c0 += kCK) {
            for (int e = tid; e < kCK * 32; e += 256) {
                const int cc = e % kCK, j = e / kCK;
                const int64_t row = srow[j];
                const int c = c0 + cc;
                Xs[cc * S + j] = (row >= 0 && c < K) ? (Tc)in[row + c] : Tc(0);
            }
            for (int e = tid; e < kCK * KP; e += 256) {
                const int cc = e / KP, k = e - cc * KP;
                const int c = c0 + cc;
                Ts_[e] = (c < K && k < K) ? tabo[(size_t)c * K + k] : Tc(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int cc = 0; cc < kCK; ++cc) {
                Tc xv[4], tv[RPT];
#pragma unroll
                for (int c = 0; c < 4; ++c) xv[c] = Xs[cc * S + tx * 4 + c];
#pragma unroll
                for (int r = 0; r < RPT; ++r) tv[r] = Ts_[cc * KP + ty * RPT + r];
#pragma unroll
                for (int r = 0; r < RPT; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += tv[r] * xv[c];
            }
            __syncthreads();
        }
    }
    Ts *out = reinterpret_cast<Ts *>(a.out);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = tx * 4 + c;
        const int slot = j / B, bb = j - slot * B;
        if (slot >= a.nbox || obox[slot] < 0) continue;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int k = ty * RPT + r;
            if (k >= K) continue;
            Ts *o = out + (obox[slot] * B + bb) * a.ldk + k;
            const bool update = a.kind == 1 || a.kind == 2;
            *o = update ? (Ts)((Tc)*o + acc[r][c]) : (Ts)acc[r][c];
        }
    }
}

template <class Ts, class Tc, int RPT>
gf_status launch_xlate(const XArgs &a, int64_t tiles, int ny, cudaStream_t st) {
    const size_t shm = sizeof(Tc) * (kCK * XStride<Tc>::v + kCK * 32 * RPT);
    GF_TRY(ensure_smem(xlate_simt<Ts, Tc, RPT>, shm));
    xlate_simt<Ts, Tc, RPT><<<dim3((unsigned)tiles, ny), 256, shm, st>>>(a);
    GF_KERNEL_DONE();
    return GF_OK;
}

template <class T, int RPT>
gf_status launch_simt(const M2LArgs &a, int64_t max_tiles, cudaStream_t st) {
    const size_t shm = sizeof(T) * (kCK * XStride<T>::v + kCK * 32 * RPT);
    GF_TRY(ensure_smem(m2l_simt<T, RPT>, shm));
    m2l_simt<T, RPT><<<dim3((unsigned)max_tiles, 8), 256, shm, st>>>(a);
    GF_KERNEL_DONE();
    return GF_OK;
}

// ---------------------------------------------------------------- tcgen05
// Tensor-core translations (mixed precision): the M2L, and with the same
// machinery the M2M (8 child positions per parent) and the L2L (one step
// from the parent, operator chosen by the box's position in its parent).
// For the M2L, a CTA owns 128 target columns --
// (box, batch member) pairs of one parity class of one level -- and, offset
// by offset, computes D_o[col][k_out] = sum_k_in ME[t + o][k_in] T_o[k_out][k_in]
// on the tensor cores from FP16 parts, A_hi B_hi + A_hi B_lo + A_lo B_hi
// (K = 16 per MMA), with FP32 accumulation.  Both operands are scaled by
// powers of two so that every part that matters is a normal FP16 number:
// the inputs of a level by 2^sh (largest |input| into (2^14, 2^15]), each
// output column of the operator images by its own factor; the write-back
// divides both out exactly.  The inputs are split once per level by a small
// kernel before the M2L; the M2M, L2L and P2M kinds split FP32 inputs into
// TF32 parts in the kernel (3xTF32, K = 8 per MMA).  Inputs come in chunks
// (32 FP16 or 16 TF32 inputs; an FP16 stage holds two chunks) through a ring
// of shared-memory stages (64-byte swizzle), filled by warp-specialised
// producers:
//   warps 0-3   A producers, with 16-byte asynchronous copies: FP16 parts go
//               straight into the stage (eight lanes per row's 128 contiguous
//               bytes), and the stage is signalled once they have landed;
//               FP32 values (thread r: column r) go into a private ring three
//               chunks ahead, then are split into TF32 parts and stored
//               swizzled;
//   warp 4      one thread issues the MMAs of a stage and commits them to the
//               stage's "empty" barrier (and, after an offset's last chunk,
//               to the bank's "full" barrier);
//   warp 5      one thread bulk-copies the pre-split, pre-swizzled operator
//               image of each stage (transaction count on the same "full"
//               barrier the producers arrive on, so the issuer checks one
//               barrier per stage);
//   warps 6-13  promoters: after each offset they read the finished bank of
//               tensor memory and add it into FP32 registers (two banks
//               alternate, so the tensor cores never accumulate more than one
//               offset: their FP32 accumulation rounds differently from
//               IEEE and long chains over zero-mean data lose digits).
// Offsets whose source boxes are all missing are skipped by every role (a
// per-tile list built first).  Every wait is bounded and watches an abort
// flag; a wait that gives up sets status[1], and the CTA then drains its
// copies and MMAs (bounded) and frees its tensor memory.

// Translation kinds run by the kernel: the M2L (offsets of the interaction
// list, all levels in one launch), the M2M into one level (the 8 child
// positions; targets = every parent box of the dense block, one class) and
// the L2L into one level (one step: the parent; targets = observer boxes
// grouped by their position in the parent, which selects the operator);
// and the P2M (one step: the leaf's b^3 voxel masses times the P2M matrix).
enum TcKind { kTcM2L = 0, kTcM2M = 1, kTcL2L = 2, kTcP2M = 3 };

struct TcLevel {
    const float *me;      // input rows (M2L: ME_l or adjoint LE_l duals; M2M: ME_{l+1}; L2L: LE_{l-1})
    float *le;            // output rows (M2L: LE_l or adjoint ME_l duals; M2M: ME_l; L2L: LE_l, added to)
    const int32_t *order;
    const uint64_t *tkey;
    int64_t blo[3], bn[3];
    int64_t cls_off[9];
    int adj;
    const int32_t *imap;
    int64_t mlo[3], mn[3];
    int64_t clo[3], cn[3];       // M2M: child source block
    const int32_t *tparent;      // L2L: parent of each observer box
    const uint32_t *amax;        // M2L: largest |input| of the level (float bits)
    const unsigned char *split;  // M2L: the level's inputs split into scaled FP16 parts
    int64_t tfirst;              // P2M: index of the first leaf of the targets
    int shift;                   // M2L: level - 2 (source partition test)
    // P2M into level L-1 reading the density grid itself (TcArgs::grid): grid
    // voxel (i, j, k) of leaf (x, y, z) is i = gb x - goff[0] + (voxel in the
    // leaf), likewise j, k; leaves lie wholly inside or outside the grid
    int64_t goff[3], gn[3], gnvox;
    int gb;
    // M2M and P2M kinds (forward, mixed): the largest |value| written into
    // the target boxes [amax_lo, amax_hi) -- the z-slabs of the output level
    // that its M2L reads -- as float bits combined with atomicMax into
    // amax_out (the level's M2L input scale; null: not collected here)
    uint32_t *amax_out;
    int64_t amax_lo, amax_hi;
};

struct TcArgs {
    const TcLevel *lv;          // device array indexed by level
    int lmin, nent;             // entries e = (level - lmin) * 8 + class
    int tile_begin[kMaxLevels * 8 + 1];
    int K, ldk, B, Npad, nck, nst;
    int S;                      // input chunks per pipeline stage
    int le_f64;                 // M2L: the output rows are FP64 (an FP64 plan's local expansions)
    int kind, noff;             // TcKind; offsets per target (189, 8 or 1)
    int ntiles;                 // tiles of the launch (persistent kinds)
    int kin, ldin;              // input coefficients per row and input row stride
    const unsigned char *img;   // operator images, one [hi|lo] tile pair per (slot, chunk)
    const float *cs;            // M2L: column scales of the image ([Npad] scale, [Npad] inverse)
    int *status;
    long wait_tries;            // bound of every barrier wait (kWaitTries)
    uint32_t part_lo, part_hi;  // M2L forward: source partition (in_source_part)
    // M2L forward with msplit = 2: each tile's active offsets are shared by two
    // CTAs (blockIdx 2 t and 2 t + 1); each writes its partial rows to mpart
    // (slot = blockIdx, [128][Npad]) and counts itself in mcnt ([tile][8]
    // promoter warps, zero at launch); the second to arrive adds the other's
    // rows to its own and writes the tile.
    int msplit;
    float *mpart;
    int *mcnt;
    int test_stall;             // testing aid: the MMA issuer first waits on a barrier that
                                // nothing completes, so the bounded-wait failure path runs
    // M2M kind over leaf masses taken straight from the FP32 density grid:
    // the grid, and the element steps of its y and z rows (an input chunk is
    // one z-layer of a leaf, four rows of four voxels)
    const float *grid;
    int64_t gstep[2];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand with the 64-byte
// swizzle (8-row atoms of 512 bytes).
__device__ __forceinline__ uint64_t umma_desc64(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused, swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset: one 8-row atom
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)4 << 61;             // 64-byte swizzle
    return d;
}

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    // D = FP32, A = B = TF32, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    // D = FP32, A = B = FP16 (format 0), both K-major
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Power-of-two scale sig = 2^sh that brings the largest |input| m of an
// M2L level into (2^14, 2^15] (the top of the FP16 range, far from its
// subnormals), from the bits of m: ceil(log2 m) = E + (mantissa != 0) for
// m = 1.mantissa * 2^E.  sh is clamped to [-126, 126]; m = 0 gives 1.
__device__ __forceinline__ void input_scale(uint32_t mbits, float &sig, float &inv) {
    int sh = 0;
    if (mbits != 0u) {
        const int eb = (int)(mbits >> 23);   // biased exponent (0: subnormal)
        const int cl = (eb == 0 ? -126 : eb - 127) + ((mbits & 0x7FFFFFu) != 0u ? 1 : 0);
        sh = min(126, max(-126, 15 - cl));
    }
    sig = __int_as_float((127 + sh) << 23);
    inv = __int_as_float((127 - sh) << 23);
}

// Input chunk that an offset processes at step j of its nck steps: the
// highest chunk first (see the MMA issue order).
__host__ __device__ __forceinline__ int chunk_of(int nck, int j) { return nck - 1 - j; }

constexpr long kWaitTries = 1l << 24;
constexpr long kTestWaitTries = 1l << 12;   // wait bound under GF_FLAG_TEST_WAIT_TIMEOUT

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(addr), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier that also gives up when
// another role has set the abort flag; a timeout sets the flag.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t addr, uint32_t parity, volatile int *abort_flag,
                                             long tries) {
    for (long it = 0; it < tries; ++it) {
        if (mbar_try(addr, parity)) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// Bounded wait that ignores the abort flag (used to drain in-flight work).
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long tries) {
    for (long it = 0; it < tries; ++it)
        if (mbar_try(addr, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit_to(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Read 8 accumulator columns starting at address ta (this warp's 32 lanes).
__device__ __forceinline__ void tmem_ld8(uint32_t ta, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

constexpr int kTcWarps = 14;
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kTcMaxStages = 8;
constexpr uint32_t kTcCols = 512;           // two banks of 256 columns
constexpr uint32_t kTcA = 2u * 8192u;       // A hi + lo: 128 rows x 64 bytes each

constexpr int kTcRaw = 4;                   // input chunks in flight per producer thread (TF32 kinds)

__host__ __device__ constexpr uint32_t tc_stage_bytes(int Npad) { return kTcA + 2u * (uint32_t)Npad * 64u; }
// raw FP32 input ring of the TF32 producers: [kTcRaw][128 rows][16 floats]
__host__ __device__ constexpr uint32_t tc_raw_bytes(bool h16) { return h16 ? 0u : kTcRaw * 128u * 64u; }
constexpr size_t kTcSmemBudget = 227 * 1024 - 2048;
// Chunks per pipeline stage: the FP16 M2L moves two 32-input chunks per
// stage (12 MMAs per barrier wait); the TF32 kinds two 16-input chunks
// when two such stages fit in shared memory, else one.
inline int tc_chunks_per_stage(int Npad, bool h16) {
    if (h16) return 2;
    const size_t two = 2u * (size_t)tc_stage_bytes(Npad);
    return (kTcSmemBudget - tc_raw_bytes(false)) / two >= 2 ? 2 : 1;
}
inline int tc_stages(int Npad, bool h16) {
    const int n = (int)((kTcSmemBudget - tc_raw_bytes(h16)) /
                        ((size_t)tc_chunks_per_stage(Npad, h16) * tc_stage_bytes(Npad)));
    return n > kTcMaxStages ? kTcMaxStages : n;
}
size_t tc_smem_bytes(int Npad, bool h16) {
    return (size_t)tc_stages(Npad, h16) * tc_chunks_per_stage(Npad, h16) * tc_stage_bytes(Npad) +
           tc_raw_bytes(h16) + 1024;
}

// 16-byte asynchronous global -> shared copy; nbytes = 0 fills zeros.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t nbytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}

// NS >= Npad / 2: FP32 sums held per promoter thread.  H16: the M2L with
// FP16 operands, 32 inputs per stage (K = 16 per MMA); otherwise TF32, 16
// inputs per stage (K = 8 per MMA).
template <int NS, bool H16>
__global__ void __launch_bounds__(kTcThreads, 1)
m2l_tc(TcArgs a) {
    extern __shared__ unsigned char dsm[];
    unsigned char *base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);
    // afull: the stage's A operand has landed (128 producer arrivals); bfull:
    // its operator image has landed (the copy's own transaction count, so the
    // copying thread can always wait for its copies, whatever the producers do)
    __shared__ __align__(8) uint64_t afull[kTcMaxStages], bfull[kTcMaxStages], empty[kTcMaxStages];
    __shared__ __align__(8) uint64_t stall_bar;
    __shared__ __align__(8) uint64_t bank_full[2], bank_empty[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ uint32_t omask[6];   // M2L: offsets with at least one source box in this tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int B = a.B, Npad = a.Npad, nck = a.nck, NST = a.nst;
    const int nsum = Npad / 2;
    const uint32_t b_bytes = 2u * (uint32_t)Npad * 64u;
    constexpr int SH = 2;                  // chunks per stage of the FP16 M2L
    const int S = H16 ? SH : a.S;          // chunks per stage
    const uint32_t stage_bytes = S * tc_stage_bytes(Npad);   // [A: S x (hi, lo)][B: S x (hi, lo)]
    volatile int *abortp = &abort_flag;
    const int nbox = 128 / B;
    const int noff = a.noff;

    // The M2L takes one tile per CTA (its offsets are skipped where a whole
    // tile has no source); the other kinds are persistent: CTA b takes tiles
    // b, b + gridDim.x, ... and runs every offset of each.
    const bool persist = a.kind != kTcM2L;
    const int ntl = persist ? (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 1;
    const int msplit = persist ? 1 : max(1, a.msplit);
    const int utile = (int)blockIdx.x / msplit, uhalf = (int)blockIdx.x - utile * msplit;   // M2L: tile, share
    struct Ctx {
        const TcLevel *L;
        int cls, tile;
        int64_t cbeg, ccnt;
    };
    // (level, class, tile within the class) of this CTA's j-th tile
    auto ctx_of = [&](int j) -> Ctx {
        const int t = persist ? (int)blockIdx.x + j * (int)gridDim.x : utile;
        int e = 0;
        while (e + 1 < a.nent && a.tile_begin[e + 1] <= t) ++e;
        Ctx c;
        c.L = &a.lv[a.lmin + e / 8];
        c.cls = e % 8;
        c.tile = t - a.tile_begin[e];
        c.cbeg = c.L->cls_off[c.cls];
        c.ccnt = c.L->cls_off[c.cls + 1] - c.cbeg;
        return c;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            // 128 producer threads; the operator copy's expect-tx arrival
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[i])), "r"(128));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bfull[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bank_full[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bank_empty[i])), "r"(8));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&stall_bar)), "r"(1));
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < 6) omask[tid] = 0;

    // producer role: column `row` of the current tile
    const int row = tid & 127;
    const int slot = row / B, bb = row - slot * B;
    Ctx pc = ctx_of(0);
    int64_t tbox = -1, tc0 = 0, tc1 = 0, tc2 = 0;
    int64_t qbn0 = 0, qbn1 = 0, qbn2 = 0;   // the level's source block extent, kept in registers
    // M2M kind: the row of this parent's first child (position 0), the row
    // steps of a child move along x, y and z, and which of the 8 children exist
    int64_t qbase = 0, qsx = 0, qsy = 0, qsz = 0;
    uint32_t qmask = 0;
    int qadj = 0;
    auto set_target = [&]() {
        tbox = -1;
        tc0 = tc1 = tc2 = 0;
        const TcLevel &L = *pc.L;
        qbn0 = L.bn[0];
        qbn1 = L.bn[1];
        qbn2 = L.bn[2];
        qadj = L.adj;
        const int64_t sidx = (int64_t)pc.tile * nbox + slot;
        if (warp >= 4 || slot >= nbox || sidx >= pc.ccnt) return;
        if (a.kind == kTcP2M) {
            tbox = L.tfirst + sidx;
        } else if (a.kind == kTcM2M) {
            tbox = sidx;
            tc0 = sidx % L.bn[0];
            tc1 = (sidx / L.bn[0]) % L.bn[1];
            tc2 = sidx / (L.bn[0] * L.bn[1]);
            const int64_t c0 = 2 * (tc0 + L.blo[0]) - L.clo[0], c1 = 2 * (tc1 + L.blo[1]) - L.clo[1],
                          c2 = 2 * (tc2 + L.blo[2]) - L.clo[2];
            uint32_t v0 = 0, v1 = 0, v2 = 0;   // bit d: the child at step d along the axis exists
            for (int d = 0; d < 2; ++d) {
                bool ok0 = c0 + d >= 0 && c0 + d < L.cn[0], ok1 = c1 + d >= 0 && c1 + d < L.cn[1],
                     ok2 = c2 + d >= 0 && c2 + d < L.cn[2];
                if (a.grid) {   // and its first voxel lies in the density grid
                    const int64_t i = (L.clo[0] + c0 + d) * L.gb - L.goff[0], j = (L.clo[1] + c1 + d) * L.gb - L.goff[1],
                                  k = (L.clo[2] + c2 + d) * L.gb - L.goff[2];
                    ok0 = ok0 && i >= 0 && i < L.gn[0];
                    ok1 = ok1 && j >= 0 && j < L.gn[1];
                    ok2 = ok2 && k >= 0 && k < L.gn[2];
                }
                v0 |= (uint32_t)ok0 << d;
                v1 |= (uint32_t)ok1 << d;
                v2 |= (uint32_t)ok2 << d;
            }
            qmask = 0;
            for (int oi = 0; oi < 8; ++oi)
                if (((v0 >> (oi & 1)) & (v1 >> ((oi >> 1) & 1)) & (v2 >> (oi >> 2))) & 1u) qmask |= 1u << oi;
            if (a.grid) {   // the child leaf's first voxel in the density grid
                const int64_t i0 = (L.clo[0] + c0) * L.gb - L.goff[0], j0 = (L.clo[1] + c1) * L.gb - L.goff[1],
                              k0 = (L.clo[2] + c2) * L.gb - L.goff[2];
                qbase = bb * L.gnvox + (k0 * L.gn[1] + j0) * L.gn[0] + i0;
                qsx = L.gb;
                qsy = (int64_t)L.gb * L.gn[0];
                qsz = qsy * L.gn[1];
            } else {
                qsx = (int64_t)B * a.ldin;
                qsy = L.cn[0] * qsx;
                qsz = L.cn[1] * qsy;
                qbase = ((c2 * L.cn[1] + c1) * L.cn[0] + c0) * qsx + (int64_t)bb * a.ldin;
            }
        } else if (a.kind == kTcL2L) {
            tbox = L.order[pc.cbeg + sidx];
        } else if (!L.adj) {
            tbox = L.order[pc.cbeg + sidx];
            const uint64_t key = L.tkey[tbox];
            tc0 = dm(key, 0) - L.blo[0];
            tc1 = dm(key, 1) - L.blo[1];
            tc2 = dm(key, 2) - L.blo[2];
        } else {
            class_box(pc.cls, L.blo, L.bn, sidx, tc0, tc1, tc2);
            tbox = (tc2 * L.bn[1] + tc1) * L.bn[0] + tc0;
        }
    };
    set_target();
    // input row of this column at offset oi of the current tile (-1: none)
    auto src_row = [&](int oi) -> int64_t {
        if (tbox < 0) return -1;
        const TcLevel &L = *pc.L;
        if (a.kind == kTcM2M)   // child at position oi of this parent
            return ((qmask >> oi) & 1u) ? qbase + (oi & 1) * qsx + ((oi >> 1) & 1) * qsy + (oi >> 2) * qsz : -1;
        if (a.kind == kTcL2L) return ((int64_t)L.tparent[tbox] * B + bb) * a.ldin;
        if (a.kind == kTcP2M) return (tbox * B + bb) * a.ldin;
        const int cls = pc.cls;
        const int64_t sx = tc0 + c_il[cls][oi][0], sy = tc1 + c_il[cls][oi][1], sz = tc2 + c_il[cls][oi][2];
        if (!qadj) {
            if (sx >= 0 && sy >= 0 && sz >= 0 && sx < qbn0 && sy < qbn1 && sz < qbn2 &&
                in_source_part(sx + L.blo[0], sy + L.blo[1], sz + L.blo[2], L.shift, a.part_lo, a.part_hi))
                return (((sz * qbn1 + sy) * qbn0 + sx) * B + bb) * a.ldin;
            return -1;
        }
        const int64_t wx = sx + L.blo[0] - L.mlo[0], wy = sy + L.blo[1] - L.mlo[1], wz = sz + L.blo[2] - L.mlo[2];
        if (wx >= 0 && wy >= 0 && wz >= 0 && wx < L.mn[0] && wy < L.mn[1] && wz < L.mn[2]) {
            const int32_t m = L.imap[(wz * L.mn[1] + wy) * L.mn[0] + wx];
            if (m >= 0) return ((int64_t)m * B + bb) * a.ldin;
        }
        return -1;
    };
    __syncthreads();
    if (!persist && warp < 4) {
        for (int w = 0; w * 32 < noff; ++w) {
            uint32_t bits = 0;
            for (int b = 0; b < 32 && 32 * w + b < noff; ++b)
                if (src_row(32 * w + b) >= 0) bits |= 1u << b;
            bits = __reduce_or_sync(0xffffffffu, bits);
            if (lane == 0 && bits) atomicOr(&omask[w], bits);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (msplit > 1) {
        // keep this CTA's share of the tile's active offsets: ranks
        // [uhalf tot / msplit, (uhalf + 1) tot / msplit) in offset order
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < 6; ++w) tot += __popc(omask[w]);
            const int lo = uhalf * tot / msplit, hi = (uhalf + 1) * tot / msplit;
            int rank = 0;
            for (int w = 0; w < 6; ++w) {
                uint32_t m = omask[w], keep = 0;
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    if (rank >= lo && rank < hi) keep |= 1u << b;
                    ++rank;
                }
                omask[w] = keep;
            }
        }
        __syncthreads();
    }
    const uint32_t tmem = tslot;
    int G = noff;   // offsets per tile
    if (!persist) {
        G = 0;
        for (int w = 0; w < 6; ++w) G += __popc(omask[w]);
    }
    const int offs = G * ntl;        // offsets run by this CTA
    const int nsp = (nck + S - 1) / S;   // stages per offset
    const int iters = offs * nsp;    // stages run by this CTA
    // the next offset to run after oi within a tile (noff when none is left)
    auto next_off = [&](int oi) -> int {
        for (++oi; oi < noff; ++oi)
            if (persist || (omask[oi >> 5] & (1u << (oi & 31)))) return oi;
        return noff;
    };

    if (warp < 4) {
        // ---------------- A producers
        int qj = 0, qo = next_off(-1), qc = 0;
        int64_t qs = qo < noff ? src_row(qo) : -1;
        auto take = [&](int &c_out, int64_t &s_out) {   // next chunk in sequence
            c_out = qc;
            s_out = qs;
            if (++qc == nck) {
                qc = 0;
                qo = next_off(qo);
                if (qo >= noff && ++qj < ntl) {
                    pc = ctx_of(qj);
                    set_target();
                    qo = next_off(-1);
                }
                qs = (qj < ntl && qo < noff) ? src_row(qo) : -1;
            }
        };
        if (H16) {
            // FP16 inputs, scaled and split in advance: once a stage is free,
            // each thread copies its row's 64-byte high and low pieces of the
            // stage's chunks straight into it (16-byte asynchronous copies to
            // the swizzled positions; a missing source copies zeros), waits for
            // them and signals the stage.  The copies overlap the MMAs of the
            // previous stage.
            const unsigned char *spl = pc.L->split;   // every tile of a launch reads the same levels
            int s = 0;
            uint32_t ph = 0;
            for (int it = 0; it < iters; ++it) {
                if (it >= NST && !mbar_wait_ab(smem_u32(&empty[s]), ph ^ 1, abortp, a.wait_tries)) break;
                unsigned char *stage = base + (size_t)s * stage_bytes;
                int c0 = 0, nc = SH;
#pragma unroll
                for (int q = 0; q < SH; ++q) {
                    if (q > 0 && c0 + q >= nck) break;   // the offset's last stage may hold fewer chunks
                    int cc;
                    int64_t sr;
                    take(cc, sr);
                    if (q == 0) {
                        c0 = cc;
                        nc = min(SH, nck - c0);
                    }
                    // chunks run from the highest inputs down (chunk_of), and the
                    // stage keeps its chunks in ascending order
                    const int pc = chunk_of(nck, cc);
                    // the warp's 32 rows in 8 passes of 4: eight lanes copy one
                    // row's 128 contiguous bytes (pieces 0-3 high, 4-7 low)
                    const uint32_t sub = smem_u32(stage + (nc - 1 - q) * kTcA);
                    const int k = lane & 7;
                    const uint32_t kpart = k < 4 ? 0u : 8192u;
                    const int kk = 8 * (k & 3);
#pragma unroll
                    for (int pp = 0; pp < 8; ++pp) {
                        const int rl = 4 * pp + (lane >> 3);
                        const int64_t srp = __shfl_sync(0xffffffffu, (long long)sr, rl);
                        const int r = (row & ~31) + rl;
                        const unsigned char *src = srp >= 0 ? spl + (size_t)srp * 4 + (size_t)pc * 128 + 16 * k : spl;
                        cp_async16(sub + kpart + swz64h(r, kk), src, srp >= 0 ? 16u : 0u);
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&afull[s]));
                if (++s == NST) {
                    s = 0;
                    ph ^= 1;
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");   // no copy outlives the loop (abort)
        } else {
            // TF32 inputs, split here
            constexpr int kW = 16;     // inputs per chunk
            constexpr int kV = kW / 4; // 16-byte pieces per row and chunk
            const float *me = a.grid ? a.grid : pc.L->me;   // every tile of a launch reads the same input array
            // Each thread copies its own row's chunks kTcRaw - 1 chunks ahead into
            // a raw ring (16-byte pieces XOR-swizzled by row, so that a warp's
            // reads of one piece hit distinct banks); a missing source copies
            // zeros.  Only the copying thread reads them back.
            unsigned char *raw = base + (size_t)NST * stage_bytes + (size_t)row * (kW * 4);
            auto issue = [&](int64_t j) {
                int cc;
                int64_t sr;
                take(cc, sr);
                const uint32_t d0 = smem_u32(raw + (size_t)(j % kTcRaw) * 128 * (kW * 4));
                // a chunk is 16 contiguous inputs, or (density grid) the leaf's
                // z-layer: four rows of four voxels a y-step apart
                const int ck = chunk_of(nck, cc);
                const float *src = sr < 0 ? me : (a.grid ? me + sr + ck * a.gstep[1] : me + sr + kW * ck);
                const int64_t qs = sr < 0 ? 0 : (a.grid ? a.gstep[0] : 4);
#pragma unroll
                for (int q = 0; q < kV; ++q)
                    cp_async16(d0 + ((q ^ (row & (kV - 1))) << 4), src + q * qs, sr >= 0 ? 16u : 0u);
            };
            // chunks are issued and consumed in take() order: stage `it` holds
            // the chunks at positions [c0, c0 + nc) of its offset (the offset's
            // last stage may hold fewer), slot nc - 1 - q for the q-th
            const int64_t nchunks = (int64_t)offs * nck;
#pragma unroll 1
            for (int j = 0; j < kTcRaw - 1; ++j) {
                if (j < nchunks) issue(j);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            int s = 0;
            uint32_t ph = 0;
            bool bad = false;   // a non-finite input (densities read from the grid)
            int64_t jc = 0;     // next chunk to consume
            bool stop = false;
            for (int it = 0; it < iters && !stop; ++it) {
                const int c0 = (it % nsp) * S;
                const int nc = min(S, nck - c0);
                unsigned char *stage = base + (size_t)s * stage_bytes;
                for (int q = 0; q < nc; ++q, ++jc) {
                    if (jc + kTcRaw - 1 < nchunks) issue(jc + kTcRaw - 1);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group %0;" ::"n"(kTcRaw - 1) : "memory");   // chunk jc has landed
                    if (q == 0 && it >= NST && !mbar_wait_ab(smem_u32(&empty[s]), ph ^ 1, abortp, a.wait_tries)) {
                        stop = true;
                        break;
                    }
                    const int cin = chunk_of(nck, c0 + q);   // input chunk
                    float4 cur[kV];
                    {
                        const float4 *rr =
                            reinterpret_cast<const float4 *>(raw + (size_t)(jc % kTcRaw) * 128 * (kW * 4));
#pragma unroll
                        for (int v = 0; v < kV; ++v) cur[v] = rr[v ^ (row & (kV - 1))];
                    }
                    unsigned char *sub = stage + (size_t)(nc - 1 - q) * kTcA;
                    // inputs past kin (the last chunk) read as zero; densities read
                    // from the grid are checked for non-finite values
                    auto split = [&](auto tail, auto check) {
                        constexpr bool kTail = decltype(tail)::value, kCheck = decltype(check)::value;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float x4[4] = {cur[v].x, cur[v].y, cur[v].z, cur[v].w};
                            uint32_t h[4], l[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float x = (!kTail || 16 * cin + 4 * v + j < a.kin) ? x4[j] : 0.f;
                                if (kCheck) bad |= !isfinite(x);
                                h[j] = to_tf32_int(x);
                                l[j] = to_tf32_int(x - __uint_as_float(h[j]));
                            }
                            const uint32_t o = swz64(row, 4 * v);
                            *reinterpret_cast<uint4 *>(sub + o) = make_uint4(h[0], h[1], h[2], h[3]);
                            *reinterpret_cast<uint4 *>(sub + 8192 + o) = make_uint4(l[0], l[1], l[2], l[3]);
                        }
                    };
                    if (16 * (cin + 1) > a.kin)
                        split(std::true_type{}, std::true_type{});
                    else if (a.grid)
                        split(std::false_type{}, std::true_type{});
                    else
                        split(std::false_type{}, std::false_type{});
                }
                if (stop) break;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&afull[s]));
                if (++s == NST) {
                    s = 0;
                    ph ^= 1;
                }
            }
            asm volatile("cp.async.wait_all;" ::: "memory");   // no copy outlives the loop (abort)
            if (bad && a.grid) atomicOr(a.status, 1);
        }
    } else if (warp == 4) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = H16 ? idesc_f16(128, Npad) : idesc_tf32(128, Npad);
            int s = 0, c0 = 0, g = 0;
            uint32_t ph = 0;
            int last = -1;
            // testing aid: a wait that nothing completes runs out, sets the abort
            // flag, and every role stops, drains and reports through status[1]
            const bool stalled = a.test_stall && !mbar_wait_ab(smem_u32(&stall_bar), 0, abortp, a.wait_tries);
            for (int it = 0; it < (stalled ? 0 : iters); ++it) {
                if (!mbar_wait_ab(smem_u32(&afull[s]), ph, abortp, a.wait_tries)) break;
                if (!mbar_wait_ab(smem_u32(&bfull[s]), ph, abortp, a.wait_tries)) break;
                if (c0 == 0 && g >= 2 &&
                    !mbar_wait_ab(smem_u32(&bank_empty[g & 1]), ((g - 2) >> 1) & 1, abortp, a.wait_tries))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned char *stage = base + (size_t)s * stage_bytes;
                const uint32_t d = tmem + (uint32_t)(g & 1) * 256u;
                const int nc = min(S, nck - c0);
                // Inputs in descending order: the stage's chunks from the last
                // slot down, each chunk's k-steps from the last down, and in each
                // k-step the two small cross products before the main one.  The
                // accumulator adds of the tensor cores truncate, so every add made
                // once the sum has its full size costs up to an ulp of it, all of
                // the same sign; leading with the small high-order terms leaves
                // only the last few adds at full size.
                for (int q = 0; q < nc; ++q) {
                    const int sl = nc - 1 - q;
                    const int c = chunk_of(nck, c0 + nc - 1) + sl;   // the input chunk in slot sl
                    const uint32_t sa = smem_u32(stage + sl * kTcA);
                    const uint32_t sb = smem_u32(stage + S * kTcA + sl * b_bytes);
                    // k-steps of 32 bytes (8 TF32 or 16 FP16 inputs) holding inputs
                    const int nks = H16 ? min(2, (a.kin - 32 * c + 15) / 16) : min(2, (a.kin - 16 * c + 7) / 8);
                    for (int ks = nks - 1; ks >= 0; --ks) {
                        const uint32_t ko = ks * 32;
                        const uint64_t ah = umma_desc64(sa + ko), al = umma_desc64(sa + 8192 + ko);
                        const uint64_t bh = umma_desc64(sb + ko), bl = umma_desc64(sb + (uint32_t)Npad * 64 + ko);
                        const uint32_t acc = (c0 > 0 || q > 0 || ks < nks - 1) ? 1u : 0u;
                        if (H16) {
                            mma_f16(d, ah, bl, idesc, acc);
                            mma_f16(d, al, bh, idesc, 1u);
                            mma_f16(d, ah, bh, idesc, 1u);
                        } else {
                            mma_tf32(d, ah, bl, idesc, acc);
                            mma_tf32(d, al, bh, idesc, 1u);
                            mma_tf32(d, ah, bh, idesc, 1u);
                        }
                    }
                }
                commit_to(&empty[s]);
                last = it;
                c0 += S;
                if (c0 >= nck) {
                    commit_to(&bank_full[g & 1]);
                    c0 = 0;
                    ++g;
                }
                if (++s == NST) {
                    s = 0;
                    ph ^= 1;
                }
            }
            // drain: the last commit covers every MMA issued
            if (last >= 0) mbar_wait(smem_u32(&empty[last % NST]), (uint32_t)((last / NST) & 1), a.wait_tries);
        }
    } else if (warp == 5) {
        // ---------------- operator images
        if (lane == 0) {
            int s = 0, c0 = 0, bj = 0;
            int oi = next_off(-1);
            int bcls = pc.cls;
            uint32_t ph = 0;
            int last = -1;
            for (int it = 0; it < iters; ++it) {
                if (it >= NST && !mbar_wait_ab(smem_u32(&empty[s]), ph ^ 1, abortp, a.wait_tries)) break;
                int slot_off;
                if (a.kind == kTcM2L) {
                    const int dx = c_il[bcls][oi][0], dy = c_il[bcls][oi][1], dz = c_il[bcls][oi][2];
                    slot_off = (dz + 3) * 49 + (dy + 3) * 7 + (dx + 3);
                } else if (a.kind == kTcM2M) {
                    slot_off = oi;     // child position
                } else if (a.kind == kTcL2L) {
                    slot_off = bcls;   // the box's own position in its parent
                } else {
                    slot_off = 0;
                }
                unsigned char *stage = base + (size_t)s * stage_bytes;
                // the stage's chunks of the operator image are contiguous
                // (ascending, the lowest being that of the stage's last chunk)
                const int ncs = min(S, nck - c0);
                const uint32_t nbytes = (uint32_t)ncs * b_bytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bfull[s])),
                             "r"(nbytes));
                const unsigned char *srcimg = a.img + ((size_t)slot_off * nck + chunk_of(nck, c0 + ncs - 1)) * b_bytes;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(stage + S * kTcA)),
                    "l"(srcimg), "r"(nbytes), "r"(smem_u32(&bfull[s]))
                    : "memory");
                last = it;
                c0 += S;
                if (c0 >= nck) {
                    c0 = 0;
                    oi = next_off(oi);
                    if (oi >= noff && ++bj < ntl) {
                        bcls = ctx_of(bj).cls;
                        oi = next_off(-1);
                    }
                }
                if (++s == NST) {
                    s = 0;
                    ph ^= 1;
                }
            }
            // drain: every copy issued must have landed before the CTA exits;
            // the last NST stages may still have copies in flight (earlier ones
            // were consumed by MMAs before their stage was reused), and each
            // stage's copy completes its own barrier
            for (int j = last - NST + 1 > 0 ? last - NST + 1 : 0; j <= last; ++j)
                mbar_wait(smem_u32(&bfull[j % NST]), (uint32_t)((j / NST) & 1), a.wait_tries);
        }
    }
    // ---------------- promoters (warps 6-13) and the write-back of each tile
    const int pw = warp - 6;
    const int pq = warp & 3, ph_half = pw >> 2;   // TMEM lane quarter, column half
    bool ok = true;
    if (pw >= 0) {
        float acc[NS];
        int gg = 0;   // offsets promoted so far (bank gg & 1)
        for (int j = 0; j < ntl && ok; ++j) {
#pragma unroll
            for (int q = 0; q < NS; ++q) acc[q] = 0.f;
            for (int g = 0; g < G; ++g, ++gg) {
                bool w_ok = mbar_wait_ab(smem_u32(&bank_full[gg & 1]), (gg >> 1) & 1, abortp, a.wait_tries);
                w_ok = __all_sync(0xffffffffu, w_ok);   // tcgen05.ld is warp-collective
                if (!w_ok) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t tb =
                    tmem + ((uint32_t)(pq * 32) << 16) + (uint32_t)(gg & 1) * 256u + (uint32_t)(ph_half * nsum);
#pragma unroll
                for (int j0 = 0; j0 < NS; j0 += 8) {
                    if (j0 < nsum) {
                        float t[8];
                        tmem_ld8(tb + j0, t);
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc[j0 + q] += t[q];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&bank_empty[gg & 1]));
            }
            if (!ok || *abortp) {
                ok = false;
                break;
            }
            // write this tile's rows
            const Ctx oc = ctx_of(j);
            const TcLevel &L = *oc.L;
            const int r = pq * 32 + lane;
            const int oslot = r / B, obb = r - oslot * B;
            const int64_t os = (int64_t)oc.tile * nbox + oslot;
            bool write = true;
            if (H16) {
                // undo the column scales of the image and the input scale
                float sig, sig_inv;
                input_scale(*L.amax, sig, sig_inv);
                const float4 *ci = reinterpret_cast<const float4 *>(a.cs + Npad + ph_half * nsum);
#pragma unroll
                for (int q = 0; q < NS; q += 4)
                    if (q < nsum) {
                        const float4 c4 = __ldg(ci + q / 4);
                        acc[q] = acc[q] * c4.x * sig_inv;
                        acc[q + 1] = acc[q + 1] * c4.y * sig_inv;
                        acc[q + 2] = acc[q + 2] * c4.z * sig_inv;
                        acc[q + 3] = acc[q + 3] * c4.w * sig_inv;
                    }
                if (msplit > 1) {
                    // this warp's slice of the tile (32 rows, half the columns):
                    // partial rows out, then the second CTA to arrive adds the
                    // other's rows (a + b = b + a, so the sum does not depend on
                    // which CTA is second) and writes the tile
                    float4 *mine = reinterpret_cast<float4 *>(a.mpart + ((size_t)blockIdx.x * 128 + r) * Npad +
                                                              ph_half * nsum);
#pragma unroll
                    for (int q = 0; q < NS; q += 4)
                        if (q < nsum) mine[q / 4] = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
                    __threadfence();
                    __syncwarp();
                    int second = 0;
                    if (lane == 0) second = atomicAdd(a.mcnt + (size_t)utile * 8 + pw, 1) == msplit - 1;
                    second = __shfl_sync(0xffffffffu, second, 0);
                    write = second != 0;
                    if (write) {
                        __threadfence();
                        const float4 *other = reinterpret_cast<const float4 *>(
                            a.mpart + ((size_t)(utile * msplit + (1 - uhalf)) * 128 + r) * Npad + ph_half * nsum);
#pragma unroll
                        for (int q = 0; q < NS; q += 4)
                            if (q < nsum) {
                                const float4 o4 = __ldcg(other + q / 4);
                                acc[q] += o4.x;
                                acc[q + 1] += o4.y;
                                acc[q + 2] += o4.z;
                                acc[q + 3] += o4.w;
                            }
                    }
                }
            }
            float am = 0.f;   // this row's largest |value| (M2M / P2M kinds with amax_out)
            if (write && oslot < nbox && os < oc.ccnt) {
                int64_t obox;
                if (a.kind == kTcM2M) {   // dense targets
                    obox = os;
                } else if (a.kind == kTcP2M) {
                    obox = L.tfirst + os;
                } else if (!L.adj) {
                    obox = L.order[oc.cbeg + os];
                } else {
                    int64_t ox, oy, oz;
                    class_box(oc.cls, L.blo, L.bn, os, ox, oy, oz);
                    obox = (oz * L.bn[1] + oy) * L.bn[0] + ox;
                }
                // 16-byte stores of the whole half row: columns from K up to
                // Npad hold zeros (the operator images are zero there) and stay
                // inside the row's padding (Npad <= ldk)
                float4 *dst = reinterpret_cast<float4 *>(L.le + (obox * B + obb) * a.ldk + ph_half * nsum);
                if (a.kind == kTcL2L) {
#pragma unroll
                    for (int q = 0; q < NS; q += 4)
                        if (q < nsum) {
                            float4 v = dst[q / 4];
                            v.x += acc[q];
                            v.y += acc[q + 1];
                            v.z += acc[q + 2];
                            v.w += acc[q + 3];
                            dst[q / 4] = v;
                        }
                } else if (H16) {   // rows already unscaled (above)
                    if (a.le_f64) {
                        // an FP64 plan's local expansions: rows of ldk >= Npad doubles
                        double *dd = reinterpret_cast<double *>(L.le) + (obox * B + obb) * a.ldk + ph_half * nsum;
#pragma unroll
                        for (int q = 0; q < NS; q += 4)
                            if (q < nsum) {
                                dd[q] = (double)acc[q];
                                dd[q + 1] = (double)acc[q + 1];
                                dd[q + 2] = (double)acc[q + 2];
                                dd[q + 3] = (double)acc[q + 3];
                            }
                    } else {
#pragma unroll
                        for (int q = 0; q < NS; q += 4)
                            if (q < nsum) dst[q / 4] = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < NS; q += 4)
                        if (q < nsum) dst[q / 4] = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
                    if (L.amax_out && obox >= L.amax_lo && obox < L.amax_hi) {
#pragma unroll
                        for (int q = 0; q < NS; ++q)
                            if (q < nsum && ph_half * nsum + q < a.K) am = fmaxf(am, fabsf(acc[q]));
                    }
                }
            }
            if (!H16 && L.amax_out) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
                if (lane == 0 && am > 0.f) atomicMax(L.amax_out, __float_as_uint(am));
            }
        }
    }
    const bool failed = __syncthreads_or(!ok || abort_flag);
    if (failed && tid == 0) atomicOr(a.status + 1, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

}  // namespace

// Bytes of the split FP16 inputs of levels 2..l-1 (the start of level l in
// the split buffer), for the plan's largest batch.
static size_t split_offset(const FmmPlan *F, int adj, int l) {
    size_t off = 0;
    for (int k = 2; k < l; ++k) off += (size_t)(adj ? F->lev[k].nt : F->lev[k].ns) * F->B * F->KS * sizeof(float);
    return off;
}

gf_status m2l_tc_prepare_adj(gf_plan_s *plan) {
    FmmPlan *F = plan->fmm;
    if (!F->mixed || !F->tab->m2l_tc) return GF_OK;
    GF_TRY(plan->arena.alloc((void **)&F->tc_split_adj, std::max<size_t>(16, split_offset(F, 1, F->L + 1))));
    for (int adj = 1; adj < 2; ++adj) {
        std::vector<TcLevel> h(F->L + 1);
        memset(h.data(), 0, h.size() * sizeof(TcLevel));
        for (int l = 2; l <= F->L; ++l) {
            const FmmLevel &lv = F->lev[l];
            TcLevel &t = h[l];
            t.me = (const float *)(adj ? lv.le : lv.me);
            t.le = (float *)(adj ? lv.me : lv.le);
            t.order = lv.m2l_order;
            t.tkey = lv.tkey;
            t.adj = adj;
            t.imap = F->imap[l];
            for (int d = 0; d < 3; ++d) {
                t.blo[d] = lv.slo[d];
                t.bn[d] = lv.sn[d];
                t.mlo[d] = F->mlo[l][d];
                t.mn[d] = F->mn[l][d];
            }
            for (int c = 0; c <= 8; ++c) t.cls_off[c] = adj ? F->scls_off[l][c] : lv.cls_off[c];
            t.amax = F->tc_amax + (adj ? kMaxLevels + 1 : 0) + l;
            t.split = (adj ? F->tc_split_adj : F->tc_split) + split_offset(F, adj, l);
            t.shift = l - 2;
        }
        std::vector<unsigned char> &hb = adj ? F->tc_levels_adj_host : F->tc_levels_host;
        void *&dev = adj ? F->tc_levels_adj : F->tc_levels;
        hb.assign(reinterpret_cast<unsigned char *>(h.data()), reinterpret_cast<unsigned char *>(h.data() + h.size()));
        GF_TRY(plan->arena.alloc(&dev, hb.size()));
        GF_TRY(upload_small(dev, hb.data(), hb.size(), plan->arena.stream));
    }
    return GF_OK;
}

gf_status m2l_tc_prepare(gf_plan_s *plan) {
    FmmPlan *F = plan->fmm;
    if (!(F->mixed || F->m2l_tc64) || !F->tab->m2l_tc) return GF_OK;
    GF_TRY(plan->arena.alloc((void **)&F->tc_amax, 2 * (kMaxLevels + 1) * sizeof(uint32_t)));
    GF_TRY(plan->arena.alloc((void **)&F->tc_split, std::max<size_t>(16, split_offset(F, 0, F->L + 1))));
    {
        // partial rows of the forward M2L's tiles when two CTAs share each
        // (tiles counted for the plan's largest batch: the most tiles)
        const int nbox = 128 / std::max(1, std::min(F->B, 128));
        int64_t tiles = 0;
        for (int l = 2; l <= F->L; ++l)
            for (int c = 0; c < 8; ++c) {
                const int64_t cnt = F->lev[l].nt > 0 ? F->lev[l].cls_off[c + 1] - F->lev[l].cls_off[c] : 0;
                tiles += (cnt + nbox - 1) / nbox;
            }
        if (tiles > 0 && 2 * tiles <= (int64_t)sm_count()) {
            GF_TRY(plan->arena.alloc((void **)&F->m2l_part, (size_t)tiles * 2 * 128 * F->tab->tc_npad * sizeof(float)));
            GF_TRY(plan->arena.alloc((void **)&F->m2l_cnt, (size_t)tiles * 8 * sizeof(int)));
            F->m2l_part_tiles = (int)tiles;
        }
    }
    for (int adj = 0; adj < 1; ++adj) {
        std::vector<TcLevel> h(F->L + 1);
        memset(h.data(), 0, h.size() * sizeof(TcLevel));
        for (int l = 2; l <= F->L; ++l) {
            const FmmLevel &lv = F->lev[l];
            TcLevel &t = h[l];
            t.me = (const float *)(adj ? lv.le : lv.me);
            t.le = (float *)(adj ? lv.me : lv.le);
            t.order = lv.m2l_order;
            t.tkey = lv.tkey;
            t.adj = adj;
            t.imap = F->imap[l];
            for (int d = 0; d < 3; ++d) {
                t.blo[d] = lv.slo[d];
                t.bn[d] = lv.sn[d];
                t.mlo[d] = F->mlo[l][d];
                t.mn[d] = F->mn[l][d];
            }
            for (int c = 0; c <= 8; ++c) t.cls_off[c] = adj ? F->scls_off[l][c] : lv.cls_off[c];
            t.amax = F->tc_amax + (adj ? kMaxLevels + 1 : 0) + l;
            t.split = (adj ? F->tc_split_adj : F->tc_split) + split_offset(F, adj, l);
            t.shift = l - 2;
        }
        std::vector<unsigned char> &hb = adj ? F->tc_levels_adj_host : F->tc_levels_host;
        void *&dev = adj ? F->tc_levels_adj : F->tc_levels;
        hb.assign(reinterpret_cast<unsigned char *>(h.data()), reinterpret_cast<unsigned char *>(h.data() + h.size()));
        GF_TRY(plan->arena.alloc(&dev, hb.size()));
        GF_TRY(upload_small(dev, hb.data(), hb.size(), plan->arena.stream));
    }
    // M2M into level l (entries [0, L]), L2L into level l (entries [L+1, 2L+1]),
    // the P2M of every leaf (entry 2L+2), the P2M into level L-1 straight
    // from the leaf masses (entry 2L+3) and the P2M of the leaves in the
    // z-slabs the leaf level's M2L reads (entry 2L+4)
    if (F->mixed && F->tab->m2m_tc && F->tab->l2l_tc) {
        // the output level's M2L-reachable boxes (the rows input_absmax reads)
        auto set_amax = [&](TcLevel &t, int l) {
            const FmmLevel &lv = F->lev[l];
            const int64_t slab = lv.sn[0] * lv.sn[1];
            t.amax_out = F->tc_amax + l;
            t.amax_lo = lv.m2l_z1 >= lv.m2l_z0 ? lv.m2l_z0 * slab : 0;
            t.amax_hi = lv.m2l_z1 >= lv.m2l_z0 ? (lv.m2l_z1 + 1) * slab : 0;
        };
        std::vector<TcLevel> h(2 * (F->L + 1) + 3);
        memset(h.data(), 0, h.size() * sizeof(TcLevel));
        for (int l = 2; l <= F->L; ++l) {
            if (l < F->L) {
                const FmmLevel &pa = F->lev[l], &ch = F->lev[l + 1];
                TcLevel &t = h[l];
                t.me = (const float *)ch.me;
                t.le = (float *)pa.me;
                for (int d = 0; d < 3; ++d) {
                    t.blo[d] = pa.slo[d];
                    t.bn[d] = pa.sn[d];
                    t.clo[d] = ch.slo[d];
                    t.cn[d] = ch.sn[d];
                }
                t.cls_off[0] = 0;
                for (int c = 1; c <= 8; ++c) t.cls_off[c] = pa.ns;
                set_amax(t, l);
            }
            if (l > 2) {
                const FmmLevel &lv = F->lev[l], &pa = F->lev[l - 1];
                TcLevel &t = h[F->L + 1 + l];
                t.me = (const float *)pa.le;
                t.le = (float *)lv.le;
                t.order = lv.m2l_order;
                t.tkey = lv.tkey;
                t.tparent = lv.tparent;
                for (int d = 0; d < 3; ++d) {
                    t.blo[d] = lv.slo[d];
                    t.bn[d] = lv.sn[d];
                }
                for (int c = 0; c <= 8; ++c) t.cls_off[c] = lv.cls_off[c];
            }
        }
        {
            const FmmLevel &lv = F->lev[F->L];
            TcLevel &t = h[2 * (F->L + 1)];
            t.me = (const float *)F->mass;
            t.le = (float *)lv.me;
            t.cls_off[0] = 0;
            for (int c = 1; c <= 8; ++c) t.cls_off[c] = lv.ns;
            set_amax(t, F->L);
            if ((F->b * F->b * F->b) % 16 == 0) GF_TRY(get_p2m_tc(plan, plan->arena.stream));
            TcLevel &r = h[2 * (F->L + 1) + 2];
            r = t;
            const int64_t slab = lv.sn[0] * lv.sn[1];
            const int64_t nz = lv.m2l_z1 >= lv.m2l_z0 ? lv.m2l_z1 - lv.m2l_z0 + 1 : 0;
            r.tfirst = nz > 0 ? lv.m2l_z0 * slab : 0;
            for (int c = 1; c <= 8; ++c) r.cls_off[c] = nz * slab;
        }
        if (F->L - 1 > 2) {
            const FmmLevel &pa = F->lev[F->L - 1], &ch = F->lev[F->L];
            TcLevel &t = h[2 * (F->L + 1) + 1];
            t.me = (const float *)F->mass;
            t.le = (float *)pa.me;
            for (int d = 0; d < 3; ++d) {
                t.blo[d] = pa.slo[d];
                t.bn[d] = pa.sn[d];
                t.clo[d] = ch.slo[d];
                t.cn[d] = ch.sn[d];
            }
            t.cls_off[0] = 0;
            for (int c = 1; c <= 8; ++c) t.cls_off[c] = pa.ns;
            t.gb = F->b;
            set_amax(t, F->L - 1);
            t.gnvox = plan->nvox;
            for (int d = 0; d < 3; ++d) {
                t.goff[d] = F->voff[d];
                t.gn[d] = plan->grid.n[d];
            }
        }
        F->tc_xlate_host.assign(reinterpret_cast<unsigned char *>(h.data()),
                                reinterpret_cast<unsigned char *>(h.data() + h.size()));
        GF_TRY(plan->arena.alloc(&F->tc_xlate, F->tc_xlate_host.size()));
        GF_TRY(upload_small(F->tc_xlate, F->tc_xlate_host.data(), F->tc_xlate_host.size(), plan->arena.stream));
    }
    return GF_OK;
}

namespace {

// Largest |x| over the first kin components of every row of each level's
// M2L input (forward: ME_l; adjoint: the LE_l duals), as the bits of a
// non-negative float, combined with atomicMax (out[] zeroed before).
struct AmaxArgs {
    const float4 *in[kMaxLevels + 1];   // FP32 rows, or (f64) FP64 rows read through in64
    const double *in64[kMaxLevels + 1];
    int64_t rows[kMaxLevels + 1];
    uint32_t *out;
    int lmin, ld4, kin;
    int f64;                            // inputs are FP64 rows of 4 ld4 doubles
};

__global__ void __launch_bounds__(256) input_absmax(AmaxArgs a) {
    const int l = a.lmin + (int)blockIdx.y;
    if (a.f64) {
        // FP64 rows: element by element
        const double *p = a.in64[l];
        const int ld = 4 * a.ld4;
        const int64_t n = a.rows[l] * ld;
        float m = 0.f;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            if ((int)(i % ld) < a.kin) m = fmaxf(m, fabsf((float)__ldg(p + i)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(a.out + l, __float_as_uint(m));
        return;
    }
    const float4 *p = a.in[l];
    const int64_t n = a.rows[l] * a.ld4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = i + u * stride < n ? __ldg(p + i + u * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = (int)((i + u * stride) % a.ld4) * 4;
            if (c < a.kin) m = fmaxf(m, fabsf(v[u].x));
            if (c + 1 < a.kin) m = fmaxf(m, fabsf(v[u].y));
            if (c + 2 < a.kin) m = fmaxf(m, fabsf(v[u].z));
            if (c + 3 < a.kin) m = fmaxf(m, fabsf(v[u].w));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(a.out + l, __float_as_uint(m));
}

// Split every M2L input row into the FP16 operand parts the tensor-core
// M2L copies: x s = hi + lo + O(2^-22 |x s|), s = the level's input scale;
// per row and 32-wide chunk, 64 bytes of hi then 64 bytes of lo (inputs
// beyond kin are zero).
struct SplitArgs {
    unsigned char *out[kMaxLevels + 1];
};

__global__ void __launch_bounds__(256) input_split(AmaxArgs a, SplitArgs o, int nck) {
    const int l = a.lmin + (int)blockIdx.y;
    float sig, sig_inv;
    input_scale(a.out[l], sig, sig_inv);
    const int64_t items = a.rows[l] * nck;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nck;
        const int c = (int)(i - r * nck);
        float4 v[8];
        if (a.f64) {
            // FP64 rows (4 ld4 doubles): 32 inputs rounded to FP32 (the parts carry 22 bits)
            const double2 *s2 = reinterpret_cast<const double2 *>(a.in64[l] + r * 4 * a.ld4 + 32 * c);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const double2 d0 = __ldg(s2 + 2 * q), d1 = __ldg(s2 + 2 * q + 1);
                v[q] = make_float4((float)d0.x, (float)d0.y, (float)d1.x, (float)d1.y);
            }
        } else {
            const float4 *src = a.in[l] + r * a.ld4 + 8 * c;
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldg(src + q);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(o.out[l] + (size_t)i * 128);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float x8[8] = {v[2 * q].x,     v[2 * q].y,     v[2 * q].z,     v[2 * q].w,
                                 v[2 * q + 1].x, v[2 * q + 1].y, v[2 * q + 1].z, v[2 * q + 1].w};
            uint32_t h[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int kin = 32 * c + 8 * q + 2 * j;
                const float x0 = kin < a.kin ? x8[2 * j] * sig : 0.f;
                const float x1 = kin + 1 < a.kin ? x8[2 * j + 1] * sig : 0.f;
                const __half2 hh = __floats2half2_rn(x0, x1);
                const float2 hf = __half22float2(hh);
                const __half2 ll = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
                memcpy(&h[j], &hh, 4);
                memcpy(&lo[j], &ll, 4);
            }
            dst[q] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[4 + q] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

gf_status tc_launch(TcArgs &a, int tiles, cudaStream_t st) {
    if (tiles == 0) return GF_OK;
    a.ntiles = tiles;
    // the M2L runs one tile per CTA; the other kinds loop over tiles, one CTA per SM
    const int grid = a.kind == kTcM2L ? tiles * std::max(1, a.msplit) : std::min(tiles, 152);
    const bool h16 = a.kind == kTcM2L;
    const size_t shm = tc_smem_bytes(a.Npad, h16);
    a.nst = tc_stages(a.Npad, h16);
    a.S = tc_chunks_per_stage(a.Npad, h16);
    const int nsum = a.Npad / 2;
#define GF_TC_LAUNCH(NS)                                                  \
    do {                                                                  \
        if (a.kind == kTcM2L) {                                           \
            GF_TRY((ensure_smem(m2l_tc<NS, true>, shm)));                 \
            m2l_tc<NS, true><<<grid, kTcThreads, shm, st>>>(a);           \
        } else {                                                          \
            GF_TRY((ensure_smem(m2l_tc<NS, false>, shm)));                \
            m2l_tc<NS, false><<<grid, kTcThreads, shm, st>>>(a);          \
        }                                                                 \
    } while (0)
    if (nsum <= 32)
        GF_TC_LAUNCH(32);
    else if (nsum <= 64)
        GF_TC_LAUNCH(64);
    else if (nsum <= 96)
        GF_TC_LAUNCH(96);
    else
        GF_TC_LAUNCH(128);
#undef GF_TC_LAUNCH
    GF_KERNEL_DONE();
    return GF_OK;
}

TcArgs tc_args(gf_plan_s *plan, int B) {
    FmmPlan *F = plan->fmm;
    const Tables *T = F->tab;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.K = F->K;
    a.ldk = F->KS;
    a.B = B;
    a.Npad = T->tc_npad;
    a.nck = T->tc_nck;
    a.kin = F->K;
    a.ldin = F->KS;
    a.status = plan->d_status;
    a.wait_tries = kWaitTries;
    a.part_lo = 0;
    a.part_hi = 64;
    a.msplit = 1;
    return a;
}

gf_status m2l_run_tc(gf_plan_s *plan, int B, bool adj, cudaStream_t st, cudaEvent_t fork) {
    FmmPlan *F = plan->fmm;
    const Tables *T = F->tab;
    TcArgs a = tc_args(plan, B);
    a.lv = reinterpret_cast<const TcLevel *>(adj ? F->tc_levels_adj : F->tc_levels);
    a.lmin = 2;
    a.kind = kTcM2L;
    a.noff = 189;
    a.nck = T->tc_nck_h;
    a.img = (const unsigned char *)(adj ? T->am2l_tc : T->m2l_tc);
    a.cs = adj ? T->am2l_cs : T->m2l_cs;
    a.le_f64 = F->m2l_tc64 ? 1 : 0;
    a.part_lo = adj ? 0u : plan->part_lo;
    a.part_hi = adj ? 64u : plan->part_hi;
    if (plan->opt.reserved0 & GF_FLAG_TEST_WAIT_TIMEOUT) {
        a.test_stall = 1;
        a.wait_tries = kTestWaitTries;
    }
    if (F->L < 2) return GF_OK;
    // the largest |input| of every level, for the FP16 input scales
    {
        AmaxArgs m;
        memset(&m, 0, sizeof(m));
        m.out = F->tc_amax + (adj ? kMaxLevels + 1 : 0);
        m.lmin = 2;
        m.ld4 = F->KS / 4;
        m.kin = F->K;
        m.f64 = F->m2l_tc64 ? 1 : 0;
        int64_t most = 0;
        // forward: only the z-slabs of each level's source block that an
        // interaction list reaches (rows run x fastest, then y, then z)
        int64_t row0[kMaxLevels + 1] = {};
        for (int l = 2; l <= F->L; ++l) {
            const FmmLevel &lv = F->lev[l];
            int64_t r0 = 0, nr = (adj ? lv.nt : lv.ns) * B;
            if (!adj) {
                const int64_t slab = lv.sn[0] * lv.sn[1] * B;
                r0 = lv.m2l_z1 >= lv.m2l_z0 ? lv.m2l_z0 * slab : 0;
                nr = lv.m2l_z1 >= lv.m2l_z0 ? (lv.m2l_z1 - lv.m2l_z0 + 1) * slab : 0;
            }
            row0[l] = r0;
            m.in[l] = (const float4 *)(adj ? lv.le : lv.me) + r0 * m.ld4;
            m.in64[l] = (const double *)(adj ? lv.le : lv.me) + r0 * 4 * m.ld4;
            m.rows[l] = nr;
            most = std::max(most, m.rows[l] * m.ld4);
        }
        const int gx = (int)std::min<int64_t>(8 * 152, std::max<int64_t>(1, (most + 1023) / 1024));
        if (adj || !F->amax_fused) {   // else the kernels that wrote the expansions took it
            GF_CUDA(cudaMemsetAsync(m.out, 0, (kMaxLevels + 1) * sizeof(uint32_t), st));
            input_absmax<<<dim3(gx, F->L - 1), 256, 0, st>>>(m);
            GF_KERNEL_DONE();
        }
        SplitArgs o;
        memset(&o, 0, sizeof(o));
        for (int l = 2; l <= F->L; ++l)
            o.out[l] = (adj ? F->tc_split_adj : F->tc_split) + split_offset(F, adj, l) + (size_t)row0[l] * F->KS * 4;
        input_split<<<dim3(gx, F->L - 1), 256, 0, st>>>(m, o, T->tc_nck_h);
        GF_KERNEL_DONE();
    }
    if (!adj) stage_mark(plan, 4, st);
    const int nbox = 128 / B;
    int tiles = 0, e = 0;
    for (int l = 2; l <= F->L; ++l)
        for (int c = 0; c < 8; ++c, ++e) {
            a.tile_begin[e] = tiles;
            const int64_t *off = adj ? F->scls_off[l] : F->lev[l].cls_off;
            const int64_t cnt = (adj || F->lev[l].nt > 0) ? off[c + 1] - off[c] : 0;
            tiles += (int)((cnt + nbox - 1) / nbox);
        }
    a.tile_begin[e] = tiles;
    a.nent = e;
    // when two CTAs per tile still fit the SMs at once, every tile's offsets
    // are shared by two: each chain of offsets is half as long (and each
    // FP32 sum of offsets half as deep)
    if (!adj && F->m2l_part && tiles <= F->m2l_part_tiles && 2 * tiles <= sm_count()) {
        a.msplit = 2;
        a.mpart = F->m2l_part;
        a.mcnt = F->m2l_cnt;
        GF_CUDA(cudaMemsetAsync(F->m2l_cnt, 0, (size_t)tiles * 8 * sizeof(int), st));
    }
    if (fork) GF_CUDA(cudaEventRecord(fork, st));
    return tc_launch(a, tiles, st);
}

gf_status p2m_run_tc_impl(gf_plan_s *plan, int B, bool slabs, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    TcArgs a = tc_args(plan, B);
    const int b3 = F->b * F->b * F->b;
    const int entry = 2 * (F->L + 1) + (slabs ? 2 : 0);
    a.lv = reinterpret_cast<const TcLevel *>(F->tc_xlate) + entry;
    a.lmin = 0;
    a.kind = kTcP2M;
    a.noff = 1;
    a.kin = b3;
    a.ldin = b3;
    a.nck = b3 / 16;
    a.img = (const unsigned char *)F->p2m_tc;
    const int nbox = 128 / B;
    const int64_t ns = reinterpret_cast<const TcLevel *>(F->tc_xlate_host.data())[entry].cls_off[1];
    const int tiles = (int)((ns + nbox - 1) / nbox);
    a.tile_begin[0] = 0;
    for (int c = 1; c <= 8; ++c) a.tile_begin[c] = tiles;
    a.nent = 8;
    return tc_launch(a, tiles, st);
}

// P2M into level L-1: the M2M kind over the leaf masses (8 child positions,
// b^3 inputs each) with the composite operators Q_o.
gf_status p2m_up_run_tc_impl(gf_plan_s *plan, int B, const float *grid, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    TcArgs a = tc_args(plan, B);
    if (grid) {
        a.grid = grid;
        a.gstep[0] = plan->grid.n[0];
        a.gstep[1] = plan->grid.n[0] * plan->grid.n[1];
    }
    const int b3 = F->b * F->b * F->b;
    const int entry = 2 * (F->L + 1) + 1;
    a.lv = reinterpret_cast<const TcLevel *>(F->tc_xlate) + entry;
    a.lmin = 0;
    a.kind = kTcM2M;
    a.noff = 8;
    a.kin = b3;
    a.ldin = b3;
    a.nck = b3 / 16;
    a.img = (const unsigned char *)F->p2m_up_tc;
    const int nbox = 128 / B;
    const int64_t np = F->lev[F->L - 1].ns;
    const int tiles = (int)((np + nbox - 1) / nbox);
    a.tile_begin[0] = 0;
    for (int c = 1; c <= 8; ++c) a.tile_begin[c] = tiles;
    a.nent = 8;
    return tc_launch(a, tiles, st);
}

// M2M (kind 0) or L2L (kind 1) into `level` on the tensor cores.
gf_status xlate_run_tc(gf_plan_s *plan, int level, int kind, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const Tables *T = F->tab;
    TcArgs a = tc_args(plan, B);
    const TcLevel *base = reinterpret_cast<const TcLevel *>(F->tc_xlate);
    a.lv = base + (kind == 0 ? 0 : F->L + 1);
    a.lmin = level;
    a.kind = kind == 0 ? kTcM2M : kTcL2L;
    a.noff = kind == 0 ? 8 : 1;
    a.img = (const unsigned char *)(kind == 0 ? T->m2m_tc : T->l2l_tc);
    const TcLevel &h = reinterpret_cast<const TcLevel *>(F->tc_xlate_host.data())[(kind == 0 ? 0 : F->L + 1) + level];
    const int nbox = 128 / B;
    int tiles = 0;
    for (int c = 0; c < 8; ++c) {
        a.tile_begin[c] = tiles;
        tiles += (int)((h.cls_off[c + 1] - h.cls_off[c] + nbox - 1) / nbox);
    }
    a.tile_begin[8] = tiles;
    a.nent = 8;
    return tc_launch(a, tiles, st);
}

}  // namespace

template <class T>
gf_status m2l_level(gf_plan_s *plan, int level, int B, bool adj, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const FmmLevel &lv = F->lev[level];
    M2LArgs a;
    a.me = adj ? lv.le : lv.me;
    a.le = adj ? lv.me : lv.le;
    a.K = F->K;
    a.ldk = F->KS;
    a.B = B;
    a.nbox = std::max(1, 32 / B);
    a.order = lv.m2l_order;
    a.adj = adj ? 1 : 0;
    a.imap = F->imap[level];
    a.shift = level - 2;
    a.part_lo = adj ? 0u : plan->part_lo;
    a.part_hi = adj ? 64u : plan->part_hi;
    int64_t maxc = 0;
    for (int c = 0; c <= 8; ++c) a.cls_off[c] = adj ? F->scls_off[level][c] : lv.cls_off[c];
    for (int c = 0; c < 8; ++c) maxc = std::max<int64_t>(maxc, a.cls_off[c + 1] - a.cls_off[c]);
    a.tkey = lv.tkey;
    for (int d = 0; d < 3; ++d) {
        a.blo[d] = lv.slo[d];
        a.bn[d] = lv.sn[d];
        a.mlo[d] = F->mlo[level][d];
        a.mn[d] = F->mn[level][d];
    }
    if (adj)
        a.tab = sizeof(T) == 8 ? (const void *)F->tab->am2l_d : (const void *)F->tab->am2l_f;
    else
        a.tab = sizeof(T) == 8 ? (const void *)F->tab->m2l_d : (const void *)F->tab->m2l_f;
    if (B > 32) {
        set_error("M2L supports at most 32 batch members");
        return GF_ERR_UNSUPPORTED;
    }
    const int64_t tiles = (maxc + a.nbox - 1) / a.nbox;
    if (tiles == 0) return GF_OK;
    const int rpt = (F->K + 31) / 32;
    switch (rpt) {
        case 1: return launch_simt<T, 1>(a, tiles, st);
        case 2: return launch_simt<T, 2>(a, tiles, st);
        case 3: return launch_simt<T, 3>(a, tiles, st);
        case 4: return launch_simt<T, 4>(a, tiles, st);
        case 5: return launch_simt<T, 5>(a, tiles, st);
        case 6: return launch_simt<T, 6>(a, tiles, st);
        case 7: return launch_simt<T, 7>(a, tiles, st);
        case 8: return launch_simt<T, 8>(a, tiles, st);
        case 9: return launch_simt<T, 9>(a, tiles, st);
        case 10: return launch_simt<T, 10>(a, tiles, st);
        default:
            set_error("expansion degree too large for the M2L kernel");
            return GF_ERR_UNSUPPORTED;
    }
}

bool p2m_tc_ok(const gf_plan_s *plan, int B) {
    const FmmPlan *F = plan->fmm;
    return F && F->mixed && F->p2m_tc && F->tc_xlate && !(plan->opt.reserved0 & GF_FLAG_M2L_SIMT) && B <= 128 &&
           tc_stages(F->tab->tc_npad, false) >= 2;
}

bool p2m_up_ok(const gf_plan_s *plan, int B) {
    const FmmPlan *F = plan->fmm;
    return p2m_tc_ok(plan, B) && F->p2m_up_tc && F->L - 1 > 2 && F->b * F->b * F->b == 64;
}

gf_status p2m_run_tc(gf_plan_s *plan, int B, cudaStream_t st) {
    return p2m_run_tc_impl(plan, B, p2m_up_ok(plan, B), st);
}

bool p2m_up_grid_ok(const gf_plan_s *plan, const void *rho, int rho_dtype) {
    const FmmPlan *F = plan->fmm;
    if (rho_dtype != GF_DTYPE_F32 || ((uintptr_t)rho & 15) != 0 || F->b != 4) return false;
    for (int d = 0; d < 3; ++d)
        if (plan->grid.n[d] % 4 != 0 || F->voff[d] % 4 != 0) return false;
    return true;
}

gf_status p2m_up_run_tc(gf_plan_s *plan, int B, const float *grid, cudaStream_t st) {
    return p2m_up_run_tc_impl(plan, B, grid, st);
}

template <class Ts, class Tc>
gf_status translate_run(gf_plan_s *plan, int level, int kind, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    // mixed precision: forward M2M / L2L on the tensor cores (3xTF32)
    if (sizeof(Ts) == 4 && sizeof(Tc) == 4 && (kind == 0 || kind == 1) && F->tc_xlate &&
        !(plan->opt.reserved0 & GF_FLAG_M2L_SIMT) && B <= 128 && tc_stages(F->tab->tc_npad, false) >= 2)
        return xlate_run_tc(plan, level, kind, B, st);
    XArgs a;
    a.K = F->K;
    a.ldk = F->KS;
    a.B = B;
    a.nbox = std::max(1, 32 / B);
    a.kind = kind;
    int64_t tiles;
    int ny = 1;
    a.child = nullptr;
    if (kind == 2) {   // M2M^T into `level` (children) from level - 1
        const FmmLevel &ch = F->lev[level], &pa = F->lev[level - 1];
        a.in = pa.me;
        a.out = ch.me;
        a.nout = ch.ns;
        for (int d = 0; d < 3; ++d) {
            a.plo[d] = pa.slo[d];
            a.pn[d] = pa.sn[d];
            a.clo[d] = ch.slo[d];
            a.cn[d] = ch.sn[d];
        }
        for (int c = 0; c <= 8; ++c) a.cls_off[c] = F->scls_off[level][c];
        a.order = nullptr;
        a.tparent = nullptr;
        a.tab = sizeof(Tc) == 8 ? (const void *)F->tab->am2m_d : (const void *)F->tab->am2m_f;
        int64_t maxc = 0;
        for (int c = 0; c < 8; ++c) maxc = std::max<int64_t>(maxc, a.cls_off[c + 1] - a.cls_off[c]);
        tiles = (maxc + a.nbox - 1) / a.nbox;
        ny = 8;
    } else if (kind == 3) {   // L2L^T into `level` (parents) from level + 1
        const FmmLevel &lv = F->lev[level], &ch = F->lev[level + 1];
        if (lv.nt == 0) return GF_OK;
        a.in = ch.le;
        a.out = lv.le;
        a.nout = lv.nt;
        a.child = F->child[level];
        a.order = nullptr;
        a.tparent = nullptr;
        a.tab = sizeof(Tc) == 8 ? (const void *)F->tab->al2l_d : (const void *)F->tab->al2l_f;
        tiles = (lv.nt + a.nbox - 1) / a.nbox;
    } else if (kind == 0) {   // M2M into `level` from level + 1
        const FmmLevel &pa = F->lev[level], &ch = F->lev[level + 1];
        a.in = ch.me;
        a.out = pa.me;
        a.nout = pa.ns;
        for (int d = 0; d < 3; ++d) {
            a.plo[d] = pa.slo[d];
            a.pn[d] = pa.sn[d];
            a.clo[d] = ch.slo[d];
            a.cn[d] = ch.sn[d];
        }
        a.order = nullptr;
        a.tparent = nullptr;
        a.tab = sizeof(Tc) == 8 ? (const void *)F->tab->m2m_d : (const void *)F->tab->m2m_f;
        tiles = (pa.ns + a.nbox - 1) / a.nbox;
    } else {           // L2L into `level` from level - 1
        const FmmLevel &lv = F->lev[level], &pa = F->lev[level - 1];
        if (lv.nt == 0) return GF_OK;
        a.in = pa.le;
        a.out = lv.le;
        a.nout = lv.nt;
        a.order = lv.m2l_order;
        for (int c = 0; c <= 8; ++c) a.cls_off[c] = lv.cls_off[c];
        a.tparent = lv.tparent;
        a.tab = sizeof(Tc) == 8 ? (const void *)F->tab->l2l_d : (const void *)F->tab->l2l_f;
        int64_t maxc = 0;
        for (int c = 0; c < 8; ++c) maxc = std::max<int64_t>(maxc, lv.cls_off[c + 1] - lv.cls_off[c]);
        tiles = (maxc + a.nbox - 1) / a.nbox;
        ny = 8;
    }
    if (tiles == 0) return GF_OK;
    switch ((F->K + 31) / 32) {
        case 1: return launch_xlate<Ts, Tc, 1>(a, tiles, ny, st);
        case 2: return launch_xlate<Ts, Tc, 2>(a, tiles, ny, st);
        case 3: return launch_xlate<Ts, Tc, 3>(a, tiles, ny, st);
        case 4: return launch_xlate<Ts, Tc, 4>(a, tiles, ny, st);
        case 5: return launch_xlate<Ts, Tc, 5>(a, tiles, ny, st);
        case 6: return launch_xlate<Ts, Tc, 6>(a, tiles, ny, st);
        case 7: return launch_xlate<Ts, Tc, 7>(a, tiles, ny, st);
        case 8: return launch_xlate<Ts, Tc, 8>(a, tiles, ny, st);
        case 9: return launch_xlate<Ts, Tc, 9>(a, tiles, ny, st);
        case 10: return launch_xlate<Ts, Tc, 10>(a, tiles, ny, st);
        default:
            set_error("expansion degree too large for the translation kernel");
            return GF_ERR_UNSUPPORTED;
    }
}

template gf_status translate_run<float, float>(gf_plan_s *, int, int, int, cudaStream_t);
template gf_status translate_run<float, double>(gf_plan_s *, int, int, int, cudaStream_t);
template gf_status translate_run<double, double>(gf_plan_s *, int, int, int, cudaStream_t);

template <class T>
gf_status m2l_run(gf_plan_s *plan, int B, bool adj, cudaStream_t st, cudaEvent_t fork) {
    FmmPlan *F = plan->fmm;
    const bool tc = (sizeof(T) == 4 || (F->m2l_tc64 && !adj)) && F->tab->m2l_tc && (adj ? F->tc_levels_adj : F->tc_levels) &&
                    !(plan->opt.reserved0 & GF_FLAG_M2L_SIMT) && B <= 128 &&
                    tc_stages(F->tab->tc_npad, true) >= 2;
    if (tc) return m2l_run_tc(plan, B, adj, st, fork);
    if (!adj) stage_mark(plan, 4, st);   // no input split on this path
    if (fork) GF_CUDA(cudaEventRecord(fork, st));
    for (int l = 2; l <= F->L; ++l) {
        if (F->lev[l].nt == 0 && !adj) continue;   // the adjoint writes every source box
        GF_TRY(m2l_level<T>(plan, l, B, adj, st));
    }
    return GF_OK;
}

template gf_status m2l_run<float>(gf_plan_s *, int, bool, cudaStream_t, cudaEvent_t);
template gf_status m2l_run<double>(gf_plan_s *, int, bool, cudaStream_t, cudaEvent_t);

}  // namespace gf
