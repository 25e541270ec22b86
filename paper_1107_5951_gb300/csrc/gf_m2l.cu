// gf_m2l.cu -- M2L over the interaction list, as a batched dense contraction.
//
// Observer boxes of a level are grouped by parity class (their position in
// the parent), because the 189 interaction-list offsets depend only on that
// class.  A block takes up to 32 columns -- (box, batch member) pairs of one
// class -- and, offset by offset, multiplies the K x K operator T_o by the
// K x 32 matrix of gathered source expansions ME[t + o], accumulating the
// K x 32 result in registers.  Sources outside the source block contribute
// zero columns.  Each output is written once, so the result is deterministic.
#include <algorithm>

#include "gf_m2l.cuh"

namespace gf {

__constant__ signed char c_il[8][189][3];

gf_status m2l_upload_offsets(const signed char h_il[8][189][3]) {
    GF_CUDA(cudaMemcpyToSymbol(c_il, h_il, sizeof(signed char) * 8 * 189 * 3));
    return GF_OK;
}

gf_status m2l_prepare_tables(Tables *, cudaStream_t) { return GF_OK; }

namespace {

struct M2LArgs {
    const void *me;
    void *le;
    int K, B, nbox;
    const int32_t *order;
    int64_t cls_off[9];
    const uint64_t *tkey;
    int64_t blo[3], bn[3];
    const void *tab;   // [343][K][K], input component major
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
            const int64_t t = a.order[cbeg + s];
            tbox[tid] = t;
            const uint64_t key = a.tkey[t];
            tc[tid][0] = (int)(dm(key, 0) - a.blo[0]);
            tc[tid][1] = (int)(dm(key, 1) - a.blo[1]);
            tc[tid][2] = (int)(dm(key, 2) - a.blo[2]);
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
                if (sx >= 0 && sy >= 0 && sz >= 0 && sx < a.bn[0] && sy < a.bn[1] && sz < a.bn[2])
                    row = (((sz * a.bn[1] + sy) * a.bn[0] + sx) * B + bb) * K;
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
            if (k < K) le[(tbox[slot] * B + bb) * K + k] = acc[r][c];
        }
    }
}

template <class T, int RPT>
gf_status launch_simt(const M2LArgs &a, int64_t max_tiles, cudaStream_t st) {
    const size_t shm = sizeof(T) * (kCK * XStride<T>::v + kCK * 32 * RPT);
    GF_TRY(ensure_smem(m2l_simt<T, RPT>, shm));
    m2l_simt<T, RPT><<<dim3((unsigned)max_tiles, 8), 256, shm, st>>>(a);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace

template <class T>
gf_status m2l_level(gf_plan_s *plan, int level, int B, cudaStream_t st) {
    FmmPlan *F = plan->fmm;
    const FmmLevel &lv = F->lev[level];
    M2LArgs a;
    a.me = lv.me;
    a.le = lv.le;
    a.K = F->K;
    a.B = B;
    a.nbox = std::max(1, 32 / B);
    a.order = lv.m2l_order;
    int64_t maxc = 0;
    for (int c = 0; c <= 8; ++c) a.cls_off[c] = lv.cls_off[c];
    for (int c = 0; c < 8; ++c) maxc = std::max<int64_t>(maxc, lv.cls_off[c + 1] - lv.cls_off[c]);
    a.tkey = lv.tkey;
    for (int d = 0; d < 3; ++d) {
        a.blo[d] = lv.slo[d];
        a.bn[d] = lv.sn[d];
    }
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

template gf_status m2l_level<float>(gf_plan_s *, int, int, cudaStream_t);
template gf_status m2l_level<double>(gf_plan_s *, int, int, cudaStream_t);

}  // namespace gf
