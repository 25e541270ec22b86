// gf_prim.cu -- exclusive scan, stable LSD radix sort and a bounding-box
// reduction, written for the octree build.
#include <float.h>
#include <string.h>

#include <algorithm>

#include "gf_prim.cuh"

namespace gf {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;   // 1024

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 keys per block
constexpr int kRadix = 256;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one 1024-element tile per block; block totals to sums.
__global__ void __launch_bounds__(kScanThreads)
scan_tiles(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
           int64_t *__restrict__ sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        loc += v[i];
    }
    const int64_t incl = warp_incl_scan(loc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        const int64_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int64_t run = warp_tot[warp] + incl - loc;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void add_tile_offsets(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanTile];
}

__global__ void write_total(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs,
                            const int64_t *__restrict__ sums, int64_t nb) {
    out[n] = offs[nb - 1] + sums[nb - 1];
}

// Whole scan in one block (n <= kSmallScan): thread t takes the run of up
// to 32 consecutive items starting at t * ceil(n / 1024); a first sweep sums
// the run (independent, unrolled loads), one block-wide scan of the run
// totals gives every run its offset, and a second sweep writes the run.
// Also the total into out[n] when asked.  (`in` may alias `out`: the
// second sweep reads each item before writing it.)
constexpr int kSmallThreads = 1024;
constexpr int kSmallItems = 32;
constexpr int64_t kSmallScan = (int64_t)kSmallItems * kSmallThreads;

__global__ void __launch_bounds__(kSmallThreads)
scan_small(const int64_t *in, int64_t *out, int64_t n, int write_tot) {
    __shared__ int64_t warp_tot[kSmallThreads / 32 + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (int)((n + kSmallThreads - 1) / kSmallThreads);
    const int64_t b0 = (int64_t)threadIdx.x * per;
    int64_t loc = 0;
#pragma unroll
    for (int i = 0; i < kSmallItems; ++i)
        if (i < per && b0 + i < n) loc += in[b0 + i];
    const int64_t incl = warp_incl_scan(loc);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = warp_tot[lane];
        const int64_t wi = warp_incl_scan(w);
        warp_tot[lane] = wi - w;
        if (lane == 31) warp_tot[32] = wi;
    }
    __syncthreads();
    int64_t run = warp_tot[warp] + incl - loc;
#pragma unroll 8
    for (int i = 0; i < kSmallItems; ++i)
        if (i < per && b0 + i < n) {
            const int64_t v = in[b0 + i];
            out[b0 + i] = run;
            run += v;
        }
    if (threadIdx.x == 0 && write_tot) out[n] = warp_tot[32];
}

gf_status scan_rec(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch, cudaStream_t st,
                   bool write_tot) {
    if (n <= 0) {
        if (write_tot) GF_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return GF_OK;
    }
    if (n <= kSmallScan) {
        scan_small<<<1, kSmallThreads, 0, st>>>(in, out, n, write_tot ? 1 : 0);
        GF_KERNEL_DONE();
        return GF_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = scratch;            // [nb]
    int64_t *offs = scratch + nb;       // [nb + 1]
    scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
    GF_KERNEL_DONE();
    if (nb > 1) {
        GF_TRY(scan_rec(sums, offs, nb, scratch + 2 * nb + 1, st, false));
        add_tile_offsets<<<ceil_div(n, 256), 256, 0, st>>>(out, n, offs);
        GF_KERNEL_DONE();
    } else {
        GF_CUDA(cudaMemsetAsync(offs, 0, sizeof(int64_t), st));
    }
    if (write_tot) {
        write_total<<<1, 1, 0, st>>>(out, n, offs, sums, nb);
        GF_KERNEL_DONE();
    }
    return GF_OK;
}

// -------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kSortThreads)
radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int64_t nblocks,
           int64_t *__restrict__ hist) {
    __shared__ int cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: keys of the tile are ranked in index order (round-major,
// thread-minor), so equal digits keep their relative order.
__global__ void __launch_bounds__(kSortThreads)
radix_scatter(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t n,
              int shift, int64_t nblocks, const int64_t *__restrict__ offs,
              uint64_t *__restrict__ keys_out, int32_t *__restrict__ vals_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int64_t run[kRadix];
    __shared__ int wcnt[kWarps][kRadix];
    __shared__ int total[kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        uint64_t k = valid ? keys[i] : 0;
        int32_t v = valid ? vals[i] : 0;
        const int d = valid ? (int)((k >> shift) & 0xff) : kRadix;  // invalid -> sentinel
        for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
        const int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // exclusive prefix over warps for digit threadIdx.x
            int acc = 0;
            for (int w = 0; w < kWarps; ++w) {
                const int c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = acc;
                acc += c;
            }
            total[threadIdx.x] = acc;
        }
        __syncthreads();
        if (valid) {
            const int64_t pos = run[d] + wcnt[warp][d] + rank;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
        run[threadIdx.x] += total[threadIdx.x];
        __syncthreads();
    }
}

// -------------------------------------------------------------- bbox
// Bounding box on the integer units: a double's bits map to an unsigned key
// with the same order (negative values: all bits flipped; others: the sign
// bit set), so min/max are integer operations (FP64 is slow on this GPU)
// and the blocks combine with 64-bit atomics.
__device__ __forceinline__ unsigned long long order_key(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void bbox_keys(const double *__restrict__ p, int64_t n, unsigned long long *__restrict__ out) {
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long k = order_key(p[3 * i + a]);
            mn[a] = k < mn[a] ? k : mn[a];
            mx[a] = k > mx[a] ? k : mx[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, mn[a], o), y = __shfl_xor_sync(0xffffffffu, mx[a], o);
            mn[a] = x < mn[a] ? x : mn[a];
            mx[a] = y > mx[a] ? y : mx[a];
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(out + a, mn[a]);
            atomicMax(out + 3 + a, mx[a]);
        }
}

// keys back to doubles
__global__ void bbox_decode(const unsigned long long *__restrict__ k, double *__restrict__ out) {
    if (threadIdx.x < 6) {
        const unsigned long long u = k[threadIdx.x];
        out[threadIdx.x] = __longlong_as_double((long long)((u >> 63) ? (u & 0x7fffffffffffffffull) : ~u));
    }
}

__global__ void bbox_init(unsigned long long *__restrict__ k) {
    if (threadIdx.x < 6) k[threadIdx.x] = threadIdx.x < 3 ? ~0ull : 0ull;
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
    size_t tot = 0;
    int64_t m = n;
    do {
        const int64_t nb = (m + kScanTile - 1) / kScanTile;
        tot += (size_t)(2 * nb + 1);
        m = nb;
    } while (m > 1);
    return (tot + 16) * sizeof(int64_t);
}

size_t sort_scratch_bytes(int64_t n) {
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    const int64_t h = nb * kRadix;
    return (size_t)(h + 1) * sizeof(int64_t) + scan_scratch_bytes(h) + 256;
}

gf_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st) {
    return scan_rec(in, out, n, reinterpret_cast<int64_t *>(scratch), st, true);
}

gf_status radix_sort_u64(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt, int64_t n,
                         int bits, void *scratch, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return GF_OK;
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    const int64_t h = nb * kRadix;
    int64_t *hist = reinterpret_cast<int64_t *>(scratch);
    int64_t *scan_scr = hist + h + 1;
    uint64_t *ka = keys, *kb = keys_alt;
    int32_t *va = vals, *vb = vals_alt;
    const int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        radix_hist<<<(unsigned)nb, kSortThreads, 0, st>>>(ka, n, shift, nb, hist);
        GF_KERNEL_DONE();
        GF_TRY(scan_rec(hist, hist, h, scan_scr, st, false));
        radix_scatter<<<(unsigned)nb, kSortThreads, 0, st>>>(ka, va, n, shift, nb, hist, kb, vb);
        GF_KERNEL_DONE();
        uint64_t *tk = ka;
        ka = kb;
        kb = tk;
        int32_t *tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != keys) {
        GF_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        GF_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return GF_OK;
}

// Small host arrays travel to the device as kernel arguments (pieces of
// kUploadWords words), not as host-to-device copies: a plan build then
// never queues behind a large copy the caller has in flight on another
// stream, and the host memory may be reused as soon as the call returns.
namespace {
constexpr int kUploadWords = 960;
struct UploadPiece {
    uint32_t w[kUploadWords];
};
__global__ void upload_piece(UploadPiece pc, int nw, uint32_t *__restrict__ dst) {
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = pc.w[i];
}
}  // namespace

gf_status upload_small(void *dst, const void *src, size_t nbytes, cudaStream_t st) {
    if (nbytes % 4 != 0 || ((uintptr_t)dst & 3) != 0) {
        set_error("upload_small: %zu bytes to %p (whole aligned words only)", nbytes, dst);
        return GF_ERR_INVALID_ARG;
    }
    const size_t nw = nbytes / 4;
    const unsigned char *s8 = static_cast<const unsigned char *>(src);
    uint32_t *d = static_cast<uint32_t *>(dst);
    for (size_t w0 = 0; w0 < nw; w0 += kUploadWords) {
        UploadPiece pc;
        const int n = (int)std::min<size_t>(kUploadWords, nw - w0);
        memcpy(pc.w, s8 + 4 * w0, 4 * (size_t)n);
        upload_piece<<<1, 256, 0, st>>>(pc, n, d + w0);
        GF_KERNEL_DONE();
    }
    return GF_OK;
}

gf_status bbox3(const double *pts, int64_t n, double *out, cudaStream_t st) {
    // out must have room for 12 doubles: the integer keys follow the result
    if (n <= 0) return GF_OK;
    unsigned long long *k = reinterpret_cast<unsigned long long *>(out + 6);
    bbox_init<<<1, 32, 0, st>>>(k);
    GF_KERNEL_DONE();
    const int nb = (int)std::min<int64_t>(4 * 152, (n + 255) / 256);
    bbox_keys<<<nb, 256, 0, st>>>(pts, n, k);
    GF_KERNEL_DONE();
    bbox_decode<<<1, 32, 0, st>>>(k, out);
    GF_KERNEL_DONE();
    return GF_OK;
}

}  // namespace gf
