// gf_prim.cuh -- device-wide primitives used by the tree build:
// exclusive scan and a stable LSD radix sort of (uint64 key, int32 value).
#pragma once

#include "gf_internal.cuh"

namespace gf {

// Scratch needed by exclusive_scan_i64 / radix_sort for n items.
size_t scan_scratch_bytes(int64_t n);
size_t sort_scratch_bytes(int64_t n);

// out[i] = sum_{j<i} in[i] (int64), out[n] = total.  `in` and `out` may
// alias.  scratch: scan_scratch_bytes(n) bytes of device memory.
gf_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch,
                             cudaStream_t st);

// Stable sort of keys (the low `bits` bits matter) carrying vals.  Results
// end in keys/vals; keys_alt/vals_alt are ping-pong buffers of size n.
gf_status radix_sort_u64(uint64_t *keys, int32_t *vals, uint64_t *keys_alt, int32_t *vals_alt,
                         int64_t n, int bits, void *scratch, cudaStream_t st);

// min/max of the three coordinates of n points [n][3] (FP64) into out[6]
// (min x,y,z, max x,y,z); out must hold 12 doubles (6 of scratch).
gf_status bbox3(const double *pts, int64_t n, double *out, cudaStream_t st);

}  // namespace gf
