// gf_m2l.cuh -- the multipole-to-local stage (Sec. 2.3: an ME is turned
// into an LE for every box of the interaction list).
#pragma once

#include "gf_fmm.cuh"

namespace gf {

gf_status m2l_upload_offsets(const signed char h_il[8][189][3]);
gf_status m2l_prepare_tables(Tables *T, cudaStream_t st);

// LE_l[t] = sum over the interaction list of box t of T_o * ME_l[t + o],
// for every observer box t of every level (overwrites each LE_l).  Mixed
// precision runs on the tensor cores (tcgen05, 3xTF32) unless the plan asks
// for the SIMT kernel; FP64 runs on the SIMT kernel.
template <class T>
gf_status m2l_run(gf_plan_s *plan, int B, cudaStream_t st);
template <class T>
gf_status m2l_level(gf_plan_s *plan, int level, int B, cudaStream_t st);

// Batched M2M (kind 0: into `level` from level + 1) or L2L (kind 1: into
// `level` from level - 1) on the SIMT cores; Ts = storage, Tc = arithmetic.
template <class Ts, class Tc>
gf_status translate_run(gf_plan_s *plan, int level, int kind, int B, cudaStream_t st);

// Plan-time set-up of the tensor-core path (level descriptors on the device).
gf_status m2l_tc_prepare(gf_plan_s *plan);

}  // namespace gf
