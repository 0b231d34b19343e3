// Small device helpers shared by the stage kernels.
#pragma once

#include "common.cuh"

namespace mq {

// Whether this instance does nothing in this launch.
__device__ __forceinline__ bool stage_skips(const InstState& s, const StageArgs& A) {
    if (A.field_only) return false;
    if (s.done) return true;
    if (A.kind == KIND_DP45 && A.stage == 0 && s.have_k1) return true;
    return false;
}

// DP45: stage 1 lives in k1slot (first-same-as-last swap between buffers 0 and 6)
__device__ __forceinline__ int k_slot(const InstState& s, int j) { return j == 0 ? s.k1slot : j; }

}  // namespace mq
