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

// Asynchronous global -> shared copies (cp.async, sm_80+): the loads are in
// flight without holding registers; cp_async_wait_all() waits for this
// thread's copies (a barrier must follow before other threads read them).
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
// The same with the destination given as a shared-window address.
__device__ __forceinline__ void cp_async8s(unsigned dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Hint: bring [src, src + bytes) into L2 (bulk prefetch, sm_90+).  src must be
// 16-byte aligned, bytes a multiple of 16, and the range inside an allocation.
__device__ __forceinline__ void prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}

// DP45: stage 1 lives in k1slot (first-same-as-last swap between buffers 0 and 6)
__device__ __forceinline__ int k_slot(const InstState& s, int j) { return j == 0 ? s.k1slot : j; }

}  // namespace mq
