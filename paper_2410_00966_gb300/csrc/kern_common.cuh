// Small device helpers shared by the stage kernels.
#pragma once

#include "common.cuh"

namespace mq {

// Host side: launch a stage-chain kernel; cluster > 1 groups consecutive
// blocks along x into clusters of that size.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain_cl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   int cluster, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cluster > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                Args... args) {
    return launch_chain_cl(kernel, grid, block, smem, s, 1, args...);
}

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

// ---- bulk tensor copies (TMA) completing on an mbarrier --------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Order this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same memory, and make an mbarrier
// initialisation visible to them.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Arrive on `bar` expecting `bytes` from bulk copies, then copy the box at
// coordinates (c0, c1, c2, c3) (innermost first) of the 4-D tensor map into
// shared memory at `dst` (128-byte aligned); the copy completes on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const TensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Wait until the phase of `bar` with the given parity has completed, for at
// most `limit_ns` nanoseconds; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit_ns) {
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (int it = 0;; it++) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = global_ns();
        else if (global_ns() - t0 > limit_ns) return false;
    }
}

// *p += v for a float2 in global memory: a device-scope atomic add whose
// result is not used, so the add is done where the line lives (L2) and no
// value comes back to the thread.
__device__ __forceinline__ void red_add_f2(float2* p, float2 v) {
    atomicAdd(p, v);
}

// ---- thread-block clusters ----------------------------------------------------
// Barrier over every thread of every block of the cluster (hardware barrier;
// release / acquire order the shared-memory writes before it against the
// reads after it, across the blocks).  All threads of a warp must reach it
// together.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// The shared-window address `a` of this block mapped into block `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_map(unsigned a, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster_f2(unsigned a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

// DP45: stage 1 lives in k1slot (first-same-as-last swap between buffers 0 and 6)
__device__ __forceinline__ int k_slot(const InstState& s, int j) { return j == 0 ? s.k1slot : j; }

}  // namespace mq
