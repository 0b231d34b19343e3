// Shapes shared by the two x passes (stage.cu: x forward, xinv.cu: x inverse).
#pragma once

#include "common.cuh"
#include "fftreg.cuh"

namespace mq {

// Shared-memory pitch of the x passes: 3 R lines rounded up to an odd count,
// so that consecutive cells (stride one pitch) fall in different banks.
__host__ __device__ constexpr int xpass_ld(int R) { return (3 * R) | 1; }

// Threads of an x-pass block: 3 R lines x N1 threads per line with R = 64 / N1
// rows (fewer when the grid has fewer rows), so never more than 192.
constexpr int XPASS_THREADS = 192;
// Resident blocks asked of the compiler: 5 (64 registers) while a thread
// holds 16 points of the x transform, 3 when it holds 32 (L >= 512).
constexpr int xpass_min_blocks(int L) { return L >= 512 ? 3 : 5; }

static inline int xthreads(const Plan& P) { return 3 * P.R * col_threads_per_column(P.L); }

// Rows per block: 64 lines of the transform per block, 3 R lines x N1 threads.
__host__ __device__ constexpr int xpass_rows(int L) {
    return L <= 16 ? 64 : (L <= 256 ? 64 / (L / 16) : (64 / (L / 32) > 0 ? 64 / (L / 32) : 1));
}

// Lengths with a fixed-shape instantiation of the x passes, and whether a plan
// has that shape: rows of L cells, whole blocks of xpass_rows(L) rows, 8-column
// tiles (so L / 8 + 1 tiles over the L + 1 half-spectrum values).
#define MMCQ_XFIXED(F) F(256) F(512) F(1024)
static inline bool xpass_fixed(const Plan& P) {
    return (P.L == 256 || P.L == 512 || P.L == 1024) && P.nx == P.L && P.TX == 8 && P.R == xpass_rows(P.L) &&
           P.nrows % P.R == 0 && P.NT == P.L / 8 + 1 && P.px == 2 * P.L;
}

// Shared memory of the x inverse: the half-spectrum lines.
static inline size_t xinv_smem(const Plan& P) { return (size_t)(P.L + 1) * xpass_ld(P.R) * sizeof(float2); }

#define MMCQ_XCASES(F) F(1) F(2) F(4) F(8) F(16) F(32) F(64) F(128) F(256) F(512) F(1024)

}  // namespace mq
