// Shapes shared by the two x passes (stage.cu: x forward, xinv.cu: x inverse).
#pragma once

#include "common.cuh"
#include "fftreg.cuh"

namespace mq {

// Shared-memory pitch of the x passes: 3 R lines rounded up to an odd count,
// so that consecutive cells (stride one pitch) fall in different banks.
__host__ __device__ constexpr int xpass_ld(int R) { return (3 * R) | 1; }

// Lines of L = 1024 points use the three-factor transform (16 points per
// thread, 64 threads per line, ColShape3); shorter lines the register
// four-step (ColShape).
__host__ __device__ constexpr bool xpass_f3(int L) { return L == 1024; }
// Threads per line of the x transform.
__host__ __device__ constexpr int xpass_line_threads(int L) {
    return xpass_f3(L) ? L / 16 : (L <= 16 ? 1 : (L <= 256 ? L / 16 : L / 32));
}
// Shared-memory rows of the x transform: the line, plus the swizzle padding
// of the three-factor transpose (PADS = 4 per 64-row group).
constexpr int XPASS_F3_PADS = 4;
__host__ __device__ constexpr int xpass_fft_rows(int L) { return xpass_f3(L) ? L + 16 * XPASS_F3_PADS : L; }

// Threads of an x-pass block: 3 R lines x N1 threads per line with R = 64 / N1
// rows (fewer when the grid has fewer rows), so never more than 192.
constexpr int XPASS_THREADS = 192;
// Resident blocks asked of the compiler: 5 (64 registers) while a thread
// holds 16 points of the x transform, 3 when it holds 32 (L = 512).
constexpr int xpass_min_blocks(int L) { return (L >= 512 && !xpass_f3(L)) ? 3 : 5; }

static inline int xthreads(const Plan& P) { return 3 * P.R * xpass_line_threads(P.L); }

// Rows per block: 64 lines of the transform per block, 3 R lines x N1 threads.
__host__ __device__ constexpr int xpass_rows(int L) {
    return 64 / xpass_line_threads(L) > 0 ? 64 / xpass_line_threads(L) : 1;
}

// Lengths with a fixed-shape instantiation of the x passes, and whether a plan
// has that shape: rows of L cells, whole blocks of xpass_rows(L) rows, 8-column
// tiles (so L / 8 + 1 tiles over the L + 1 half-spectrum values).
#define MMCQ_XFIXED(F) F(256) F(512) F(1024)
static inline bool xpass_fixed(const Plan& P) {
    return (P.L == 256 || P.L == 512 || P.L == 1024) && P.nx == P.L && P.TX == 8 && P.R == xpass_rows(P.L) &&
           P.nrows % P.R == 0 && P.NT == P.L / 8 + 1 && P.px == 2 * P.L;
}

// Shared memory of the x inverse: the half-spectrum lines (L + 1 rows), or
// the transform's rows if more.
static inline size_t xinv_smem(const Plan& P) {
    const int rows = xpass_fft_rows(P.L) > P.L + 1 ? xpass_fft_rows(P.L) : P.L + 1;
    return (size_t)rows * xpass_ld(P.R) * sizeof(float2);
}

#define MMCQ_XCASES(F) F(1) F(2) F(4) F(8) F(16) F(32) F(64) F(128) F(256) F(512) F(1024)

}  // namespace mq
