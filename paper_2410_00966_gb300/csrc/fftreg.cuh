// Register FFTs for the convolution passes (FP32).
//
// fft_reg<N>: an N-point (N <= 32) complex DFT held entirely in one thread's
// registers: radix-2 decimation in frequency, every loop unrolled at compile
// time so twiddle indices are constants and the final bit-reversal is a
// register renaming.
//
// col_fft<P>: a P-point transform of one column shared by N1 = P / NPT
// threads (NPT = 16 or 32 points each, see ColShape), by the four-step factorisation
// P = N1 * NPT: thread j transforms x[j + N1 n2] over n2 (fft_reg<NPT>),
// multiplies by W_P^{j k2}, the block transposes through shared memory, and
// each thread finishes NPT / N1 transforms of length N1 (needs N1 <= NPT,
// i.e. P <= 1024).  Output element i of thread j is frequency
// k2 + NPT * k1 with k2 = j (NPT / N1) + i / N1 and k1 = i % N1.
#pragma once

#include <math.h>

#include "common.cuh"
#include "fft.cuh"

namespace mq {

// exp(-2 pi i k / 32); one copy per translation unit, filled by upload_tw32()
static __constant__ float2 c_tw32[32];

inline cudaError_t upload_tw32() {
    float2 t[32];
    for (int k = 0; k < 32; k++) {
        double a = -2.0 * 3.14159265358979323846 * k / 32.0;
        t[k] = make_float2((float)cos(a), (float)sin(a));
    }
    return cudaMemcpyToSymbol(c_tw32, t, sizeof(t));
}

template <int N>
__host__ __device__ constexpr int bit_reverse(int k) {
    int r = 0;
    for (int b = 1; b < N; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

template <int N>
__host__ __device__ constexpr int ilog2(int n = N) {
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

template <int N, bool INV>
__device__ __forceinline__ void fft_reg(float2* v) {
    if constexpr (N > 1) {
#pragma unroll
    for (int len = N; len >= 2; len >>= 1) {
#pragma unroll
        for (int s0 = 0; s0 < N; s0 += len) {
#pragma unroll
            for (int k = 0; k < len / 2; k++) {
                float2 a = v[s0 + k], b = v[s0 + k + len / 2];
                v[s0 + k] = cadd(a, b);
                float2 d = csub(a, b);
                const int e = k * (32 / len);   // W_len^k = W_32^e
                if (e == 0) {
                    v[s0 + k + len / 2] = d;
                } else if (e == 8) {            // -i (forward) / +i (inverse)
                    v[s0 + k + len / 2] = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                } else {
                    float2 w = c_tw32[e];
                    if (INV) w.y = -w.y;
                    v[s0 + k + len / 2] = cmul(d, w);
                }
            }
        }
    }
    float2 t[N];
#pragma unroll
    for (int k = 0; k < N; k++) t[k] = v[bit_reverse<N>(k)];
#pragma unroll
    for (int k = 0; k < N; k++) v[k] = t[k];
    }
}

// Points per thread: 16 up to P = 256 (keeps the register footprint small),
// 32 above (four-step needs N1 = P / NPT <= NPT).
template <int P>
struct ColShape {
    static constexpr int NPT = P <= 16 ? P : (P <= 256 ? 16 : 32);   // points per thread
    static constexpr int N1 = P / NPT;            // threads per column
    static constexpr int Q = NPT / N1;            // length-N1 transforms per thread in step 3
};

inline int col_threads_per_column(int P) { return P <= 16 ? 1 : (P <= 256 ? P / 16 : P / 32); }

// Row of output element i of thread j (see file comment).
template <int P>
__device__ __forceinline__ int col_out_row(int j, int i) {
    constexpr int NPT = ColShape<P>::NPT, N1 = ColShape<P>::N1, Q = ColShape<P>::Q;
    if (N1 == 1) return i;
    return (j * Q + i / N1) + NPT * (i % N1);
}

// v[n2] holds x[j + N1 n2] on entry and the outputs (rows col_out_row) on
// exit.  `buf` (ld floats2 per row, at least P rows) is used for the transpose
// when N1 > 1; every thread of the block must call this (it synchronises).
// Twiddles come from `tw`, a table of exp(-2 pi i k / twn) for k < twn (a
// multiple of P), in global memory (TW_SHARED = false, read through the
// read-only cache) or in shared memory.
template <int P, bool INV, bool TW_SHARED = false>
__device__ __forceinline__ void col_fft(float2* v, float2* buf, int ld, int col, int j, const float2* __restrict__ tw,
                                        int twn) {
    constexpr int NPT = ColShape<P>::NPT, N1 = ColShape<P>::N1, Q = ColShape<P>::Q;
    fft_reg<NPT, INV>(v);
    if (N1 == 1) return;
    // twiddle W_P^{j k2}
    const int step = twn / P;
#pragma unroll
    for (int k2 = 1; k2 < NPT; k2++) {
        float2 w;
        if (TW_SHARED) {
            w = tw[j * k2 * step];
            if (INV) w.y = -w.y;
        } else {
            w = twiddle(tw, j * k2 * step, INV);
        }
        v[k2] = cmul(v[k2], w);
    }
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < NPT; k2++) buf[(k2 * N1 + j) * ld + col] = v[k2];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int k2 = j * Q + q;
#pragma unroll
        for (int n1 = 0; n1 < N1; n1++) v[q * N1 + n1] = buf[(k2 * N1 + n1) * ld + col];
    }
#pragma unroll
    for (int q = 0; q < Q; q++) fft_reg<N1, INV>(v + q * N1);
    __syncthreads();   // the buffer may be reused by the caller right after
}

// ---------------------------------------------------------------------------
// Three-factor transform for the long lines (P = 256 N3, N3 = 2, 4 or 8): 16
// points per thread, so that a line of P points takes N1 = P / 16 threads
// with half the registers of the 32-point four-step above.
//   P = 16 x N1 and N1 = 16 x N3.  Input: thread j (< N1) holds
//   v[n2] = x[j + N1 n2].
//   1. 16-point DFT over n2, twiddle W_P^{j k2}, transpose through `buf`.
//   2. Thread j' = N3 a + q takes A[q + N3 n, a] (the twiddled stage-1 value
//      of thread q + N3 n at k2 = a) for n < 16: 16-point DFT over n, twiddle
//      W_N1^{q k'}.
//   3. The N3-point DFT over q runs across the N3 lanes of the group by
//      butterfly exchanges (decimation in frequency, lanes LS apart); lane q
//      ends with output index bitrev(q).
//   Element i of thread j' = (a, q) is then frequency a + 16 (i + 16 br(q)).
// The transpose buffer rows are swizzled: row r at r + PADS (r / N1), so that
// the stage-2 reads of lanes with different a spread over the banks (PADS = 4
// for three lines per pitch, 0 when a warp reads whole 8-column rows); `buf`
// needs P + 16 PADS rows.  Lanes q of a group must be LS apart inside one warp.
template <int P>
struct ColShape3 {
    static constexpr int NPT = 16;
    static constexpr int N1 = P / 16;     // threads per line
    static constexpr int N3 = P / 256;    // last factor (across lanes)
    static_assert(N3 == 2 || N3 == 4 || N3 == 8, "three-factor lengths are 512, 1024 and 2048");
};

template <int N3>
__host__ __device__ constexpr int lane_bitrev(int q) {
    return N3 == 2 ? q : (N3 == 4 ? ((q & 1) << 1) | (q >> 1) : ((q & 1) << 2) | (q & 2) | (q >> 2));
}

// Frequency held by element i of thread j (see above).
template <int P>
__device__ __forceinline__ int col3_out_row(int j, int i) {
    constexpr int N3 = ColShape3<P>::N3;
    return j / N3 + 16 * (i + 16 * lane_bitrev<N3>(j % N3));
}

template <int N1, int PADS>
__device__ __forceinline__ int col3_swz(int r) { return r + PADS * (r / N1); }

// v[k] *= w^k for k = 1..15, w = table[b]: six table values (w^1..3 and
// w^4, w^8, w^12) and one product for each of the other nine powers, so that
// every factor carries at most one rounding beyond the table's.
template <bool INV, bool TW_SHARED>
__device__ __forceinline__ void twiddle15(float2* v, const float2* __restrict__ tw, int b) {
    auto at = [&](int k) {
        float2 w = TW_SHARED ? tw[k] : __ldg(tw + k);
        if (INV) w.y = -w.y;
        return w;
    };
    const float2 lo[4] = {make_float2(1.f, 0.f), at(b), at(2 * b), at(3 * b)};
    const float2 hi[4] = {make_float2(1.f, 0.f), at(4 * b), at(8 * b), at(12 * b)};
#pragma unroll
    for (int k = 1; k < 16; k++) {
        const int a = k & 3, c = k >> 2;
        const float2 w = a == 0 ? hi[c] : (c == 0 ? lo[a] : cmul(lo[a], hi[c]));
        v[k] = cmul(v[k], w);
    }
}

// Variant of step 3 (T2): a second transpose instead of the lane exchange.
// Thread (a, q) then takes k' = q (16 / N3) + qq, qq < 16 / N3, gathers the N3
// values of each k' and runs N3-point register DFTs; element i = qq N3 + k''
// is frequency a + 16 (k' + 16 k'').  The second transpose's rows are
// swizzled so that the lane groups of a warp hit different banks both when
// they write (rows a N1 + k' N3 + q) and when they read (rows a N1 + 16 q +
// ...): with 8-column rows (PADS = 0) the low log2 N3 bits are XORed with the
// bits above the 16-row group; with three-line rows (PADS > 0) the rows are
// shifted by PADS per N1 group plus those bits.
template <int P>
__device__ __forceinline__ int col3t_out_row(int j, int i) {
    constexpr int N3 = ColShape3<P>::N3, QK = 16 / N3;
    const int a = j / N3, q = j % N3;
    return a + 16 * (q * QK + i / N3 + 16 * (i % N3));
}

template <int N1, int N3, int PADS>
__device__ __forceinline__ int col3t_swz(int r) {
    return PADS == 0 ? (r ^ ((r >> 4) & (N3 - 1))) : r + PADS * (r / N1) + ((r >> 4) & (N3 - 1));
}

template <int P, bool INV, bool TW_SHARED, int PADS, int LS, bool T2 = false>
__device__ __forceinline__ void col_fft3(float2* v, float2* buf, int ld, int col, int j, const float2* __restrict__ tw,
                                         int twn) {
    constexpr int N1 = ColShape3<P>::N1, N3 = ColShape3<P>::N3;
    auto tw_at = [&](int k) {
        float2 w = TW_SHARED ? tw[k] : __ldg(tw + k);
        if (INV) w.y = -w.y;
        return w;
    };
    // 1. 16 points at stride N1, twiddle W_P^{j k2}, transpose
    fft_reg<16, INV>(v);
    const int step = twn / P;
    twiddle15<INV, TW_SHARED>(v, tw, j * step);
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) buf[col3_swz<N1, PADS>(k2 * N1 + j) * ld + col] = v[k2];
    __syncthreads();
    // 2. thread (a, q): 16 points of column a at stride N3, twiddle W_N1^{q k'}
    const int a = j / N3, q = j % N3;
#pragma unroll
    for (int n = 0; n < 16; n++) v[n] = buf[col3_swz<N1, PADS>(a * N1 + q + N3 * n) * ld + col];
    fft_reg<16, INV>(v);
    const int step2 = twn / N1;
    twiddle15<INV, TW_SHARED>(v, tw, q * step2);
    if constexpr (T2) {
        // 3'. transpose and N3-point register DFTs
        constexpr int QK = 16 / N3;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) buf[col3t_swz<N1, N3, PADS>(a * N1 + k * N3 + q) * ld + col] = v[k];
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < QK; qq++) {
            float2 u[N3];
            const int kk = q * QK + qq;
#pragma unroll
            for (int r = 0; r < N3; r++) u[r] = buf[col3t_swz<N1, N3, PADS>(a * N1 + kk * N3 + r) * ld + col];
            fft_reg<N3, INV>(u);
#pragma unroll
            for (int r = 0; r < N3; r++) v[qq * N3 + r] = u[r];
        }
        __syncthreads();   // the buffer may be reused by the caller right after
        return;
    }
    // 3. N3 points across the lanes of the group: at each level the lower lane
    // of a pair keeps x_lo + x_hi, the upper lane (x_lo - x_hi) W_len^{p - half}
#pragma unroll
    for (int half = N3 / 2; half >= 1; half >>= 1) {
        const int p = q & (2 * half - 1);
        const bool upper = p >= half;
        const float2 w = upper ? tw_at((p - half) * (twn / (2 * half))) : make_float2(1.f, 0.f);
#pragma unroll
        for (int e = 0; e < 16; e++) {
            float2 o;
            o.x = __shfl_xor_sync(0xffffffffu, v[e].x, half * LS);
            o.y = __shfl_xor_sync(0xffffffffu, v[e].y, half * LS);
            const float2 lo = upper ? o : v[e], hi = upper ? v[e] : o;
            v[e] = upper ? cmul(csub(lo, hi), w) : cadd(lo, hi);
        }
    }
    __syncthreads();   // the buffer may be reused by the caller right after
}

}  // namespace mq
