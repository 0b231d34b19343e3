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

}  // namespace mq
