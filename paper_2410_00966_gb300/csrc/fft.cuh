// Block-cooperative complex FFT in shared memory (FP32), used by the demag
// convolution passes.  Stockham auto-sort formulation (Govindaraju et al.
// 2008): every stage reads element j + r L/R of a line, twiddles it by
// W_{Ns R}^{(j mod Ns) r}, runs a radix-R butterfly in registers and writes it
// to position (j - j mod Ns) R + j mod Ns + r Ns, so the output comes out in
// natural order without a bit-reversal pass.  Radix 4 throughout, with one
// radix-2 stage when log2(L) is odd.  All loads of a stage complete (barrier)
// before any store, so one shared buffer suffices.
#pragma once

#include "common.cuh"

namespace mq {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Complex add and subtract as paired FP32 instructions (sm_100 and later issue
// the two component adds of a float2 as one instruction, each rounded like the
// scalar add); the butterflies of every register FFT are made of these.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// exp(-+ 2 pi i k / twn) from the table; inverse transforms use the conjugate.
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int k, bool inv) {
    float2 w = __ldg(tw + k);
    return inv ? make_float2(w.x, -w.y) : w;
}

__device__ __forceinline__ void radix4(float2* v, bool inv) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
    // forward: X1 = t1 - i t3, X3 = t1 + i t3 ; inverse swaps the sign of i
    float2 mt3 = inv ? make_float2(-t3.y, t3.x) : make_float2(t3.y, -t3.x);  // (-+i) t3
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, mt3);
    v[3] = csub(t1, mt3);
}

// FFT of `nlines` lines of length L (power of two) held in shared memory:
// element k of line l sits at s[l * ls + k * es].  LINE_FAST maps consecutive
// threads to consecutive lines (good when lines are adjacent in memory),
// otherwise to consecutive elements of one line.  Unnormalised; the caller
// must have synchronised before the call, and the call ends synchronised.
// Requires nlines * L / 4 <= SLOTS * blockDim.x.
template <bool LINE_FAST, int SLOTS>
__device__ void block_fft(float2* s, int L, int nlines, int es, int ls, bool inv,
                          const float2* __restrict__ tw, int twn) {
    for (int Ns = 1; Ns < L;) {
        const int R = ((L / Ns) & 3) == 0 ? 4 : 2;
        const int tpl = L / R;                 // butterflies per line
        const int ntask = tpl * nlines;
        const int per_slot = 4 / R;            // butterflies held in one 4-value slot
        const int twstep_base = twn / (Ns * R);
        float2 v[SLOTS][4];
        int off[SLOTS][2];                 // line base of each butterfly in the slot
        int jj[SLOTS][2];
#pragma unroll
        for (int q = 0; q < SLOTS; q++) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int t = (threadIdx.x + q * blockDim.x) * per_slot + h;
                off[q][h] = -1;
                if (h < per_slot && t < ntask) {
                    int line, j;
                    if (LINE_FAST) { line = t % nlines; j = t / nlines; }
                    else { line = t / tpl; j = t - line * tpl; }
                    off[q][h] = line * ls;
                    jj[q][h] = j;
                    const float2* p = s + line * ls;
                    int jm = j & (Ns - 1);
                    int ts = jm * twstep_base;
                    if (R == 4) {
                        v[q][0] = p[j * es];
#pragma unroll
                        for (int r = 1; r < 4; r++) v[q][r] = cmul(p[(j + r * tpl) * es], twiddle(tw, r * ts, inv));
                        radix4(v[q], inv);
                    } else {
                        float2 a = p[j * es];
                        float2 b = cmul(p[(j + tpl) * es], twiddle(tw, ts, inv));
                        v[q][2 * h] = cadd(a, b);
                        v[q][2 * h + 1] = csub(a, b);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SLOTS; q++) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                if (off[q][h] >= 0) {
                    float2* p = s + off[q][h];
                    int j = jj[q][h];
                    int jm = j & (Ns - 1);
                    int d = (j - jm) * R + jm;
                    if (R == 4) {
#pragma unroll
                        for (int r = 0; r < 4; r++) p[(d + r * Ns) * es] = v[q][r];
                    } else {
                        p[d * es] = v[q][2 * h];
                        p[(d + Ns) * es] = v[q][2 * h + 1];
                    }
                }
            }
        }
        __syncthreads();
        Ns *= R;
    }
}

}  // namespace mq
