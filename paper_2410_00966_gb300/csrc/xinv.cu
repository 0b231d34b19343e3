// x inverse of the demag convolution fused with everything a stage does per
// cell (Mumax3-cQED, arXiv 2410.00966): complex-to-real inverse FFT along x
// giving B_demag, then exchange + anisotropy + Zeeman (with the Appendix C
// excitation) + cavity sum_k B_rms,k Gamma_k (Sec. 2.1 field terms, Eq. bcav),
// the LLG torque (Eq. llg), the RK bookkeeping, and FP64 block partials of the
// coupling sums X_k = V_c sum_i Ms_i m_i . B_rms,k,i (Eq. gammafinal).  The last
// block of each instance to finish reduces the partials in a fixed order and
// advances the cavity amplitudes and the step-size controller in FP64.
#include <math.h>

#include "common.cuh"
#include "fftreg.cuh"
#include "kern_common.cuh"
#include "stagecore.cuh"
#include "xpass.cuh"

namespace mq {

// ---------------------------------------------------------------------------
// x inverse + local fields + torque + RK bookkeeping + cavity reduction.
// Shared memory: xs[k][line] (k <= L, line = 3 r + comp), then m rows.
// ---------------------------------------------------------------------------
// REC: this launch records the spatial average of the state being accepted
// (the last stage of a step with recording on); NM: cavity modes compiled in
// (1, or MAX_MODES when more than one mode is enabled).  Separate
// instantiations so that the common launches carry no extra accumulators.
template <int L, bool REC, int NM>
__global__ void __launch_bounds__(XPASS_THREADS, xpass_min_blocks(L)) k_xinv(Plan P, Material mat, Buffers Bf, StageArgs A) {
    constexpr int NPT = ColShape<L>::NPT, N1 = ColShape<L>::N1;
    extern __shared__ float2 sm[];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma[NM];
    __shared__ float s_drive;
    __shared__ int s_last;
    const int b = A.inst0 + blockIdx.y;
    const InstState& st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const InstParams& ip = Bf.ip[b];
    const int TX = P.TX, nx = P.nx, lt = P.lt;
    const int row0 = blockIdx.x * P.R;
    const int nr = min(P.R, P.nrows - row0);
    const int ld = xpass_ld(P.R);
    const long long cb = (long long)b * P.N;
    const long long base = cb + (long long)row0 * nx;
    const int s = A.stage;
    const int K = A.kind;
    float2* xs = sm;                                   // [L + 1][ld]
    const int xs_n = (L + 1) * ld + (((L + 1) * ld) & 1);
    // m rows staged in shared memory while they are short; long rows
    // (L >= 512) read m through the read-only path instead, which keeps the
    // block's shared memory (and so its residency) at the half-spectrum lines
    constexpr bool STAGE_M = xinv_stages_m(L);
    float4* mrow = reinterpret_cast<float4*>(sm + xs_n);  // [row][nx] (STAGE_M)

    // which buffer holds the stage input m_s
    const float4* msrc;
    if (A.field_only || s == 0) msrc = Bf.m[st.mcur];
    else if (K == KIND_DP45 && s == 6) msrc = Bf.m[st.mcur ^ 1];
    else msrc = Bf.ms;

    // the z neighbours of this block's rows are read in the cell loop: ask L2
    // for them now (only when the whole range lies inside the instance)
    if (threadIdx.x == 0 && P.nz > 1 && (A.terms & 2)) {
        const long long pl_ = (long long)nx * P.ny;
        const unsigned bytes = (unsigned)(nr * nx * sizeof(float4));
        if (row0 >= P.ny) prefetch_l2(msrc + base - pl_, bytes);
        if (row0 + nr - 1 + P.ny < P.nrows) prefetch_l2(msrc + base + pl_, bytes);
    }

    // half-spectrum rows X[0..L] of the three components of every row
    const long long tstride = (long long)P.ny * 3 * TX;
    for (int r = 0; r < nr; r++) {
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        const float2* in = Bf.spec + (((long long)b * P.nz + z) * P.NT * P.ny + y) * 3 * TX;
        for (int idx = threadIdx.x; idx < 3 * (L + 1); idx += blockDim.x) {
            const int c = idx / (L + 1), k = idx - c * (L + 1);
            const int t = k >> lt, tx = k & (TX - 1);
            cp_async8(xs + k * ld + 3 * r + c, in + t * tstride + c * TX + tx);
        }
    }
    if (STAGE_M) {
        for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) cp_async16(mrow + i, msrc + base + i);
    } else if (threadIdx.x == 0) {
        prefetch_l2(msrc + base, (unsigned)(nr * nx * sizeof(float4)));
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < NM; q++) s_gamma[q] = stage_gamma(A, ip, st, mat, q);
        s_drive = (float)drive_factor(A, ip, st);
    }
    cp_async_wait_all();
    __syncthreads();
    // Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k / px} (X[k] - conj X[L-k]), in place by pairs
    const int twstep = P.twn / P.px;
    constexpr int HALF = L / 2 + 1;
    for (int idx = threadIdx.x; idx < 3 * nr * HALF; idx += blockDim.x) {
        const int line = idx / HALF, k = idx - line * HALF;
        const int kk = L - k;
        float2 a = xs[k * ld + line], bq = xs[kk * ld + line];
        float2 ca = conjf2(bq);
        float2 sum = cadd(a, ca), dif = csub(a, ca);
        float2 wd = cmul(twiddle(Bf.tw, k * twstep, true), dif);
        float2 zk = make_float2(sum.x - wd.y, sum.y + wd.x);   // sum + i wd
        if (k != 0 && kk != k) {
            float2 cb2 = conjf2(a);
            float2 sum2 = cadd(bq, cb2), dif2 = csub(bq, cb2);
            float2 wd2 = cmul(twiddle(Bf.tw, kk * twstep, true), dif2);
            xs[kk * ld + line] = make_float2(sum2.x - wd2.y, sum2.y + wd2.x);
        }
        xs[k * ld + line] = zk;
    }
    __syncthreads();
    {
        const int nl = 3 * P.R;
        const int line = threadIdx.x % nl, j = threadIdx.x / nl;
        float2 v[NPT];
#pragma unroll
        for (int n2 = 0; n2 < NPT; n2++) v[n2] = xs[(j + N1 * n2) * ld + line];
        col_fft<L, true>(v, xs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
        for (int i = 0; i < NPT; i++) xs[col_out_row<L>(j, i) * ld + line] = v[i];
    }
    __syncthreads();

    const bool want_demag = A.terms & 1, want_exch = A.terms & 2;
    CellUpdate<NM> cu;
    cu.init(Bf, A, st, ip, s_gamma, s_drive, cb, (long long)A.inst0 * P.N);
    const long long pl = (long long)nx * P.ny;
    double xacc[NM];
#pragma unroll
    for (int q = 0; q < NM; q++) xacc[q] = 0.0;
    double macc[REC ? 3 : 1] = {};
    float emax = 0.f;
    bool bad = false;
    for (int ii = threadIdx.x; ii < nr * nx; ii += blockDim.x) {
        const int r = (int)fdiv((unsigned)ii, P.fd_nx), x = ii - r * nx;
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        const long long i = base + ii;
        float4 m = STAGE_M ? mrow[ii] : __ldg(msrc + i);
        const float Ms = m.w;
        float Bx = 0.f, By = 0.f, Bz = 0.f;
        if (want_demag) {
            const float2* zr = xs + (x >> 1) * ld + 3 * r;
            float2 zx = zr[0], zy = zr[1], zz = zr[2];
            if (x & 1) { Bx = zx.y; By = zy.y; Bz = zz.y; }
            else { Bx = zx.x; By = zy.x; Bz = zz.x; }
        }
        if (Ms > 0.f && want_exch) {
            float hx = 0.f, hy = 0.f, hz = 0.f;
            float4 q;
#define MMCQ_NB(Q, C)                                                                   \
    q = (Q);                                                                            \
    if (q.w > 0.f) { hx += (C) * (q.x - m.x); hy += (C) * (q.y - m.y); hz += (C) * (q.z - m.z); }
            if (x > 0) { MMCQ_NB(STAGE_M ? mrow[ii - 1] : __ldg(msrc + i - 1), mat.exch[0]) }
            if (x + 1 < nx) { MMCQ_NB(STAGE_M ? mrow[ii + 1] : __ldg(msrc + i + 1), mat.exch[0]) }
            if (y > 0) {
                if (STAGE_M && r > 0) { MMCQ_NB(mrow[ii - nx], mat.exch[1]) }
                else { MMCQ_NB(__ldg(msrc + i - nx), mat.exch[1]) }
            }
            if (y + 1 < P.ny) {
                if (STAGE_M && r + 1 < nr) { MMCQ_NB(mrow[ii + nx], mat.exch[1]) }
                else { MMCQ_NB(__ldg(msrc + i + nx), mat.exch[1]) }
            }
            if (z > 0) { MMCQ_NB(__ldg(msrc + i - pl), mat.exch[2]) }
            if (z + 1 < P.nz) { MMCQ_NB(__ldg(msrc + i + pl), mat.exch[2]) }
#undef MMCQ_NB
            float inv = 1.f / Ms;
            Bx += hx * inv; By += hy * inv; Bz += hz * inv;
        }
        cu.template run<REC>(mat, Bf, i, m, Bx, By, Bz, xacc, macc, emax, bad);
    }
    if (A.field_only) return;
    stage_epilogue<REC, NM>(P, mat, Bf, A, b, blockIdx.x, P.nblk, xacc, emax, bad, s_red, s_redf, &s_last, macc);
}

cudaError_t launch_xinv(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A, int nb,
                        cudaStream_t s) {
    dim3 grid(P.nblk, nb);
    const int th = xthreads(P);
    const size_t sm = xinv_smem(P);
    const bool rec = A.record > 0 && !A.field_only && A.stage == (A.kind == KIND_RK4 ? 3 : 6);
    const bool multi = A.nmodes > 1;
    switch (P.L) {
#define MMCQ_CASE(Lv)                                                                          \
    case Lv:                                                                                   \
        if (multi) {                                                                           \
            if (rec) k_xinv<Lv, true, MAX_MODES><<<grid, th, sm, s>>>(P, mat, Bf, A);          \
            else k_xinv<Lv, false, MAX_MODES><<<grid, th, sm, s>>>(P, mat, Bf, A);             \
        } else {                                                                               \
            if (rec) k_xinv<Lv, true, 1><<<grid, th, sm, s>>>(P, mat, Bf, A);                  \
            else k_xinv<Lv, false, 1><<<grid, th, sm, s>>>(P, mat, Bf, A);                     \
        }                                                                                      \
        break;
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename K>
static cudaError_t xinv_attr(K kernel, int lim) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// Per-unit constant tables and shared-memory limits of the x-inverse kernels.
cudaError_t xinv_init() {
    cudaError_t e;
    upload_tableaux();
    if ((e = upload_tw32()) != cudaSuccess) return e;
    const int lim = 200 * 1024;
#define MMCQ_CASE(Lv)                                                                   \
    if ((e = xinv_attr(k_xinv<Lv, false, 1>, lim)) != cudaSuccess) return e;            \
    if ((e = xinv_attr(k_xinv<Lv, true, 1>, lim)) != cudaSuccess) return e;             \
    if ((e = xinv_attr(k_xinv<Lv, false, MAX_MODES>, lim)) != cudaSuccess) return e;    \
    if ((e = xinv_attr(k_xinv<Lv, true, MAX_MODES>, lim)) != cudaSuccess) return e;
    MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
    return cudaSuccess;
}

}  // namespace mq
