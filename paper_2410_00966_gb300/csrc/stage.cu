// Stage kernels of the LLG + cavity hot path (Mumax3-cQED, arXiv 2410.00966).
//
// One field evaluation (one Runge-Kutta stage) is three kinds of launch:
//   k_xfwd : stage input m_s = m0 + dt sum_j a_sj k_j (Eq. llg integrated by
//            RK4 / Dormand-Prince), M = Ms m_s, zero-padded real-to-complex FFT
//            along x, written to a tiled half-spectrum.
//   k_col  : (col.cu) FFT along y (and z) of tiles of kx columns, the
//            pointwise product with the symmetric demag kernel, inverse FFT.
//   k_xinv : complex-to-real inverse FFT along x giving B_demag, then per cell
//            exchange + anisotropy + Zeeman + cavity B_rms Gamma (Sec. 2.1
//            field terms, Eq. bcav), the LLG torque (Eq. llg), the RK
//            bookkeeping, and FP64 block partials of the coupling sum
//            X = V_c sum_i Ms_i m_i . B_rms,i (Eq. gammafinal).  The last block
//            of each instance to finish reduces the partials in a fixed order
//            and advances the cavity amplitude / step-size controller in FP64.
#include <math.h>

#include "common.cuh"
#include "fftreg.cuh"
#include "kern_common.cuh"
#include "stagecore.cuh"

namespace mq {

// Shared-memory pitch of the x passes: 3 R lines rounded up to an odd count,
// so that consecutive cells (stride one pitch) fall in different banks.
__host__ __device__ __forceinline__ int xpass_ld(int R) { return (3 * R) | 1; }

// Threads of an x-pass block: 3 R lines x N1 threads per line with R = 64 / N1
// rows (fewer when the grid has fewer rows), so never more than 192.
constexpr int XPASS_THREADS = 192;
// Resident blocks asked of the compiler: 5 (64 registers) while a thread
// holds 16 points of the x transform, 3 when it holds 32 (L >= 512).
constexpr int xpass_min_blocks(int L) { return L >= 512 ? 3 : 5; }

// ---------------------------------------------------------------------------
// x forward: stage input, M = Ms m_s, packed real FFT of length px = 2L.
// R consecutive rows per block; shared memory zs[n][line], line = 3 r + comp.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(XPASS_THREADS, xpass_min_blocks(L)) k_xfwd(Plan P, Buffers Bf, StageArgs A) {
    constexpr int NPT = ColShape<L>::NPT, N1 = ColShape<L>::N1;
    extern __shared__ float2 sm[];
    const int b = A.inst0 + blockIdx.y;
    const InstState& st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const int nx = P.nx;
    const int row0 = blockIdx.x * P.R;
    const int nr = min(P.R, P.nrows - row0);
    const int ld = xpass_ld(P.R);
    const long long base = (long long)b * P.N + (long long)row0 * nx;
    float2* zs = sm;
    float2* stw = sm + L * ld;                 // exp(-2 pi i e / px), e < px
    const int tws = P.twn / P.px;
    for (int e = threadIdx.x; e < P.px; e += blockDim.x) stw[e] = __ldg(Bf.tw + e * tws);
    // rows nx/2.. of the packed line are zero padding (rows below are all written)
    for (int i = (nx >> 1) * ld + threadIdx.x; i < L * ld; i += blockDim.x) zs[i] = make_float2(0.f, 0.f);
    __syncthreads();

    const float4* m0 = Bf.m[st.mcur] + base;
    StageInput si;
    si.init(Bf, A, st, base);
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) {
        float4 v = m0[i];
        si.apply(Bf, v, i);
        const int r = (int)fdiv((unsigned)i, P.fd_nx), x = i - r * nx;
        float2* zr = zs + (x >> 1) * ld + 3 * r;
        float Mx = v.w * v.x, My = v.w * v.y, Mz = v.w * v.z;
        if (x & 1) { zr[0].y = Mx; zr[1].y = My; zr[2].y = Mz; }
        else { zr[0].x = Mx; zr[1].x = My; zr[2].x = Mz; }
    }
    __syncthreads();
    {
        const int nl = 3 * P.R;
        const int line = threadIdx.x % nl, j = threadIdx.x / nl;
        float2 v[NPT];
#pragma unroll
        for (int n2 = 0; n2 < NPT; n2++) v[n2] = zs[(j + N1 * n2) * ld + line];
        col_fft<L, false, true>(v, zs, ld, line, j, stw, P.px);
#pragma unroll
        for (int i = 0; i < NPT; i++) zs[col_out_row<L>(j, i) * ld + line] = v[i];
    }
    __syncthreads();

    // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2, O = -i (Z[k] - conj Z[L-k]) / 2
    const int TX = P.TX, lt = P.lt;
    const long long tstride = (long long)P.ny * 3 * TX;
    const int W3 = P.NT * 3 * TX;
    for (int r = 0; r < nr; r++) {
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        float2* out = Bf.spec + (((long long)b * P.nz + z) * P.NT * P.ny + y) * 3 * TX;
        for (int idx = threadIdx.x; idx < W3; idx += blockDim.x) {
            const int t = (idx >> lt) / 3;
            const int ctx = idx - t * 3 * TX;
            const int c = ctx >> lt, tx = ctx & (TX - 1);
            const int k = t * TX + tx;
            const int line = 3 * r + c;
            float2 X = make_float2(0.f, 0.f);
            if (k <= L) {
                float2 Zk = zs[(k == L ? 0 : k) * ld + line];
                float2 Zc = conjf2(zs[(k == 0 ? 0 : L - k) * ld + line]);
                float2 E = make_float2(0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y));
                float2 D = make_float2(0.5f * (Zk.x - Zc.x), 0.5f * (Zk.y - Zc.y));
                float2 wD = cmul(stw[k], D);
                X = make_float2(E.x + wD.y, E.y - wD.x);
            }
            out[t * tstride + ctx] = X;
        }
    }
}

// ---------------------------------------------------------------------------
// x inverse + local fields + torque + RK bookkeeping + cavity reduction.
// Shared memory: xs[k][line] (k <= L, line = 3 r + comp), then m rows.
// ---------------------------------------------------------------------------
// REC: this launch records the spatial average of the state being accepted
// (the last stage of a step with recording on); a separate instantiation so
// that the common launches carry no extra accumulators.
template <int L, bool REC>
__global__ void __launch_bounds__(XPASS_THREADS, xpass_min_blocks(L)) k_xinv(Plan P, Material mat, Buffers Bf, StageArgs A) {
    constexpr int NPT = ColShape<L>::NPT, N1 = ColShape<L>::N1;
    extern __shared__ float2 sm[];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma;
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
    float4* mrow = reinterpret_cast<float4*>(sm + xs_n);  // [row][nx]

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
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) cp_async16(mrow + i, msrc + base + i);
    if (threadIdx.x == 0) {
        s_gamma = stage_gamma(A, ip, st, mat);
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
    CellUpdate cu;
    cu.init(Bf, A, st, ip, (float)s_gamma, s_drive, cb);
    const long long pl = (long long)nx * P.ny;
    double xacc = 0.0;
    double macc[REC ? 3 : 1] = {};
    float emax = 0.f;
    bool bad = false;
    for (int ii = threadIdx.x; ii < nr * nx; ii += blockDim.x) {
        const int r = (int)fdiv((unsigned)ii, P.fd_nx), x = ii - r * nx;
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        const long long i = base + ii;
        float4 m = mrow[ii];
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
            if (x > 0) { MMCQ_NB(mrow[ii - 1], mat.exch[0]) }
            if (x + 1 < nx) { MMCQ_NB(mrow[ii + 1], mat.exch[0]) }
            if (y > 0) {
                if (r > 0) { MMCQ_NB(mrow[ii - nx], mat.exch[1]) }
                else { MMCQ_NB(__ldg(msrc + i - nx), mat.exch[1]) }
            }
            if (y + 1 < P.ny) {
                if (r + 1 < nr) { MMCQ_NB(mrow[ii + nx], mat.exch[1]) }
                else { MMCQ_NB(__ldg(msrc + i + nx), mat.exch[1]) }
            }
            if (z > 0) { MMCQ_NB(__ldg(msrc + i - pl), mat.exch[2]) }
            if (z + 1 < P.nz) { MMCQ_NB(__ldg(msrc + i + pl), mat.exch[2]) }
#undef MMCQ_NB
            float inv = 1.f / Ms;
            Bx += hx * inv; By += hy * inv; Bz += hz * inv;
        }
        cu.run<REC>(mat, Bf, i, m, Bx, By, Bz, xacc, macc, emax, bad);
    }
    if (A.field_only) return;
    stage_epilogue<REC>(P, mat, Bf, A, b, blockIdx.x, P.nblk, xacc, emax, bad, s_red, s_redf, &s_last, macc);
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

// m of one instance (or all) from an N x 3 float array: FP64 normalisation,
// zero in empty cells, Ms into w.  A non-finite direction is stored as zero
// and raises FLAG_NAN (reported by the next synchronising call).
__global__ void k_set_m(float4* m, const float* src, const float* ms, long long N, int b0, int nb, int* flags) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x = src[3 * i], y = src[3 * i + 1], zz = src[3 * i + 2];
    double r = sqrt(x * x + y * y + zz * zz);
    if (!isfinite(r)) { atomicOr(flags, FLAG_NAN); r = 0.0; }
    float w = ms[i];
    float4 v;
    if (w > 0.f && r > 0.0) v = make_float4((float)(x / r), (float)(y / r), (float)(zz / r), w);
    else v = make_float4(0.f, 0.f, 0.f, w > 0.f ? w : 0.f);
    for (int b = b0; b < b0 + nb; b++) m[(long long)b * N + i] = v;
}

__global__ void k_get_m(const float4* m, float* dst, long long N) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 v = m[i];
    dst[3 * i] = v.x; dst[3 * i + 1] = v.y; dst[3 * i + 2] = v.z;
}

// new Ms map: rescale w, zero m where Ms = 0 (cells that gain Ms keep direction +x)
__global__ void k_apply_ms(float4* m, const float* ms, long long N, int B) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float w = ms[i];
    for (int b = 0; b < B; b++) {
        float4 v = m[(long long)b * N + i];
        if (!(w > 0.f)) v = make_float4(0.f, 0.f, 0.f, 0.f);
        else {
            if (v.x == 0.f && v.y == 0.f && v.z == 0.f) v.x = 1.f;
            v.w = w;
        }
        m[(long long)b * N + i] = v;
    }
}

__global__ void k_get_field(const float4* f, float* dst, long long N) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 v = f[i];
    dst[3 * i] = v.x; dst[3 * i + 1] = v.y; dst[3 * i + 2] = v.z;
}

// X = V_c sum Ms m . B_rms of each instance at its accepted state (read-out
// only): one block per instance, fixed-order reduction.
__global__ void k_coupling_sum(const float4* m0, const float4* m1, const InstState* st, const InstParams* ip,
                               const float4* prof, long long N, double vc, int b0, double* out) {
    __shared__ double red[32];
    const int b = b0 + blockIdx.x;
    const float4* m = (st[b].mcur ? m1 : m0) + (long long)b * N;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        float4 v = m[i];
        double px = 0, py = 1, pz = 0;
        if (prof) { float4 p = prof[i]; px = p.x; py = p.y; pz = p.z; }
        acc += (double)v.w * (v.x * px + v.y * py + v.z * pz);
    }
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = ip[b].cav_on ? acc * ip[b].brms_scale * vc : 0.0;
}

// Trapezoid-weighted Fourier transform of one component of the recorded
// spatial averages (t_n, <m>_n), n < ns (Appendix C: the broadband response
// is the numerical Fourier transform of the averaged m):
// S(w) = sum_n c_n (y_n - ybar) exp(-i w t_n), c_n the trapezoid weights of
// the sample times, ybar the time average.  One block per frequency (grid
// stride), FP64, fixed-order reductions.
__global__ void k_spectrum(const double* mh, long long ns, int comp, const double* w, int nw, double* out) {
    __shared__ double red[32];
    auto weight = [&](long long q) {
        if (ns < 2) return 0.0;
        const double tl = mh[4 * (q > 0 ? q - 1 : q)], tr = mh[4 * (q + 1 < ns ? q + 1 : q)];
        return 0.5 * (tr - tl);
    };
    double cs = 0.0, cy = 0.0;
    for (long long q = threadIdx.x; q < ns; q += blockDim.x) {
        const double c = weight(q);
        cs += c;
        cy += c * mh[4 * q + 1 + comp];
    }
    cs = block_sum_d(cs, red);
    cy = block_sum_d(cy, red);
    __shared__ double s_ybar;
    if (threadIdx.x == 0) s_ybar = cs > 0.0 ? cy / cs : 0.0;
    __syncthreads();
    const double ybar = s_ybar;
    for (int k = blockIdx.x; k < nw; k += gridDim.x) {
        double re = 0.0, im = 0.0;
        for (long long q = threadIdx.x; q < ns; q += blockDim.x) {
            const double v = weight(q) * (mh[4 * q + 1 + comp] - ybar);
            double sn, c;
            sincos(w[k] * mh[4 * q], &sn, &c);
            re += v * c;
            im -= v * sn;
        }
        re = block_sum_d(re, red);
        im = block_sum_d(im, red);
        if (threadIdx.x == 0) { out[2 * k] = re; out[2 * k + 1] = im; }
    }
}

__global__ void k_set_dt(InstState* st, int B, double dt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) st[b].dt = dt;
}

// ---------------------------------------------------------------------------
// host-side launchers (called from the C ABI)
// ---------------------------------------------------------------------------
// Rows per x-pass block: R lines of 3 components times N1 = L / 32 threads
// each, aiming at ~192 threads per block.
int rows_per_block(int L, int nrows) {
    int n1 = col_threads_per_column(L);
    int R = 64 / n1;
    if (R < 1) R = 1;
    if (R > nrows) R = nrows;
    return R;
}

static int xthreads(const Plan& P) { return 3 * P.R * col_threads_per_column(P.L); }

// shared memory of the x passes: x forward: the packed lines and the
// px-entry twiddle table; x inverse: the half-spectrum lines and the m rows
size_t xfwd_smem(const Plan& P) { return ((size_t)P.L * xpass_ld(P.R) + P.px) * sizeof(float2); }

size_t xinv_smem(const Plan& P) {
    size_t n2 = (size_t)(P.L + 1) * xpass_ld(P.R);
    n2 += n2 & 1;
    return n2 * sizeof(float2) + (size_t)P.nx * P.R * sizeof(float4);
}

bool x_fits(const Plan& P) { return P.L <= 1024 && xthreads(P) <= 512 && xinv_smem(P) <= 200 * 1024; }

#define MMCQ_XCASES(F) F(1) F(2) F(4) F(8) F(16) F(32) F(64) F(128) F(256) F(512) F(1024)

cudaError_t launch_xfwd(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s) {
    dim3 grid(P.nblk, nb);
    const int th = xthreads(P);
    const size_t sm = xfwd_smem(P);
    switch (P.L) {
#define MMCQ_CASE(Lv) case Lv: k_xfwd<Lv><<<grid, th, sm, s>>>(P, Bf, A); break;
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_xinv(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A, int nb,
                        cudaStream_t s) {
    dim3 grid(P.nblk, nb);
    const int th = xthreads(P);
    const size_t sm = xinv_smem(P);
    const bool rec = A.record > 0 && !A.field_only && A.stage == (A.kind == KIND_RK4 ? 3 : 6);
    switch (P.L) {
#define MMCQ_CASE(Lv)                                                      \
    case Lv:                                                               \
        if (rec) k_xinv<Lv, true><<<grid, th, sm, s>>>(P, mat, Bf, A);    \
        else k_xinv<Lv, false><<<grid, th, sm, s>>>(P, mat, Bf, A);       \
        break;
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const double* mh, long long ns, int comp, const double* w, int nw, double* out,
                            cudaStream_t s) {
    const int blocks = nw < 1024 ? nw : 1024;
    if (blocks < 1) return cudaSuccess;
    k_spectrum<<<blocks, 256, 0, s>>>(mh, ns, comp, w, nw, out);
    return cudaGetLastError();
}

cudaError_t launch_set_m(float4* m, const float* src, const float* ms, long long N, int b0, int nb, int* flags,
                         cudaStream_t s) {
    k_set_m<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(m, src, ms, N, b0, nb, flags);
    return cudaGetLastError();
}
cudaError_t launch_get_m(const float4* m, float* dst, long long N, cudaStream_t s) {
    k_get_m<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(m, dst, N);
    return cudaGetLastError();
}
cudaError_t launch_apply_ms(float4* m, const float* ms, long long N, int B, cudaStream_t s) {
    k_apply_ms<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(m, ms, N, B);
    return cudaGetLastError();
}
cudaError_t launch_get_field(const float4* f, float* dst, long long N, cudaStream_t s) {
    k_get_field<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, dst, N);
    return cudaGetLastError();
}
cudaError_t launch_coupling_sum(const Buffers& Bf, long long N, double vc, int b0, int nb, double* out,
                                cudaStream_t s) {
    k_coupling_sum<<<nb, 1024, 0, s>>>(Bf.m[0], Bf.m[1], Bf.st, Bf.ip, Bf.prof, N, vc, b0, out);
    return cudaGetLastError();
}
cudaError_t launch_set_dt(InstState* st, int B, double dt, cudaStream_t s) {
    k_set_dt<<<(B + 127) / 128, 128, 0, s>>>(st, B, dt);
    return cudaGetLastError();
}

cudaError_t col_init();

cudaError_t set_smem_limits() {
    cudaError_t e;
    upload_tableaux();
    if ((e = upload_tw32()) != cudaSuccess) return e;
    const int lim = 200 * 1024;
#define MMCQ_CASE(Lv)                                                                                         \
    if ((e = cudaFuncSetAttribute(k_xfwd<Lv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) \
        return e;                                                                                             \
    if ((e = cudaFuncSetAttribute(k_xinv<Lv, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=        \
        cudaSuccess)                                                                                               \
        return e;                                                                                                  \
    if ((e = cudaFuncSetAttribute(k_xinv<Lv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) \
        return e;
    MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
    return col_init();
}

}  // namespace mq
