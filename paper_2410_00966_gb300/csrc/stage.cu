// Stage kernels of the LLG + cavity hot path (Mumax3-cQED, arXiv 2410.00966).
//
// One field evaluation (one Runge-Kutta stage) is three kinds of launch:
//   k_xfwd : stage input m_s = m0 + dt sum_j a_sj k_j (Eq. llg integrated by
//            RK4 / Dormand-Prince), M = Ms m_s, zero-padded real-to-complex FFT
//            along x, written to a tiled half-spectrum.
//   k_col  : (col.cu) FFT along y (and z) of tiles of kx columns, the
//            pointwise product with the symmetric demag kernel, inverse FFT.
//   k_xinv : (xinv.cu) complex-to-real inverse FFT along x giving B_demag, then per cell
//            exchange + anisotropy + Zeeman + cavity B_rms Gamma (Sec. 2.1
//            field terms, Eq. bcav), the LLG torque (Eq. llg), the RK
//            bookkeeping, and block partials of the coupling sum
//            X = V_c sum_i Ms_i m_i . B_rms,i (Eq. gammafinal).  The last block
//            of each instance to finish reduces the partials in a fixed order
//            and advances the cavity amplitude / step-size controller in FP64.
#include <math.h>

#include "common.cuh"
#include "fftreg.cuh"
#include "kern_common.cuh"
#include "stagecore.cuh"
#include "xpass.cuh"

namespace mq {

// ---------------------------------------------------------------------------
// x forward: stage input, M = Ms m_s, packed real FFT of length px = 2L.
// R consecutive rows per block; shared memory zs[n][line], line = 3 r + comp.
// ---------------------------------------------------------------------------
// FX: the fixed shape of the large grids (see xpass_fixed) at compile time.
template <int L, bool FX>
__global__ void __launch_bounds__(XPASS_THREADS, xpass_min_blocks(L)) k_xfwd(Plan P, Buffers Bf, StageArgs A) {
    constexpr bool F3 = xpass_f3(L);
    constexpr int NPT = F3 ? 16 : ColShape<L>::NPT, N1 = xpass_line_threads(L);
    constexpr int RF = xpass_rows(L);
    extern __shared__ float2 sm[];
    const int b = A.inst0 + blockIdx.y;
    const InstState& st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const int Rb = FX ? RF : P.R;
    const int nx = FX ? L : P.nx;
    const int px = FX ? 2 * L : P.px;
    const int nthr = FX ? 3 * RF * N1 : (int)blockDim.x;
    const int row0 = blockIdx.x * Rb;
    const int nr = FX ? RF : min(P.R, P.nrows - row0);
    const int ld = xpass_ld(Rb);
    const long long base = (long long)b * P.N + (long long)row0 * nx;
    const float4* m0 = Bf.m[st.mcur] + base;
    StageInput si;
    si.init(Bf, A, st, base);
    if (threadIdx.x == 0) {
        // the block's rows of m0 and of every k it combines: in flight while
        // the shared tables are set up
        const unsigned bytes = (unsigned)(nr * nx * sizeof(float4));
        prefetch_l2(m0, bytes);
        si.prefetch(Bf, bytes);
    }
    float2* zs = sm;
    // exp(-2 pi i e / px), e < px: a shared copy for the four-step transform;
    // the three-factor one (L = 1024) reads the global table through L1
    float2* stw = sm + xpass_fft_rows(L) * ld;
    const int tws = P.twn / px;
    if constexpr (!F3)
        for (int e = threadIdx.x; e < px; e += nthr) stw[e] = __ldg(Bf.tw + e * tws);
    // rows nx/2.. of the packed line are zero padding (rows below are all
    // written).  FX (nx = L): they are not stored, the transform takes its
    // points n2 >= NPT / 2 as zeros.
    if constexpr (!FX)
        for (int i = (nx >> 1) * ld + threadIdx.x; i < L * ld; i += nthr) zs[i] = make_float2(0.f, 0.f);
    __syncthreads();


    for (int i = threadIdx.x; i < nr * nx; i += nthr) {
        float4 v = m0[i];
        si.apply(Bf, v, i);
        const int r = FX ? i / L : (int)fdiv((unsigned)i, P.fd_nx), x = i - r * nx;
        // z_n = x_2n + i x_2n+1: cell x is the real (even x) or imaginary part
        float* zr = reinterpret_cast<float*>(zs + (x >> 1) * ld + 3 * r) + (x & 1);
        zr[0] = v.w * v.x;
        zr[2] = v.w * v.y;
        zr[4] = v.w * v.z;
    }
    __syncthreads();
    {
        // three-factor: a line's 64 threads are consecutive (lane groups of
        // the last factor inside one warp); otherwise lines are fastest
        const int nl = 3 * Rb;
        const int line = F3 ? threadIdx.x / N1 : threadIdx.x % nl;
        const int j = F3 ? threadIdx.x % N1 : threadIdx.x / nl;
        float2 v[NPT];
#pragma unroll
        for (int n2 = 0; n2 < NPT; n2++)
            v[n2] = (!FX || n2 < NPT / 2) ? zs[(j + N1 * n2) * ld + line] : make_float2(0.f, 0.f);
        if constexpr (F3) {
            col_fft3<L, false, false, XPASS_F3_PADS, 1>(v, zs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
            for (int i = 0; i < NPT; i++) zs[col3_out_row<L>(j, i) * ld + line] = v[i];
        } else {
            col_fft<L, false, true>(v, zs, ld, line, j, stw, px);
#pragma unroll
            for (int i = 0; i < NPT; i++) zs[col_out_row<L>(j, i) * ld + line] = v[i];
        }
    }
    __syncthreads();

    // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2, O = -i (Z[k] - conj Z[L-k]) / 2
    const int TX = FX ? 8 : P.TX, lt = FX ? 3 : P.lt;
    const int NT = FX ? L / 8 + 1 : P.NT;
    const long long tstride = (long long)P.ny * 3 * TX;
    auto unpack = [&](int k, int line) {
        float2 X = make_float2(0.f, 0.f);
        if (k <= L) {
            float2 Zk = zs[(k == L ? 0 : k) * ld + line];
            float2 Zc = conjf2(zs[(k == 0 ? 0 : L - k) * ld + line]);
            float2 E = make_float2(0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y));
            float2 D = make_float2(0.5f * (Zk.x - Zc.x), 0.5f * (Zk.y - Zc.y));
            float2 wD = cmul(F3 ? __ldg(Bf.tw + k * tws) : stw[k], D);
            X = make_float2(E.x + wD.y, E.y - wD.x);
        }
        return X;
    };
    // tile t of a row holds the 3 TX values (c, tx) contiguously; when 3 TX
    // divides the block, a thread keeps one (c, tx) and steps over the tiles
    const int w3 = 3 * TX;
    if (nthr % w3 == 0) {
        const int e = threadIdx.x % w3, t0 = threadIdx.x / w3, dtt = nthr / w3;
        const int c = e >> lt, tx = e & (TX - 1);
        for (int r = 0; r < nr; r++) {
            const int row = row0 + r;
            const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
            float2* out = Bf.spec + (((long long)b * P.nz + z) * NT * P.ny + y) * 3 * TX + e;
            for (int t = t0; t < NT; t += dtt) out[t * tstride] = unpack(t * TX + tx, 3 * r + c);
        }
        return;
    }
    const int W3 = NT * 3 * TX;
    for (int r = 0; r < nr; r++) {
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        float2* out = Bf.spec + (((long long)b * P.nz + z) * NT * P.ny + y) * 3 * TX;
        for (int idx = threadIdx.x; idx < W3; idx += nthr) {
            const int t = (idx >> lt) / 3;
            const int ctx = idx - t * 3 * TX;
            const int c = ctx >> lt, tx = ctx & (TX - 1);
            out[t * tstride + ctx] = unpack(t * TX + tx, 3 * r + c);
        }
    }
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
// and gradient path), all in FP64.  Pass 1: cpart_n blocks per instance, each
// a contiguous chunk of at most CSUM_THREADS x CSUM_CELLS cells, spread over
// the whole GPU (FP64 issues at a small fraction of the FP32 rate, so one
// block per instance would leave it to a few SMs).  Pass 2: one block per
// instance sums its partials in a fixed order.
constexpr int CSUM_THREADS = 256, CSUM_CELLS = 16;
__global__ void __launch_bounds__(CSUM_THREADS) k_coupling_part(const float4* m0, const float4* m1,
                                                                const InstState* st, const float4* prof, long long N,
                                                                int b0, double* part, int nblk) {
    __shared__ double red[32];
    const int b = b0 + blockIdx.y;
    const float4* m = (st[b].mcur ? m1 : m0) + (long long)b * N;
    const long long chunk = (N + nblk - 1) / nblk;
    const long long i0 = blockIdx.x * chunk;
    const long long i1 = i0 + chunk < N ? i0 + chunk : N;
    double acc = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += CSUM_THREADS) {
        const float4 v = m[i];
        const float4 p = prof ? prof[i] : make_float4(0.f, 1.f, 0.f, 0.f);
        acc += (double)v.w * ((double)v.x * p.x + (double)v.y * p.y + (double)v.z * p.z);
    }
    const double s = block_sum_d(acc, red);
    if (threadIdx.x == 0) part[(long long)blockIdx.y * nblk + blockIdx.x] = s;
}

__global__ void __launch_bounds__(CSUM_THREADS) k_coupling_fin(const InstParams* ip, const double* part, int nblk,
                                                               double vc, int b0, int k, double* out) {
    __shared__ double red[32];
    const int b = b0 + blockIdx.x;
    double acc = 0.0;
    for (int q = threadIdx.x; q < nblk; q += CSUM_THREADS) acc += part[(long long)blockIdx.x * nblk + q];
    acc = block_sum_d(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = ip[b].cav_on[k] ? acc * ip[b].brms_scale[k] * vc : 0.0;
}

// Blocks per instance of the coupling sum (host side, for the allocation).
int coupling_blocks(long long N) {
    const long long per = (long long)CSUM_THREADS * CSUM_CELLS;
    return (int)((N + per - 1) / per);
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
    int n1 = xpass_line_threads(L);
    int R = 64 / n1;
    if (R < 1) R = 1;
    if (R > nrows) R = nrows;
    return R;
}


// shared memory of the x forward: the packed lines and (four-step lengths) the
// px-entry twiddle table
size_t xfwd_smem(const Plan& P) {
    const size_t table = xpass_f3(P.L) ? 0 : (size_t)P.px;   // the three-factor transform reads the global table
    return ((size_t)xpass_fft_rows(P.L) * xpass_ld(P.R) + table) * sizeof(float2);
}


bool x_fits(const Plan& P) { return P.L <= 1024 && xthreads(P) <= 512 && xinv_smem(P) <= 200 * 1024; }


cudaError_t launch_xfwd(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s) {
    dim3 grid(P.nblk, nb);
    const int th = xthreads(P);
    const size_t sm = xfwd_smem(P);
    if (xpass_fixed(P)) {
        switch (P.L) {
#define MMCQ_CASE(Lv) case Lv: return launch_chain(k_xfwd<Lv, true>, grid, th, sm, s, P, Bf, A);
            MMCQ_XFIXED(MMCQ_CASE)
#undef MMCQ_CASE
            default: break;
        }
    }
    switch (P.L) {
#define MMCQ_CASE(Lv) case Lv: return launch_chain(k_xfwd<Lv, false>, grid, th, sm, s, P, Bf, A);
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
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
cudaError_t launch_coupling_sum(const Buffers& Bf, long long N, double vc, int b0, int nb, int k, double* out,
                                cudaStream_t s) {
    k_coupling_part<<<dim3(Bf.cpart_n, nb), CSUM_THREADS, 0, s>>>(Bf.m[0], Bf.m[1], Bf.st, Bf.prof[k], N, b0,
                                                                  Bf.cpart, Bf.cpart_n);
    k_coupling_fin<<<nb, CSUM_THREADS, 0, s>>>(Bf.ip, Bf.cpart, Bf.cpart_n, vc, b0, k, out);
    return cudaGetLastError();
}
cudaError_t launch_set_dt(InstState* st, int B, double dt, cudaStream_t s) {
    k_set_dt<<<(B + 127) / 128, 128, 0, s>>>(st, B, dt);
    return cudaGetLastError();
}

cudaError_t col_init();
cudaError_t xinv_init();

cudaError_t set_smem_limits() {
    cudaError_t e;
    upload_tableaux();
    if ((e = upload_tw32()) != cudaSuccess) return e;
    const int lim = 200 * 1024;
#define MMCQ_CASE(Lv)                                                                                \
    if ((e = cudaFuncSetAttribute(k_xfwd<Lv, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != \
        cudaSuccess)                                                                                        \
        return e;
    MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
#define MMCQ_CASE(Lv)                                                                               \
    if ((e = cudaFuncSetAttribute(k_xfwd<Lv, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != \
        cudaSuccess)                                                                                       \
        return e;
    MMCQ_XFIXED(MMCQ_CASE)
#undef MMCQ_CASE
    if ((e = xinv_init()) != cudaSuccess) return e;
    return col_init();
}

}  // namespace mq
