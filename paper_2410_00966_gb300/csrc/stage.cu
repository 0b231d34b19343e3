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

namespace mq {

// Shared-memory pitch of the x passes: 3 R lines rounded up to an odd count,
// so that consecutive cells (stride one pitch) fall in different banks.
__host__ __device__ __forceinline__ int xpass_ld(int R) { return (3 * R) | 1; }

// Butcher tableaux: [kind][stage][j].
__constant__ float c_af[2][MAX_STAGES][MAX_STAGES];
__constant__ double c_ad[2][MAX_STAGES][MAX_STAGES];
__constant__ float c_bf[2][MAX_STAGES];    // weights of the propagated solution
__constant__ double c_bd[2][MAX_STAGES];
__constant__ double c_cd[2][MAX_STAGES];   // stage times
__constant__ float c_ef[MAX_STAGES];       // DP45 error weights b5 - b4

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
// Fixed-shape block reductions (deterministic for a given blockDim).
__device__ double block_sum_d(double v, double* red) {
    v = warp_sum_d(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    double r = 0.0;
    if (w == 0) {
        r = l < nw ? red[l] : 0.0;
        r = warp_sum_d(r);
    }
    __syncthreads();
    return r;  // valid in thread 0
}
__device__ float block_max_f(float v, float* red) {
    v = warp_max_f(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    float r = 0.f;
    if (w == 0) {
        r = l < nw ? red[l] : 0.f;
        r = warp_max_f(r);
    }
    __syncthreads();
    return r;
}

// Gamma(t) from the P-mode accumulators, Eq. (gammadiscretefinal).
__device__ double gamma_p(const InstParams& ip, const InstState& s, double tc, double hbar) {
    double e = exp(-ip.kappa * tc);
    double sn, cs;
    sincos(ip.wc * tc, &sn, &cs);
    return e * cs * (ip.x0 - 2.0 * s.S / hbar) - e * sn * (ip.p0 - 2.0 * s.C / hbar);
}

// FP64 scalar work after the last block of an instance has finished a stage:
// cavity amplitude (E-mode: d alpha/dt = -(kappa + i omega_c) alpha + i X / hbar,
// Eq. eqmotionaclasical with omega_c -> omega_c - i kappa), accumulators
// (P-mode, Eq. Sdiscrete / Cdiscrete), time, accept / reject and step size.
__device__ void finish_stage(const Plan& P, const Material& mat, const StageArgs& A, const InstParams& ip,
                             InstState& s, double Xsum, float errmax, double* hist, int hcap, int* flags) {
    const double X = Xsum * mat.vc;
    const int k = A.stage;
    const bool ecav = ip.cav_on && A.mode == CAV_E;
    const bool pcav = ip.cav_on && A.mode == CAV_P;
    const int K = A.kind;
    const double dt = s.dt;
    s.X = X;
    if (ecav) {
        // derivative of alpha at this stage
        s.ka_re[k] = -ip.kappa * s.as_re + ip.wc * s.as_im;
        s.ka_im[k] = -ip.kappa * s.as_im - ip.wc * s.as_re + X / mat.hbar;
    }
    const int nst = K == KIND_RK4 ? 4 : 7;
    const bool last = k == nst - 1;
    if (!last) {
        if (ecav) {
            // alpha of the next stage (DP45 stage 7 takes the 5th-order weights)
            const bool to_b = (K == KIND_DP45 && k + 1 == 6);
            double re = s.a_re, im = s.a_im;
            for (int j = 0; j <= k; j++) {
                double w = to_b ? c_bd[1][j] : c_ad[K][k + 1][j];
                re += dt * w * s.ka_re[j];
                im += dt * w * s.ka_im[j];
            }
            s.as_re = re;
            s.as_im = im;
        }
        if (K == KIND_DP45 && k == 0) s.have_k1 = 1;
        return;
    }
    int accept = 1;
    if (K == KIND_DP45) {
        float tol = A.tol;
        accept = errmax <= tol;
        if (!(errmax == errmax)) { accept = 0; atomicOr(flags, FLAG_NAN); }
    }
    if (accept) {
        if (K == KIND_RK4) {
            if (ecav) {
                double re = s.a_re, im = s.a_im;
                for (int j = 0; j < 4; j++) {
                    re += dt * c_bd[0][j] * s.ka_re[j];
                    im += dt * c_bd[0][j] * s.ka_im[j];
                }
                s.a_re = re; s.a_im = im;
            }
        } else {
            s.mcur ^= 1;
            s.k1slot = s.k1slot == 0 ? 6 : 0;
            if (ecav) {
                s.a_re = s.as_re; s.a_im = s.as_im;   // alpha5
                s.ka_re[0] = s.ka_re[6]; s.ka_im[0] = s.ka_im[6];
            }
            if (A.mode == CAV_P) s.have_k1 = 0;   // Gamma at t_n changes with S_n, C_n
        }
        s.t += dt;
        s.tcav += dt;
        s.nacc++;
        if (s.nhist < hcap) hist[s.nhist] = dt;
        else atomicOr(flags, FLAG_HIST_FULL);
        s.nhist++;
        if (pcav) {
            double e = exp(ip.kappa * s.tcav), sn, cs;
            sincos(ip.wc * s.tcav, &sn, &cs);
            s.S += e * sn * X * dt;
            s.C += e * cs * X * dt;
        }
    } else {
        s.nrej++;
    }
    if (K == KIND_DP45) {
        double err = (double)errmax;
        double f = err > 0.0 ? 0.9 * pow((double)A.tol / err, 0.2) : 5.0;
        if (!(f == f)) f = 0.2;
        f = fmin(5.0, fmax(0.2, f));
        double nd = dt * f;
        s.err = err;
        if (s.t_end > 0.0) {
            if (s.t >= s.t_end * (1.0 - 1e-14)) s.done = 1;
            else if (s.t + nd > s.t_end) nd = s.t_end - s.t;
        }
        if (nd < 1e-20 && !s.done) { atomicOr(flags, FLAG_DT_UNDERFLOW); s.done = 1; }
        s.dt = nd;
    }
    if (ecav) {
        if (K == KIND_DP45) {
            s.as_re = s.a_re + s.dt * c_ad[1][1][0] * s.ka_re[0];
            s.as_im = s.a_im + s.dt * c_ad[1][1][0] * s.ka_im[0];
        } else {
            s.as_re = s.a_re; s.as_im = s.a_im;
        }
    }
}

// ---------------------------------------------------------------------------
// x forward: stage input, M = Ms m_s, packed real FFT of length px = 2L.
// R consecutive rows per block; shared memory zs[n][line], line = 3 r + comp.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(512) k_xfwd(Plan P, Buffers Bf, StageArgs A) {
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
    for (int i = threadIdx.x; i < L * ld; i += blockDim.x) zs[i] = make_float2(0.f, 0.f);
    __syncthreads();

    const float4* m0 = Bf.m[st.mcur] + base;
    const int s = A.stage;
    const float dt = (float)st.dt;
    const bool form = !A.field_only && s > 0;
    const bool dp_last = A.kind == KIND_DP45 && s == 6 && !A.field_only;
    const float4* kp[MAX_STAGES - 1];
    float kw[MAX_STAGES - 1], ke[MAX_STAGES - 1];
    int nk = 0;
#pragma unroll
    for (int q = 0; q < MAX_STAGES - 1; q++) { kp[q] = Bf.k[0]; kw[q] = 0.f; ke[q] = 0.f; }
    if (form) {
        for (int j = 0; j < s; j++) {
            float w = dp_last ? c_bf[1][j] : c_af[A.kind][s][j];
            float e = dp_last ? c_ef[j] : 0.f;
            if (w == 0.f && e == 0.f) continue;
            kp[nk] = Bf.k[A.kind == KIND_DP45 ? k_slot(st, j) : j] + base;
            kw[nk] = dt * w;
            ke[nk] = dt * e;
            nk++;
        }
    }
    float4* ms_out = dp_last ? Bf.m[st.mcur ^ 1] + base : Bf.ms + base;
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) {
        float4 v = m0[i];
        if (form) {
            float ax = 0.f, ay = 0.f, az = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
            for (int q = 0; q < MAX_STAGES - 1; q++) {
                if (q < nk) {
                    float4 kj = kp[q][i];
                    ax += kw[q] * kj.x; ay += kw[q] * kj.y; az += kw[q] * kj.z;
                    ex += ke[q] * kj.x; ey += ke[q] * kj.y; ez += ke[q] * kj.z;
                }
            }
            v.x += ax; v.y += ay; v.z += az;
            if (dp_last) {
                // 5th-order solution, renormalised: stage 7 is evaluated there
                float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
                float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                v.x *= inv; v.y *= inv; v.z *= inv;
                Bf.e6[base + i] = make_float4(ex, ey, ez, 0.f);
            }
            ms_out[i] = v;
        }
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
        col_fft<L, false>(v, zs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
        for (int i = 0; i < NPT; i++) zs[col_out_row<L>(j, i) * ld + line] = v[i];
    }
    __syncthreads();

    // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2, O = -i (Z[k] - conj Z[L-k]) / 2
    const int TX = P.TX, lt = P.lt;
    const long long tstride = (long long)P.ny * 3 * TX;
    const int twstep = P.twn / P.px;
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
                float2 wD = cmul(twiddle(Bf.tw, k * twstep, false), D);
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
template <int L>
__global__ void __launch_bounds__(512) k_xinv(Plan P, Material mat, Buffers Bf, StageArgs A) {
    constexpr int NPT = ColShape<L>::NPT, N1 = ColShape<L>::N1;
    extern __shared__ float2 sm[];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma;
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

    // half-spectrum rows X[0..L] of the three components of every row
    const long long tstride = (long long)P.ny * 3 * TX;
    for (int r = 0; r < nr; r++) {
        const int row = row0 + r;
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        const float2* in = Bf.spec + (((long long)b * P.nz + z) * P.NT * P.ny + y) * 3 * TX;
        for (int idx = threadIdx.x; idx < 3 * (L + 1); idx += blockDim.x) {
            const int c = (int)fdiv((unsigned)idx, P.fd_L1), k = idx - c * (L + 1);
            const int t = k >> lt, tx = k & (TX - 1);
            xs[k * ld + 3 * r + c] = in[t * tstride + c * TX + tx];
        }
    }
    for (int i = threadIdx.x; i < nr * nx; i += blockDim.x) mrow[i] = msrc[base + i];
    if (threadIdx.x == 0) {
        double G = 0.0;
        if (ip.cav_on) {
            if (A.mode == CAV_E) G = 2.0 * (A.field_only ? st.a_re : st.as_re);
            else G = gamma_p(ip, st, st.tcav + (A.field_only ? 0.0 : c_cd[K][s] * st.dt), mat.hbar);
        }
        s_gamma = G;
    }
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

    const bool want_demag = A.terms & 1, want_exch = A.terms & 2, want_anis = A.terms & 4,
               want_zee = A.terms & 8, want_cav = A.terms & 16;
    const float G = (float)s_gamma;
    const float bs = (float)ip.brms_scale;
    const float dt = (float)st.dt;
    const bool cav_on = ip.cav_on != 0;
    // outputs of this stage
    const int k1slot = st.k1slot;
    float4* const kout = K == KIND_RK4 ? (s < 3 ? Bf.k[s] : nullptr)
                                       : (s < 6 ? Bf.k[s == 0 ? k1slot : s] : Bf.k[k1slot == 0 ? 6 : 0]);
    const float bex = (float)ip.bext[0], bey = (float)ip.bext[1], bez = (float)ip.bext[2];
    const long long pl = (long long)nx * P.ny;
    double xacc = 0.0;
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
        float px_ = 0.f, py_ = 0.f, pz_ = 0.f;   // coupling profile at this cell
        if (Ms > 0.f) {
            if (want_exch) {
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
            if (want_anis) {
                float mu = m.x * mat.u[0] + m.y * mat.u[1] + m.z * mat.u[2];
                float f = mat.two_ku / Ms * mu;
                Bx += f * mat.u[0]; By += f * mat.u[1]; Bz += f * mat.u[2];
            }
            if (want_zee) { Bx += bex; By += bey; Bz += bez; }
            if (cav_on) {
                if (Bf.prof) { float4 p = __ldg(Bf.prof + (i - cb)); px_ = bs * p.x; py_ = bs * p.y; pz_ = bs * p.z; }
                else { py_ = bs; }
                if (want_cav) { Bx += G * px_; By += G * py_; Bz += G * pz_; }
            }
        }
        if (A.field_only) {
            Bf.fout[i - cb] = make_float4(Bx, By, Bz, 0.f);
            continue;
        }
        // LLG torque, Eq. (llg)
        float cx = m.y * Bz - m.z * By, cy = m.z * Bx - m.x * Bz, cz = m.x * By - m.y * Bx;
        float dx = m.y * cz - m.z * cy, dy = m.z * cx - m.x * cz, dz = m.x * cy - m.y * cx;
        float4 kk = make_float4(mat.pre * (cx + mat.alpha * dx), mat.pre * (cy + mat.alpha * dy),
                                mat.pre * (cz + mat.alpha * dz), 0.f);
        if (!(Ms > 0.f)) kk = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!isfinite(kk.x) || !isfinite(kk.y) || !isfinite(kk.z)) bad = true;
        // m used for the coupling sum of this launch
        float4 mx = m;
        if (K == KIND_RK4) {
            if (s < 3) {
                kout[i] = kk;
            } else {
                float4 m0 = Bf.m[0][i];
                float4 k0 = Bf.k[0][i], k1 = Bf.k[1][i], k2 = Bf.k[2][i];
                float h = dt * (1.f / 6.f);
                float4 mn;
                mn.x = m0.x + h * (k0.x + 2.f * k1.x + 2.f * k2.x + kk.x);
                mn.y = m0.y + h * (k0.y + 2.f * k1.y + 2.f * k2.y + kk.y);
                mn.z = m0.z + h * (k0.z + 2.f * k1.z + 2.f * k2.z + kk.z);
                float r2 = mn.x * mn.x + mn.y * mn.y + mn.z * mn.z;
                float inv = (Ms > 0.f && r2 > 0.f) ? rsqrtf(r2) : 0.f;
                mn.x *= inv; mn.y *= inv; mn.z *= inv;
                mn.w = m0.w;
                Bf.m[0][i] = mn;
                if (A.mode == CAV_P) mx = mn;
            }
        } else {
            if (s < 6) {
                kout[i] = kk;
            } else {
                kout[i] = kk;
                float4 e = Bf.e6[i];
                float c7 = c_ef[6] * dt;
                float exx = e.x + c7 * kk.x, eyy = e.y + c7 * kk.y, ezz = e.z + c7 * kk.z;
                emax = fmaxf(emax, sqrtf(exx * exx + eyy * eyy + ezz * ezz));
            }
        }
        // per-cell product in FP32, accumulated in FP64 (the sum over cells is
        // the quantity that needs the range; FP64 arithmetic is ~1/64 rate here)
        if (cav_on) xacc += (double)(Ms * (mx.x * px_ + mx.y * py_ + mx.z * pz_));
    }
    if (A.field_only) return;
    if (bad) atomicOr(Bf.flags, FLAG_NAN);
    // block partials, then the last block of this instance finishes the stage
    double xb = block_sum_d(xacc, s_red);
    float eb = block_max_f(emax, s_redf);
    const long long pb = (long long)b * P.nblk;
    if (threadIdx.x == 0) {
        Bf.xpart[pb + blockIdx.x] = xb;
        Bf.epart[pb + blockIdx.x] = eb;
        __threadfence();
        unsigned prev = atomicAdd(Bf.counter + b, 1u);
        s_last = prev == (unsigned)(P.nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double xsum = 0.0;
    float em = 0.f;
    for (int r = threadIdx.x; r < P.nblk; r += blockDim.x) {
        xsum += __ldcg(Bf.xpart + pb + r);
        em = fmaxf(em, __ldcg(Bf.epart + pb + r));
    }
    xsum = block_sum_d(xsum, s_red);
    em = block_max_f(em, s_redf);
    if (threadIdx.x == 0) {
        InstState ns = Bf.st[b];
        finish_stage(P, mat, A, ip, ns, xsum, em, Bf.hist + (long long)b * Bf.hcap, Bf.hcap, Bf.flags);
        Bf.st[b] = ns;
        Bf.counter[b] = 0u;
    }
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

// m of one instance (or all) from an N x 3 float array: FP64 normalisation,
// zero in empty cells, Ms into w.
__global__ void k_set_m(float4* m, const float* src, const float* ms, long long N, int b0, int nb) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double x = src[3 * i], y = src[3 * i + 1], zz = src[3 * i + 2];
    double r = sqrt(x * x + y * y + zz * zz);
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

__global__ void k_set_dt(InstState* st, int B, double dt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) st[b].dt = dt;
}

// ---------------------------------------------------------------------------
// host-side launchers (called from the C ABI)
// ---------------------------------------------------------------------------
void upload_tableaux() {
    float af[2][MAX_STAGES][MAX_STAGES] = {};
    double ad[2][MAX_STAGES][MAX_STAGES] = {};
    float bf[2][MAX_STAGES] = {};
    double bd[2][MAX_STAGES] = {};
    double cd[2][MAX_STAGES] = {};
    float ef[MAX_STAGES] = {};
    // classic RK4
    ad[0][1][0] = 0.5; ad[0][2][1] = 0.5; ad[0][3][2] = 1.0;
    double b4[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    double c4[4] = {0.0, 0.5, 0.5, 1.0};
    for (int j = 0; j < 4; j++) { bd[0][j] = b4[j]; cd[0][j] = c4[j]; }
    // Dormand & Prince (1980) RK5(4)7FM
    const double A5[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {1.0 / 5, 0, 0, 0, 0, 0},
        {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
        {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
        {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
        {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
        {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
    const double B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
    const double B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};
    const double C5[7] = {0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1, 1};
    for (int s = 0; s < 7; s++)
        for (int j = 0; j < 6; j++) ad[1][s][j] = A5[s][j];
    for (int j = 0; j < 7; j++) { bd[1][j] = B5[j]; cd[1][j] = C5[j]; ef[j] = (float)(B5[j] - B4[j]); }
    for (int k = 0; k < 2; k++) {
        for (int s = 0; s < 7; s++) for (int j = 0; j < 7; j++) af[k][s][j] = (float)ad[k][s][j];
        for (int j = 0; j < 7; j++) bf[k][j] = (float)bd[k][j];
    }
    cudaMemcpyToSymbol(c_af, af, sizeof(af));
    cudaMemcpyToSymbol(c_ad, ad, sizeof(ad));
    cudaMemcpyToSymbol(c_bf, bf, sizeof(bf));
    cudaMemcpyToSymbol(c_bd, bd, sizeof(bd));
    cudaMemcpyToSymbol(c_cd, cd, sizeof(cd));
    cudaMemcpyToSymbol(c_ef, ef, sizeof(ef));
}

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

size_t xfwd_smem(const Plan& P) { return (size_t)P.L * xpass_ld(P.R) * sizeof(float2); }

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
    switch (P.L) {
#define MMCQ_CASE(Lv) case Lv: k_xinv<Lv><<<grid, th, sm, s>>>(P, mat, Bf, A); break;
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_set_m(float4* m, const float* src, const float* ms, long long N, int b0, int nb, cudaStream_t s) {
    k_set_m<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(m, src, ms, N, b0, nb);
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
    if ((e = upload_tw32()) != cudaSuccess) return e;
    const int lim = 200 * 1024;
#define MMCQ_CASE(Lv)                                                                                         \
    if ((e = cudaFuncSetAttribute(k_xfwd<Lv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) \
        return e;                                                                                             \
    if ((e = cudaFuncSetAttribute(k_xinv<Lv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) \
        return e;
    MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
    return col_init();
}

}  // namespace mq
