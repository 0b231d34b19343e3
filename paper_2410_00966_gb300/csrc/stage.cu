// Stage kernels of the LLG + cavity hot path (Mumax3-cQED, arXiv 2410.00966).
//
// One field evaluation (one Runge-Kutta stage) is three kinds of launch:
//   k_xfwd : stage input m_s = m0 + dt sum_j a_sj k_j (Eq. llg integrated by
//            RK4 / Dormand-Prince), M = Ms m_s, zero-padded real-to-complex FFT
//            along x, written to a tiled half-spectrum.
//   k_col  : FFT along y (and z) of a tile of kx columns, the pointwise product
//            with the symmetric demag kernel H = N M (6 real components,
//            mirror-reduced storage), inverse FFT.  2-D grids do everything
//            in one launch; 3-D grids use y-forward, z-convolve, y-inverse.
//   k_xinv : complex-to-real inverse FFT along x giving B_demag, then per cell
//            exchange + anisotropy + Zeeman + cavity B_rms Gamma (Sec. 2.1
//            field terms, Eq. bcav), the LLG torque (Eq. llg), the RK
//            bookkeeping, and FP64 block partials of the coupling sum
//            X = V_c sum_i Ms_i m_i . B_rms,i (Eq. gammafinal).  The last block
//            of each instance to finish reduces the partials in a fixed order
//            and advances the cavity amplitude / step-size controller in FP64.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"

namespace mq {

// Butcher tableaux: [kind][stage][j].
__constant__ float c_af[2][MAX_STAGES][MAX_STAGES];
__constant__ double c_ad[2][MAX_STAGES][MAX_STAGES];
__constant__ float c_bf[2][MAX_STAGES];    // weights of the propagated solution
__constant__ double c_bd[2][MAX_STAGES];
__constant__ double c_cd[2][MAX_STAGES];   // stage times
__constant__ float c_ef[MAX_STAGES];       // DP45 error weights b5 - b4

// Whether this instance does nothing in this launch.
__device__ __forceinline__ bool stage_skips(const InstState& s, const StageArgs& A) {
    if (A.field_only) return false;
    if (s.done) return true;
    if (A.kind == KIND_DP45 && A.stage == 0 && s.have_k1) return true;
    return false;
}

__device__ __forceinline__ int k_slot(const InstState& s, int j) {
    // DP45: stage 1 lives in k1slot (FSAL swap between buffers 0 and 6)
    return j == 0 ? s.k1slot : j;
}

// ---------------------------------------------------------------------------
// x forward: stage input, M = Ms m_s, packed real FFT of length px.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MAX_THREADS) k_xfwd(Plan P, Buffers Bf, StageArgs A) {
    extern __shared__ float2 sm[];
    const int row = blockIdx.x;
    const int b = A.inst0 + blockIdx.y;
    const InstState st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const int L = P.L;
    const int y = row % P.ny, z = row / P.ny;
    const long long base = (long long)b * P.N + (long long)row * P.nx;
    float2* zs = sm;  // [3][L]
    for (int i = threadIdx.x; i < 3 * L; i += blockDim.x) zs[i] = make_float2(0.f, 0.f);
    __syncthreads();

    const float4* m0 = Bf.m[st.mcur] + base;
    const int s = A.stage;
    const float dt = (float)st.dt;
    const bool form = !A.field_only && s > 0;
    const bool dp_last = A.kind == KIND_DP45 && s == 6 && !A.field_only;
    for (int x = threadIdx.x; x < P.nx; x += blockDim.x) {
        float4 v = m0[x];
        if (form) {
            float ax = 0.f, ay = 0.f, az = 0.f;
            float ex = 0.f, ey = 0.f, ez = 0.f;
            for (int j = 0; j < s; j++) {
                float w = dp_last ? c_bf[1][j] : c_af[A.kind][s][j];
                float e = dp_last ? c_ef[j] : 0.f;
                if (w == 0.f && e == 0.f) continue;   // uniform: skips the load
                float4 kj = Bf.k[A.kind == KIND_DP45 ? k_slot(st, j) : j][base + x];
                ax += w * kj.x; ay += w * kj.y; az += w * kj.z;
                ex += e * kj.x; ey += e * kj.y; ez += e * kj.z;
            }
            v.x += dt * ax; v.y += dt * ay; v.z += dt * az;
            if (dp_last) {
                // 5th-order solution, renormalised: stage 7 is evaluated there
                float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
                float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                v.x *= inv; v.y *= inv; v.z *= inv;
                Bf.m[st.mcur ^ 1][base + x] = v;
                Bf.e6[base + x] = make_float4(dt * ex, dt * ey, dt * ez, 0.f);
            } else {
                Bf.ms[base + x] = v;
            }
        }
        float Mx = v.w * v.x, My = v.w * v.y, Mz = v.w * v.z;
        int n = x >> 1;
        if (x & 1) { zs[n].y = Mx; zs[L + n].y = My; zs[2 * L + n].y = Mz; }
        else { zs[n].x = Mx; zs[L + n].x = My; zs[2 * L + n].x = Mz; }
    }
    __syncthreads();
    block_fft<false>(zs, L, 3, 1, L, false, Bf.tw, P.twn);

    // X[k] = E[k] + W^k O[k], E = (Z[k] + conj Z[L-k]) / 2, O = -i (Z[k] - conj Z[L-k]) / 2
    const int TX = P.TX;
    float2* out = Bf.spec + (((long long)b * P.nz + z) * P.NT * P.ny + y) * 3 * TX;
    const long long tstride = (long long)P.ny * 3 * TX;
    const int twstep = P.twn / P.px;
    const int W3 = P.NT * 3 * TX;
    for (int idx = threadIdx.x; idx < W3; idx += blockDim.x) {
        int t = idx / (3 * TX);
        int rem = idx - t * 3 * TX;
        int c = rem / TX;
        int tx = rem - c * TX;
        int k = t * TX + tx;
        float2 X = make_float2(0.f, 0.f);
        if (k <= L) {
            float2 Zk = zs[c * L + (k == L ? 0 : k)];
            float2 Zc = conjf2(zs[c * L + (k == 0 ? 0 : L - k)]);
            float2 E = make_float2(0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y));
            float2 D = make_float2(0.5f * (Zk.x - Zc.x), 0.5f * (Zk.y - Zc.y));
            float2 wD = cmul(twiddle(Bf.tw, k * twstep, false), D);
            X = make_float2(E.x + wD.y, E.y - wD.x);
        }
        out[t * tstride + c * TX + tx] = X;
    }
}

// ---------------------------------------------------------------------------
// column FFT / demag product along y or z on a tile of TX kx columns.
// ---------------------------------------------------------------------------
struct ColArgs {
    const float2* in;
    float2* out;
    long long in_b, in_o, in_t, in_r;    // strides (float2) of instance, outer index, tile, row
    long long out_b, out_o, out_t, out_r;
    int P;          // transform length
    int n_in;       // rows read (the rest are zero padding)
    int n_out;      // rows written
    int fwd, mult, inv;
    int ncomp;      // 3: all components per block (needed for the product); 1: one each
    int ky_is_row;  // product index: (ky, kz) = (row, 0) if set, else (outer, row)
};

__device__ __forceinline__ void demag_product(const Plan& P, const float* __restrict__ kern, int kx, int ky,
                                              int kz, float2& mx, float2& my, float2& mz) {
    if (kx >= P.hx) { mx = my = mz = make_float2(0.f, 0.f); return; }
    float sy = 1.f, sz = 1.f;
    int kyr = ky, kzr = kz;
    if (ky > P.py / 2) { kyr = P.py - ky; sy = -1.f; }
    if (kz > P.pz / 2) { kzr = P.pz - kz; sz = -1.f; }
    const float* K = kern + (((long long)kzr * P.hyk + kyr) * (P.NT * P.TX) + kx) * 6;
    float xx = __ldg(K), yy = __ldg(K + 1), zz = __ldg(K + 2);
    float xy = sy * __ldg(K + 3), xz = sz * __ldg(K + 4), yz = sy * sz * __ldg(K + 5);
    float2 hx = make_float2(xx * mx.x + xy * my.x + xz * mz.x, xx * mx.y + xy * my.y + xz * mz.y);
    float2 hy = make_float2(xy * mx.x + yy * my.x + yz * mz.x, xy * mx.y + yy * my.y + yz * mz.y);
    float2 hz = make_float2(xz * mx.x + yz * my.x + zz * mz.x, xz * mx.y + yz * my.y + zz * mz.y);
    mx = hx; my = hy; mz = hz;
}

__global__ void __launch_bounds__(MAX_THREADS) k_col(Plan P, Buffers Bf, StageArgs A, ColArgs C) {
    extern __shared__ float2 sm[];
    const int t = blockIdx.x;
    const int outer = blockIdx.y;
    const int bz = blockIdx.z;
    const int b = A.inst0 + (C.ncomp == 3 ? bz : bz / 3);
    const int c0 = C.ncomp == 3 ? 0 : bz % 3;
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = P.TX;
    const int rw = C.ncomp * TX;   // float2 per row in shared memory
    const float2* in = C.in + b * C.in_b + outer * C.in_o + t * C.in_t + c0 * TX;
    float2* out = C.out + b * C.out_b + outer * C.out_o + t * C.out_t + c0 * TX;
    // load rows (contiguous rw values per row), zero-pad to P rows
    for (int i = threadIdx.x; i < C.P * rw; i += blockDim.x) {
        int r = i / rw, e = i - r * rw;
        sm[i] = r < C.n_in ? in[r * C.in_r + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (C.fwd) block_fft<true>(sm, C.P, rw, rw, 1, false, Bf.tw, P.twn);
    if (C.mult) {
        for (int i = threadIdx.x; i < C.P * TX; i += blockDim.x) {
            int r = i / TX, tx = i - r * TX;
            float2* p = sm + r * rw + tx;
            float2 mx = p[0], my = p[TX], mz = p[2 * TX];
            int ky = C.ky_is_row ? r : outer;
            int kz = C.ky_is_row ? 0 : r;
            demag_product(P, Bf.kern, t * TX + tx, ky, kz, mx, my, mz);
            p[0] = mx; p[TX] = my; p[2 * TX] = mz;
        }
        __syncthreads();
    }
    if (C.inv) block_fft<true>(sm, C.P, rw, rw, 1, true, Bf.tw, P.twn);
    for (int i = threadIdx.x; i < C.n_out * rw; i += blockDim.x) {
        int r = i / rw, e = i - r * rw;
        out[r * C.out_r + e] = sm[i];
    }
}

// ---------------------------------------------------------------------------
// x inverse + local fields + torque + RK bookkeeping + cavity reduction.
// ---------------------------------------------------------------------------
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

__global__ void __launch_bounds__(MAX_THREADS) k_xinv(Plan P, Material mat, Buffers Bf, StageArgs A) {
    extern __shared__ float2 sm[];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma;
    __shared__ int s_last;
    const int row = blockIdx.x;
    const int b = A.inst0 + blockIdx.y;
    const InstState st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const InstParams ip = Bf.ip[b];
    const int L = P.L, TX = P.TX, nx = P.nx;
    const int y = row % P.ny, z = row / P.ny;
    const long long cb = (long long)b * P.N;
    const long long base = cb + (long long)row * nx;
    const int s = A.stage;
    const int K = A.kind;
    float2* xs = sm;                                   // [3][L+1]
    float4* mrow = reinterpret_cast<float4*>(sm + 3 * (L + 1) + ((3 * (L + 1)) & 1));  // [nx]

    // which buffer holds the stage input m_s
    const float4* msrc;
    if (A.field_only || s == 0) msrc = Bf.m[st.mcur];
    else if (K == KIND_DP45 && s == 6) msrc = Bf.m[st.mcur ^ 1];
    else msrc = Bf.ms;

    // load the half spectrum row X[0..L] of the three components
    const float2* in = Bf.spec + (((long long)b * P.nz + z) * P.NT * P.ny + y) * 3 * TX;
    const long long tstride = (long long)P.ny * 3 * TX;
    for (int idx = threadIdx.x; idx < 3 * (L + 1); idx += blockDim.x) {
        int c = idx / (L + 1), k = idx - c * (L + 1);
        int t = k / TX, tx = k - t * TX;
        xs[idx] = in[t * tstride + c * TX + tx];
    }
    for (int x = threadIdx.x; x < nx; x += blockDim.x) mrow[x] = msrc[base + x];
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
    for (int idx = threadIdx.x; idx < 3 * (L / 2 + 1); idx += blockDim.x) {
        int c = idx / (L / 2 + 1), k = idx - c * (L / 2 + 1);
        float2* X = xs + c * (L + 1);
        int kk = L - k;
        float2 a = X[k], bq = X[kk];
        // Z[k]
        float2 ca = conjf2(bq);
        float2 sum = cadd(a, ca), dif = csub(a, ca);
        float2 w = twiddle(Bf.tw, k * twstep, true);
        float2 wd = cmul(w, dif);
        float2 zk = make_float2(sum.x - wd.y, sum.y + wd.x);   // sum + i wd
        if (k != 0 && kk != k) {
            float2 cb2 = conjf2(a);
            float2 sum2 = cadd(bq, cb2), dif2 = csub(bq, cb2);
            float2 w2 = twiddle(Bf.tw, kk * twstep, true);
            float2 wd2 = cmul(w2, dif2);
            X[kk] = make_float2(sum2.x - wd2.y, sum2.y + wd2.x);
        }
        X[k] = zk;
    }
    __syncthreads();
    block_fft<false>(xs, L, 3, 1, L + 1, true, Bf.tw, P.twn);

    const bool want_demag = A.terms & 1, want_exch = A.terms & 2, want_anis = A.terms & 4,
               want_zee = A.terms & 8, want_cav = A.terms & 16;
    const float G = (float)s_gamma;
    const float bs = (float)ip.brms_scale;
    const float dt = (float)st.dt;
    double xacc = 0.0;
    float emax = 0.f;
    bool bad = false;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const long long i = base + x;
        float4 m = mrow[x];
        const float Ms = m.w;
        float Bx = 0.f, By = 0.f, Bz = 0.f;
        if (want_demag) {
            float2 zx = xs[x >> 1], zy = xs[(L + 1) + (x >> 1)], zz = xs[2 * (L + 1) + (x >> 1)];
            if (x & 1) { Bx = zx.y; By = zy.y; Bz = zz.y; }
            else { Bx = zx.x; By = zy.x; Bz = zz.x; }
        }
        float px_ = 0.f, py_ = 0.f, pz_ = 0.f;   // coupling profile at this cell
        if (Ms > 0.f) {
            if (want_exch) {
                float hx = 0.f, hy = 0.f, hz = 0.f;
                float4 q;
                if (x > 0) { q = mrow[x - 1]; if (q.w > 0.f) { hx += mat.exch[0] * (q.x - m.x); hy += mat.exch[0] * (q.y - m.y); hz += mat.exch[0] * (q.z - m.z); } }
                if (x + 1 < nx) { q = mrow[x + 1]; if (q.w > 0.f) { hx += mat.exch[0] * (q.x - m.x); hy += mat.exch[0] * (q.y - m.y); hz += mat.exch[0] * (q.z - m.z); } }
                if (y > 0) { q = __ldg(msrc + i - nx); if (q.w > 0.f) { hx += mat.exch[1] * (q.x - m.x); hy += mat.exch[1] * (q.y - m.y); hz += mat.exch[1] * (q.z - m.z); } }
                if (y + 1 < P.ny) { q = __ldg(msrc + i + nx); if (q.w > 0.f) { hx += mat.exch[1] * (q.x - m.x); hy += mat.exch[1] * (q.y - m.y); hz += mat.exch[1] * (q.z - m.z); } }
                const long long pl = (long long)nx * P.ny;
                if (z > 0) { q = __ldg(msrc + i - pl); if (q.w > 0.f) { hx += mat.exch[2] * (q.x - m.x); hy += mat.exch[2] * (q.y - m.y); hz += mat.exch[2] * (q.z - m.z); } }
                if (z + 1 < P.nz) { q = __ldg(msrc + i + pl); if (q.w > 0.f) { hx += mat.exch[2] * (q.x - m.x); hy += mat.exch[2] * (q.y - m.y); hz += mat.exch[2] * (q.z - m.z); } }
                float inv = 1.f / Ms;
                Bx += hx * inv; By += hy * inv; Bz += hz * inv;
            }
            if (want_anis) {
                float mu = m.x * mat.u[0] + m.y * mat.u[1] + m.z * mat.u[2];
                float f = mat.two_ku / Ms * mu;
                Bx += f * mat.u[0]; By += f * mat.u[1]; Bz += f * mat.u[2];
            }
            if (want_zee) {
                Bx += (float)ip.bext[0]; By += (float)ip.bext[1]; Bz += (float)ip.bext[2];
            }
            if (ip.cav_on) {
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
                Bf.k[s][i] = kk;
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
                Bf.k[k_slot(st, s)][i] = kk;
            } else {
                Bf.k[st.k1slot == 0 ? 6 : 0][i] = kk;
                float4 e = Bf.e6[i];
                float c7 = c_ef[6] * dt;
                float exx = e.x + c7 * kk.x, eyy = e.y + c7 * kk.y, ezz = e.z + c7 * kk.z;
                emax = fmaxf(emax, sqrtf(exx * exx + eyy * eyy + ezz * ezz));
            }
        }
        if (ip.cav_on) xacc += (double)Ms * ((double)mx.x * px_ + (double)mx.y * py_ + (double)mx.z * pz_);
    }
    if (A.field_only) return;
    if (bad) atomicOr(Bf.flags, FLAG_NAN);
    // block partials, then the last block of this instance finishes the stage
    double xb = block_sum_d(xacc, s_red);
    float eb = block_max_f(emax, s_redf);
    const long long pb = (long long)b * P.nrows;
    if (threadIdx.x == 0) {
        Bf.xpart[pb + row] = xb;
        Bf.epart[pb + row] = eb;
        __threadfence();
        unsigned prev = atomicAdd(Bf.counter + b, 1u);
        s_last = prev == (unsigned)(P.nrows - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double xsum = 0.0;
    float em = 0.f;
    for (int r = threadIdx.x; r < P.nrows; r += blockDim.x) {
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

static int threads_for(int nlines, int L, int minimum) {
    int slots = (nlines * L + 3) / 4;
    int t = (slots + 1) / 2;
    t = ((t + 31) / 32) * 32;
    if (t < minimum) t = minimum;
    if (t > MAX_THREADS) t = MAX_THREADS;
    return t;
}

bool fft_fits(int nlines, int L) { return (nlines * L + 3) / 4 <= MAX_SLOTS * MAX_THREADS; }

size_t xinv_smem(const Plan& P) {
    size_t n2 = 3 * (size_t)(P.L + 1);
    n2 += n2 & 1;
    return n2 * sizeof(float2) + (size_t)P.nx * sizeof(float4);
}

cudaError_t launch_xfwd(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s) {
    int th = threads_for(3, P.L, 64);
    size_t sm = 3 * (size_t)P.L * sizeof(float2);
    dim3 grid(P.nrows, nb);
    k_xfwd<<<grid, th, sm, s>>>(P, Bf, A);
    return cudaGetLastError();
}

cudaError_t launch_xinv(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A, int nb,
                        cudaStream_t s) {
    int th = threads_for(3, P.L, 64);
    dim3 grid(P.nrows, nb);
    k_xinv<<<grid, th, xinv_smem(P), s>>>(P, mat, Bf, A);
    return cudaGetLastError();
}

static cudaError_t launch_col(const Plan& P, const Buffers& Bf, const StageArgs& A, const ColArgs& C,
                              int outer, int nb, cudaStream_t s) {
    int rw = C.ncomp * P.TX;
    int th = threads_for(rw, C.P, 32);
    size_t sm = (size_t)C.P * rw * sizeof(float2);
    dim3 grid(P.NT, outer, nb * (C.ncomp == 3 ? 1 : 3));
    k_col<<<grid, th, sm, s>>>(P, Bf, A, C);
    return cudaGetLastError();
}

// Layout strides of the tiled spectra.
static void spec_strides(const Plan& P, int rows, long long& sb, long long& sz, long long& st, long long& sr) {
    sr = 3LL * P.TX;                    // one row (ky or y) of a tile
    st = (long long)rows * sr;          // one tile
    sz = (long long)P.NT * st;          // one z plane
    sb = (long long)P.nz * sz;          // one instance
}

// One launch of the demag convolution: part 0 = 2-D (fwd y, product, inv y);
// 3-D: part 1 = forward y, 2 = z forward / product / z inverse, 3 = inverse y.
cudaError_t launch_conv_part(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s, int part) {
    long long sb, sz, st, sr, tb, tz, tt, tr;
    spec_strides(P, P.ny, sb, sz, st, sr);
    spec_strides(P, P.py, tb, tz, tt, tr);
    ColArgs C{};
    int outer = 1;
    if (part == 0) {
        C.in = Bf.spec; C.out = Bf.spec;
        C.in_b = C.out_b = sb; C.in_o = C.out_o = 0; C.in_t = C.out_t = st; C.in_r = C.out_r = sr;
        C.P = P.py; C.n_in = P.ny; C.n_out = P.ny;
        C.fwd = 1; C.mult = 1; C.inv = 1; C.ncomp = 3; C.ky_is_row = 1;
    } else if (part == 1) {
        C.in = Bf.spec; C.out = Bf.spec2;
        C.in_b = sb; C.in_o = sz; C.in_t = st; C.in_r = sr;
        C.out_b = tb; C.out_o = tz; C.out_t = tt; C.out_r = tr;
        C.P = P.py; C.n_in = P.ny; C.n_out = P.py; C.fwd = 1; C.ncomp = 1;
        outer = P.nz;
    } else if (part == 2) {
        C.in = Bf.spec2; C.out = Bf.spec2;
        C.in_b = C.out_b = tb; C.in_o = C.out_o = tr; C.in_t = C.out_t = tt; C.in_r = C.out_r = tz;
        C.P = P.pz; C.n_in = P.nz; C.n_out = P.nz; C.fwd = 1; C.mult = 1; C.inv = 1; C.ncomp = 3; C.ky_is_row = 0;
        outer = P.py;
    } else {
        C.in = Bf.spec2; C.out = Bf.spec;
        C.in_b = tb; C.in_o = tz; C.in_t = tt; C.in_r = tr;
        C.out_b = sb; C.out_o = sz; C.out_t = st; C.out_r = sr;
        C.P = P.py; C.n_in = P.py; C.n_out = P.ny; C.inv = 1; C.ncomp = 1;
        outer = P.nz;
    }
    return launch_col(P, Bf, A, C, outer, nb, s);
}

cudaError_t launch_convolution(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s) {
    if (P.nz == 1) return launch_conv_part(P, Bf, A, nb, s, 0);
    cudaError_t e;
    for (int part = 1; part <= 3; part++)
        if ((e = launch_conv_part(P, Bf, A, nb, s, part)) != cudaSuccess) return e;
    return cudaSuccess;
}

int convolution_launches(const Plan& P) { return P.nz == 1 ? 1 : 3; }

bool col_fits(const Plan& P) {
    if (P.nz == 1) return fft_fits(3 * P.TX, P.py) && (size_t)P.py * 3 * P.TX * 8 <= 200 * 1024;
    return fft_fits(P.TX, P.py) && (size_t)P.py * P.TX * 8 <= 200 * 1024 && fft_fits(3 * P.TX, P.pz) &&
           (size_t)P.pz * 3 * P.TX * 8 <= 200 * 1024;
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

cudaError_t set_smem_limits() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_xfwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_xinv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_col, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace mq
