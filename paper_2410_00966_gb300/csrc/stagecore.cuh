// Device code shared by the stage kernels (stage.cu): Runge-Kutta
// tableaux, the per-cell field / torque / RK update, the FP64 block
// reductions and the per-instance finisher.  Included by each translation
// unit; constant-memory tables are per unit and filled by upload_tableaux().
#pragma once

#include <math.h>

#include "common.cuh"
#include "kern_common.cuh"

namespace mq {

// Butcher tableaux: [kind][stage][j].
static __constant__ float c_af[2][MAX_STAGES][MAX_STAGES];
static __constant__ double c_ad[2][MAX_STAGES][MAX_STAGES];
static __constant__ float c_bf[2][MAX_STAGES];    // weights of the propagated solution
static __constant__ double c_bd[2][MAX_STAGES];
static __constant__ double c_cd[2][MAX_STAGES];   // stage times
static __constant__ float c_ef[MAX_STAGES];       // DP45 error weights b5 - b4

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
// Fixed-shape block reductions (deterministic for a given blockDim).
static __device__ double block_sum_d(double v, double* red) {
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
static __device__ float block_max_f(float v, float* red) {
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

// Gamma_k(t) from the P-mode accumulators, Eq. (gammadiscretefinal).
static __device__ double gamma_p(const InstParams& ip, const InstState& s, int k, double tc, double hbar) {
    double e = exp(-ip.kappa[k] * tc);
    double sn, cs;
    sincos(ip.wc[k] * tc, &sn, &cs);
    return e * cs * (ip.x0[k] - 2.0 * s.S[k] / hbar) - e * sn * (ip.p0[k] - 2.0 * s.C[k] / hbar);
}

// FP64 scalar work after the last block of an instance has finished a stage:
// for every cavity mode k the amplitude (E-mode: d alpha_k/dt =
// -(kappa_k + i omega_k) alpha_k + i X_k / hbar, Eq. eqmotionaclasical with
// omega_c -> omega_c - i kappa) or the accumulators (P-mode, Eq. Sdiscrete /
// Cdiscrete); then time, accept / reject and step size.  Xsum[k] holds the
// coupling sums without V_c.
static __device__ void finish_stage(const Plan& P, const Material& mat, const StageArgs& A, const InstParams& ip,
                             InstState& s, const double* Xsum, float errmax, double* hist, int hcap, int* flags,
                             const double* msum = nullptr, double* mhist = nullptr) {
    const int k = A.stage;
    const int K = A.kind;
    const int nm = A.nmodes;
    const double dt = s.dt;
    for (int q = 0; q < nm; q++) {
        const double X = Xsum[q] * mat.vc;
        s.X[q] = X;
        if (ip.cav_on[q] && A.mode == CAV_E) {
            // derivative of alpha_q at this stage
            s.ka_re[q][k] = -ip.kappa[q] * s.as_re[q] + ip.wc[q] * s.as_im[q];
            s.ka_im[q][k] = -ip.kappa[q] * s.as_im[q] - ip.wc[q] * s.as_re[q] + X / mat.hbar;
        }
    }
    const int nst = K == KIND_RK4 ? 4 : 7;
    const bool last = k == nst - 1;
    if (!last) {
        // alpha of the next stage (DP45 stage 7 takes the 5th-order weights)
        const bool to_b = (K == KIND_DP45 && k + 1 == 6);
        for (int q = 0; q < nm; q++) {
            if (!ip.cav_on[q] || A.mode != CAV_E) continue;
            double re = s.a_re[q], im = s.a_im[q];
            for (int j = 0; j <= k; j++) {
                double w = to_b ? c_bd[1][j] : c_ad[K][k + 1][j];
                re += dt * w * s.ka_re[q][j];
                im += dt * w * s.ka_im[q][j];
            }
            s.as_re[q] = re;
            s.as_im[q] = im;
        }
        if (K == KIND_DP45 && k == 0) s.have_k1 = 1;
        return;
    }
    int accept = 1;
    if (K == KIND_DP45) {
        float tol = A.tol;
        if (s.poison || !(errmax == errmax)) errmax = INFINITY;
        accept = errmax <= tol;
    }
    if (accept) {
        if (K == KIND_RK4) {
            for (int q = 0; q < nm; q++) {
                if (!ip.cav_on[q] || A.mode != CAV_E) continue;
                double re = s.a_re[q], im = s.a_im[q];
                for (int j = 0; j < 4; j++) {
                    re += dt * c_bd[0][j] * s.ka_re[q][j];
                    im += dt * c_bd[0][j] * s.ka_im[q][j];
                }
                s.a_re[q] = re; s.a_im[q] = im;
            }
        } else {
            s.mcur ^= 1;
            s.k1slot = s.k1slot == 0 ? 6 : 0;
            for (int q = 0; q < nm; q++) {
                if (!ip.cav_on[q] || A.mode != CAV_E) continue;
                s.a_re[q] = s.as_re[q]; s.a_im[q] = s.as_im[q];   // alpha5
                s.ka_re[q][0] = s.ka_re[q][6]; s.ka_im[q][0] = s.ka_im[q][6];
            }
            if (A.mode == CAV_P) s.have_k1 = 0;   // Gamma at t_n changes with S_n, C_n
        }
        s.t += dt;
        s.tcav += dt;
        s.nacc++;
        if (s.nhist < hcap) hist[s.nhist] = dt;
        else atomicOr(flags, FLAG_HIST_FULL);
        s.nhist++;
        if (A.record > 0 && msum && mhist && s.nacc % A.record == 0) {
            if (s.nmh < hcap) {
                double* e = mhist + 4 * s.nmh;
                e[0] = s.t;
                for (int c = 0; c < 3; c++) e[1 + c] = msum[c] * ip.inv_nmag;
            } else {
                atomicOr(flags, FLAG_HIST_FULL);
            }
            s.nmh++;
        }
        if (A.mode == CAV_P) {
            for (int q = 0; q < nm; q++) {
                if (!ip.cav_on[q]) continue;
                double e = exp(ip.kappa[q] * s.tcav), sn, cs;
                sincos(ip.wc[q] * s.tcav, &sn, &cs);
                s.S[q] += e * sn * s.X[q] * dt;
                s.C[q] += e * cs * s.X[q] * dt;
            }
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
        s.poison = 0;
        if (s.t_end > 0.0) {
            if (s.t >= s.t_end * (1.0 - 1e-14)) s.done = 1;
            else if (s.t + nd > s.t_end) nd = s.t_end - s.t;
        }
        if (nd < 1e-20 && !s.done) { atomicOr(flags, FLAG_DT_UNDERFLOW); s.done = 1; }
        s.dt = nd;
    }
    for (int q = 0; q < nm; q++) {
        if (!ip.cav_on[q] || A.mode != CAV_E) continue;
        if (K == KIND_DP45) {
            s.as_re[q] = s.a_re[q] + s.dt * c_ad[1][1][0] * s.ka_re[q][0];
            s.as_im[q] = s.a_im[q] + s.dt * c_ad[1][1][0] * s.ka_im[q][0];
        } else {
            s.as_re[q] = s.a_re[q]; s.as_im[q] = s.a_im[q];
        }
    }
}

static void upload_tableaux() {
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


// Stage input m_s = m0 + dt sum_j a_sj k_j of the Runge-Kutta stage being
// evaluated (Eq. llg integrated by RK4 / Dormand-Prince).  At the last
// Dormand-Prince stage the 5th-order solution is formed, renormalised and
// stored as the candidate, with the partial error dt sum_j e_j k_j.
// Weights are indexed by compile-time stage numbers only (registers, no
// stack), and the k buffers are read through the kernel's parameter block.
struct StageInput {
    float kw[MAX_STAGES - 1], ke[MAX_STAGES - 1];
    const float4* k0;    // buffer of stage 1 (DP45: first-same-as-last slot)
    long long base;
    bool form, dp_last;
    float4* out;         // where m_s is written (stage > 0)
    float4* e6;

    // apply() takes the cell index relative to `base` (the block's first cell).
    __device__ __forceinline__ void init(const Buffers& Bf, const StageArgs& A, const InstState& st, long long base_) {
        const int s = A.stage;
        const float dt = (float)st.dt;
        base = base_;
        form = !A.field_only && s > 0;
        dp_last = A.kind == KIND_DP45 && s == 6 && !A.field_only;
#pragma unroll
        for (int j = 0; j < MAX_STAGES - 1; j++) {
            const bool on = form && j < s;
            kw[j] = on ? dt * (dp_last ? c_bf[1][j] : c_af[A.kind][s][j]) : 0.f;
            ke[j] = on && dp_last ? dt * c_ef[j] : 0.f;
        }
        k0 = (A.kind == KIND_DP45 ? Bf.k[st.k1slot] : Bf.k[0]) + base;
        out = (dp_last ? Bf.m[st.mcur ^ 1] : Bf.ms) + base;
        e6 = Bf.e6 + base;
    }

    // Ask L2 for the k rows this block will read ([base, base + bytes) of each).
    __device__ __forceinline__ void prefetch(const Buffers& Bf, unsigned bytes) const {
        if (!form) return;
#pragma unroll
        for (int q = 0; q < MAX_STAGES - 1; q++)
            if (kw[q] != 0.f || ke[q] != 0.f) prefetch_l2(q == 0 ? k0 : Bf.k[q] + base, bytes);
    }

    // v = m0[i] on entry; m_s on return (written to out, and e6 at the last DP stage)
    __device__ __forceinline__ void apply(const Buffers& Bf, float4& v, int i) const {
        if (!form) return;
        float ax = 0.f, ay = 0.f, az = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
        for (int q = 0; q < MAX_STAGES - 1; q++) {
            if (kw[q] != 0.f || ke[q] != 0.f) {
                const float4 kj = q == 0 ? k0[i] : Bf.k[q][base + i];
                ax += kw[q] * kj.x; ay += kw[q] * kj.y; az += kw[q] * kj.z;
                ex += ke[q] * kj.x; ey += ke[q] * kj.y; ez += ke[q] * kj.z;
            }
        }
        v.x += ax; v.y += ay; v.z += az;
        if (dp_last) {
            float r2 = v.x * v.x + v.y * v.y + v.z * v.z;
            float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
            v.x *= inv; v.y *= inv; v.z *= inv;
            e6[i] = make_float4(ex, ey, ez, 0.f);
        }
        out[i] = v;
    }
};

// Everything a stage needs per cell once demag and exchange are known:
// anisotropy, Zeeman (with the Appendix C excitation) and cavity fields, the
// LLG torque (Eq. llg), the RK bookkeeping of this stage, and the cell's
// share of the coupling sums and of the DP45 error.  NM: cavity modes
// compiled in (1: the paper's single mode; MAX_MODES: up to A.nmodes).
// Material constants and buffer pointers are read from the kernel's
// parameter block at each use.
template <int NM>
struct CellUpdate {
    float G[NM], bs[NM];
    bool on[NM];
    float dt, bex, bey, bez, D;
    bool want_demag, want_exch, want_anis, want_zee, want_cav, field_only;
    int K, s, mode, nm;
    long long cb, fb;    // first cell of this instance; of the launch's first instance (field output)
    float4* kout;

    // fb_: first cell of the launch's first instance; a field evaluation writes
    // fout[i - fb_], so a launch over several instances fills [instances][N]
    __device__ __forceinline__ void init(const Buffers& Bf, const StageArgs& A, const InstState& st,
                                         const InstParams& ip, const double* gam, float drive, long long cb_,
                                         long long fb_) {
        nm = NM == 1 ? 1 : A.nmodes;
#pragma unroll
        for (int q = 0; q < NM; q++) {
            G[q] = (float)gam[q];
            bs[q] = (float)ip.brms_scale[q];
            on[q] = q < nm && ip.cav_on[q] != 0;
        }
        D = drive;
        dt = (float)st.dt;
        bex = (float)ip.bext[0]; bey = (float)ip.bext[1]; bez = (float)ip.bext[2];
        want_demag = A.terms & 1; want_exch = A.terms & 2;
        want_anis = A.terms & 4; want_zee = A.terms & 8; want_cav = A.terms & 16;
        field_only = A.field_only != 0;
        K = A.kind; s = A.stage; mode = A.mode;
        cb = cb_;
        fb = fb_;
        const int k1slot = st.k1slot;
        kout = K == KIND_RK4 ? (s < 3 ? Bf.k[s] : nullptr)
                             : (s < 6 ? Bf.k[s == 0 ? k1slot : s] : Bf.k[k1slot == 0 ? 6 : 0]);
    }

    // (Bx, By, Bz) holds demag + exchange on entry
    template <bool REC>
    __device__ __forceinline__ void run(const Material& mat, const Buffers& Bf, long long i, float4 m, float Bx,
                                        float By, float Bz, double (&xacc)[NM], double (&macc)[REC ? 3 : 1],
                                        float& emax, bool& bad) const {
        const float Ms = m.w;
        float px_[NM], py_[NM], pz_[NM];
#pragma unroll
        for (int q = 0; q < NM; q++) px_[q] = py_[q] = pz_[q] = 0.f;
        if (Ms > 0.f) {
            if (want_anis) {
                float mu = m.x * mat.u[0] + m.y * mat.u[1] + m.z * mat.u[2];
                float f = mat.two_ku * __fdividef(mu, Ms);
                Bx += f * mat.u[0]; By += f * mat.u[1]; Bz += f * mat.u[2];
            }
            if (want_zee) { Bx += bex; By += bey; Bz += bez; }
#pragma unroll
            for (int q = 0; q < NM; q++) {
                // the excitation (Appendix C) uses the map of mode 0
                if (!(on[q] || (q == 0 && D != 0.f))) continue;
                if (Bf.prof[q]) {
                    float4 p = __ldg(Bf.prof[q] + (i - cb));
                    px_[q] = bs[q] * p.x; py_[q] = bs[q] * p.y; pz_[q] = bs[q] * p.z;
                } else {
                    py_[q] = bs[q];
                }
                if (on[q] && want_cav) { Bx += G[q] * px_[q]; By += G[q] * py_[q]; Bz += G[q] * pz_[q]; }
                if (q == 0 && want_zee) { Bx += D * px_[0]; By += D * py_[0]; Bz += D * pz_[0]; }
            }
        }
        if (field_only) {
            Bf.fout[i - fb] = make_float4(Bx, By, Bz, 0.f);
            return;
        }
        float cx = m.y * Bz - m.z * By, cy = m.z * Bx - m.x * Bz, cz = m.x * By - m.y * Bx;
        float dx = m.y * cz - m.z * cy, dy = m.z * cx - m.x * cz, dz = m.x * cy - m.y * cx;
        float4 kk = make_float4(mat.pre * (cx + mat.alpha * dx), mat.pre * (cy + mat.alpha * dy),
                                mat.pre * (cz + mat.alpha * dz), 0.f);
        if (!(Ms > 0.f)) kk = make_float4(0.f, 0.f, 0.f, 0.f);
        // a NaN or infinite component makes the sum non-finite (so does a
        // component sum beyond the float range, itself an overflowing torque)
        if (!(fabsf(kk.x + kk.y + kk.z) <= 3.0e38f)) bad = true;
        float4 mx = m;   // m used for the coupling sums of this launch
        float4 mrec = m; // state being accepted (recorded spatial average)
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
                if (mode == CAV_P) mx = mn;
                mrec = mn;
            }
        } else {
            kout[i] = kk;
            if (s == 6) {
                float4 e = Bf.e6[i];
                float c7 = c_ef[6] * dt;
                float exx = e.x + c7 * kk.x, eyy = e.y + c7 * kk.y, ezz = e.z + c7 * kk.z;
                const float en = sqrtf(exx * exx + eyy * eyy + ezz * ezz);
                if (!(en <= 3.0e38f)) bad = true;    // fmaxf would drop a NaN
                emax = fmaxf(emax, en);
            }
        }
        // the coupling sums: each cell's product in FP32, promoted and
        // accumulated in FP64 (thread, block and instance sums)
#pragma unroll
        for (int q = 0; q < NM; q++)
            if (on[q]) xacc[q] += (double)(Ms * (mx.x * px_[q] + mx.y * py_[q] + mx.z * pz_[q]));
        if constexpr (REC) {
            if (Ms > 0.f) { macc[0] += mrec.x; macc[1] += mrec.y; macc[2] += mrec.z; }
        }
    }
};

// Factor of the Appendix C excitation at this launch's stage time (simulation
// time t + c_s dt): drv_amp sinc(drv_wcut (t - drv_t0)), sinc(0) = 1.
static __device__ double drive_factor(const StageArgs& A, const InstParams& ip, const InstState& st) {
    if (!ip.drv_on) return 0.0;
    const double ts = st.t + (A.field_only ? 0.0 : c_cd[A.kind][A.stage] * st.dt);
    const double x = ip.drv_wcut * (ts - ip.drv_t0);
    return ip.drv_amp * (x == 0.0 ? 1.0 : sin(x) / x);
}

// Gamma_k(t) for the stage of this launch (E-mode: 2 Re alpha_k of the stage;
// P-mode: Eq. gammadiscretefinal at the stage time).
static __device__ double stage_gamma(const StageArgs& A, const InstParams& ip, const InstState& st,
                                     const Material& mat, int k) {
    if (!ip.cav_on[k]) return 0.0;
    if (A.mode == CAV_E) return 2.0 * (A.field_only ? st.a_re[k] : st.as_re[k]);
    return gamma_p(ip, st, k, st.tcav + (A.field_only ? 0.0 : c_cd[A.kind][A.stage] * st.dt), mat.hbar);
}

// Block partials of X_k and of the DP45 error; the last block of the instance
// to arrive reduces all partials in a fixed order and runs finish_stage.
// `nparts` = blocks per instance, `part` = this block's index among them.
// Partials of mode k live at xpart[(k B + b) nparts + part].
template <bool REC, int NM>
static __device__ void stage_epilogue(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A,
                                      int b, int part, int nparts, const double (&xacc)[NM], float emax, bool bad,
                                      double* s_red, float* s_redf, int* s_last, const double* macc) {
    // RK4: a non-finite torque is an error.  DP45: it marks the attempt, which
    // is then rejected with the smallest step factor (an overflowing trial
    // step); a state that stays non-finite ends in step-size underflow.
    if (bad) {
        if (A.kind == KIND_DP45) atomicOr(&Bf.st[b].poison, 1);
        else atomicOr(Bf.flags, FLAG_NAN);
    }
    const int nm = NM == 1 ? 1 : A.nmodes;
    double xb[NM];
#pragma unroll
    for (int q = 0; q < NM; q++) xb[q] = q < nm ? block_sum_d(xacc[q], s_red) : 0.0;
    float eb = block_max_f(emax, s_redf);
    const long long pb = (long long)b * nparts;
    double mb[3] = {0.0, 0.0, 0.0};
    if (REC)
        for (int c = 0; c < 3; c++) mb[c] = block_sum_d(macc[c], s_red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NM; q++)
            if (q < nm) Bf.xpart[((long long)q * P.B + b) * nparts + part] = xb[q];
        Bf.epart[pb + part] = eb;
        if (REC)
            for (int c = 0; c < 3; c++) Bf.mpart[3 * (pb + part) + c] = mb[c];
        __threadfence();
        unsigned prev = atomicAdd(Bf.counter + b, 1u);
        *s_last = prev == (unsigned)(nparts - 1);
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    double xs[MAX_MODES] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nm; q++) {
        double v = 0.0;
        const double* xp = Bf.xpart + ((long long)q * P.B + b) * nparts;
        for (int r = threadIdx.x; r < nparts; r += blockDim.x) v += __ldcg(xp + r);
        xs[q] = block_sum_d(v, s_red);
    }
    float em = 0.f;
    for (int r = threadIdx.x; r < nparts; r += blockDim.x) em = fmaxf(em, __ldcg(Bf.epart + pb + r));
    em = block_max_f(em, s_redf);
    double msum[3] = {0.0, 0.0, 0.0};
    if (REC) {
        for (int c = 0; c < 3; c++) {
            double v = 0.0;
            for (int r = threadIdx.x; r < nparts; r += blockDim.x) v += __ldcg(Bf.mpart + 3 * (pb + r) + c);
            msum[c] = block_sum_d(v, s_red);
        }
    }
    if (threadIdx.x == 0) {
        InstState ns = Bf.st[b];
        finish_stage(P, mat, A, Bf.ip[b], ns, xs, em, Bf.hist + (long long)b * Bf.hcap, Bf.hcap, Bf.flags,
                     REC ? msum : nullptr, REC ? Bf.mhist + 4LL * b * Bf.hcap : nullptr);
        Bf.st[b] = ns;
        Bf.counter[b] = 0u;
    }
}

}  // namespace mq
