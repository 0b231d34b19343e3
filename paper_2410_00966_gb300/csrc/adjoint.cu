// Element-wise and stencil kernels of the discrete adjoint of the RK4 path
// (gradients of J = w . <m>(T) + wn |alpha(T)|^2; the host side is
// mmcq_adjoint_rk4 in capi.cu).  The demag convolution of the adjoint field
// reuses the forward passes (the tensor is symmetric, so the convolution is
// its own transpose).  Per-cell arithmetic in FP32 like the forward path,
// sums over cells in FP64 with fixed-order block reductions.
//
// State buffers are float4 [B][N] with Ms in w, like the forward path.
#include <math.h>

#include "adjoint.cuh"
#include "common.cuh"
#include "stagecore.cuh"

namespace mq {

// k = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)] (Eq. llg) at the stage
// state Y with field Bf; optionally the next stage state Yn = Y1 + cdt k.
__global__ void k_adj_torque(const float4* Y, const float4* Bfield, const float4* Y1, float4* K, float4* Yn,
                             float cdt, float pre, float alpha, long long total) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float4 m = Y[i], B = Bfield[i];
    float4 k = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m.w > 0.f) {
        float cx = m.y * B.z - m.z * B.y, cy = m.z * B.x - m.x * B.z, cz = m.x * B.y - m.y * B.x;
        float dx = m.y * cz - m.z * cy, dy = m.z * cx - m.x * cz, dz = m.x * cy - m.y * cx;
        k = make_float4(pre * (cx + alpha * dx), pre * (cy + alpha * dy), pre * (cz + alpha * dz), 0.f);
    }
    K[i] = k;
    if (Yn) {
        const float4 a = Y1[i];
        Yn[i] = make_float4(a.x + cdt * k.x, a.y + cdt * k.y, a.z + cdt * k.z, a.w);
    }
}

// Cotangent through the end-of-step renormalisation m = m'/|m'| with
// m' = Y1 + dt sum_s b_s K_s: lp = (lam - (lam . mh) mh) / |m'|; also starts
// the next adjoint state nl = lp and the stage-4 cotangent lk = dt b_4 lp.
__global__ void k_adj_norm(const float4* Y1, const float4* K0, const float4* K1, const float4* K2,
                           const float4* K3, const float4* lam, float4* lp, float4* nl, float4* lk, float dt,
                           long long total) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float4 y = Y1[i];
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (y.w > 0.f) {
        const float4 a = K0[i], b = K1[i], c = K2[i], d = K3[i];
        const float h = dt * (1.f / 6.f);
        const float mx = y.x + h * (a.x + 2.f * b.x + 2.f * c.x + d.x);
        const float my = y.y + h * (a.y + 2.f * b.y + 2.f * c.y + d.y);
        const float mz = y.z + h * (a.z + 2.f * b.z + 2.f * c.z + d.z);
        const float r = sqrtf(mx * mx + my * my + mz * mz);
        if (r > 0.f) {
            const float ir = 1.f / r;
            const float hx = mx * ir, hy = my * ir, hz = mz * ir;
            const float4 l = lam[i];
            const float dd = l.x * hx + l.y * hy + l.z * hz;
            out = make_float4((l.x - dd * hx) * ir, (l.y - dd * hy) * ir, (l.z - dd * hz) * ir, 0.f);
        }
    }
    lp[i] = out;
    nl[i] = out;
    const float w = dt * (1.f / 6.f);
    lk[i] = make_float4(w * out.x, w * out.y, w * out.z, 0.f);
}

// Local part of the vector-Jacobian product of the right-hand side at the
// stage state (Y, field B) with cotangent u = lk of dm/dt:
//   lB = pre [(u x m) + alpha ((u.m) m - |m|^2 u)]                (of the field)
//   gd = pre [(B x u) + alpha ((m.B) u + (u.m) B - 2 (u.B) m)]   (of m, at fixed B)
//        + lX V_c Ms B_rms                                         (through X)
// lB carries w = 1 on magnetised cells (the multiplier of the demag input).
// Block partials (FP64) per instance: sum lB (x, y, z) and sum B_rms . lB.
__global__ void k_adj_local(const float4* Y, const float4* Bfield, const float4* lk, const double* lX,
                            const InstParams* ip, const float4* prof, float4* lB, float4* gd, double* part,
                            float pre, float alpha, double vc, long long N) {
    __shared__ double red[32];
    const int b = blockIdx.y;
    const long long base = (long long)b * N;
    const float bs = (float)ip[b].brms_scale[0];
    const float cX = (float)(lX[b] * vc);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const long long i = base + c;
        const float4 m = Y[i];
        float4 lb = make_float4(0.f, 0.f, 0.f, 0.f), g = lb;
        if (m.w > 0.f) {
            const float4 B = Bfield[i], u = lk[i];
            const float mb = m.x * B.x + m.y * B.y + m.z * B.z;
            const float um = u.x * m.x + u.y * m.y + u.z * m.z;
            const float ub = u.x * B.x + u.y * B.y + u.z * B.z;
            const float mm = m.x * m.x + m.y * m.y + m.z * m.z;
            const float bxu_x = B.y * u.z - B.z * u.y, bxu_y = B.z * u.x - B.x * u.z, bxu_z = B.x * u.y - B.y * u.x;
            const float uxm_x = u.y * m.z - u.z * m.y, uxm_y = u.z * m.x - u.x * m.z, uxm_z = u.x * m.y - u.y * m.x;
            float px = 0.f, py = bs, pz = 0.f;
            if (prof) { const float4 p = prof[c]; px = bs * p.x; py = bs * p.y; pz = bs * p.z; }
            g.x = pre * (bxu_x + alpha * (mb * u.x + um * B.x - 2.f * ub * m.x)) + cX * m.w * px;
            g.y = pre * (bxu_y + alpha * (mb * u.y + um * B.y - 2.f * ub * m.y)) + cX * m.w * py;
            g.z = pre * (bxu_z + alpha * (mb * u.z + um * B.z - 2.f * ub * m.z)) + cX * m.w * pz;
            lb.x = pre * (uxm_x + alpha * (um * m.x - mm * u.x));
            lb.y = pre * (uxm_y + alpha * (um * m.y - mm * u.y));
            lb.z = pre * (uxm_z + alpha * (um * m.z - mm * u.z));
            lb.w = 1.f;
            s0 += lb.x; s1 += lb.y; s2 += lb.z;
            s3 += (double)(px * lb.x + py * lb.y + pz * lb.z);
        }
        lB[i] = lb;
        gd[i] = g;
    }
    s0 = block_sum_d(s0, red);
    s1 = block_sum_d(s1, red);
    s2 = block_sum_d(s2, red);
    s3 = block_sum_d(s3, red);
    if (threadIdx.x == 0) {
        double* p = part + ((long long)b * gridDim.x + blockIdx.x) * 4;
        p[0] = s0; p[1] = s1; p[2] = s2; p[3] = s3;
    }
}

// The field terms are linear in m; their transposes applied to lB:
//   demag: Ms_i D(lB)_i (D symmetric, D = the field-only pass on lB, given here)
//   exchange: sum_j w_ij (c_j lB_j - c_i lB_i), c = 2A/Ms, both cells magnetised
//   anisotropy: (2 Ku / Ms_i)(lB_i . u) u
// g = gd + those; then nl += g and lk = dtb * lp + cdt * g (next stage's cotangent).
// With gms: the Ms-map cotangent (mask and B_rms map fixed) accumulates
//   m_i . D(lB)_i - lB_i . (B_exch,i + B_anis,i) / Ms_i + lX V_c m_i . B_rms,i.
__global__ void k_adj_combine(const float4* Y, const float4* lB, const float4* Dl, const float4* gd,
                              const float4* lp, float4* nl, float4* lk, Material mat, float dtb, float cdt,
                              int nx, int ny, int nz, float* gms, const double* lX, const InstParams* ip,
                              const float4* prof) {
    const long long N = (long long)nx * ny * nz;
    const int b = blockIdx.y;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const long long i = (long long)b * N + c;
    const float4 m = Y[i];
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m.w > 0.f) {
        const float4 l = lB[i], d = Dl[i], q = gd[i];
        g.x = q.x + m.w * d.x; g.y = q.y + m.w * d.y; g.z = q.z + m.w * d.z;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const float ci = 1.f / m.w;
        const long long st[3] = {1, nx, (long long)nx * ny};
        const int pos[3] = {x, y, z}, ext[3] = {nx, ny, nz};
        float hx = 0.f, hy = 0.f, hz = 0.f;      // sum_j exch (m_j - m_i): Ms_i B_exch,i
        for (int a = 0; a < 3; a++) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const int pn = pos[a] + sgn;
                if (pn < 0 || pn >= ext[a]) continue;
                const long long j = i + sgn * st[a];
                const float4 mj = Y[j];
                if (!(mj.w > 0.f)) continue;
                const float4 lj = lB[j];
                const float cj = 1.f / mj.w;
                g.x += mat.exch[a] * (cj * lj.x - ci * l.x);
                g.y += mat.exch[a] * (cj * lj.y - ci * l.y);
                g.z += mat.exch[a] * (cj * lj.z - ci * l.z);
                hx += mat.exch[a] * (mj.x - m.x);
                hy += mat.exch[a] * (mj.y - m.y);
                hz += mat.exch[a] * (mj.z - m.z);
            }
        }
        const float lu = l.x * mat.u[0] + l.y * mat.u[1] + l.z * mat.u[2];
        const float f = mat.two_ku / m.w * lu;
        g.x += f * mat.u[0]; g.y += f * mat.u[1]; g.z += f * mat.u[2];
        if (gms) {
            const float mu = m.x * mat.u[0] + m.y * mat.u[1] + m.z * mat.u[2];
            const float an = mat.two_ku * mu;    // Ms_i B_anis,i = an u
            float px = 0.f, py = 1.f, pz = 0.f;
            if (prof) { const float4 p = prof[c]; px = p.x; py = p.y; pz = p.z; }
            const float bs = (float)ip[b].brms_scale[0];
            const float xs = (float)(lX[b] * mat.vc) * bs * (m.x * px + m.y * py + m.z * pz);
            const float ex = l.x * (hx + an * mat.u[0]) + l.y * (hy + an * mat.u[1]) + l.z * (hz + an * mat.u[2]);
            gms[i] += m.x * d.x + m.y * d.y + m.z * d.z - ex * ci * ci + xs;
        }
    }
    float4 a = nl[i];
    nl[i] = make_float4(a.x + g.x, a.y + g.y, a.z + g.z, 0.f);
    const float4 p = lp[i];
    lk[i] = make_float4(dtb * p.x + cdt * g.x, dtb * p.y + cdt * g.y, dtb * p.z + cdt * g.z, 0.f);
}

// Terminal cotangent of J = w . <m>: w / (magnetised cells) on magnetised cells.
__global__ void k_adj_terminal(const float4* Y, float4* lam, float wx, float wy, float wz, long long total) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    lam[i] = Y[i].w > 0.f ? make_float4(wx, wy, wz, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---- FP64 scalar steps (one thread or block per instance) -------------------
static __device__ const double ADJ_C[4] = {0.0, 0.5, 0.5, 1.0};
static __device__ const double ADJ_B[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};

// Cursor of the reversed loop in device memory, so that one captured step
// serves every step: cur[0] = q - c0 (the step within its checkpoint segment),
// cur[1] = c0.
__global__ void k_adj_set_cursor(long long* cur, long long qrel, long long c0) {
    cur[0] = qrel;
    cur[1] = c0;
}
__global__ void k_adj_next(long long* cur) { cur[0] -= 1; }

// Inputs of reversed step q from the segment arrays at the cursor: the state
// m_q into Ybase and Y0 (the first stage input), the instance states of steps
// q and q + 1.
__global__ void k_adj_step_inputs(const float4* seg, const InstState* segst, float4* Ybase, float4* Y0,
                                  InstState* stq, InstState* stq1, const long long* cur, long long BN, int B) {
    const long long qrel = cur[0];
    const float4* src = seg + qrel * BN;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < BN; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        Ybase[i] = v;
        Y0[i] = v;
    }
    if (blockIdx.x == 0) {
        for (int b = threadIdx.x; b < B; b += blockDim.x) {
            stq[b] = segst[qrel * B + b];
            stq1[b] = segst[(qrel + 1) * B + b];
        }
    }
}

// The averaged photon number sees alpha at step q + 1 (q from the cursor;
// only steps with q + 1 >= wstart count): J += c |alpha|^2 and its cotangent
// 2 c alpha.
__global__ void k_adj_window(AdjScalars* S, const InstState* st, double c, int B, const long long* cur,
                             long long wstart) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (cur[1] + cur[0] + 1 < wstart) return;
    const double ar = st[b].a_re[0], ai = st[b].a_im[0];
    S[b].J += c * (ar * ar + ai * ai);
    S[b].la_re += 2.0 * c * ar;
    S[b].la_im += 2.0 * c * ai;
}

// Start of a reversed step from its state: the field evaluations read their
// cavity amplitude from adst (E-mode, field only).
__global__ void k_adj_begin_step(AdjScalars* S, InstState* adst, const InstState* st, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    InstState x = st[b];
    x.mcur = 0;
    x.as_re[0] = x.a_re[0];
    x.as_im[0] = x.a_im[0];
    adst[b] = x;
    S[b].a0_re = S[b].as_re[0] = x.a_re[0];
    S[b].a0_im = S[b].as_im[0] = x.a_im[0];
}

// Stage s of the recomputation: d alpha/dt = -(kappa + i omega) alpha + i X / hbar,
// then the amplitude of stage s + 1 for the next field evaluation.
__global__ void k_adj_alpha_stage(AdjScalars* S, InstState* adst, const InstParams* ip, const double* X, int s,
                                  double dt, double hbar, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    AdjScalars& q = S[b];
    const double re = q.as_re[s], im = q.as_im[s];
    const bool on = ip[b].cav_on[0] != 0;
    q.X[s] = X[b];
    q.ka_re[s] = on ? -ip[b].kappa[0] * re + ip[b].wc[0] * im : 0.0;
    q.ka_im[s] = on ? -ip[b].kappa[0] * im - ip[b].wc[0] * re + X[b] / hbar : 0.0;
    if (s < 3) {
        const double nr = q.a0_re + ADJ_C[s + 1] * dt * q.ka_re[s];
        const double ni = q.a0_im + ADJ_C[s + 1] * dt * q.ka_im[s];
        q.as_re[s + 1] = nr;
        q.as_im[s + 1] = ni;
        adst[b].a_re[0] = adst[b].as_re[0] = nr;
        adst[b].a_im[0] = adst[b].as_im[0] = ni;
    }
}

// Start of the stage cotangents: y' = y + dt sum b_s k_s.
__global__ void k_adj_begin_vjp(AdjScalars* S, const InstParams* ip, double* lX, double dt, double hbar, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    AdjScalars& q = S[b];
    q.lp_re = q.nl_re = q.la_re;
    q.lp_im = q.nl_im = q.la_im;
    q.lk_re = dt * ADJ_B[3] * q.lp_re;
    q.lk_im = dt * ADJ_B[3] * q.lp_im;
    lX[b] = ip[b].cav_on[0] ? q.lk_im / hbar : 0.0;
}

// After the local products of stage s: the block partials (sum lB, sum B_rms . lB)
// reduced in a fixed order, the amplitude cotangent through
// d alpha/dt = -(kappa + i omega) alpha + i X / hbar and B_cav = B_rms 2 Re alpha,
// the parameter cotangents, and the next stage's d alpha/dt cotangent.
__global__ void k_adj_scalar_vjp(AdjScalars* S, const double* part, int nblk, const InstParams* ip, double* lX, int s,
                                 double dt, double hbar) {
    __shared__ double red[32];
    const int b = blockIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nblk; k += blockDim.x)
        for (int c = 0; c < 4; c++) v[c] += part[((long long)b * nblk + k) * 4 + c];
    for (int c = 0; c < 4; c++) v[c] = block_sum_d(v[c], red);
    if (threadIdx.x != 0) return;
    AdjScalars& q = S[b];
    const bool on = ip[b].cav_on[0] != 0;
    const double re = q.as_re[s], im = q.as_im[s], nr = q.lk_re, ni = q.lk_im, lx = lX[b];
    const double gr = on ? -ip[b].kappa[0] * nr - ip[b].wc[0] * ni + 2.0 * v[3] : 0.0;
    const double gi = on ? ip[b].wc[0] * nr - ip[b].kappa[0] * ni : 0.0;
    q.grad[0] += v[0]; q.grad[1] += v[1]; q.grad[2] += v[2];
    if (on) {
        q.grad[3] += 2.0 * re * v[3] + lx * q.X[s];
        q.grad[4] += nr * im - ni * re;
        q.grad[5] += -nr * re - ni * im;
    }
    q.nl_re += gr;
    q.nl_im += gi;
    if (s > 0) {
        q.lk_re = dt * ADJ_B[s - 1] * q.lp_re + ADJ_C[s] * dt * gr;
        q.lk_im = dt * ADJ_B[s - 1] * q.lp_im + ADJ_C[s] * dt * gi;
        lX[b] = on ? q.lk_im / hbar : 0.0;
    }
}

__global__ void k_adj_end_step(AdjScalars* S, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    S[b].la_re = S[b].nl_re;
    S[b].la_im = S[b].nl_im;
}

// ---------------------------------------------------------------------------
static unsigned blocks_for(long long n, int th) { return (unsigned)((n + th - 1) / th); }

cudaError_t launch_adj_torque(const float4* Y, const float4* Bf, const float4* Y1, float4* K, float4* Yn, float cdt,
                              float pre, float alpha, long long total, cudaStream_t s) {
    k_adj_torque<<<blocks_for(total, 256), 256, 0, s>>>(Y, Bf, Y1, K, Yn, cdt, pre, alpha, total);
    return cudaGetLastError();
}
cudaError_t launch_adj_norm(const float4* Y1, const float4* const* K, const float4* lam, float4* lp, float4* nl,
                            float4* lk, float dt, long long total, cudaStream_t s) {
    k_adj_norm<<<blocks_for(total, 256), 256, 0, s>>>(Y1, K[0], K[1], K[2], K[3], lam, lp, nl, lk, dt, total);
    return cudaGetLastError();
}
int adj_local_blocks(long long N) {
    long long b = (N + 255) / 256;
    return (int)(b < 128 ? b : 128);
}
cudaError_t launch_adj_local(const float4* Y, const float4* Bf, const float4* lk, const double* lX,
                             const InstParams* ip, const float4* prof, float4* lB, float4* gd, double* part, float pre,
                             float alpha, double vc, long long N, int B, cudaStream_t s) {
    dim3 grid(adj_local_blocks(N), B);
    k_adj_local<<<grid, 256, 0, s>>>(Y, Bf, lk, lX, ip, prof, lB, gd, part, pre, alpha, vc, N);
    return cudaGetLastError();
}
cudaError_t launch_adj_combine(const float4* Y, const float4* lB, const float4* Dl, const float4* gd,
                               const float4* lp, float4* nl, float4* lk, const Material& mat, float dtb, float cdt,
                               int nx, int ny, int nz, int B, float* gms, const double* lX, const InstParams* ip,
                               const float4* prof, cudaStream_t s) {
    const long long N = (long long)nx * ny * nz;
    dim3 grid(blocks_for(N, 256), B);
    k_adj_combine<<<grid, 256, 0, s>>>(Y, lB, Dl, gd, lp, nl, lk, mat, dtb, cdt, nx, ny, nz, gms, lX, ip, prof);
    return cudaGetLastError();
}
cudaError_t launch_adj_terminal(const float4* Y, float4* lam, const double w[3], long long total, cudaStream_t s) {
    k_adj_terminal<<<blocks_for(total, 256), 256, 0, s>>>(Y, lam, (float)w[0], (float)w[1], (float)w[2], total);
    return cudaGetLastError();
}

static unsigned small_blocks(int B) { return (unsigned)((B + 63) / 64); }
cudaError_t launch_adj_window(AdjScalars* S, const InstState* st, double c, int B, const long long* cur,
                              long long wstart, cudaStream_t s) {
    k_adj_window<<<small_blocks(B), 64, 0, s>>>(S, st, c, B, cur, wstart);
    return cudaGetLastError();
}
cudaError_t launch_adj_set_cursor(long long* cur, long long qrel, long long c0, cudaStream_t s) {
    k_adj_set_cursor<<<1, 1, 0, s>>>(cur, qrel, c0);
    return cudaGetLastError();
}
cudaError_t launch_adj_next(long long* cur, cudaStream_t s) {
    k_adj_next<<<1, 1, 0, s>>>(cur);
    return cudaGetLastError();
}
cudaError_t launch_adj_step_inputs(const float4* seg, const InstState* segst, float4* Ybase, float4* Y0,
                                   InstState* stq, InstState* stq1, const long long* cur, long long BN, int B,
                                   cudaStream_t s) {
    k_adj_step_inputs<<<blocks_for(BN, 256), 256, 0, s>>>(seg, segst, Ybase, Y0, stq, stq1, cur, BN, B);
    return cudaGetLastError();
}
cudaError_t launch_adj_begin_step(AdjScalars* S, InstState* adst, const InstState* st, int B, cudaStream_t s) {
    k_adj_begin_step<<<small_blocks(B), 64, 0, s>>>(S, adst, st, B);
    return cudaGetLastError();
}
cudaError_t launch_adj_alpha_stage(AdjScalars* S, InstState* adst, const InstParams* ip, const double* X, int st,
                                   double dt, double hbar, int B, cudaStream_t s) {
    k_adj_alpha_stage<<<small_blocks(B), 64, 0, s>>>(S, adst, ip, X, st, dt, hbar, B);
    return cudaGetLastError();
}
cudaError_t launch_adj_begin_vjp(AdjScalars* S, const InstParams* ip, double* lX, double dt, double hbar, int B,
                                 cudaStream_t s) {
    k_adj_begin_vjp<<<small_blocks(B), 64, 0, s>>>(S, ip, lX, dt, hbar, B);
    return cudaGetLastError();
}
cudaError_t launch_adj_scalar_vjp(AdjScalars* S, const double* part, int nblk, const InstParams* ip, double* lX,
                                  int st, double dt, double hbar, int B, cudaStream_t s) {
    k_adj_scalar_vjp<<<B, 128, 0, s>>>(S, part, nblk, ip, lX, st, dt, hbar);
    return cudaGetLastError();
}
cudaError_t launch_adj_end_step(AdjScalars* S, int B, cudaStream_t s) {
    k_adj_end_step<<<small_blocks(B), 64, 0, s>>>(S, B);
    return cudaGetLastError();
}

}  // namespace mq

