// C ABI of the mmcq library (declarations and argument contracts in
// include/mmcq.h).  Host code only sets things up and enqueues kernels;
// every step of the time integration runs in the kernels of stage.cu.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "adjoint.cuh"
#include "common.cuh"
#include "mmcq.h"

namespace mq {
cudaError_t set_smem_limits();
cudaError_t launch_xfwd(const Plan&, const Buffers&, const StageArgs&, int, cudaStream_t);
cudaError_t launch_xinv(const Plan&, const Material&, const Buffers&, const StageArgs&, int, cudaStream_t,
                        const SpecMap*, const Tune*);
cudaError_t launch_convolution(const Plan&, const Buffers&, const StageArgs&, int, cudaStream_t, const Tune*);
cudaError_t launch_conv_part(const Plan&, const Buffers&, const StageArgs&, int, cudaStream_t, int, const Tune*);
void conv_tunables(const Plan&, int*, int*, int*, int*, int*);
int convolution_launches(const Plan&);
bool col_fits(const Plan&);
bool fft_fits(int, int);
int rows_per_block(int, int);
int coupling_blocks(long long);
bool x_fits(const Plan&);
cudaError_t launch_set_m(float4*, const float*, const float*, long long, int, int, int*, cudaStream_t);
cudaError_t launch_get_m(const float4*, float*, long long, cudaStream_t);
cudaError_t launch_apply_ms(float4*, const float*, long long, int, cudaStream_t);
cudaError_t launch_get_field(const float4*, float*, long long, cudaStream_t);
cudaError_t launch_coupling_sum(const Buffers&, long long, double, int, int, int, double*, cudaStream_t);
cudaError_t launch_set_dt(InstState*, int, double, cudaStream_t);
cudaError_t launch_spectrum(const double*, long long, int, const double*, int, double*, cudaStream_t);
cudaError_t launch_adj_torque(const float4*, const float4*, const float4*, float4*, float4*, float, float, float,
                              long long, cudaStream_t);
cudaError_t launch_adj_norm(const float4*, const float4* const*, const float4*, float4*, float4*, float4*, float,
                            long long, cudaStream_t);
int adj_local_blocks(long long);
cudaError_t launch_adj_local(const float4*, const float4*, const float4*, const double*, const InstParams*,
                             const float4*, float4*, float4*, double*, float, float, double, long long, int,
                             cudaStream_t);
cudaError_t launch_adj_combine(const float4*, const float4*, const float4*, const float4*, const float4*, float4*,
                               float4*, const Material&, float, float, int, int, int, int, float*, const double*,
                               const InstParams*, const float4*, cudaStream_t);
cudaError_t launch_adj_terminal(const float4*, float4*, const double*, long long, cudaStream_t);
cudaError_t launch_adj_window(AdjScalars*, const InstState*, double, int, const long long*, long long, cudaStream_t);
cudaError_t launch_adj_set_cursor(long long*, long long, long long, cudaStream_t);
cudaError_t launch_adj_next(long long*, cudaStream_t);
cudaError_t launch_adj_step_inputs(const float4*, const InstState*, float4*, float4*, InstState*, InstState*,
                                   const long long*, long long, int, cudaStream_t);
cudaError_t launch_adj_begin_step(AdjScalars*, InstState*, const InstState*, int, cudaStream_t);
cudaError_t launch_adj_alpha_stage(AdjScalars*, InstState*, const InstParams*, const double*, int, double, double, int,
                                   cudaStream_t);
cudaError_t launch_adj_begin_vjp(AdjScalars*, const InstParams*, double*, double, double, int, cudaStream_t);
cudaError_t launch_adj_scalar_vjp(AdjScalars*, const double*, int, const InstParams*, double*, int, double, double,
                                  int, cudaStream_t);
cudaError_t launch_adj_end_step(AdjScalars*, int, cudaStream_t);
cudaError_t build_demag_kernel(const Plan&, double, double, double, double, float*, double2*, cudaStream_t);
}  // namespace mq

using namespace mq;

struct mmcq {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mmcq_alloc_fn alloc = nullptr;
    mmcq_free_fn freefn = nullptr;
    void* actx = nullptr;
    Plan P{};
    Material mat{};
    Buffers Bf{};
    double dx = 0, dy = 0, dz = 0, gamma = 0, mu0 = 0, hbar = 0;
    int kind = KIND_RK4;
    double tol = 1e-6;
    int mode = CAV_E;
    std::vector<InstParams> ip;
    std::vector<double> g;          // [B][MAX_MODES] coupling strength (profile_is_brms = 0)
    std::vector<int> g_mode;        // [B][MAX_MODES] 1: scale from g, 0: profile is B_rms
    int nmodes = 1;                 // cavity modes in use: highest configured mode + 1
    std::vector<float> ms_host;
    float* ms_dev = nullptr;
    float* stage3 = nullptr;
    double* dscratch = nullptr;
    std::vector<void*> allocs;
    size_t bytes = 0;
    double setup_ms = 0;
    std::string err;
    bool k1_dirty = true;   // some instance may need its first DP45 stage recomputed
    int record = 0;         // record <m> every `record` accepted steps (0: off)
    double* spec_buf = nullptr;   // device scratch of mmcq_spectrum (frequencies + result)
    int spec_cap = 0;             // frequencies it holds
    // measurement
    int64_t launches = 0;
    bool profiling = false;
    struct Rec { int cls; int ev; double bytes; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> events;   // pool, two per record
    // pipelined cavity read-out: a ring of pinned host slots, each holding the
    // instance states, the coupling sums and the error flags as of one post
    struct Post { void* host = nullptr; cudaEvent_t ev = nullptr; };
    std::vector<Post> posts;
    int post_head = 0, post_count = 0;
    SpecMap spec_map{};     // TMA map of the x-half-spectrum (pipelined x inverse)
    Tune tune{{0, 0, 0, 0}, -1, -1, {-1, -1}};   // launch parameters chosen by mmcq_autotune (default: the fixed rules)
    int rows_rule = 1;      // x-pass rows per block of the fixed rule
    int64_t tune_epoch = 0; // bumped when the launch parameters change (groups capture again)
};

enum { CLS_XFWD = 0, CLS_CONV2D, CLS_YFWD, CLS_ZCONV, CLS_YINV, CLS_XINV, NCLS };
static const char* CLS_NAMES[NCLS] = {"x_forward", "conv_2d", "y_forward", "z_convolve", "y_inverse", "x_inverse"};

namespace {

int fail(mmcq_t* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

int cuda_fail(mmcq_t* h, cudaError_t e, const char* where) {
    return fail(h, MMCQ_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);     \
    } while (0)

void* dev_alloc(mmcq_t* h, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (h->alloc) p = h->alloc(bytes, h->actx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) { h->allocs.push_back(p); h->bytes += bytes; }
    return p;
}

void dev_release(mmcq_t* h, void* p);

// Release one allocation now (it leaves the list freed at destroy).
void dev_free_now(mmcq_t* h, void* p) {
    if (!p) return;
    for (size_t q = 0; q < h->allocs.size(); q++)
        if (h->allocs[q] == p) { h->allocs.erase(h->allocs.begin() + q); break; }
    dev_release(h, p);
}

void dev_release(mmcq_t* h, void* p) {
    if (!p) return;
    if (h->freefn) h->freefn(p, h->actx);
    else if (!h->alloc) cudaFree(p);
}

int pow2_at_least(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

bool valid_inst(mmcq_t* h, int inst, bool allow_all) {
    return (allow_all && inst == -1) || (inst >= 0 && inst < h->P.B);
}

// Host read-modify-write of instance states (not on the hot path).
template <typename F>
int edit_state(mmcq_t* h, int inst, F fn) {
    int b0 = inst < 0 ? 0 : inst, nb = inst < 0 ? h->P.B : 1;
    std::vector<InstState> s(nb);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(s.data(), h->Bf.st + b0, sizeof(InstState) * nb, cudaMemcpyDeviceToHost));
    for (int i = 0; i < nb; i++) fn(s[i], b0 + i);
    CK(h, cudaMemcpy(h->Bf.st + b0, s.data(), sizeof(InstState) * nb, cudaMemcpyHostToDevice));
    h->k1_dirty = true;
    return MMCQ_OK;
}

int upload_params(mmcq_t* h) {
    CK(h, cudaMemcpyAsync(h->Bf.ip, h->ip.data(), sizeof(InstParams) * h->P.B, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return MMCQ_OK;
}

double ms_sum(mmcq_t* h) {
    double s = 0;
    for (float v : h->ms_host) s += v > 0 ? v : 0;
    return s;
}

void refresh_scales(mmcq_t* h) {
    double sm = ms_sum(h);
    long long nmag = 0;
    for (float v : h->ms_host) nmag += v > 0;
    for (int b = 0; b < h->P.B; b++) {
        for (int k = 0; k < MAX_MODES; k++)
            if (h->g_mode[b * MAX_MODES + k])
                h->ip[b].brms_scale[k] =
                    sm > 0 ? h->g[b * MAX_MODES + k] * std::sqrt(2.0 * h->hbar / (h->gamma * h->mat.vc * sm)) : 0.0;
        h->ip[b].inv_nmag = nmag > 0 ? 1.0 / (double)nmag : 0.0;
    }
}

// Every mode back to alpha_k(0) = (x0_k - i p0_k)/2 with empty accumulators at
// t_cav = 0 (ResetMemoryTerm).
void reset_memory(const InstParams& ip, InstState& s) {
    s.tcav = 0;
    for (int k = 0; k < MAX_MODES; k++) {
        s.S[k] = s.C[k] = 0;
        s.a_re[k] = s.as_re[k] = 0.5 * ip.x0[k];
        s.a_im[k] = s.as_im[k] = -0.5 * ip.p0[k];
    }
    s.have_k1 = 0;
}

StageArgs step_args(const mmcq_t* h) {
    StageArgs A{};
    A.kind = h->kind;
    A.mode = h->mode;
    A.terms = MMCQ_TERM_ALL;
    A.field_only = 0;
    A.inst0 = 0;
    A.tol = (float)h->tol;
    A.record = h->record;
    A.nmodes = h->nmodes;
    return A;
}

// Algorithmic (compulsory) bytes of one launch of class cls for nb instances.
double launch_bytes(const mmcq_t* h, int cls, const StageArgs& A, int nb) {
    const Plan& P = h->P;
    const double N = (double)P.N;
    const double cplx = 8.0;
    // spectra and kernel count the px/2 + 1 half-spectrum columns the method
    // needs, not the tile padding beyond them
    const double xrow = (double)P.nrows * P.hx * 3 * cplx;      // one instance's x half-spectrum
    const double yrow = (double)P.nz * P.py * P.hx * 3 * cplx;  // after the y transform
    const double kern = (double)P.hzk * P.hyk * P.hx * 6 * 4;
    static const int dp_kreads[7] = {0, 1, 2, 3, 4, 5, 5};
    const int s = A.stage;
    double per = 0.0;
    switch (cls) {
        case CLS_XFWD: {
            int kr = A.field_only || s == 0 ? 0 : (A.kind == KIND_RK4 ? 1 : dp_kreads[s]);
            int wr = A.field_only || s == 0 ? 0 : ((A.kind == KIND_DP45 && s == 6) ? 2 : 1);
            per = N * 16.0 * (1 + kr + wr) + xrow;
            break;
        }
        case CLS_CONV2D: return nb * 2.0 * xrow + kern;
        case CLS_YFWD: per = xrow + yrow; break;
        case CLS_ZCONV: return nb * 2.0 * yrow + kern;
        case CLS_YINV: per = yrow + xrow; break;
        case CLS_XINV: {
            double spec = xrow;
            double cells = 16.0;                         // stage input m_s
            if (A.field_only) cells += 16.0;             // field out
            else if (A.kind == KIND_RK4 && s == 3) cells += 16.0 * 5;  // m0, k1..k3 in, m out
            else if (A.kind == KIND_DP45 && s == 6) cells += 32.0;     // e6 in, k out
            else cells += 16.0;                          // k out
            for (int k = 0; k < h->nmodes; k++)
                if (h->Bf.prof[k]) cells += 16.0;
            per = spec + N * cells;
            break;
        }
    }
    return per * nb;
}

int launch_timed(mmcq_t* h, int cls, const StageArgs& A, int nb, int part) {
    int ev = -1;
    if (h->profiling) {
        ev = (int)h->recs.size() * 2;
        while ((int)h->events.size() < ev + 2) {
            cudaEvent_t e;
            CK(h, cudaEventCreate(&e));
            h->events.push_back(e);
        }
        CK(h, cudaEventRecord(h->events[ev], h->stream));
    }
    if (cls == CLS_XFWD) CK(h, launch_xfwd(h->P, h->Bf, A, nb, h->stream));
    else if (cls == CLS_XINV) CK(h, launch_xinv(h->P, h->mat, h->Bf, A, nb, h->stream, &h->spec_map, &h->tune));
    else CK(h, launch_conv_part(h->P, h->Bf, A, nb, h->stream, part, &h->tune));
    h->launches++;
    if (h->profiling) {
        CK(h, cudaEventRecord(h->events[ev + 1], h->stream));
        h->recs.push_back({cls, ev, launch_bytes(h, cls, A, nb)});
    }
    return MMCQ_OK;
}

int run_stage(mmcq_t* h, const StageArgs& A, int nb) {
    int r;
    if ((r = launch_timed(h, CLS_XFWD, A, nb, 0))) return r;
    if (h->P.nz == 1) {
        if ((r = launch_timed(h, CLS_CONV2D, A, nb, 0))) return r;
    } else {
        if ((r = launch_timed(h, CLS_YFWD, A, nb, 1))) return r;
        if ((r = launch_timed(h, CLS_ZCONV, A, nb, 2))) return r;
        if ((r = launch_timed(h, CLS_YINV, A, nb, 3))) return r;
    }
    return launch_timed(h, CLS_XINV, A, nb, 0);
}

int check_flags(mmcq_t* h) {
    int f = 0;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(&f, h->Bf.flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (f & FLAG_TIMEOUT)
        return fail(h, MMCQ_ERR_TIMEOUT, "a bulk copy into shared memory did not complete within its wait limit; "
                                         "the handle's state is undefined");
    if (f & (FLAG_NAN | FLAG_DT_UNDERFLOW)) {
        int z = 0;
        CK(h, cudaMemcpy(h->Bf.flags, &z, sizeof(int), cudaMemcpyHostToDevice));
        return fail(h, MMCQ_ERR_NUMERIC, (f & FLAG_NAN) ? "non-finite magnetisation or field" : "adaptive step underflow");
    }
    return MMCQ_OK;
}

// n steps (RK4) or attempts (DP45) of every instance, enqueued on h->stream.
int enqueue_steps(mmcq_t* h, int64_t n) {
    StageArgs A = step_args(h);
    const int B = h->P.B;
    for (int64_t it = 0; it < n; it++) {
        if (h->kind == KIND_RK4) {
            for (int s = 0; s < 4; s++) {
                A.stage = s;
                int r = run_stage(h, A, B);
                if (r) return r;
            }
        } else {
            for (int s = 0; s < 7; s++) {
                // stage 1 is first-same-as-last in E-mode: it only needs a launch
                // after a host-side change (P-mode recomputes it every attempt)
                if (s == 0 && h->mode == CAV_E && !h->k1_dirty) continue;
                A.stage = s;
                int r = run_stage(h, A, B);
                if (r) return r;
                if (s == 0 && h->mode == CAV_E) h->k1_dirty = false;
            }
        }
    }
    return MMCQ_OK;
}

// The 4-D tensor map of the x-half-spectrum [B nz][NT][ny][3 TX] (complex64
// values copied as 8-byte elements), box = one row: 3 TX x 1 x NT x 1.  Only
// for the shapes the pipelined x inverse takes; otherwise map.valid = false.
int encode_spec_map(mmcq_t* h) {
    const Plan& P = h->P;
    h->spec_map.valid = false;
    if (!(P.L == 1024 && P.TX == 8 && P.R == 1 && P.NT <= 256)) return MMCQ_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return fail(h, MMCQ_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t row = 3ull * P.TX;
    cuuint64_t dims[4] = {row, (cuuint64_t)P.ny, (cuuint64_t)P.NT, (cuuint64_t)P.B * P.nz};
    cuuint64_t strides[3] = {row * 8, row * 8 * P.ny, row * 8 * P.ny * P.NT};   // bytes, dims 1..3
    cuuint32_t box[4] = {(cuuint32_t)row, 1, (cuuint32_t)P.NT, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    static_assert(sizeof(CUtensorMap) == sizeof(TensorMap), "tensor map size");
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(&h->spec_map.map), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                        h->Bf.spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, MMCQ_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    h->spec_map.base = h->Bf.spec;
    h->spec_map.valid = true;
    return MMCQ_OK;
}

}  // namespace

extern "C" {

int mmcq_create(mmcq_t** out, const mmcq_grid* g, double Ms, double Aex, double alpha, double Ku,
                const double axis[3], const mmcq_opts* o) {
    if (!out) return MMCQ_ERR_ARG;
    *out = nullptr;
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || g->batch < 1 || !(g->dx > 0) || !(g->dy > 0) ||
        !(g->dz > 0) || !(Ms >= 0) || !(Aex >= 0) || !(alpha >= 0) || !std::isfinite(Ku))
        return MMCQ_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    mmcq_t* h = new mmcq();
    h->device = o ? o->device : 0;
    h->gamma = (o && o->gamma > 0) ? o->gamma : 1.7595e11;
    h->mu0 = (o && o->mu0 > 0) ? o->mu0 : 4e-7 * 3.14159265358979323846;
    h->hbar = (o && o->hbar > 0) ? o->hbar : 1.05457182e-34;
    h->alloc = o ? o->alloc : nullptr;
    h->freefn = o ? o->free : nullptr;
    h->actx = o ? o->alloc_ctx : nullptr;
    h->dx = g->dx; h->dy = g->dy; h->dz = g->dz;
    auto bail = [&](int code) { mmcq_destroy(h); return code; };
    if (cudaSetDevice(h->device) != cudaSuccess) return bail(MMCQ_ERR_CUDA);
    if (o && o->stream) h->stream = (cudaStream_t)o->stream;
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MMCQ_ERR_CUDA);
        h->own_stream = true;
    }

    Plan& P = h->P;
    P.nx = g->nx; P.ny = g->ny; P.nz = g->nz; P.B = g->batch;
    P.N = (long long)g->nx * g->ny * g->nz;
    P.px = pow2_at_least(2 * g->nx - 1); if (P.px < 2) P.px = 2;
    P.py = pow2_at_least(2 * g->ny - 1);
    P.pz = pow2_at_least(2 * g->nz - 1);
    if (P.px > 2048 || P.py > 4096 || P.pz > 4096) return bail(MMCQ_ERR_UNSUPPORTED);
    P.L = P.px / 2;
    P.hx = P.L + 1;
    P.hyk = P.py / 2 + 1;
    P.hzk = P.pz / 2 + 1;
    P.nrows = g->ny * g->nz;
    P.twn = std::max(P.px, std::max(P.py, P.pz));
    P.TX = 8;
    while (P.TX > 1 && P.TX / 2 >= P.hx) P.TX /= 2;
    while (P.TX > 1 && !col_fits(P)) P.TX /= 2;
    if (!col_fits(P)) return bail(MMCQ_ERR_UNSUPPORTED);
    P.NT = (P.hx + P.TX - 1) / P.TX;
    P.lt = 0;
    while ((1 << P.lt) < P.TX) P.lt++;
    P.R = rows_per_block(P.L, P.nrows);
    P.nblk = (P.nrows + P.R - 1) / P.R;
    h->rows_rule = P.R;
    if (!x_fits(P)) return bail(MMCQ_ERR_UNSUPPORTED);
    P.fd_nx = make_fastdiv((unsigned)P.nx);
    P.fd_ny = make_fastdiv((unsigned)P.ny);
    P.fd_nz = make_fastdiv((unsigned)P.nz);
    P.fd_L1 = make_fastdiv((unsigned)(P.L + 1));
    P.fd_half = make_fastdiv((unsigned)(P.L / 2 + 1));

    Material& M = h->mat;
    M.exch[0] = (float)(2.0 * Aex / (g->dx * g->dx));
    M.exch[1] = (float)(2.0 * Aex / (g->dy * g->dy));
    M.exch[2] = (float)(2.0 * Aex / (g->dz * g->dz));
    M.two_ku = (float)(2.0 * Ku);
    double ax[3] = {1, 0, 0};
    if (axis) { ax[0] = axis[0]; ax[1] = axis[1]; ax[2] = axis[2]; }
    double an = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
    for (int c = 0; c < 3; c++) M.u[c] = an > 0 ? (float)(ax[c] / an) : 0.f;
    M.pre = (float)(-h->gamma / (1.0 + alpha * alpha));
    M.alpha = (float)alpha;
    M.vc = g->dx * g->dy * g->dz;
    M.hbar = h->hbar;

    const long long BN = (long long)P.B * P.N;
    Buffers& Bf = h->Bf;
    bool ok = true;
    auto A = [&](size_t bytes) { void* p = dev_alloc(h, bytes); if (!p) ok = false; return p; };
    Bf.m[0] = (float4*)A(sizeof(float4) * BN);
    Bf.m[1] = (float4*)A(sizeof(float4) * BN);
    Bf.ms = (float4*)A(sizeof(float4) * BN);
    for (int k = 0; k < MAX_STAGES; k++) Bf.k[k] = (float4*)A(sizeof(float4) * BN);
    Bf.e6 = (float4*)A(sizeof(float4) * BN);
    const long long spec_n = (long long)P.B * P.nz * P.NT * P.ny * 3 * P.TX;
    Bf.spec = (float2*)A(sizeof(float2) * spec_n);
    if (P.nz > 1) Bf.spec2 = (float2*)A(sizeof(float2) * (long long)P.B * P.nz * P.NT * P.py * 3 * P.TX);
    Bf.kern = (float*)A(sizeof(float) * 6LL * P.hzk * P.hyk * P.NT * P.TX);
    for (int k = 0; k < MAX_MODES; k++) Bf.prof[k] = nullptr;
    Bf.ip = (InstParams*)A(sizeof(InstParams) * P.B);
    Bf.st = (InstState*)A(sizeof(InstState) * P.B);
    // block partials: room for one row per block (the autotuner may lower P.R)
    Bf.xpart = (double*)A(sizeof(double) * MAX_MODES * (long long)P.B * P.nrows);
    Bf.mpart = (double*)A(sizeof(double) * 3LL * P.B * P.nrows);
    Bf.mhist = nullptr;   // allocated by mmcq_set_recording
    Bf.epart = (float*)A(sizeof(float) * (long long)P.B * P.nrows);
    Bf.counter = (unsigned*)A(sizeof(unsigned) * P.B);
    Bf.hcap = 1 << 16;
    Bf.hist = (double*)A(sizeof(double) * (long long)P.B * Bf.hcap);
    Bf.flags = (int*)A(sizeof(int));
    float2* tw = (float2*)A(sizeof(float2) * P.twn);
    Bf.tw = tw;
    Bf.fout = (float4*)A(sizeof(float4) * P.N);
    h->ms_dev = (float*)A(sizeof(float) * P.N);
    h->stage3 = (float*)A(sizeof(float) * 3 * P.N);
    h->dscratch = (double*)A(sizeof(double) * P.B);
    Bf.cpart_n = coupling_blocks(P.N);
    Bf.cpart = (double*)A(sizeof(double) * (long long)P.B * Bf.cpart_n);
    if (!ok) { h->err = "device allocation failed"; return bail(MMCQ_ERR_CUDA); }

    if (set_smem_limits() != cudaSuccess) return bail(MMCQ_ERR_CUDA);
    if (encode_spec_map(h) != MMCQ_OK) return bail(MMCQ_ERR_CUDA);
    {
        std::vector<float2> t(P.twn);
        for (int k = 0; k < P.twn; k++) {
            double a = -2.0 * 3.14159265358979323846 * k / P.twn;
            t[k] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        if (cudaMemcpy(tw, t.data(), sizeof(float2) * P.twn, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(MMCQ_ERR_CUDA);
    }
    // demag kernel, FP64 on the device
    {
        size_t sbytes = sizeof(double2) * (size_t)P.px * P.py * P.pz;
        void* scratch = nullptr;
        if (h->alloc) scratch = h->alloc((sbytes + 255) & ~(size_t)255, h->actx);
        else if (cudaMalloc(&scratch, sbytes) != cudaSuccess) scratch = nullptr;
        if (!scratch) { h->err = "scratch allocation failed"; return bail(MMCQ_ERR_CUDA); }
        cudaError_t e = build_demag_kernel(P, g->dx, g->dy, g->dz, h->mu0, Bf.kern, (double2*)scratch, h->stream);
        if (h->freefn) h->freefn(scratch, h->actx);
        else if (!h->alloc) cudaFree(scratch);
        if (e != cudaSuccess) { h->err = std::string("demag kernel: ") + cudaGetErrorString(e); return bail(MMCQ_ERR_CUDA); }
    }
    // initial state
    h->ms_host.assign(P.N, (float)Ms);
    h->ip.assign(P.B, InstParams{});
    h->g.assign((size_t)P.B * MAX_MODES, 0.0);
    h->g_mode.assign((size_t)P.B * MAX_MODES, 0);
    refresh_scales(h);
    std::vector<InstState> st(P.B);
    for (auto& s : st) {
        std::memset(&s, 0, sizeof(s));
    }
    if (cudaMemcpy(h->ms_dev, h->ms_host.data(), sizeof(float) * P.N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(Bf.st, st.data(), sizeof(InstState) * P.B, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(Bf.ip, h->ip.data(), sizeof(InstParams) * P.B, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(Bf.counter, 0, sizeof(unsigned) * P.B) != cudaSuccess ||
        cudaMemset(Bf.flags, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(Bf.spec, 0, sizeof(float2) * spec_n) != cudaSuccess)
        return bail(MMCQ_ERR_CUDA);
    {
        std::vector<float> m3(3 * P.N, 0.f);
        for (long long i = 0; i < P.N; i++) m3[3 * i] = 1.f;
        if (cudaMemcpy(h->stage3, m3.data(), sizeof(float) * 3 * P.N, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(MMCQ_ERR_CUDA);
        for (int k = 0; k < 2; k++)
            if (launch_set_m(Bf.m[k], h->stage3, h->ms_dev, P.N, 0, P.B, Bf.flags, h->stream) != cudaSuccess)
                return bail(MMCQ_ERR_CUDA);
        for (int k = 0; k < MAX_STAGES; k++)
            if (cudaMemsetAsync(Bf.k[k], 0, sizeof(float4) * BN, h->stream) != cudaSuccess) return bail(MMCQ_ERR_CUDA);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(MMCQ_ERR_CUDA);
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return MMCQ_OK;
}

void mmcq_destroy(mmcq_t* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) dev_release(h, p);
    for (auto e : h->events) cudaEventDestroy(e);
    for (auto& q : h->posts) {
        if (q.host) cudaFreeHost(q.host);
        if (q.ev) cudaEventDestroy(q.ev);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* mmcq_last_error(const mmcq_t* h) { return h ? h->err.c_str() : "null handle"; }

int mmcq_info_get(mmcq_t* h, mmcq_info* out) {
    if (!h || !out) return MMCQ_ERR_ARG;
    out->px = h->P.px; out->py = h->P.py; out->pz = h->P.pz;
    out->tile = h->P.TX;
    out->device_bytes = h->bytes;
    out->setup_ms = h->setup_ms;
    out->launches_per_step = (int64_t)(h->kind == KIND_RK4 ? 4 : 6) * (2 + convolution_launches(h->P));
    return MMCQ_OK;
}

int mmcq_set_ms_map(mmcq_t* h, const float* ms, int where) {
    if (!h || !ms) return MMCQ_ERR_ARG;
    const long long N = h->P.N;
    if (where == MMCQ_DEVICE) {
        CK(h, cudaMemcpyAsync(h->ms_dev, ms, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->ms_host.data(), ms, sizeof(float) * N, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    } else if (where == MMCQ_HOST) {
        std::memcpy(h->ms_host.data(), ms, sizeof(float) * N);
        CK(h, cudaMemcpyAsync(h->ms_dev, ms, sizeof(float) * N, cudaMemcpyHostToDevice, h->stream));
    } else return MMCQ_ERR_ARG;
    for (auto& v : h->ms_host) if (!(v > 0)) v = 0;
    for (int k = 0; k < 2; k++) CK(h, launch_apply_ms(h->Bf.m[k], h->ms_dev, N, h->P.B, h->stream));
    refresh_scales(h);
    int r = upload_params(h);
    if (r) return r;
    return edit_state(h, -1, [](InstState& s, int) { s.have_k1 = 0; });
}

int mmcq_set_bias(mmcq_t* h, int inst, const double B[3]) {
    if (!h || !B || !valid_inst(h, inst, true)) return MMCQ_ERR_ARG;
    for (int b = 0; b < h->P.B; b++)
        if (inst < 0 || b == inst)
            for (int c = 0; c < 3; c++) h->ip[b].bext[c] = B[c];
    int r = upload_params(h);
    if (r) return r;
    return edit_state(h, inst, [](InstState& s, int) { s.have_k1 = 0; });
}

int mmcq_set_m(mmcq_t* h, int inst, const float* m, int where) {
    if (!h || !m || !valid_inst(h, inst, true) || (where != MMCQ_HOST && where != MMCQ_DEVICE)) return MMCQ_ERR_ARG;
    const long long N = h->P.N;
    const float* src = m;
    if (where == MMCQ_HOST) {
        CK(h, cudaMemcpyAsync(h->stage3, m, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, h->stream));
        src = h->stage3;
    }
    int b0 = inst < 0 ? 0 : inst, nb = inst < 0 ? h->P.B : 1;
    for (int k = 0; k < 2; k++) CK(h, launch_set_m(h->Bf.m[k], src, h->ms_dev, N, b0, nb, h->Bf.flags, h->stream));
    return edit_state(h, inst, [](InstState& s, int) { s.have_k1 = 0; });
}

int mmcq_get_m(mmcq_t* h, int inst, float* out, int where) {
    if (!h || !out || !valid_inst(h, inst, false) || (where != MMCQ_HOST && where != MMCQ_DEVICE)) return MMCQ_ERR_ARG;
    int r = check_flags(h);
    InstState s;
    CK(h, cudaMemcpy(&s, h->Bf.st + inst, sizeof(InstState), cudaMemcpyDeviceToHost));
    const long long N = h->P.N;
    const float4* src = h->Bf.m[s.mcur] + (long long)inst * N;
    if (where == MMCQ_DEVICE) {
        CK(h, launch_get_m(src, out, N, h->stream));
    } else {
        CK(h, launch_get_m(src, h->stage3, N, h->stream));
        CK(h, cudaMemcpyAsync(out, h->stage3, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return r;
}

int mmcq_set_cavity_mode(mmcq_t* h, int inst, int mode, double omega_c, double kappa, double g,
                         const float* profile, int profile_is_brms) {
    if (!h || !valid_inst(h, inst, true) || mode < 0 || mode >= MAX_MODES || !std::isfinite(omega_c) ||
        !std::isfinite(kappa) || !std::isfinite(g))
        return MMCQ_ERR_ARG;
    const long long N = h->P.N;
    if (profile) {
        if (!h->Bf.prof[mode]) {
            h->Bf.prof[mode] = (float4*)dev_alloc(h, sizeof(float4) * N);
            if (!h->Bf.prof[mode]) return fail(h, MMCQ_ERR_CUDA, "profile allocation failed");
        }
        std::vector<float4> p(N);
        for (long long i = 0; i < N; i++) p[i] = make_float4(profile[3 * i], profile[3 * i + 1], profile[3 * i + 2], 0.f);
        CK(h, cudaStreamSynchronize(h->stream));
        CK(h, cudaMemcpy(h->Bf.prof[mode], p.data(), sizeof(float4) * N, cudaMemcpyHostToDevice));
    }
    for (int b = 0; b < h->P.B; b++) {
        if (inst >= 0 && b != inst) continue;
        h->ip[b].wc[mode] = omega_c;
        h->ip[b].kappa[mode] = kappa;
        h->ip[b].cav_on[mode] = 1;
        h->g[b * MAX_MODES + mode] = g;
        h->g_mode[b * MAX_MODES + mode] = profile_is_brms ? 0 : 1;
        if (profile_is_brms) h->ip[b].brms_scale[mode] = 1.0;
    }
    if (mode + 1 > h->nmodes) h->nmodes = mode + 1;
    refresh_scales(h);
    int r = upload_params(h);
    if (r) return r;
    std::vector<InstParams> ip = h->ip;
    return edit_state(h, inst, [&](InstState& s, int b) { reset_memory(ip[b], s); });
}

int mmcq_set_cavity(mmcq_t* h, int inst, double omega_c, double kappa, double g, const float* profile,
                    int profile_is_brms) {
    return mmcq_set_cavity_mode(h, inst, 0, omega_c, kappa, g, profile, profile_is_brms);
}

int mmcq_set_cavity_init_mode(mmcq_t* h, int inst, int mode, double x0, double p0) {
    if (!h || !valid_inst(h, inst, true) || mode < 0 || mode >= MAX_MODES || !std::isfinite(x0) ||
        !std::isfinite(p0))
        return MMCQ_ERR_ARG;
    for (int b = 0; b < h->P.B; b++)
        if (inst < 0 || b == inst) { h->ip[b].x0[mode] = x0; h->ip[b].p0[mode] = p0; }
    int r = upload_params(h);
    if (r) return r;
    std::vector<InstParams> ip = h->ip;
    return edit_state(h, inst, [&](InstState& s, int b) {
        s.a_re[mode] = s.as_re[mode] = 0.5 * ip[b].x0[mode];
        s.a_im[mode] = s.as_im[mode] = -0.5 * ip[b].p0[mode];
        s.have_k1 = 0;
    });
}

int mmcq_set_cavity_init(mmcq_t* h, int inst, double x0, double p0) {
    return mmcq_set_cavity_init_mode(h, inst, 0, x0, p0);
}

int mmcq_reset_cavity(mmcq_t* h, int inst) {
    if (!h || !valid_inst(h, inst, true)) return MMCQ_ERR_ARG;
    std::vector<InstParams> ip = h->ip;
    return edit_state(h, inst, [&](InstState& s, int b) { reset_memory(ip[b], s); });
}

int mmcq_disable_cavity(mmcq_t* h, int inst) {
    if (!h || !valid_inst(h, inst, true)) return MMCQ_ERR_ARG;
    for (int b = 0; b < h->P.B; b++)
        if (inst < 0 || b == inst)
            for (int k = 0; k < MAX_MODES; k++) h->ip[b].cav_on[k] = 0;
    int r = upload_params(h);
    if (r) return r;
    return edit_state(h, inst, [](InstState& s, int) { s.have_k1 = 0; });
}

int mmcq_set_integrator(mmcq_t* h, int kind, double tol, int cavity_mode) {
    if (!h || (kind != MMCQ_RK4 && kind != MMCQ_DP45) || (cavity_mode != MMCQ_CAVITY_E && cavity_mode != MMCQ_CAVITY_P) ||
        (kind == MMCQ_DP45 && !(tol > 0)))
        return MMCQ_ERR_ARG;
    h->kind = kind;
    h->tol = tol;
    h->mode = cavity_mode;
    // the accepted state moves to buffer 0 (RK4 keeps it there)
    const int B = h->P.B;
    const long long N = h->P.N;
    std::vector<InstState> st(B);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(st.data(), h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToHost));
    for (int b = 0; b < B; b++)
        if (st[b].mcur == 1)
            CK(h, cudaMemcpyAsync(h->Bf.m[0] + (long long)b * N, h->Bf.m[1] + (long long)b * N, sizeof(float4) * N,
                                  cudaMemcpyDeviceToDevice, h->stream));
    return edit_state(h, -1, [](InstState& s, int) {
        s.mcur = 0;
        s.have_k1 = 0;
        s.k1slot = 0;
        for (int k = 0; k < MAX_MODES; k++) {
            s.as_re[k] = s.a_re[k];
            s.as_im[k] = s.a_im[k];
        }
    });
}

int mmcq_set_horizon(mmcq_t* h, int inst, double t_end) {
    if (!h || !valid_inst(h, inst, true) || !std::isfinite(t_end)) return MMCQ_ERR_ARG;
    return edit_state(h, inst, [&](InstState& s, int) {
        s.t_end = t_end > 0 ? t_end : 0.0;
        s.done = (s.t_end > 0 && s.t >= s.t_end) ? 1 : 0;
        if (s.t_end > 0 && s.dt > 0 && s.t + s.dt > s.t_end) s.dt = s.t_end - s.t;
    });
}

int mmcq_step(mmcq_t* h, int64_t n, double dt) {
    if (!h || n < 0 || !std::isfinite(dt)) return MMCQ_ERR_ARG;
    if (h->kind == KIND_RK4 && !(dt > 0)) return fail(h, MMCQ_ERR_ARG, "RK4 needs dt > 0");
    if (n == 0) return MMCQ_OK;
    if (dt > 0) CK(h, launch_set_dt(h->Bf.st, h->P.B, dt, h->stream));
    return enqueue_steps(h, n);
}

int mmcq_sync(mmcq_t* h) {
    if (!h) return MMCQ_ERR_ARG;
    return check_flags(h);
}

namespace {
// Cavity read-out of mode k for instances b0 .. b0 + nb - 1 from their states
// and coupling sums (Sec. 2.2; in P-mode alpha is rebuilt from S and C).
void fill_cavity(const mmcq_t* h, const InstState* st, const double* X, int b0, int nb, int k, mmcq_cavity* out) {
    for (int q = 0; q < nb; q++) {
        const InstState& s = st[q];
        const InstParams& ip = h->ip[b0 + q];
        std::complex<double> a(s.a_re[k], s.a_im[k]);
        double G = ip.cav_on[k] ? 2.0 * s.a_re[k] : 0.0;
        if (ip.cav_on[k] && h->mode == CAV_P) {
            std::complex<double> a0(0.5 * ip.x0[k], -0.5 * ip.p0[k]);
            a = std::exp(-std::complex<double>(ip.kappa[k], ip.wc[k]) * s.tcav) *
                (a0 + std::complex<double>(-s.S[k] / h->hbar, s.C[k] / h->hbar));
            double e = std::exp(-ip.kappa[k] * s.tcav);
            G = e * std::cos(ip.wc[k] * s.tcav) * (ip.x0[k] - 2.0 * s.S[k] / h->hbar) -
                e * std::sin(ip.wc[k] * s.tcav) * (ip.p0[k] - 2.0 * s.C[k] / h->hbar);
        }
        mmcq_cavity& o = out[q];
        o.t = s.t;
        o.t_cav = s.tcav;
        o.re_alpha = a.real();
        o.im_alpha = a.imag();
        o.n_photon = std::norm(a);
        o.Gamma = G;
        o.S = s.S[k];
        o.C = s.C[k];
        o.X = X[q];
        o.dt = s.dt;
        o.accepted = s.nacc;
        o.rejected = s.nrej;
        o.err = s.err;
    }
}
}  // namespace

int mmcq_get_cavity_mode(mmcq_t* h, int inst, int mode, mmcq_cavity* out) {
    if (!h || !out || !valid_inst(h, inst, true) || mode < 0 || mode >= MAX_MODES) return MMCQ_ERR_ARG;
    int r = check_flags(h);
    const int b0 = inst < 0 ? 0 : inst, nb = inst < 0 ? h->P.B : 1;
    std::vector<InstState> st(nb);
    std::vector<double> X(nb, 0.0);
    CK(h, cudaMemcpy(st.data(), h->Bf.st + b0, sizeof(InstState) * nb, cudaMemcpyDeviceToHost));
    CK(h, launch_coupling_sum(h->Bf, h->P.N, h->mat.vc, b0, nb, mode, h->dscratch, h->stream));
    CK(h, cudaMemcpyAsync(X.data(), h->dscratch, sizeof(double) * nb, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    fill_cavity(h, st.data(), X.data(), b0, nb, mode, out);
    return r;
}

int mmcq_get_cavity(mmcq_t* h, int inst, mmcq_cavity* out) { return mmcq_get_cavity_mode(h, inst, 0, out); }

// Slot layout: B InstState, B doubles (X), one int (flags).
static size_t post_bytes(const mmcq_t* h) {
    return sizeof(InstState) * h->P.B + sizeof(double) * h->P.B + sizeof(int);
}

int mmcq_post_cavity(mmcq_t* h) {
    if (!h) return MMCQ_ERR_ARG;
    if (h->post_count == MMCQ_POST_SLOTS) return fail(h, MMCQ_ERR_STATE, "post_cavity: every slot holds an untaken read-out");
    if (h->posts.empty()) {
        h->posts.resize(MMCQ_POST_SLOTS);
        for (auto& q : h->posts) {
            CK(h, cudaMallocHost(&q.host, post_bytes(h)));
            CK(h, cudaEventCreateWithFlags(&q.ev, cudaEventDisableTiming));
        }
    }
    const int B = h->P.B;
    mmcq::Post& q = h->posts[(h->post_head + h->post_count) % MMCQ_POST_SLOTS];
    char* p = static_cast<char*>(q.host);
    CK(h, launch_coupling_sum(h->Bf, h->P.N, h->mat.vc, 0, B, 0, h->dscratch, h->stream));
    CK(h, cudaMemcpyAsync(p, h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToHost, h->stream));
    p += sizeof(InstState) * B;
    CK(h, cudaMemcpyAsync(p, h->dscratch, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream));
    p += sizeof(double) * B;
    CK(h, cudaMemcpyAsync(p, h->Bf.flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaEventRecord(q.ev, h->stream));
    h->post_count++;
    return MMCQ_OK;
}

int mmcq_take_cavity(mmcq_t* h, mmcq_cavity* out) {
    if (!h || !out) return MMCQ_ERR_ARG;
    if (h->post_count == 0) return fail(h, MMCQ_ERR_STATE, "take_cavity: nothing posted");
    const int B = h->P.B;
    mmcq::Post& q = h->posts[h->post_head];
    CK(h, cudaEventSynchronize(q.ev));
    h->post_head = (h->post_head + 1) % MMCQ_POST_SLOTS;
    h->post_count--;
    const char* p = static_cast<const char*>(q.host);
    const InstState* st = reinterpret_cast<const InstState*>(p);
    const double* X = reinterpret_cast<const double*>(p + sizeof(InstState) * B);
    int f = 0;
    std::memcpy(&f, p + sizeof(InstState) * B + sizeof(double) * B, sizeof(int));
    fill_cavity(h, st, X, 0, B, 0, out);
    if (f & (FLAG_NAN | FLAG_DT_UNDERFLOW | FLAG_TIMEOUT)) return check_flags(h);
    return MMCQ_OK;
}

int mmcq_get_dt_history(mmcq_t* h, int inst, double* out, int64_t max, int64_t* n) {
    if (!h || !valid_inst(h, inst, false) || max < 0 || (max > 0 && !out)) return MMCQ_ERR_ARG;
    int r = check_flags(h);
    InstState s;
    CK(h, cudaMemcpy(&s, h->Bf.st + inst, sizeof(InstState), cudaMemcpyDeviceToHost));
    if (n) *n = s.nhist;
    long long c = s.nhist < h->Bf.hcap ? s.nhist : h->Bf.hcap;
    if (c > max) c = max;
    if (c > 0)
        CK(h, cudaMemcpy(out, h->Bf.hist + (long long)inst * h->Bf.hcap, sizeof(double) * c, cudaMemcpyDeviceToHost));
    if (s.nhist > h->Bf.hcap && r == MMCQ_OK) return fail(h, MMCQ_ERR_STATE, "step history overflowed its capacity");
    return r;
}

int mmcq_eval_field(mmcq_t* h, int inst, int terms, float* out, int where) {
    if (!h || !out || !valid_inst(h, inst, false) || (where != MMCQ_HOST && where != MMCQ_DEVICE) ||
        terms < 0 || terms > MMCQ_TERM_ALL)
        return MMCQ_ERR_ARG;
    StageArgs A = step_args(h);
    A.terms = terms; A.field_only = 1; A.inst0 = inst; A.stage = 0; A.record = 0;
    int r = run_stage(h, A, 1);
    if (r) return r;
    const long long N = h->P.N;
    if (where == MMCQ_DEVICE) {
        CK(h, launch_get_field(h->Bf.fout, out, N, h->stream));
    } else {
        CK(h, launch_get_field(h->Bf.fout, h->stage3, N, h->stream));
        CK(h, cudaMemcpyAsync(out, h->stage3, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return MMCQ_OK;
}

int mmcq_profile(mmcq_t* h, int enable) {
    if (!h) return MMCQ_ERR_ARG;
    if (enable) {
        CK(h, cudaStreamSynchronize(h->stream));
        h->recs.clear();
    }
    h->profiling = enable != 0;
    return MMCQ_OK;
}

int mmcq_profile_read(mmcq_t* h, mmcq_kernel_stat* out, int max, int* n) {
    if (!h || !out || max < 0) return MMCQ_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    double ms[NCLS] = {0}, by[NCLS] = {0};
    int64_t cnt[NCLS] = {0};
    for (const auto& r : h->recs) {
        float t = 0.f;
        CK(h, cudaEventElapsedTime(&t, h->events[r.ev], h->events[r.ev + 1]));
        ms[r.cls] += t;
        by[r.cls] += r.bytes;
        cnt[r.cls]++;
    }
    int k = 0;
    for (int c = 0; c < NCLS && k < max; c++) {
        if (!cnt[c]) continue;
        std::memset(&out[k], 0, sizeof(mmcq_kernel_stat));
        std::snprintf(out[k].name, sizeof(out[k].name), "%s", CLS_NAMES[c]);
        out[k].launches = cnt[c];
        out[k].total_ms = ms[c];
        out[k].bytes = by[c];
        k++;
    }
    if (n) *n = k;
    return MMCQ_OK;
}

int64_t mmcq_launch_count(const mmcq_t* h) { return h ? h->launches : -1; }

// ---- excitation and spectra (Appendix C) --------------------------------------
int mmcq_set_drive(mmcq_t* h, int inst, double amp, double omega_cut, double t0) {
    if (!h || !valid_inst(h, inst, true) || !std::isfinite(amp) || !std::isfinite(omega_cut) ||
        !std::isfinite(t0))
        return MMCQ_ERR_ARG;
    for (int b = 0; b < h->P.B; b++)
        if (inst < 0 || b == inst) {
            h->ip[b].drv_on = amp != 0.0;
            h->ip[b].drv_amp = amp;
            h->ip[b].drv_wcut = omega_cut;
            h->ip[b].drv_t0 = t0;
        }
    return upload_params(h);
}

int mmcq_set_recording(mmcq_t* h, int every) {
    if (!h || every < 0) return MMCQ_ERR_ARG;
    if (every > 0 && !h->Bf.mhist) {
        h->Bf.mhist = (double*)dev_alloc(h, sizeof(double) * 4LL * h->P.B * h->Bf.hcap);
        if (!h->Bf.mhist) return fail(h, MMCQ_ERR_CUDA, "device allocation failed");
    }
    h->record = every;
    return MMCQ_OK;
}

int mmcq_get_mavg_history(mmcq_t* h, int inst, double* out, int64_t max, int64_t* n) {
    if (!h || !valid_inst(h, inst, false) || max < 0 || (max > 0 && !out)) return MMCQ_ERR_ARG;
    int r = check_flags(h);
    InstState s;
    CK(h, cudaMemcpy(&s, h->Bf.st + inst, sizeof(InstState), cudaMemcpyDeviceToHost));
    if (n) *n = s.nmh;
    long long c = s.nmh < h->Bf.hcap ? s.nmh : h->Bf.hcap;
    if (c > max) c = max;
    if (c > 0 && h->Bf.mhist)
        CK(h, cudaMemcpy(out, h->Bf.mhist + 4LL * inst * h->Bf.hcap, sizeof(double) * 4 * c,
                         cudaMemcpyDeviceToHost));
    if (s.nmh > h->Bf.hcap && r == MMCQ_OK) return fail(h, MMCQ_ERR_STATE, "m-average history overflowed its capacity");
    return r;
}

int mmcq_spectrum(mmcq_t* h, int inst, int comp, const double* omega, int nw, double* out) {
    if (!h || !valid_inst(h, inst, false) || comp < 0 || comp > 2 || nw < 0 || (nw > 0 && (!omega || !out)))
        return MMCQ_ERR_ARG;
    if (nw == 0) return MMCQ_OK;
    int r = check_flags(h);
    if (r) return r;
    if (!h->Bf.mhist) return fail(h, MMCQ_ERR_STATE, "recording was never enabled");
    InstState s;
    CK(h, cudaMemcpy(&s, h->Bf.st + inst, sizeof(InstState), cudaMemcpyDeviceToHost));
    const long long ns = s.nmh < h->Bf.hcap ? s.nmh : h->Bf.hcap;
    if (nw > h->spec_cap) {
        h->spec_buf = (double*)dev_alloc(h, sizeof(double) * 3LL * nw);
        if (!h->spec_buf) { h->spec_cap = 0; return fail(h, MMCQ_ERR_CUDA, "device allocation failed"); }
        h->spec_cap = nw;
    }
    double* dw = h->spec_buf;
    double* dout = h->spec_buf + nw;
    CK(h, cudaMemcpyAsync(dw, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_spectrum(h->Bf.mhist + 4LL * inst * h->Bf.hcap, ns, comp, dw, nw, dout, h->stream));
    CK(h, cudaMemcpyAsync(out, dout, sizeof(double) * 2 * nw, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return MMCQ_OK;
}

// ---- autotuning of the launch parameters -------------------------------------------
namespace {

// Choices found per device and shape, reused by later handles of the process.
std::mutex g_tune_mu;
std::map<std::string, mmcq_tuning> g_tune_cache;

std::string tune_key(const mmcq_t* h) {
    const Plan& P = h->P;
    return std::to_string(h->device) + ":" + std::to_string(P.nx) + "x" + std::to_string(P.ny) + "x" +
           std::to_string(P.nz) + "b" + std::to_string(P.B) + "t" + std::to_string(P.TX);
}

void tune_read(const mmcq_t* h, mmcq_tuning* t) {
    int gmax[4], zc, zr, yc, yr[2];
    conv_tunables(h->P, gmax, &zc, &zr, &yc, yr);
    t->x_rows = h->P.R;
    for (int k = 0; k < 4; k++) t->col_groups[k] = gmax[k] ? (h->tune.col_g[k] > 0 ? h->tune.col_g[k] : gmax[k]) : 0;
    t->z_split = zc ? (h->tune.z_split < 0 ? zr : h->tune.z_split) : -1;
    t->x_pipe = h->spec_map.valid ? (h->tune.x_pipe < 0 ? 1 : h->tune.x_pipe) : -1;
    for (int k = 0; k < 2; k++) t->y_split[k] = yc ? (h->tune.y_split[k] < 0 ? yr[k] : h->tune.y_split[k]) : -1;
}

// Apply a plan; false (nothing changed) if it is not one of this grid's choices.
bool tune_apply(mmcq_t* h, const mmcq_tuning* t) {
    int gmax[4], zc, zr, yc, yr[2];
    conv_tunables(h->P, gmax, &zc, &zr, &yc, yr);
    if (!t) {
        h->tune = Tune{{0, 0, 0, 0}, -1, -1, {-1, -1}};
        h->P.R = h->rows_rule;
    } else {
        if (t->x_rows < 1 || t->x_rows > h->rows_rule) return false;
        for (int k = 0; k < 4; k++)
            if (t->col_groups[k] < 0 || (gmax[k] == 0 && t->col_groups[k] != 0) || t->col_groups[k] > gmax[k])
                return false;
        if (t->z_split < -1 || t->z_split > 1 || (!zc && t->z_split == 1)) return false;
        if (t->x_pipe < -1 || t->x_pipe > 1 || (!h->spec_map.valid && t->x_pipe == 1)) return false;
        for (int k = 0; k < 2; k++)
            if (t->y_split[k] < -1 || t->y_split[k] > 1 || (!yc && t->y_split[k] == 1)) return false;
        for (int k = 0; k < 4; k++) h->tune.col_g[k] = t->col_groups[k];
        for (int k = 0; k < 2; k++) h->tune.y_split[k] = t->y_split[k];
        h->tune.z_split = t->z_split;
        h->tune.x_pipe = t->x_pipe;
        h->P.R = t->x_rows;
    }
    h->P.nblk = (h->P.nrows + h->P.R - 1) / h->P.R;
    h->tune_epoch++;
    return true;
}

}  // namespace

int mmcq_set_tuning(mmcq_t* h, const mmcq_tuning* t) {
    if (!h) return MMCQ_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    if (!tune_apply(h, t)) return fail(h, MMCQ_ERR_ARG, "set_tuning: not a plan of this grid");
    return MMCQ_OK;
}

int mmcq_get_tuning(mmcq_t* h, mmcq_tuning* out) {
    if (!h || !out) return MMCQ_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    tune_read(h, out);
    return MMCQ_OK;
}

int mmcq_autotune(mmcq_t* h, int reps, mmcq_tuning* out) {
    if (!h || !out || reps < 1) return MMCQ_ERR_ARG;
    const std::string key = tune_key(h);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            mmcq_tuning t = it->second;
            if (!tune_apply(h, &t)) return fail(h, MMCQ_ERR_STATE, "autotune: cached plan does not fit");
            *out = t;
            out->candidates = 0;
            return MMCQ_OK;
        }
    }
    int r = check_flags(h);
    if (r) return r;
    const Plan& P = h->P;
    const int B = P.B;
    // timed: one middle Runge-Kutta stage of the whole batch (stage input,
    // transforms, field, torque, coupling sums and the per-instance finish),
    // which writes only that stage's scratch buffers and the instance states;
    // the states are put back afterwards, so the integration is unchanged
    std::vector<InstState> saved(B);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(saved.data(), h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToHost));
    StageArgs A = step_args(h);
    A.stage = h->kind == KIND_RK4 ? 1 : 3;
    A.record = 0;
    // passes of one stage: 0 = x forward, 1..4 = column parts 0..3, 5 = x inverse;
    // events bracket each pass so that a knob is judged on the passes it changes
    const int parts0 = P.nz == 1 ? 0 : 1, parts1 = P.nz == 1 ? 0 : 3;
    std::vector<cudaEvent_t> ev;
    int err = MMCQ_OK;
    auto cleanup = [&]() -> int {
        for (auto e : ev) cudaEventDestroy(e);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
            cudaMemcpy(h->Bf.st, saved.data(), sizeof(InstState) * B, cudaMemcpyHostToDevice) != cudaSuccess)
            return MMCQ_ERR_CUDA;
        return MMCQ_OK;
    };
    const int nev = 2 + (parts1 - parts0 + 1) + 1;    // start, after x forward, after each part, after x inverse
    for (int q = 0; q < nev; q++) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cleanup();
            return fail(h, MMCQ_ERR_CUDA, "autotune: event creation failed");
        }
        ev.push_back(e);
    }
    int ncand = 0;
    auto eval = [&](bool timed) -> cudaError_t {
        cudaError_t e;
        int q = 0;
        if (timed && (e = cudaEventRecord(ev[q++], h->stream)) != cudaSuccess) return e;
        if ((e = launch_xfwd(h->P, h->Bf, A, B, h->stream)) != cudaSuccess) return e;
        if (timed && (e = cudaEventRecord(ev[q++], h->stream)) != cudaSuccess) return e;
        for (int part = parts0; part <= parts1; part++) {
            if ((e = launch_conv_part(h->P, h->Bf, A, B, h->stream, part, &h->tune)) != cudaSuccess) return e;
            if (timed && (e = cudaEventRecord(ev[q++], h->stream)) != cudaSuccess) return e;
        }
        if ((e = launch_xinv(h->P, h->mat, h->Bf, A, B, h->stream, &h->spec_map, &h->tune)) != cudaSuccess) return e;
        if (timed && (e = cudaEventRecord(ev[q++], h->stream)) != cudaSuccess) return e;
        return cudaSuccess;
    };
    // median time per pass over `reps` stages, after one untimed; pass k is
    // slot 0 (x forward), 1 + part, or 5 (x inverse)
    auto measure = [&](double (&ms)[6]) -> int {
        std::vector<std::vector<float>> t(6, std::vector<float>(reps, 0.f));
        if (eval(false) != cudaSuccess) return MMCQ_ERR_CUDA;
        for (int q = 0; q < reps; q++) {
            if (eval(true) != cudaSuccess || cudaEventSynchronize(ev[nev - 1]) != cudaSuccess) return MMCQ_ERR_CUDA;
            std::vector<int> slot;
            slot.push_back(0);
            for (int part = parts0; part <= parts1; part++) slot.push_back(1 + part);
            slot.push_back(5);
            for (size_t k = 0; k < slot.size(); k++)
                if (cudaEventElapsedTime(&t[slot[k]][q], ev[k], ev[k + 1]) != cudaSuccess) return MMCQ_ERR_CUDA;
        }
        for (int k = 0; k < 6; k++) {
            std::sort(t[k].begin(), t[k].end());
            ms[k] = t[k][reps / 2];
        }
        ncand++;
        return MMCQ_OK;
    };
    auto total = [](const double (&ms)[6]) { return ms[0] + ms[1] + ms[2] + ms[3] + ms[4] + ms[5]; };
    mmcq_tuning best{};
    tune_apply(h, nullptr);
    tune_read(h, &best);
    double rule[6], cur[6];
    if ((err = measure(rule))) {
        cleanup();
        return fail(h, err, "autotune: timing failed");
    }
    std::copy(rule, rule + 6, cur);
    // one knob at a time, the others at their best so far, judged on the
    // passes that knob changes (slots)
    auto trial = [&](const mmcq_tuning& c, std::initializer_list<int> slots) -> int {
        mmcq_tuning t = c;
        if (!tune_apply(h, &t)) return MMCQ_OK;
        double ms[6];
        int e = measure(ms);
        if (e) return e;
        double a = 0, b = 0;
        for (int k : slots) { a += ms[k]; b += cur[k]; }
        if (a < b) {
            best = t;
            for (int k : slots) cur[k] = ms[k];
        }
        tune_apply(h, &best);
        return MMCQ_OK;
    };
    for (int R = h->rows_rule / 2; R >= 1 && R >= h->rows_rule / 4 && !err; R /= 2) {
        mmcq_tuning c = best;
        c.x_rows = R;
        err = trial(c, {0, 5});
    }
    int gmax[4], zc, zr, yc, yr[2];
    conv_tunables(P, gmax, &zc, &zr, &yc, yr);
    if (zc && !err) {
        mmcq_tuning c = best;
        c.z_split = 1 - zr;
        err = trial(c, {3});
    }
    for (int k = 0; k < 2 && yc && !err; k++) {
        mmcq_tuning c = best;
        c.y_split[k] = 1 - yr[k];
        err = trial(c, {k == 0 ? 2 : 4});
    }
    for (int k = 0; k < 4 && !err; k++) {
        for (int G = 1; G < gmax[k] && !err; G *= 2) {
            mmcq_tuning c = best;
            c.col_groups[k] = G;
            err = trial(c, {1 + k});
        }
    }
    if (h->spec_map.valid && !err) {
        mmcq_tuning c = best;
        c.x_pipe = 0;
        err = trial(c, {5});
    }
    const double rule_ms = total(rule), best_ms = total(cur);
    if (cleanup() != MMCQ_OK) err = MMCQ_ERR_CUDA;
    if (err) {
        tune_apply(h, nullptr);
        return fail(h, err, "autotune: timing failed");
    }
    tune_apply(h, &best);
    best.eval_ms = best_ms;
    best.rule_ms = rule_ms;
    best.candidates = ncand;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    *out = best;
    return MMCQ_OK;
}

// ---- discrete adjoint of the RK4 path ---------------------------------------------
namespace {

// One field evaluation of every instance at the states in Bq.m[0] (Ms in w),
// with cavity amplitudes from Bq.st[b].a_re, written to Bq.fout [B][N].
int adj_field(mmcq_t* h, const Buffers& Bq, int terms) {
    StageArgs A = step_args(h);
    A.kind = KIND_RK4; A.mode = CAV_E; A.stage = 0; A.field_only = 1; A.terms = terms; A.inst0 = 0;
    A.record = 0; A.nmodes = 1;
    const int B = h->P.B;
    CK(h, launch_xfwd(h->P, Bq, A, B, h->stream));
    CK(h, launch_convolution(h->P, Bq, A, B, h->stream, &h->tune));
    CK(h, launch_xinv(h->P, h->mat, Bq, A, B, h->stream, &h->spec_map, &h->tune));
    return MMCQ_OK;
}

// A reversed adjoint step captured once and replayed (falls back to direct
// launches when the stream cannot be captured).
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;
    int capture(mmcq_t* h, const std::function<int()>& enqueue) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return MMCQ_OK;
        }
        const int r = enqueue();
        const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (r != MMCQ_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            failed = true;
            return r;
        }
        if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
            exec = nullptr;
            cudaGetLastError();
            failed = true;
        }
        cudaGraphDestroy(g);
        return MMCQ_OK;
    }
    ~StepGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

struct AdjScratch {
    std::vector<void*> bufs;
    mmcq_t* h;
    explicit AdjScratch(mmcq_t* h_) : h(h_) {}
    void* get(size_t bytes) {
        void* p = dev_alloc(h, bytes);
        if (p) bufs.push_back(p);
        return p;
    }
    ~AdjScratch() {
        for (void* p : bufs) dev_free_now(h, p);
    }
};

}  // namespace

int mmcq_adjoint_rk4(mmcq_t* h, int64_t nsteps, double dt, const mmcq_objective* obj, int64_t ckpt_every,
                     double* J, double* grad, float* grad_ms) {
    if (!h || nsteps < 1 || !(dt > 0) || !std::isfinite(dt) || !obj || !grad || ckpt_every < 0) return MMCQ_ERR_ARG;
    const double* w = obj->w;
    const double wn = obj->wn, wavg = obj->wavg;
    if (!std::isfinite(w[0]) || !std::isfinite(w[1]) || !std::isfinite(w[2]) || !std::isfinite(wn) ||
        !std::isfinite(wavg))
        return MMCQ_ERR_ARG;
    int64_t window = obj->window < 1 ? 1 : (obj->window > nsteps ? nsteps : obj->window);
    const int64_t K = ckpt_every < 1 ? 1 : (ckpt_every > nsteps ? nsteps : ckpt_every);
    if (h->mode != CAV_E || h->nmodes != 1) return fail(h, MMCQ_ERR_UNSUPPORTED, "adjoint: E-mode, one cavity mode");
    for (const InstParams& q : h->ip)
        if (q.drv_on) return fail(h, MMCQ_ERR_UNSUPPORTED, "adjoint: drive on");
    const int B = h->P.B;
    const long long N = h->P.N, BN = (long long)B * N;
    const size_t sv = sizeof(float4) * BN;
    const int kind0 = h->kind;
    const double tol0 = h->tol;
    int r = mmcq_set_integrator(h, MMCQ_RK4, tol0, MMCQ_CAVITY_E);
    if (r) return r;
    const int64_t nck = (nsteps + K - 1) / K;          // checkpoints at q = 0, K, 2K, ...
    AdjScratch sc(h);
    float4* ck = (float4*)sc.get(sv * nck);
    InstState* ckst = (InstState*)sc.get(sizeof(InstState) * B * nck);
    float4* seg = (float4*)sc.get(sv * K);              // states q of the current segment
    InstState* segst = (InstState*)sc.get(sizeof(InstState) * B * (K + 1));
    float4* mfin = (float4*)sc.get(sv);                  // the state at step nsteps
    InstState* stfin = (InstState*)sc.get(sizeof(InstState) * B);
    float4 *Y[4], *Bs[4], *Kb[4];
    for (int q = 0; q < 4; q++) {
        Y[q] = (float4*)sc.get(sv);
        Bs[q] = (float4*)sc.get(sv);
        Kb[q] = (float4*)sc.get(sv);
    }
    float4* lam = (float4*)sc.get(sv);
    float4* lp = (float4*)sc.get(sv);
    float4* nl = (float4*)sc.get(sv);
    float4* lk = (float4*)sc.get(sv);
    float4* lB = (float4*)sc.get(sv);
    float4* gd = (float4*)sc.get(sv);
    float4* Dl = (float4*)sc.get(sv);
    float* gms = (float*)sc.get(sizeof(float) * BN);
    InstState* adst = (InstState*)sc.get(sizeof(InstState) * B);
    double* dX = (double*)sc.get(sizeof(double) * B);
    double* dlX = (double*)sc.get(sizeof(double) * B);
    const int nblk = adj_local_blocks(N);
    double* part = (double*)sc.get(sizeof(double) * 4 * B * nblk);
    AdjScalars* S = (AdjScalars*)sc.get(sizeof(AdjScalars) * B);
    float4* Ybase = (float4*)sc.get(sv);                // m_q of the reversed step
    InstState* stq = (InstState*)sc.get(sizeof(InstState) * B);
    InstState* stq1 = (InstState*)sc.get(sizeof(InstState) * B);
    long long* cur = (long long*)sc.get(sizeof(long long) * 2);
    if (sc.bufs.size() != (size_t)(6 + 12 + 8 + 5 + 4)) return fail(h, MMCQ_ERR_CUDA, "adjoint: device allocation failed");
    CK(h, cudaMemsetAsync(gms, 0, sizeof(float) * BN, h->stream));

    // forward: checkpoint every K steps (m and the instance states)
    CK(h, launch_set_dt(h->Bf.st, B, dt, h->stream));
    for (int64_t q = 0; q < nsteps; q++) {
        if (q % K == 0) {
            CK(h, cudaMemcpyAsync(ck + (q / K) * BN, h->Bf.m[0], sv, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, cudaMemcpyAsync(ckst + (q / K) * B, h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToDevice,
                                  h->stream));
        }
        r = enqueue_steps(h, 1);
        if (r) return r;
    }
    CK(h, cudaMemcpyAsync(mfin, h->Bf.m[0], sv, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(stfin, h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToDevice, h->stream));
    // objective at the final state
    std::vector<float4> mf(BN);
    std::vector<InstState> st(B);
    CK(h, cudaMemcpyAsync(mf.data(), mfin, sv, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(st.data(), stfin, sizeof(InstState) * B, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    r = check_flags(h);
    if (r) return r;
    long long nmag = 0;
    for (float v : h->ms_host) nmag += v > 0;
    const double wv[3] = {nmag ? w[0] / nmag : 0.0, nmag ? w[1] / nmag : 0.0, nmag ? w[2] / nmag : 0.0};
    const double cav = wavg / (double)window;          // weight of each |alpha_n|^2 in the average
    std::vector<double> la_re(B), la_im(B), Jv(B);
    for (int b = 0; b < B; b++) {
        double a[3] = {0, 0, 0};
        for (long long i = 0; i < N; i++) {
            const float4 v = mf[b * N + i];
            if (v.w > 0.f) { a[0] += v.x; a[1] += v.y; a[2] += v.z; }
        }
        const double ar = st[b].a_re[0], ai = st[b].a_im[0];
        Jv[b] = wv[0] * a[0] + wv[1] * a[1] + wv[2] * a[2] + wn * (ar * ar + ai * ai);
        la_re[b] = 2.0 * wn * ar;
        la_im[b] = 2.0 * wn * ai;
        for (int c = 0; c < 6; c++) grad[6 * b + c] = 0.0;
    }
    CK(h, launch_adj_terminal(mfin, lam, wv, BN, h->stream));
    {
        std::vector<AdjScalars> Sh(B);
        for (int b = 0; b < B; b++) {
            std::memset(&Sh[b], 0, sizeof(AdjScalars));
            Sh[b].la_re = la_re[b];
            Sh[b].la_im = la_im[b];
        }
        CK(h, cudaMemcpyAsync(S, Sh.data(), sizeof(AdjScalars) * B, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }

    const double cc[4] = {0.0, 0.5, 0.5, 1.0}, bb[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    const double vc = h->mat.vc, hbar = h->hbar;
    // One reversed step q (q and the segment from the device cursor), enqueued
    // with fixed pointers only, so that it is captured once as a CUDA graph and
    // replayed for every step.
    auto back_step = [&]() -> int {
        int rr;
        CK(h, launch_adj_step_inputs(seg, segst, Ybase, Y[0], stq, stq1, cur, BN, B, h->stream));
        // the averaged photon number sees alpha at step q + 1
        CK(h, launch_adj_window(S, stq1, cav, B, cur, nsteps - window + 1, h->stream));
        CK(h, launch_adj_begin_step(S, adst, stq, B, h->stream));
        for (int s = 0; s < 4; s++) {
            Buffers Bq = h->Bf;
            Bq.m[0] = Bq.m[1] = Y[s];
            Bq.st = adst;
            Bq.fout = Bs[s];
            if ((rr = adj_field(h, Bq, MMCQ_TERM_ALL))) return rr;
            CK(h, launch_coupling_sum(Bq, N, vc, 0, B, 0, dX, h->stream));
            CK(h, launch_adj_alpha_stage(S, adst, h->Bf.ip, dX, s, dt, hbar, B, h->stream));
            CK(h, launch_adj_torque(Y[s], Bs[s], Ybase, Kb[s], s < 3 ? Y[s + 1] : nullptr,
                                    (float)(cc[s < 3 ? s + 1 : 0] * dt), h->mat.pre, h->mat.alpha, BN, h->stream));
        }
        // renormalisation and the stage cotangents
        CK(h, launch_adj_norm(Ybase, Kb, lam, lp, nl, lk, (float)dt, BN, h->stream));
        CK(h, launch_adj_begin_vjp(S, h->Bf.ip, dlX, dt, hbar, B, h->stream));
        for (int s = 3; s >= 0; s--) {
            CK(h, launch_adj_local(Y[s], Bs[s], lk, dlX, h->Bf.ip, h->Bf.prof[0], lB, gd, part, h->mat.pre,
                                   h->mat.alpha, vc, N, B, h->stream));
            Buffers Bq = h->Bf;
            Bq.m[0] = Bq.m[1] = lB;
            Bq.st = adst;
            Bq.fout = Dl;
            if ((rr = adj_field(h, Bq, MMCQ_TERM_DEMAG))) return rr;
            const float dtb = s > 0 ? (float)(dt * bb[s - 1]) : 0.f;
            const float cdt = s > 0 ? (float)(cc[s] * dt) : 0.f;
            CK(h, launch_adj_combine(Y[s], lB, Dl, gd, lp, nl, lk, h->mat, dtb, cdt, h->P.nx, h->P.ny, h->P.nz, B,
                                     grad_ms ? gms : nullptr, dlX, h->Bf.ip, h->Bf.prof[0], h->stream));
            CK(h, launch_adj_scalar_vjp(S, part, nblk, h->Bf.ip, dlX, s, dt, hbar, B, h->stream));
        }
        CK(h, launch_adj_end_step(S, B, h->stream));
        // lambda of step q is what the stages accumulated
        CK(h, cudaMemcpyAsync(lam, nl, sv, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, launch_adj_next(cur, h->stream));
        return MMCQ_OK;
    };
    StepGraph step_graph;
    for (int64_t c0 = (nck - 1) * K; c0 >= 0; c0 -= K) {
        const int64_t c1 = std::min(c0 + K, nsteps);
        // recompute the states of steps c0 .. c1 - 1 from checkpoint c0 (the state
        // of step c1 is the next checkpoint or the final state)
        CK(h, cudaMemcpyAsync(h->Bf.m[0], ck + (c0 / K) * BN, sv, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, cudaMemcpyAsync(h->Bf.st, ckst + (c0 / K) * B, sizeof(InstState) * B, cudaMemcpyDeviceToDevice,
                              h->stream));
        for (int64_t q = c0; q < c1; q++) {
            CK(h, cudaMemcpyAsync(seg + (q - c0) * BN, h->Bf.m[0], sv, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, cudaMemcpyAsync(segst + (q - c0) * B, h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToDevice,
                                  h->stream));
            if (q + 1 < c1) {
                r = enqueue_steps(h, 1);
                if (r) return r;
            }
        }
        CK(h, cudaMemcpyAsync(segst + (c1 - c0) * B, c1 < nsteps ? ckst + (c1 / K) * B : stfin,
                              sizeof(InstState) * B, cudaMemcpyDeviceToDevice, h->stream));
        CK(h, launch_adj_set_cursor(cur, c1 - 1 - c0, c0, h->stream));
        for (int64_t q = c1 - 1; q >= c0; q--) {
            if (!step_graph.exec && !step_graph.failed) {
                r = step_graph.capture(h, back_step);
                if (r) return r;
            }
            if (step_graph.exec) CK(h, cudaGraphLaunch(step_graph.exec, h->stream));
            else if ((r = back_step())) return r;
        }
    }
    {
        std::vector<AdjScalars> Sh(B);
        CK(h, cudaMemcpyAsync(Sh.data(), S, sizeof(AdjScalars) * B, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (int b = 0; b < B; b++) {
            Jv[b] += Sh[b].J;
            for (int c = 0; c < 6; c++) grad[6 * b + c] = Sh[b].grad[c];
        }
    }
    if (J) for (int b = 0; b < B; b++) J[b] = Jv[b];
    // the handle back at step nsteps
    CK(h, cudaMemcpyAsync(h->Bf.m[0], mfin, sv, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->Bf.m[1], mfin, sv, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->Bf.st, stfin, sizeof(InstState) * B, cudaMemcpyDeviceToDevice, h->stream));
    if (grad_ms) CK(h, cudaMemcpyAsync(grad_ms, gms, sizeof(float) * BN, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    r = check_flags(h);
    if (r) return r;
    // back to the integrator the caller had
    if (kind0 != KIND_RK4) return mmcq_set_integrator(h, kind0, tol0, MMCQ_CAVITY_E);
    return MMCQ_OK;
}

// ---- checkpoint / resume ---------------------------------------------------
// Snapshot: SnapHeader, then B InstState, B InstParams, B x MAX_MODES g
// (double), B x MAX_MODES g_mode (int32), then m of every instance (B x N
// float4) and the kept first DP45 stage (B x N float4).
namespace {
struct SnapHeader {
    char magic[8];
    int32_t version, nx, ny, nz, B, kind, mode, pad;
    double tol;
    int64_t N, st_bytes, ip_bytes;
};
const char SNAP_MAGIC[8] = {'M', 'M', 'C', 'Q', 'S', 'N', 'A', 'P'};

int64_t snap_size(const mmcq_t* h) {
    const int64_t B = h->P.B;
    return (int64_t)sizeof(SnapHeader) + B * (int64_t)(sizeof(InstState) + sizeof(InstParams) + 12 * MAX_MODES) +
           2 * B * h->P.N * (int64_t)sizeof(float4);
}
}  // namespace

int mmcq_get_state(mmcq_t* h, void* buf, int64_t cap, int64_t* size) {
    if (!h || cap < 0) return MMCQ_ERR_ARG;
    const int64_t need = snap_size(h);
    if (size) *size = need;
    if (!buf) return MMCQ_OK;
    if (cap < need) return fail(h, MMCQ_ERR_ARG, "snapshot buffer too small");
    const int B = h->P.B;
    const long long N = h->P.N;
    std::vector<InstState> st(B);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(st.data(), h->Bf.st, sizeof(InstState) * B, cudaMemcpyDeviceToHost));
    char* p = static_cast<char*>(buf);
    SnapHeader hd{};
    std::memcpy(hd.magic, SNAP_MAGIC, 8);
    hd.version = 2;
    hd.nx = h->P.nx; hd.ny = h->P.ny; hd.nz = h->P.nz; hd.B = B;
    hd.kind = h->kind; hd.mode = h->mode; hd.tol = h->tol;
    hd.N = N; hd.st_bytes = sizeof(InstState); hd.ip_bytes = sizeof(InstParams);
    std::memcpy(p, &hd, sizeof(hd)); p += sizeof(hd);
    std::memcpy(p, st.data(), sizeof(InstState) * B); p += sizeof(InstState) * B;
    std::memcpy(p, h->ip.data(), sizeof(InstParams) * B); p += sizeof(InstParams) * B;
    std::memcpy(p, h->g.data(), sizeof(double) * B * MAX_MODES); p += sizeof(double) * B * MAX_MODES;
    for (int q = 0; q < B * MAX_MODES; q++) { int32_t v = h->g_mode[q]; std::memcpy(p, &v, 4); p += 4; }
    const size_t row = sizeof(float4) * N;
    for (int b = 0; b < B; b++, p += row)
        CK(h, cudaMemcpy(p, h->Bf.m[st[b].mcur] + (long long)b * N, row, cudaMemcpyDeviceToHost));
    for (int b = 0; b < B; b++, p += row)
        CK(h, cudaMemcpy(p, h->Bf.k[st[b].k1slot] + (long long)b * N, row, cudaMemcpyDeviceToHost));
    return MMCQ_OK;
}

int mmcq_set_state(mmcq_t* h, const void* buf, int64_t size) {
    if (!h || !buf || size < (int64_t)sizeof(SnapHeader)) return MMCQ_ERR_ARG;
    const char* p = static_cast<const char*>(buf);
    SnapHeader hd;
    std::memcpy(&hd, p, sizeof(hd)); p += sizeof(hd);
    const int B = h->P.B;
    const long long N = h->P.N;
    if (std::memcmp(hd.magic, SNAP_MAGIC, 8) != 0 || hd.version != 2)
        return fail(h, MMCQ_ERR_ARG, "not an mmcq snapshot");
    if (hd.nx != h->P.nx || hd.ny != h->P.ny || hd.nz != h->P.nz || hd.B != B || hd.N != N ||
        hd.st_bytes != (int64_t)sizeof(InstState) || hd.ip_bytes != (int64_t)sizeof(InstParams))
        return fail(h, MMCQ_ERR_ARG, "snapshot of another grid, batch or build");
    if (size != snap_size(h)) return fail(h, MMCQ_ERR_ARG, "snapshot size mismatch");
    if ((hd.kind != KIND_RK4 && hd.kind != KIND_DP45) || (hd.mode != CAV_E && hd.mode != CAV_P))
        return fail(h, MMCQ_ERR_ARG, "snapshot integrator fields invalid");
    std::vector<InstState> st(B);
    std::memcpy(st.data(), p, sizeof(InstState) * B); p += sizeof(InstState) * B;
    for (const InstState& s : st)
        if ((s.k1slot != 0 && s.k1slot != MAX_STAGES - 1) || (s.mcur != 0 && s.mcur != 1))
            return fail(h, MMCQ_ERR_ARG, "snapshot state fields invalid");
    std::vector<InstParams> ip(B);
    std::memcpy(ip.data(), p, sizeof(InstParams) * B); p += sizeof(InstParams) * B;
    std::vector<double> g((size_t)B * MAX_MODES);
    std::memcpy(g.data(), p, sizeof(double) * B * MAX_MODES); p += sizeof(double) * B * MAX_MODES;
    std::vector<int> gm((size_t)B * MAX_MODES);
    for (int q = 0; q < B * MAX_MODES; q++) { int32_t v; std::memcpy(&v, p, 4); p += 4; gm[q] = v; }
    CK(h, cudaStreamSynchronize(h->stream));
    const size_t row = sizeof(float4) * N;
    for (int b = 0; b < B; b++, p += row)
        for (int k = 0; k < 2; k++) CK(h, cudaMemcpy(h->Bf.m[k] + (long long)b * N, p, row, cudaMemcpyHostToDevice));
    for (int b = 0; b < B; b++, p += row)
        CK(h, cudaMemcpy(h->Bf.k[st[b].k1slot] + (long long)b * N, p, row, cudaMemcpyHostToDevice));
    for (InstState& s : st) { s.mcur = 0; s.nhist = 0; }
    CK(h, cudaMemcpy(h->Bf.st, st.data(), sizeof(InstState) * B, cudaMemcpyHostToDevice));
    h->ip = ip;
    h->g = g;
    h->g_mode = gm;
    for (const InstParams& q : ip)
        for (int k = 0; k < MAX_MODES; k++)
            if (q.cav_on[k] && k + 1 > h->nmodes) h->nmodes = k + 1;
    h->kind = hd.kind;
    h->mode = hd.mode;
    h->tol = hd.tol;
    h->k1_dirty = true;
    return upload_params(h);
}


// ---- groups ------------------------------------------------------------------
struct mmcq_group {
    std::vector<mmcq_t*> hs;
    int chunk = 1;
    int device = 0;
    cudaStream_t origin = nullptr;          // graph launch stream
    std::vector<cudaStream_t> side;         // capture branch of each handle
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join, in;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> cap_kind, cap_mode, cap_record, cap_nmodes;
    std::vector<int64_t> cap_epoch;         // tuning epoch of each handle at the capture
    std::vector<double> cap_tol;
    std::vector<int64_t> cap_launches;      // kernel launches per replay, per handle
    int64_t replays = 0;
    std::string err;
};

namespace {

int gfail(mmcq_group_t* g, int code, const std::string& msg) {
    g->err = msg;
    return code;
}

#define GCK(g, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return gfail((g), MMCQ_ERR_CUDA, std::string(#call) + ": " +   \
                                                                     cudaGetErrorString(e_)); \
    } while (0)

bool group_stale(const mmcq_group_t* g) {
    if (!g->exec) return true;
    for (size_t i = 0; i < g->hs.size(); i++) {
        const mmcq_t* h = g->hs[i];
        if (h->kind != g->cap_kind[i] || h->mode != g->cap_mode[i] || h->tol != g->cap_tol[i] ||
            h->record != g->cap_record[i] || h->nmodes != g->cap_nmodes[i] || h->tune_epoch != g->cap_epoch[i])
            return true;
    }
    return false;
}

// Capture `chunk` steps of every handle, each on its own branch, into g->exec.
// The handles' streams are swapped for the branch streams while capturing.
int group_capture(mmcq_group_t* g) {
    if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
    const size_t nh = g->hs.size();
    std::vector<cudaStream_t> saved(nh);
    std::vector<int64_t> before(nh);
    for (size_t i = 0; i < nh; i++) {
        saved[i] = g->hs[i]->stream;
        before[i] = g->hs[i]->launches;
    }
    GCK(g, cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeThreadLocal));
    int r = MMCQ_OK;
    cudaError_t e = cudaEventRecord(g->fork, g->origin);
    for (size_t i = 0; i < nh && e == cudaSuccess && r == MMCQ_OK; i++) {
        e = cudaStreamWaitEvent(g->side[i], g->fork, 0);
        if (e != cudaSuccess) break;
        g->hs[i]->stream = g->side[i];
        r = enqueue_steps(g->hs[i], g->chunk);
        g->hs[i]->stream = saved[i];
        if (r == MMCQ_OK) e = cudaEventRecord(g->join[i], g->side[i]);
        if (r == MMCQ_OK && e == cudaSuccess) e = cudaStreamWaitEvent(g->origin, g->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(g->origin, &graph);
    for (size_t i = 0; i < nh; i++) {
        g->hs[i]->stream = saved[i];
        g->cap_launches[i] = g->hs[i]->launches - before[i];
        g->hs[i]->launches = before[i];
        g->cap_kind[i] = g->hs[i]->kind;
        g->cap_mode[i] = g->hs[i]->mode;
        g->cap_tol[i] = g->hs[i]->tol;
        g->cap_record[i] = g->hs[i]->record;
        g->cap_nmodes[i] = g->hs[i]->nmodes;
        g->cap_epoch[i] = g->hs[i]->tune_epoch;
    }
    if (r != MMCQ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return gfail(g, r, "capture: a handle failed to enqueue its steps");
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return gfail(g, MMCQ_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->exec = nullptr;
        return gfail(g, MMCQ_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    return MMCQ_OK;
}

}  // namespace

int mmcq_group_create(mmcq_group_t** out, mmcq_t* const* handles, int n, int chunk) {
    if (!out) return MMCQ_ERR_ARG;
    *out = nullptr;
    if (!handles || n < 1 || chunk < 1) return MMCQ_ERR_ARG;
    for (int i = 0; i < n; i++) {
        if (!handles[i] || handles[i]->device != handles[0]->device) return MMCQ_ERR_ARG;
        for (int j = 0; j < i; j++)
            if (handles[j] == handles[i]) return MMCQ_ERR_ARG;
    }
    mmcq_group_t* g = new mmcq_group();
    g->hs.assign(handles, handles + n);
    g->chunk = chunk;
    g->device = handles[0]->device;
    g->side.assign(n, nullptr);
    g->join.assign(n, nullptr);
    g->in.assign(n, nullptr);
    g->cap_kind.assign(n, -1);
    g->cap_mode.assign(n, -1);
    g->cap_tol.assign(n, -1.0);
    g->cap_epoch.assign(n, -1);
    g->cap_record.assign(n, -1);
    g->cap_nmodes.assign(n, -1);
    g->cap_launches.assign(n, 0);
    bool ok = cudaSetDevice(g->device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < n && ok; i++)
        ok = cudaStreamCreateWithFlags(&g->side[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->in[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        mmcq_group_destroy(g);
        return MMCQ_ERR_CUDA;
    }
    *out = g;
    return MMCQ_OK;
}

int mmcq_group_step(mmcq_group_t* g, int64_t n, double dt) {
    if (!g || n < 0 || !std::isfinite(dt)) return MMCQ_ERR_ARG;
    for (mmcq_t* h : g->hs)
        if (h->kind == KIND_RK4 && !(dt > 0)) return gfail(g, MMCQ_ERR_ARG, "RK4 needs dt > 0");
    if (n == 0) return MMCQ_OK;
    GCK(g, cudaSetDevice(g->device));
    bool eager = n < g->chunk;
    for (mmcq_t* h : g->hs) {
        if (dt > 0 && launch_set_dt(h->Bf.st, h->P.B, dt, h->stream) != cudaSuccess)
            return gfail(g, MMCQ_ERR_CUDA, "set_dt launch failed");
        // the first DP45 stage after a host-side change runs before the graph
        // (the captured attempts reuse it, first-same-as-last)
        if (h->kind == KIND_DP45 && h->mode == CAV_E && h->k1_dirty) {
            StageArgs A = step_args(h);
            A.stage = 0;
            int r = run_stage(h, A, h->P.B);
            if (r) return gfail(g, r, "first stage launch failed");
            h->k1_dirty = false;
        }
        if (h->profiling) eager = true;
    }
    if (eager) {
        for (mmcq_t* h : g->hs) {
            int r = enqueue_steps(h, n);
            if (r) return gfail(g, r, "step launch failed");
        }
        return MMCQ_OK;
    }
    if (group_stale(g)) {
        int r = group_capture(g);
        if (r) return r;
    }
    const size_t nh = g->hs.size();
    for (size_t i = 0; i < nh; i++) {
        GCK(g, cudaEventRecord(g->in[i], g->hs[i]->stream));
        GCK(g, cudaStreamWaitEvent(g->origin, g->in[i], 0));
    }
    const int64_t reps = n / g->chunk;
    for (int64_t q = 0; q < reps; q++) GCK(g, cudaGraphLaunch(g->exec, g->origin));
    g->replays += reps;
    GCK(g, cudaEventRecord(g->done, g->origin));
    for (size_t i = 0; i < nh; i++) {
        mmcq_t* h = g->hs[i];
        h->launches += reps * g->cap_launches[i];
        GCK(g, cudaStreamWaitEvent(h->stream, g->done, 0));
        const int64_t rem = n - reps * g->chunk;
        if (rem > 0) {
            int r = enqueue_steps(h, rem);
            if (r) return gfail(g, r, "step launch failed");
        }
    }
    return MMCQ_OK;
}

int64_t mmcq_group_replays(const mmcq_group_t* g) { return g ? g->replays : -1; }

void mmcq_group_destroy(mmcq_group_t* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->origin) cudaStreamSynchronize(g->origin);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (cudaStream_t s : g->side) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->join) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : g->in) if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->done) cudaEventDestroy(g->done);
    if (g->origin) cudaStreamDestroy(g->origin);
    delete g;
}

const char* mmcq_group_last_error(const mmcq_group_t* g) { return g ? g->err.c_str() : "null group"; }

}  // extern "C"
