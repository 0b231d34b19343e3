// x inverse of the demag convolution fused with everything a stage does per
// cell (Mumax3-cQED, arXiv 2410.00966): complex-to-real inverse FFT along x
// giving B_demag, then exchange + anisotropy + Zeeman (with the Appendix C
// excitation) + cavity sum_k B_rms,k Gamma_k (Sec. 2.1 field terms, Eq. bcav),
// the LLG torque (Eq. llg), the RK bookkeeping, and block partials of the
// coupling sums X_k = V_c sum_i Ms_i m_i . B_rms,k,i (Eq. gammafinal): each
// cell's FP32 product promoted and added in FP64.  The last block of each
// instance to finish reduces the partials in a fixed order and advances the
// cavity amplitudes and the step-size controller in FP64.
#include <math.h>

#include "common.cuh"
#include "fftreg.cuh"
#include "kern_common.cuh"
#include "stagecore.cuh"
#include "xpass.cuh"

namespace mq {

// e^{+2 pi i k / px} for the point k = j + N1 n2 of a line of L = px / 2
// complex points: with 16 points per thread (px = 32 N1) it is
// e^{+2 pi i j / px} conj(W_32^{n2}), one table value per thread times a
// constant-bank factor; otherwise one table value per point.
template <int L, int N1>
__device__ __forceinline__ float2 unpack_twiddle(const float2* __restrict__ tw, int twstep, int j, int n2) {
    if constexpr (32 * N1 == 2 * L) {
        const float2 wj = twiddle(tw, j * twstep, true);
        return n2 == 0 ? wj : cmul(wj, conjf2(c_tw32[n2]));
    } else {
        return twiddle(tw, (j + N1 * n2) * twstep, true);
    }
}

// The cells of nr rows (row r of the block at (y, z) = s_yz[r]) once the
// demag field of those rows is in xs (x_2n = Re, x_2n+1 = Im of row x / 2,
// pitch ld, line 3 r + comp): exchange, then CellUpdate (local fields,
// torque, RK bookkeeping, the cell's share of the coupling sums and error).
// Row of flat index i when blocks of one row are ordered z fastest: the rows
// that run at the same time are whole runs of z for consecutive y, so each
// row's six neighbour rows (y +- 1, z +- 1) are being read by blocks running
// alongside it and are found in L2 (in y-major order a z neighbour is a whole
// plane of the grid away and has left L2 by the time it is needed).
__device__ __forceinline__ int zfast_row(const Plan& P, int i) {
    const int y = (int)fdiv((unsigned)i, P.fd_nz);
    return (i - y * P.nz) * P.ny + y;
}

template <int NM, bool REC>
__device__ __forceinline__ void xinv_cells(const Plan& P, const Material& mat, const Buffers& Bf,
                                           const CellUpdate<NM>& cu, const float2* xs, int ld, const float4* msrc,
                                           long long base, int nx, int nr, int nthr, const int2* s_yz,
                                           double (&xacc)[NM], double (&macc)[REC ? 3 : 1], float& emax, bool& bad) {
    const bool want_demag = cu.want_demag, want_exch = cu.want_exch;
    const int pl = nx * P.ny;
    // cell ii = r nx + x of the block; (x, r) advance by the block size
    const int stepr = nthr / nx, stepx = nthr - stepr * nx;
    int r = threadIdx.x / nx, x = threadIdx.x - r * nx;
    for (int ii = threadIdx.x; ii < nr * nx; ii += nthr) {
        const int2 yz = s_yz[r];
        const int y = yz.x, z = yz.y;
        const long long i = base + ii;
        const float4* mc = msrc + i;
        const float4 m = __ldg(mc);
        const float Ms = m.w;
        float Bx = 0.f, By = 0.f, Bz = 0.f;
        if (want_demag) {
            // x_2n = Re z_n, x_2n+1 = Im z_n
            const float* zr = reinterpret_cast<const float*>(xs + (x >> 1) * ld + 3 * r) + (x & 1);
            Bx = zr[0]; By = zr[2]; Bz = zr[4];
        }
        if (want_exch) {
            // sum over the six neighbours j of w_j (m_j - m_i), w_j = C_d for
            // a non-empty neighbour and 0 for an empty one; a neighbour outside
            // the grid is read as the cell itself (m_i - m_i = 0), so every
            // load is unconditional and all six are in flight together
            const float4 q0 = __ldg(mc + (x > 0 ? -1 : 0));
            const float4 q1 = __ldg(mc + (x + 1 < nx ? 1 : 0));
            const float4 q2 = __ldg(mc + (y > 0 ? -nx : 0));
            const float4 q3 = __ldg(mc + (y + 1 < P.ny ? nx : 0));
            const float4 q4 = __ldg(mc + (z > 0 ? -pl : 0));
            const float4 q5 = __ldg(mc + (z + 1 < P.nz ? pl : 0));
            const float2 nm = make_float2(-m.x, -m.y);
            float2 hxy = make_float2(0.f, 0.f);
            float hz = 0.f;
            auto nb = [&](const float4& q, float C) {
                const float w = q.w > 0.f ? C : 0.f;
                hxy = __ffma2_rn(make_float2(w, w), __fadd2_rn(make_float2(q.x, q.y), nm), hxy);
                hz = fmaf(w, q.z - m.z, hz);
            };
            nb(q0, mat.exch[0]); nb(q1, mat.exch[0]);
            nb(q2, mat.exch[1]); nb(q3, mat.exch[1]);
            nb(q4, mat.exch[2]); nb(q5, mat.exch[2]);
            const float inv = Ms > 0.f ? __fdividef(1.f, Ms) : 0.f;
            Bx += hxy.x * inv; By += hxy.y * inv; Bz += hz * inv;
        }
        cu.template run<REC>(mat, Bf, i, m, Bx, By, Bz, xacc, macc, emax, bad);
        x += stepx;
        r += stepr;
        if (x >= nx) { x -= nx; r++; }
    }
}

// ---------------------------------------------------------------------------
// x inverse + local fields + torque + RK bookkeeping + cavity reduction.
// Shared memory: xs[k][line] (k <= L, line = 3 r + comp).
// ---------------------------------------------------------------------------
// REC: this launch records the spatial average of the state being accepted
// (the last stage of a step with recording on); NM: cavity modes compiled in
// (1, or MAX_MODES when more than one mode is enabled).  Separate
// instantiations so that the common launches carry no extra accumulators.
// FX: the fixed shape of the large grids (rows of nx = L cells, XPASS_ROWS(L)
// rows per block with none left over, tiles of 8 kx columns) at compile time.
template <int L, bool REC, int NM, bool FX>
__global__ void __launch_bounds__(XPASS_THREADS, xpass_min_blocks(L)) k_xinv(Plan P, Material mat, Buffers Bf, StageArgs A) {
    constexpr bool F3 = xpass_f3(L);
    constexpr int NPT = F3 ? 16 : ColShape<L>::NPT, N1 = xpass_line_threads(L);
    constexpr int RF = xpass_rows(L);
    extern __shared__ float2 sm[];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma[NM];
    __shared__ float s_drive;
    __shared__ int s_last;
    __shared__ int2 s_yz[64];                          // rows per block <= 64
    const int b = A.inst0 + blockIdx.y;
    const InstState& st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const InstParams& ip = Bf.ip[b];
    const int Rb = FX ? RF : P.R;
    const int TX = FX ? 8 : P.TX, nx = FX ? L : P.nx, lt = FX ? 3 : P.lt;
    const int NT = FX ? L / 8 + 1 : P.NT;
    const int nthr = FX ? 3 * RF * N1 : (int)blockDim.x;
    const int row0 = F3 ? zfast_row(P, blockIdx.x) : blockIdx.x * Rb;   // F3: one row per block
    const int nr = FX ? RF : min(P.R, P.nrows - row0);
    const int ld = xpass_ld(Rb);
    const long long cb = (long long)b * P.N;
    const long long base = cb + (long long)row0 * nx;
    const int s = A.stage;
    const int K = A.kind;
    float2* xs = sm;                                   // [L + 1][ld]

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

    // (y, z) of the block's rows, for the cell loop
    if (threadIdx.x < nr) {
        const int row = row0 + threadIdx.x;
        const int z = (int)fdiv((unsigned)row, P.fd_ny);
        s_yz[threadIdx.x] = make_int2(row - z * P.ny, z);
    }

    // half-spectrum rows X[0..L] of the three components of every row.  In the
    // spectrum, tile t of a row holds the 3 TX values (c, tx) contiguously
    // (k = t TX + tx); when 3 TX divides the block, a thread keeps one (c, tx)
    // and steps over the tiles.
    const long long tstride = (long long)P.ny * 3 * TX;
    const int w3 = 3 * TX;
    if (nthr % w3 == 0) {
        const int e = threadIdx.x % w3, t0 = threadIdx.x / w3, dtt = nthr / w3;
        const int c = e >> lt, tx = e & (TX - 1);
        // 32-bit steps: the shared-window address and the offset in the spectrum
        const unsigned sx = (unsigned)__cvta_generic_to_shared(xs) + 8u * (unsigned)((t0 * TX + tx) * ld + c);
        const unsigned sstep = 8u * (unsigned)(dtt * TX * ld);
        const int gstep = dtt * (int)tstride;
        const int nt = t0 < NT ? (NT - 1 - t0) / dtt + 1 : 0;     // tiles of this thread
        for (int r = 0; r < nr; r++) {
            const int row = row0 + r;
            const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
            const float2* in = Bf.spec + (((long long)b * P.nz + z) * NT * P.ny + y) * 3 * TX + e +
                               (long long)t0 * tstride;
            unsigned sa = sx + 8u * (unsigned)(3 * r);
            int go = 0, k = t0 * TX + tx;
            for (int n = 0; n < nt; n++) {
                if (k <= L) cp_async8s(sa, in + go);
                sa += sstep;
                go += gstep;
                k += dtt * TX;
            }
        }
    } else {
        for (int r = 0; r < nr; r++) {
            const int row = row0 + r;
            const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
            const float2* in = Bf.spec + (((long long)b * P.nz + z) * NT * P.ny + y) * 3 * TX;
            for (int idx = threadIdx.x; idx < 3 * (L + 1); idx += nthr) {
                const int c = idx / (L + 1), k = idx - c * (L + 1);
                const int t = k >> lt, tx = k & (TX - 1);
                cp_async8(xs + k * ld + 3 * r + c, in + t * tstride + c * TX + tx);
            }
        }
    }
    // the block's own rows of m are read in the cell loop (through L1, which
    // then serves the x and y neighbours as well)
    if (threadIdx.x == 0) prefetch_l2(msrc + base, (unsigned)(nr * nx * sizeof(float4)));
    if (threadIdx.x == 0) {
        for (int q = 0; q < NM; q++) s_gamma[q] = stage_gamma(A, ip, st, mat, q);
        s_drive = (float)drive_factor(A, ip, st);
    }
    cp_async_wait_all();
    __syncthreads();
    const int twstep = P.twn / P.px;
    {
        // three-factor: a line's 64 threads are consecutive (lane groups of
        // the last factor inside one warp); otherwise lines are fastest
        const int nl = 3 * Rb;
        const int line = F3 ? threadIdx.x / N1 : threadIdx.x % nl;
        const int j = F3 ? threadIdx.x % N1 : threadIdx.x / nl;
        // the C2R unpack done as the transform loads its points (k = j + N1 n2):
        // Z[k] = (X[k] + conj X[L-k]) + i e^{+2 pi i k / px} (X[k] - conj X[L-k]).
        // Every thread reads before the transform's first barrier, and no
        // thread stores into xs before it (with N1 = 1 a thread owns its line).
        float2 v[NPT];
#pragma unroll
        for (int n2 = 0; n2 < NPT; n2++) {
            const int k = j + N1 * n2;
            const float2 a = xs[k * ld + line], bq = xs[(L - k) * ld + line];
            const float2 ca = conjf2(bq);
            const float2 sum = cadd(a, ca), dif = csub(a, ca);
            const float2 wd = cmul(unpack_twiddle<L, N1>(Bf.tw, twstep, j, n2), dif);
            v[n2] = make_float2(sum.x - wd.y, sum.y + wd.x);   // sum + i wd
        }
        if constexpr (F3) {
            col_fft3<L, true, false, XPASS_F3_PADS, 1>(v, xs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
            for (int i = 0; i < NPT; i++) xs[col3_out_row<L>(j, i) * ld + line] = v[i];
        } else {
            col_fft<L, true>(v, xs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
            for (int i = 0; i < NPT; i++) xs[col_out_row<L>(j, i) * ld + line] = v[i];
        }
    }
    __syncthreads();

    CellUpdate<NM> cu;
    cu.init(Bf, A, st, ip, s_gamma, s_drive, cb, (long long)A.inst0 * P.N);
    double xacc[NM];
#pragma unroll
    for (int q = 0; q < NM; q++) xacc[q] = 0.0;
    double macc[REC ? 3 : 1] = {};
    float emax = 0.f;
    bool bad = false;
    xinv_cells<NM, REC>(P, mat, Bf, cu, xs, ld, msrc, base, nx, nr, nthr, s_yz, xacc, macc, emax, bad);
    if (A.field_only) return;
    stage_epilogue<REC, NM>(P, mat, Bf, A, b, blockIdx.x, P.nblk, xacc, emax, bad, s_red, s_redf, &s_last, macc);
}

// ---------------------------------------------------------------------------
// The same stage for rows of L = 1024 (8-column tiles, one row per pass),
// persistent and pipelined: each block takes rows blockIdx.x, + gridDim.x, ...
// of its instance in z-fastest order (zfast_row), and while it transforms and
// updates one row, the
// half-spectrum row after it is already on its way into the other of two
// shared-memory buffers by one bulk tensor copy (TMA: the 129 tiles x 24
// values of the row as one box of the 4-D map [plane][tile][y][24]),
// completing on that buffer's mbarrier.  The copy lands tile-major
// (value (c, k) at 24 (k / 8) + 8 c + k % 8); the C2R unpack runs in place
// there, the transform reads it and leaves the field in the [k][3] layout of
// the row kernel.  A wait that has not completed after XPIPE_WAIT_NS raises
// FLAG_TIMEOUT and the block returns (the handle is then unusable).
constexpr int XPIPE_BUF = (1024 + 16 * XPASS_F3_PADS) * 3;   // float2 per buffer (>= 129 * 24)
constexpr int XPIPE_BLOCKS = 4;                              // resident blocks per SM
constexpr unsigned long long XPIPE_WAIT_NS = 1000000000ull;
static int g_sms = 0;                                        // SMs of the device (set by xinv_init)

__device__ __forceinline__ int xpipe_land(int k, int c) { return 24 * (k >> 3) + 8 * c + (k & 7); }

template <bool REC, int NM, bool FX>
__global__ void __launch_bounds__(XPASS_THREADS, XPIPE_BLOCKS) k_xinv_pipe(Plan P, Material mat, Buffers Bf,
                                                                           StageArgs A,
                                                                           const __grid_constant__ TensorMap tm) {
    constexpr int L = 1024, N1 = 64, NPT = 16, ld = 3;
    extern __shared__ __align__(128) float2 sm_raw[];  // [2][XPIPE_BUF] from the first 128-byte boundary
    float2* sm = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sm_raw) + 127) & ~(uintptr_t)127);
    __shared__ __align__(8) unsigned long long s_bar[2];
    __shared__ double s_red[32];
    __shared__ float s_redf[32];
    __shared__ double s_gamma[NM];
    __shared__ float s_drive;
    __shared__ int s_last;
    __shared__ int2 s_yz[1];
    const int b = A.inst0 + blockIdx.y;
    const InstState& st = Bf.st[b];
    if (stage_skips(st, A)) return;
    const InstParams& ip = Bf.ip[b];
    const int nx = FX ? L : P.nx;
    const int nthr = XPASS_THREADS;
    const long long cb = (long long)b * P.N;
    const int s = A.stage;
    const float4* msrc;
    if (A.field_only || s == 0) msrc = Bf.m[st.mcur];
    else if (A.kind == KIND_DP45 && s == 6) msrc = Bf.m[st.mcur ^ 1];
    else msrc = Bf.ms;
    const unsigned tbytes = (unsigned)P.NT * 24u * 8u;
    const unsigned rbytes = (unsigned)(nx * sizeof(float4));
    const long long pl = (long long)nx * P.ny;

    // thread 0: the bulk copy of `row` into buffer q, and the L2 prefetch of
    // the cell rows its update will read (m, its z neighbours, the profiles)
    auto issue = [&](int row, int q) {
        const int z = (int)fdiv((unsigned)row, P.fd_ny), y = row - z * P.ny;
        fence_proxy_async();
        tma_load_4d(sm + q * XPIPE_BUF, &tm, 0, y, 0, b * P.nz + z, &s_bar[q], tbytes);
        const long long base = cb + (long long)row * nx;
        prefetch_l2(msrc + base, rbytes);
        if (z > 0) prefetch_l2(msrc + base - pl, rbytes);
        if (z + 1 < P.nz) prefetch_l2(msrc + base + pl, rbytes);
        for (int k = 0; k < NM; k++)
            if (Bf.prof[k]) prefetch_l2(Bf.prof[k] + (base - cb), rbytes);
    };
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_proxy_async();
        for (int q = 0; q < NM; q++) s_gamma[q] = stage_gamma(A, ip, st, mat, q);
        s_drive = (float)drive_factor(A, ip, st);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x < P.nrows) issue(zfast_row(P, blockIdx.x), 0);

    CellUpdate<NM> cu;
    cu.init(Bf, A, st, ip, s_gamma, s_drive, cb, (long long)A.inst0 * P.N);
    double xacc[NM];
#pragma unroll
    for (int q = 0; q < NM; q++) xacc[q] = 0.0;
    double macc[REC ? 3 : 1] = {};
    float emax = 0.f;
    bool bad = false;
    const int line = threadIdx.x / N1, j = threadIdx.x % N1;
    const int twstep = P.twn / P.px;
    int it = 0;
    for (int flat = blockIdx.x; flat < P.nrows; flat += gridDim.x, it++) {
        const int q = it & 1;
        const int row = zfast_row(P, flat);
        const int nxt = flat + gridDim.x;
        if (threadIdx.x == 0) {
            if (nxt < P.nrows) issue(zfast_row(P, nxt), q ^ 1);
            const int z = (int)fdiv((unsigned)row, P.fd_ny);
            s_yz[0] = make_int2(row - z * P.ny, z);
        }
        // the current row: buffer q, its (it / 2)-th use
        const bool late = !mbar_wait(&s_bar[q], (unsigned)((it >> 1) & 1), XPIPE_WAIT_NS);
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) {
                atomicOr(Bf.flags, FLAG_TIMEOUT);
                // the copies this block issued may still be in flight: wait
                // for them (bounded) before the block's shared memory is freed
                mbar_wait(&s_bar[q], (unsigned)((it >> 1) & 1), XPIPE_WAIT_NS);
                if (nxt < P.nrows) mbar_wait(&s_bar[q ^ 1], (unsigned)(((it + 1) >> 1) & 1), XPIPE_WAIT_NS);
            }
            return;
        }
        float2* xs = sm + q * XPIPE_BUF;
        {
            // the C2R unpack done as the transform loads its points (see
            // k_xinv), X[k] at xpipe_land(k, line)
            float2 v[NPT];
#pragma unroll
            for (int n2 = 0; n2 < NPT; n2++) {
                const int k = j + N1 * n2;
                const float2 a = xs[xpipe_land(k, line)], bq = xs[xpipe_land(L - k, line)];
                const float2 ca = conjf2(bq);
                const float2 sum = cadd(a, ca), dif = csub(a, ca);
                const float2 wd = cmul(unpack_twiddle<L, N1>(Bf.tw, twstep, j, n2), dif);
                v[n2] = make_float2(sum.x - wd.y, sum.y + wd.x);
            }
            // (the transform's first barrier comes before its first store into xs)
            col_fft3<L, true, false, XPASS_F3_PADS, 1>(v, xs, ld, line, j, Bf.tw, P.twn);
#pragma unroll
            for (int i = 0; i < NPT; i++) xs[col3_out_row<L>(j, i) * ld + line] = v[i];
        }
        __syncthreads();
        xinv_cells<NM, REC>(P, mat, Bf, cu, xs, ld, msrc, cb + (long long)row * nx, nx, 1, nthr, s_yz, xacc, macc,
                            emax, bad);
        __syncthreads();   // buffer q and s_yz are rewritten by the next rows
    }
    if (A.field_only) return;
    stage_epilogue<REC, NM>(P, mat, Bf, A, b, blockIdx.x, gridDim.x, xacc, emax, bad, s_red, s_redf, &s_last, macc);
}

// Whether the pipelined row kernel applies (see k_xinv_pipe) with this map.
static bool xpipe_applies(const Plan& P, const Buffers& Bf, const SpecMap* map) {
    return map && map->valid && map->base == Bf.spec && P.L == 1024 && P.TX == 8 && P.R == 1 && P.NT <= 256;
}

template <bool REC, int NM>
static cudaError_t launch_xpipe(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A, int nb,
                         const SpecMap* map, cudaStream_t s) {
    // persistent: XPIPE_BLOCKS per SM spread over the instances of the launch
    int per = (XPIPE_BLOCKS * g_sms + nb - 1) / nb;
    if (per > P.nrows) per = P.nrows;
    if (per < 1) per = 1;
    const size_t sm = 2 * XPIPE_BUF * sizeof(float2) + 128;   // + alignment slack
    if (P.nx == 1024) return launch_chain(k_xinv_pipe<REC, NM, true>, dim3(per, nb), dim3(XPASS_THREADS), sm, s, P, mat, Bf, A,
                                          map->map);
    return launch_chain(k_xinv_pipe<REC, NM, false>, dim3(per, nb), dim3(XPASS_THREADS), sm, s, P, mat, Bf, A, map->map);
}

cudaError_t launch_xinv(const Plan& P, const Material& mat, const Buffers& Bf, const StageArgs& A, int nb,
                        cudaStream_t s, const SpecMap* map, const Tune* T) {
    dim3 grid(P.nblk, nb);
    const int th = xthreads(P);
    const size_t sm = xinv_smem(P);
    const bool rec = A.record > 0 && !A.field_only && A.stage == (A.kind == KIND_RK4 ? 3 : 6);
    const bool multi = A.nmodes > 1;
    if (xpipe_applies(P, Bf, map) && (!T || T->x_pipe != 0)) {
        if (multi) {
            if (rec) return launch_xpipe<true, MAX_MODES>(P, mat, Bf, A, nb, map, s);
            return launch_xpipe<false, MAX_MODES>(P, mat, Bf, A, nb, map, s);
        }
        if (rec) return launch_xpipe<true, 1>(P, mat, Bf, A, nb, map, s);
        return launch_xpipe<false, 1>(P, mat, Bf, A, nb, map, s);
    }
    if (!multi && !rec && xpass_fixed(P)) {
        switch (P.L) {
#define MMCQ_CASE(Lv) \
    case Lv: return launch_chain(k_xinv<Lv, false, 1, true>, grid, th, sm, s, P, mat, Bf, A);
            MMCQ_XFIXED(MMCQ_CASE)
#undef MMCQ_CASE
            default: break;
        }
    }
    switch (P.L) {
#define MMCQ_CASE(Lv)                                                                                  \
    case Lv:                                                                                           \
        if (multi) {                                                                                   \
            if (rec) return launch_chain(k_xinv<Lv, true, MAX_MODES, false>, grid, th, sm, s, P, mat, Bf, A); \
            return launch_chain(k_xinv<Lv, false, MAX_MODES, false>, grid, th, sm, s, P, mat, Bf, A);         \
        }                                                                                              \
        if (rec) return launch_chain(k_xinv<Lv, true, 1, false>, grid, th, sm, s, P, mat, Bf, A);            \
        return launch_chain(k_xinv<Lv, false, 1, false>, grid, th, sm, s, P, mat, Bf, A);
        MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
        default: return cudaErrorInvalidValue;
    }
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
#define MMCQ_CASE(Lv)                                                                          \
    if ((e = xinv_attr(k_xinv<Lv, false, 1, false>, lim)) != cudaSuccess) return e;            \
    if ((e = xinv_attr(k_xinv<Lv, true, 1, false>, lim)) != cudaSuccess) return e;             \
    if ((e = xinv_attr(k_xinv<Lv, false, MAX_MODES, false>, lim)) != cudaSuccess) return e;    \
    if ((e = xinv_attr(k_xinv<Lv, true, MAX_MODES, false>, lim)) != cudaSuccess) return e;
    MMCQ_XCASES(MMCQ_CASE)
#undef MMCQ_CASE
#define MMCQ_CASE(Lv) \
    if ((e = xinv_attr(k_xinv<Lv, false, 1, true>, lim)) != cudaSuccess) return e;
    MMCQ_XFIXED(MMCQ_CASE)
#undef MMCQ_CASE
#define MMCQ_PIPE(R, M)                                                                 \
    if ((e = xinv_attr(k_xinv_pipe<R, M, true>, lim)) != cudaSuccess) return e;        \
    if ((e = xinv_attr(k_xinv_pipe<R, M, false>, lim)) != cudaSuccess) return e;
    MMCQ_PIPE(false, 1) MMCQ_PIPE(true, 1) MMCQ_PIPE(false, MAX_MODES) MMCQ_PIPE(true, MAX_MODES)
#undef MMCQ_PIPE
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace mq
