// Column passes of the demag convolution: FFT along y (and z) of tiles of kx
// columns of the half-spectrum, with the pointwise product by the symmetric
// demag kernel H = N M (6 real components, mirror-reduced storage) between the
// forward and the inverse transform of the last axis.  The paper lists the
// demag field among the effective-field terms (Sec. 2.1); the zero-padded
// convolution is the standard way to evaluate it.
//
// k_col_reg<P, WC>: transform length P <= 1024 in registers (fftreg.cuh);
//   a thread group owns one column and loads its strided rows straight from
//   global memory (consecutive threads = consecutive columns = contiguous
//   memory).  WC > 0: the common tile shape fixed at compile time.
// k_zconv<P> / k_zconv2<P, TXC, GC>: the z pass (pz <= 32, one thread per
//   column / pz = 16 or 32, two threads per column) with the demag product
//   between the forward and the inverse z transform.
// k_col_split<PH, FIXED>: y passes whose padded length 2 PH exceeds the
//   register path, as two PH-point register transforms per column.
// k_col_gen: any power-of-two length, shared-memory Stockham (fft.cuh); the
//   remaining long transforms.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "fftreg.cuh"
#include "kern_common.cuh"

namespace mq {

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
    int G;          // groups per block (power of two)
    int group_tiles;  // 1: groups are consecutive kx tiles; 0: consecutive outer indices
    int nouter;     // extent of the outer index
};

__device__ __forceinline__ void demag_product(const Plan& P, const float* __restrict__ kern, int kx, int ky,
                                              int kz, float2& mx, float2& my, float2& mz) {
    if (kx >= P.hx) { mx = my = mz = make_float2(0.f, 0.f); return; }
    float sy = 1.f, sz = 1.f;
    int kyr = ky, kzr = kz;
    if (ky > P.py / 2) { kyr = P.py - ky; sy = -1.f; }
    if (kz > P.pz / 2) { kzr = P.pz - kz; sz = -1.f; }
    const float2* K = reinterpret_cast<const float2*>(kern + (((long long)kzr * P.hyk + kyr) * (P.NT * P.TX) + kx) * 6);
    float2 k0 = __ldg(K), k1 = __ldg(K + 1), k2 = __ldg(K + 2);
    float xx = k0.x, yy = k0.y, zz = k1.x;
    float xy = sy * k1.y, xz = sz * k2.x, yz = sy * sz * k2.y;
    float2 hx = make_float2(xx * mx.x + xy * my.x + xz * mz.x, xx * mx.y + xy * my.y + xz * mz.y);
    float2 hy = make_float2(xy * mx.x + yy * my.x + yz * mz.x, xy * mx.y + yy * my.y + yz * mz.y);
    float2 hz = make_float2(xz * mx.x + yz * my.x + zz * mz.x, xz * mx.y + yz * my.y + zz * mz.y);
    mx = hx; my = hy; mz = hz;
}

// The product over every (row, kx column) of a block whose shared memory holds
// rows of W values laid out [group][comp][tx] (ncomp = 3).
__device__ __forceinline__ void block_product(const Plan& P, const Buffers& Bf, const ColArgs& C, float2* sm, int W,
                                              int t0, int o0) {
    const int TX = P.TX, lt = P.lt;
    const int gt = C.G * TX;          // kx columns of the block (power of two)
    const int lgt = lt + __ffs(C.G) - 1;
    const int rw = 3 * TX;
    for (int i = threadIdx.x; i < C.P * gt; i += blockDim.x) {
        int r = i >> lgt, q = i & (gt - 1);
        int g = q >> lt, tx = q & (TX - 1);
        int t = C.group_tiles ? t0 + g : t0;
        int o = C.group_tiles ? o0 : o0 + g;
        float2* p = sm + r * W + g * rw + tx;
        float2 mx = p[0], my = p[TX], mz = p[2 * TX];
        int ky = C.ky_is_row ? r : o;
        int kz = C.ky_is_row ? 0 : r;
        if (t < P.NT && o < C.nouter) demag_product(P, Bf.kern, t * TX + tx, ky, kz, mx, my, mz);
        p[0] = mx; p[TX] = my; p[2 * TX] = mz;
    }
}

// One block = G groups x ncomp x TX columns (W columns) x N1 threads per
// column.  Groups are consecutive kx tiles (y passes) or consecutive outer
// indices (z pass); in both cases consecutive columns are adjacent in memory.
// Transform lengths with a fixed-shape instantiation of k_col_reg.
constexpr bool col_fixed_len(int P) { return P >= 64 && P <= 512; }

// WC > 0: the block is one kx tile of WC / 3 columns with all three
// components (G = 1), rows WC apart in both spectra, fixed at compile time so
// that the row and shared-memory offsets are immediates.
template <int P, int WC>
__global__ void __launch_bounds__(512) k_col_reg(Plan Pl, Buffers Bf, StageArgs A, ColArgs C) {
    constexpr int NPT = ColShape<P>::NPT, N1 = ColShape<P>::N1;
    constexpr bool FIXED = WC > 0;
    extern __shared__ float2 sm[];
    const int ncomp = FIXED ? 3 : C.ncomp;
    const int b = A.inst0 + blockIdx.z;
    const int c0 = ncomp == 3 ? 0 : blockIdx.x % 3;
    const int bx = ncomp == 3 ? blockIdx.x : blockIdx.x / 3;
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = FIXED ? WC / 3 : Pl.TX;
    const int lt = FIXED ? ilog2<(FIXED ? WC / 3 : 1)>() : Pl.lt;
    const int G = FIXED ? 1 : C.G;
    const int rw = ncomp * TX;
    const int W = G * rw;
    const long long in_r = FIXED ? WC : C.in_r, out_r = FIXED ? WC : C.out_r;
    const int col = threadIdx.x % W;
    const int j = threadIdx.x / W;
    const int g = ncomp == 3 ? (col >> lt) / 3 : (col >> lt);
    const int e = col - g * rw;
    const int t0 = C.group_tiles ? bx * G : blockIdx.y;
    const int o0 = C.group_tiles ? blockIdx.y : bx * G;
    const int t = C.group_tiles ? t0 + g : t0;
    const int o = C.group_tiles ? o0 : o0 + g;
    const bool valid = t < Pl.NT && o < C.nouter;
    const float2* in = C.in + b * C.in_b + o * C.in_o + t * C.in_t + c0 * TX + e;
    float2* out = C.out + b * C.out_b + o * C.out_o + t * C.out_t + c0 * TX + e;

    float2 v[NPT];
#pragma unroll
    for (int n2 = 0; n2 < NPT; n2++) {
        const int r = j + N1 * n2;
        v[n2] = (valid && r < C.n_in) ? in[r * in_r] : make_float2(0.f, 0.f);
    }
    if (C.fwd) col_fft<P, false>(v, sm, W, col, j, Bf.tw, Pl.twn);
    if (C.mult) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NPT; i++) sm[col_out_row<P>(j, i) * W + col] = v[i];
        __syncthreads();
        block_product(Pl, Bf, C, sm, W, t0, o0);
        __syncthreads();
#pragma unroll
        for (int n2 = 0; n2 < NPT; n2++) v[n2] = sm[(j + N1 * n2) * W + col];
    }
    if (C.inv) col_fft<P, true>(v, sm, W, col, j, Bf.tw, Pl.twn);
    if (!valid) return;
    const bool transformed = C.fwd || C.inv;
#pragma unroll
    for (int i = 0; i < NPT; i++) {
        const int r = transformed ? col_out_row<P>(j, i) : j + N1 * i;
        if (r < C.n_out) out[r * out_r] = v[i];
    }
}

// z pass of the 3-D convolution for pz <= 32, one thread per (component, ky,
// kx) column holding all pz rows in registers:
//   1. forward FFT along z of the nz data rows (rows nz..pz/2-1 are read as
//      zero, rows pz/2.. are compile-time zeros, so the first butterfly
//      stage needs no additions);
//   2. the three component spectra of a (ky, kx) column meet in shared
//      memory, and the thread of component c forms row c of H m at every kz;
//   3. inverse FFT along z of that row, keeping the nz output rows.
// The mirror-reduced kernel is read once per stored kz row (kz and pz - kz
// share it, with the sign of the xz and yz entries flipped).  nz <= pz / 2
// always holds for the zero-padded convolution (pz >= 2 nz - 1, a power of 2).
template <int P>
__global__ void __launch_bounds__(256) k_zconv(Plan Pl, Buffers Bf, StageArgs A, ColArgs C) {
    extern __shared__ float2 sm[];      // [P][W]
    const int b = A.inst0 + blockIdx.z;
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = Pl.TX, lt = Pl.lt;
    const int W = C.G * 3 * TX;
    const int col = threadIdx.x;        // blockDim.x == W
    const int q = col >> lt;            // 3 g + c
    const int g = q / 3, c = q - 3 * g, tx = col & (TX - 1);
    const int t = blockIdx.y, o = blockIdx.x * C.G + g;   // tile, ky
    const float2* in = C.in + b * C.in_b + o * C.in_o + t * C.in_t + c * TX + tx;
    float2* out = C.out + b * C.out_b + o * C.out_o + t * C.out_t + c * TX + tx;

    float2 v[P];
#pragma unroll
    for (int r = 0; r < P / 2; r++) v[r] = r < C.n_in ? in[r * C.in_r] : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = P / 2; r < P; r++) v[r] = make_float2(0.f, 0.f);
    fft_reg<P, false>(v);
#pragma unroll
    for (int k = 0; k < P; k++) sm[k * W + col] = v[k];
    __syncthreads();

    // row c of the symmetric kernel [[xx xy xz] [xy yy yz] [xz yz zz]], stored
    // per (kz, ky, kx) as (xx, yy, zz, xy, xz, yz); an entry is odd in ky
    // (kz) when exactly one of its two indices is y (z).
    const int kx = t * TX + tx;
    const bool live = kx < Pl.hx;
    int kyr = o;
    float sy = 1.f;
    if (o > Pl.py / 2) { kyr = Pl.py - o; sy = -1.f; }
    const int i0 = c == 0 ? 0 : (c == 1 ? 3 : 4);
    const int i1 = c == 0 ? 3 : (c == 1 ? 1 : 5);
    const int i2 = c == 0 ? 4 : (c == 1 ? 5 : 2);
    float fp[3], fn[3];                 // signs for kz <= pz/2 and kz > pz/2
#pragma unroll
    for (int jj = 0; jj < 3; jj++) {
        const float y = ((c == 1) != (jj == 1)) ? sy : 1.f;
        fp[jj] = live ? y : 0.f;
        fn[jj] = ((c == 2) != (jj == 2)) ? -fp[jj] : fp[jj];
    }
    const long long zs = (long long)Pl.hyk * Pl.NT * TX * 6;
    const float* K = Bf.kern + ((long long)kyr * Pl.NT * TX + (live ? kx : 0)) * 6;
    const float2* mcol = sm + g * 3 * TX + tx;
#pragma unroll
    for (int kz = 0; kz <= P / 2; kz++) {
        const float* Kz = K + kz * zs;
        const float a0 = __ldg(Kz + i0), a1 = __ldg(Kz + i1), a2 = __ldg(Kz + i2);
        {
            const float2* mm = mcol + kz * W;
            const float2 mx = mm[0], my = mm[TX], mz = mm[2 * TX];
            const float c0 = a0 * fp[0], c1 = a1 * fp[1], c2 = a2 * fp[2];
            v[kz] = make_float2(c0 * mx.x + c1 * my.x + c2 * mz.x, c0 * mx.y + c1 * my.y + c2 * mz.y);
        }
        if (kz > 0 && kz < P / 2) {
            const float2* mm = mcol + (P - kz) * W;
            const float2 mx = mm[0], my = mm[TX], mz = mm[2 * TX];
            const float c0 = a0 * fn[0], c1 = a1 * fn[1], c2 = a2 * fn[2];
            v[P - kz] = make_float2(c0 * mx.x + c1 * my.x + c2 * mz.x, c0 * mx.y + c1 * my.y + c2 * mz.y);
        }
    }
    fft_reg<P, true>(v);
#pragma unroll
    for (int r = 0; r < P / 2; r++)
        if (r < C.n_out) out[r * C.out_r] = v[r];
}

// The same z pass with two threads per (component, ky, kx) column, each
// holding H = pz / 2 rows in registers (about half the registers of k_zconv,
// so about twice the resident warps).  With the data in rows < H, the DIF
// split of the P-point transform gives X[2m] = DFT_H(x)[m] and X[2m+1] =
// DFT_H(x W_P^r)[m]: thread half J = 0 takes the even, J = 1 the odd
// frequencies.  The product H m runs over the shared-memory copy of the whole
// spectrum, one (kz, ky, kx) point per thread and step.  The inverse is split
// the same way, y[n] = IDFT_H(h_even)[n] + W_P^{-n} IDFT_H(h_odd)[n] for the
// n < H rows kept; the halves add their parts through shared memory, each
// storing H / 2 rows.  Threads [0, W) form half 0, [W, 2W) half 1.
// FULL: all H rows hold data (nz = pz / 2), so no row is predicated; S: the
// integer type of the row stride rs.
template <int P, int J, bool FULL, typename S>
__device__ __forceinline__ void zsplit_forward(const ColArgs& C, float2* sm, int W, int col, const float2* in, S rs) {
    constexpr int H = P / 2;
    float2 v[H];
#pragma unroll
    for (int r = 0; r < H; r++) v[r] = (FULL || r < C.n_in) ? in[r * rs] : make_float2(0.f, 0.f);
    if (J == 1) {
#pragma unroll
        for (int r = 1; r < H; r++) {
            const int e = r * (32 / P);           // W_P^r = W_32^e
            if (e == 8) v[r] = make_float2(v[r].y, -v[r].x);
            else v[r] = cmul(v[r], c_tw32[e]);
        }
    }
    fft_reg<H, false>(v);
#pragma unroll
    for (int m = 0; m < H; m++) sm[(2 * m + J) * W + col] = v[m];
}

// The inverse runs in three phases with the block barriers between them in
// the kernel body, where every thread of the block reaches the same barrier
// instruction; each phase is a branch-free function of one half J:
//   zinv_transform: the half's H frequencies from shared memory, inverse
//     H-point DFT, and (J = 1) the twiddle W_P^{-n};
//   zinv_handoff: the rows the other half will write out (J = 0 hands over
//     rows Q..H-1, J = 1 rows 0..Q-1) go to shared memory;
//   zinv_finish: the half's own Q rows plus the other half's part, written out.
template <int P, int J>
__device__ __forceinline__ void zinv_transform(const float2* sm, int W, int col, float2 (&v)[P / 2]) {
    constexpr int H = P / 2;
#pragma unroll
    for (int m = 0; m < H; m++) v[m] = sm[(2 * m + J) * W + col];
    fft_reg<H, true>(v);
    if (J == 1) {
#pragma unroll
        for (int n = 1; n < H; n++) {
            const int e = n * (32 / P);           // W_P^{-n} = conj(W_32^e)
            if (e == 8) v[n] = make_float2(-v[n].y, v[n].x);
            else { float2 w = c_tw32[e]; w.y = -w.y; v[n] = cmul(v[n], w); }
        }
    }
}

template <int P, int J>
__device__ __forceinline__ void zinv_handoff(float2* sm, int W, int col, const float2 (&v)[P / 2]) {
    constexpr int Q = P / 4;
#pragma unroll
    for (int n = 0; n < Q; n++) sm[((J == 0 ? Q : 0) + n) * W + col] = v[(J == 0 ? Q : 0) + n];
}

template <int P, int J, bool FULL, typename S>
__device__ __forceinline__ void zinv_finish(const ColArgs& C, const float2* sm, int W, int col,
                                            const float2 (&v)[P / 2], float2* out, S rs) {
    constexpr int Q = P / 4;
#pragma unroll
    for (int n = 0; n < Q; n++) {
        const int r = (J == 0 ? 0 : Q) + n;
        const float2 u = sm[r * W + col];
        if (FULL || r < C.n_out) out[r * rs] = cadd(v[r], u);
    }
}

// TXC, GC: tile width and groups per block fixed at compile time (0: from the
// plan), so that the shared-memory offsets are immediates; with them the rows
// are all data (FULL) and the row strides fit in int.
template <int P, int TXC, int GC>
__global__ void __launch_bounds__(192, 6) k_zconv2(Plan Pl, Buffers Bf, StageArgs A, ColArgs C) {
    extern __shared__ float2 sm[];      // [P][W]
    constexpr bool FIXED = TXC > 0 && GC > 0;
    const int b = A.inst0 + blockIdx.z;
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = FIXED ? TXC : Pl.TX, lt = FIXED ? ilog2<(TXC > 0 ? TXC : 1)>() : Pl.lt;
    const int Gb = FIXED ? GC : C.G;
    const int W = Gb * 3 * TX;
    const int half = threadIdx.x >= W;
    const int col = threadIdx.x - half * W;
    const int q = col >> lt;
    const int g = q / 3, c = q - 3 * g, tx = col & (TX - 1);
    const int t = blockIdx.y, o0 = blockIdx.x * Gb;
    const long long off_in = b * C.in_b + (o0 + g) * C.in_o + t * C.in_t + c * TX + tx;
    const long long off_out = b * C.out_b + (o0 + g) * C.out_o + t * C.out_t + c * TX + tx;
    if constexpr (P <= 16) {
        // the rows of the stored kernel this thread's product reads (see
        // below), asked of L1 now so that they arrive during the forward
        // transform instead of after its barrier (P = 32 has no registers
        // to spare for the addresses)
        const int GT = Gb * TX, lgt = __ffs(GT) - 1;
        const int p = threadIdx.x & (GT - 1);
        const int ky = o0 + (p >> lt), kx = t * TX + (p & (TX - 1));
        const int kyr = ky > Pl.py / 2 ? Pl.py - ky : ky;
        if (kx < Pl.hx) {
            const float* Kb = Bf.kern + ((long long)kyr * Pl.NT * TX + kx) * 6;
            const long long zs = (long long)Pl.hyk * Pl.NT * TX * 6;
#pragma unroll
            for (int it = 0; it < (P / 2 + 6) / 6; it++) {
                const int kzr = (int)(threadIdx.x >> lgt) + 6 * it;
                if (kzr <= P / 2) asm volatile("prefetch.global.L1 [%0];\n" ::"l"(Kb + kzr * zs));
            }
        }
    }
    if (FIXED) {
        if (half == 0) zsplit_forward<P, 0, true>(C, sm, W, col, C.in + off_in, (int)C.in_r);
        else zsplit_forward<P, 1, true>(C, sm, W, col, C.in + off_in, (int)C.in_r);
    } else {
        if (half == 0) zsplit_forward<P, 0, false>(C, sm, W, col, C.in + off_in, C.in_r);
        else zsplit_forward<P, 1, false>(C, sm, W, col, C.in + off_in, C.in_r);
    }
    __syncthreads();

    // product at every (kz, g, tx) point of the block: symmetric kernel
    // (xx, yy, zz, xy, xz, yz) at (|kz|, |ky|, kx); xy is odd in ky, xz in kz,
    // yz in both.  The block has 2 W = 6 G TX threads, so a thread keeps its
    // (g, tx) point and takes every sixth mirror pair (kz, P - kz): one read
    // of the stored kernel row serves both, with xz and yz negated for P - kz.
    const int GT = Gb * TX;                       // power of two
    const int lgt = __ffs(GT) - 1;
    const long long zs = (long long)Pl.hyk * Pl.NT * TX * 6;
    const int p = threadIdx.x & (GT - 1);
    const int gg = p >> lt, xx = p & (TX - 1);
    const int ky = o0 + gg, kx = t * TX + xx;
    const bool live = kx < Pl.hx;
    const bool ny_ = ky > Pl.py / 2;
    const int kyr = ny_ ? Pl.py - ky : ky;
    const float sy = ny_ ? -1.f : 1.f;
    const float* Kb = Bf.kern + ((long long)kyr * Pl.NT * TX + (live ? kx : 0)) * 6;
    float2* pm0 = sm + gg * 3 * TX + xx;
    const int kz0 = threadIdx.x >> lgt;           // 0 .. 5
    auto apply = [&](float2* pm, float Kxx, float Kyy, float Kzz, float Kxy, float Kxz, float Kyz) {
        const float2 mx = pm[0], my = pm[TX], mz = pm[2 * TX];
        pm[0] = make_float2(Kxx * mx.x + Kxy * my.x + Kxz * mz.x, Kxx * mx.y + Kxy * my.y + Kxz * mz.y);
        pm[TX] = make_float2(Kxy * mx.x + Kyy * my.x + Kyz * mz.x, Kxy * mx.y + Kyy * my.y + Kyz * mz.y);
        pm[2 * TX] = make_float2(Kxz * mx.x + Kyz * my.x + Kzz * mz.x, Kxz * mx.y + Kyz * my.y + Kzz * mz.y);
    };
#pragma unroll
    for (int it = 0; it < (P / 2 + 6) / 6; it++) {
        const int kzr = kz0 + 6 * it;
        if (kzr > P / 2) break;
        if (live) {
            const float2* Kp = reinterpret_cast<const float2*>(Kb + kzr * zs);
            const float2 k0 = __ldg(Kp), k1 = __ldg(Kp + 1), k2 = __ldg(Kp + 2);
            const float Kxy = sy * k1.y, Kyz = sy * k2.y;
            apply(pm0 + kzr * W, k0.x, k0.y, k1.x, Kxy, k2.x, Kyz);
            if (kzr > 0 && kzr < P / 2) apply(pm0 + (P - kzr) * W, k0.x, k0.y, k1.x, Kxy, -k2.x, -Kyz);
        } else {
            const float2 z0 = make_float2(0.f, 0.f);
            float2* pm = pm0 + kzr * W;
            pm[0] = z0; pm[TX] = z0; pm[2 * TX] = z0;
            if (kzr > 0 && kzr < P / 2) {
                pm = pm0 + (P - kzr) * W;
                pm[0] = z0; pm[TX] = z0; pm[2 * TX] = z0;
            }
        }
    }
    __syncthreads();
    float2 v[P / 2];
    if (half == 0) zinv_transform<P, 0>(sm, W, col, v);
    else zinv_transform<P, 1>(sm, W, col, v);
    __syncthreads();                              // both halves have read the product
    if (half == 0) zinv_handoff<P, 0>(sm, W, col, v);
    else zinv_handoff<P, 1>(sm, W, col, v);
    __syncthreads();
    if (FIXED) {
        if (half == 0) zinv_finish<P, 0, true>(C, sm, W, col, v, C.out + off_out, (int)C.out_r);
        else zinv_finish<P, 1, true>(C, sm, W, col, v, C.out + off_out, (int)C.out_r);
    } else {
        if (half == 0) zinv_finish<P, 0, false>(C, sm, W, col, v, C.out + off_out, C.out_r);
        else zinv_finish<P, 1, false>(C, sm, W, col, v, C.out + off_out, C.out_r);
    }
}

// y passes with P = 2 PH longer than the register path holds (P = 2048): the
// zero padding leaves at most PH input rows (forward) and needs at most PH
// output rows (inverse), so the P-point transform is two PH-point register
// transforms per column (decimation in frequency):
//   forward:  X[2k] = DFT_PH(x)[k],  X[2k+1] = DFT_PH(x_r W_P^r)[k],
//   inverse:  y[n] = IDFT_PH(h_even)[n] + W_P^{-n} IDFT_PH(h_odd)[n],  n < PH.
// The same threads do both halves one after the other; in the inverse the odd
// half is added onto the rows the even half stored, by atomic adds done in L2
// (each row stays with one thread: one store, then one add).
// FIXED: one component of one 8-column tile per block (G = 1), rows 24 apart
// in both spectra, at compile time.
// F3 (FIXED with PH = 1024): the three-factor transform, 16 points per
// thread and 64 threads per column (512 threads for the 8 columns), so that
// two blocks of 16 warps fit an SM; the last factor by a second transpose.
// JS (F3 only): each half J in a block of its own (blockIdx.x = 2 (3 tile +
// component) + J), twice the blocks with half the work each.  In the forward
// the two blocks are independent.  The inverse is launched as clusters of the
// two blocks: each keeps half of the output rows (J = 0 those below PH / 2,
// J = 1 the others), hands the other half of its terms to the partner through
// its shared memory, and adds the partner's terms for its own rows, so the
// even half's rows never go to global memory and back.
template <int PH, bool FIXED, bool JS = false>
__global__ void __launch_bounds__(512, (FIXED && PH == 1024) ? 2 : 1) k_col_split(Plan Pl, Buffers Bf, StageArgs A,
                                                                                   ColArgs C) {
    constexpr bool F3 = FIXED && PH == 1024;
    static_assert(!JS || F3, "one half per block is the three-factor shape only");
    constexpr int NPT = F3 ? 16 : ColShape<PH>::NPT, N1 = F3 ? ColShape3<PH>::N1 : ColShape<PH>::N1;
    constexpr int P = 2 * PH;
    extern __shared__ float2 sm[];
    const int ncomp = FIXED ? 1 : C.ncomp;
    const int b = A.inst0 + blockIdx.z;
    const int Jb = JS ? (int)(blockIdx.x & 1) : 0;            // the block's half (JS)
    const int bxx = JS ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int c0 = ncomp == 3 ? 0 : bxx % 3;
    const int bx = ncomp == 3 ? bxx : bxx / 3;
    // the same for both blocks of a cluster (same instance)
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = FIXED ? 8 : Pl.TX, lt = FIXED ? 3 : Pl.lt;
    const int G = FIXED ? 1 : C.G;
    const long long in_r = FIXED ? 24 : C.in_r, out_r = FIXED ? 24 : C.out_r;
    const int rw = ncomp * TX;
    const int W = G * rw;
    const int col = threadIdx.x % W;
    const int j = threadIdx.x / W;
    const int g = ncomp == 3 ? (col >> lt) / 3 : (col >> lt);
    const int e = col - g * rw;
    const int t = bx * G + g, o = blockIdx.y;                  // tiles are the groups here
    const bool valid = t < Pl.NT && o < C.nouter;
    const float2* in = C.in + b * C.in_b + o * C.in_o + t * C.in_t + c0 * TX + e;
    float2* out = C.out + b * C.out_b + o * C.out_o + t * C.out_t + c0 * TX + e;
    // exp(-2 pi i e / P), e < P, after the transform buffer: the odd-half
    // twiddles W_P^r and the four-step twiddles W_PH^{j k2} = W_P^{2 j k2}
    float2* stw = sm + PH * W;
    auto fft = [&](float2 (&v)[NPT], bool inv) {
        if constexpr (F3) {
            if (inv) col_fft3<PH, true, true, 0, 8, true>(v, sm, W, col, j, stw, P);
            else col_fft3<PH, false, true, 0, 8, true>(v, sm, W, col, j, stw, P);
        } else {
            if (inv) col_fft<PH, true, true>(v, sm, W, col, j, stw, P);
            else col_fft<PH, false, true>(v, sm, W, col, j, stw, P);
        }
    };
    auto out_row = [&](int i) { return F3 ? col3t_out_row<PH>(j, i) : col_out_row<PH>(j, i); };
    {
        const int tstep = Pl.twn / P;
        for (int q = threadIdx.x; q < P; q += blockDim.x) stw[q] = __ldg(Bf.tw + q * tstep);
    }
    __syncthreads();
    if constexpr (JS) {
        if (!C.fwd) {
            // inverse, one half per block: the block's PH-point inverse, and
            // (J = 1) the twiddle W_P^{-k}, before the exchange
            const int J = Jb;
            float2 v[NPT];
#pragma unroll
            for (int n2 = 0; n2 < NPT; n2++) {
                const int r = 2 * (j + N1 * n2) + J;
                v[n2] = (valid && r < C.n_in) ? in[r * in_r] : make_float2(0.f, 0.f);
            }
            fft(v, true);
            if (J == 1) {
#pragma unroll
                for (int i = 0; i < NPT; i++) v[i] = cmul(v[i], conjf2(stw[out_row(i)]));
            }
            // element i is row a + 16 (4 q + i / 4) + (PH / 4) (i % 4): below
            // PH / 2 exactly when i % 4 < 2.  The 8 elements a block gives
            // away go to slot 2 (i / 4) + i % 2 of its own buffer [8][threads];
            // the partner thread of the same index holds the same rows.
            const int nth = (int)blockDim.x;
            float2* hand = sm;
#pragma unroll
            for (int i = 0; i < NPT; i++) {
                const bool give = ((i & 3) >= 2) == (J == 0);
                if (give) hand[(2 * (i >> 2) + (i & 1)) * nth + threadIdx.x] = v[i];
            }
            cluster_sync();
            const unsigned rem = cluster_map(smem_u32(hand), (unsigned)(J ^ 1));
#pragma unroll
            for (int i = 0; i < NPT; i++) {
                const bool give = ((i & 3) >= 2) == (J == 0);
                if (!give) {
                    const float2 u = ld_cluster_f2(rem + 8u * (unsigned)((2 * (i >> 2) + (i & 1)) * nth + threadIdx.x));
                    const int k = out_row(i);
                    if (valid && k < C.n_out) out[k * out_r] = cadd(v[i], u);
                }
            }
            cluster_sync();   // the partner has read this block's buffer
            return;
        }
    }
#pragma unroll 1
    for (int J = JS ? Jb : 0; J < (JS ? Jb + 1 : 2); J++) {
        float2 v[NPT];
        if (C.fwd) {
            // odd half: x_r W_P^r with r = j + N1 n2; for the three-factor
            // shape W_P^r = W_P^j W_32^{n2} (N1 = P / 32), one table value
            // per thread and constant-bank factors
            const float2 wj = stw[j];
#pragma unroll
            for (int n2 = 0; n2 < NPT; n2++) {
                const int r = j + N1 * n2;
                float2 x = (valid && r < C.n_in) ? in[r * in_r] : make_float2(0.f, 0.f);
                if (J == 1) x = F3 ? cmul(x, n2 == 0 ? wj : cmul(wj, c_tw32[n2])) : cmul(x, stw[r]);
                v[n2] = x;
            }
            fft(v, false);
            if (valid) {
#pragma unroll
                for (int i = 0; i < NPT; i++) out[(2 * out_row(i) + J) * out_r] = v[i];
            }
        } else {
#pragma unroll
            for (int n2 = 0; n2 < NPT; n2++) {
                const int r = 2 * (j + N1 * n2) + J;
                v[n2] = (valid && r < C.n_in) ? in[r * in_r] : make_float2(0.f, 0.f);
            }
            fft(v, true);
            if (valid) {
                if (J == 0) {
#pragma unroll
                    for (int i = 0; i < NPT; i++) {
                        const int k = out_row(i);
                        if (k < C.n_out) out[k * out_r] = v[i];
                    }
                } else {
                    // the odd half's terms are added onto the even half's rows
                    // where they are (a reduction in L2, no load back): each
                    // row holds one store and then one add, both from this
                    // thread, so the sum is the one rounding of a + y (the
                    // atomic add flushes subnormal values to zero)
#pragma unroll
                    for (int i = 0; i < NPT; i++) {
                        const int k = out_row(i);
                        const float2 y = cmul(v[i], conjf2(stw[k]));
                        if (k < C.n_out) red_add_f2(out + k * out_r, y);
                    }
                }
            }
        }
    }
}

// Generic shared-memory version (any power-of-two P up to 4096).
template <int SLOTS>
__global__ void __launch_bounds__(MAX_THREADS) k_col_gen(Plan P, Buffers Bf, StageArgs A, ColArgs C) {
    extern __shared__ float2 sm[];
    const int b = A.inst0 + blockIdx.z;
    const int c0 = C.ncomp == 3 ? 0 : blockIdx.x % 3;
    const int bx = C.ncomp == 3 ? blockIdx.x : blockIdx.x / 3;
    if (stage_skips(Bf.st[b], A)) return;
    const int TX = P.TX;
    const int rw = C.ncomp * TX;
    const int G = C.G;
    const int W = G * rw;
    const int t0 = C.group_tiles ? bx * G : blockIdx.y;
    const int o0 = C.group_tiles ? blockIdx.y : bx * G;
    const float2* in = C.in + b * C.in_b + c0 * TX;
    float2* out = C.out + b * C.out_b + c0 * TX;
    for (int i = threadIdx.x; i < C.P * W; i += blockDim.x) {
        int r = i / W, q = i - r * W;
        int g = q / rw, e = q - g * rw;
        int t = C.group_tiles ? t0 + g : t0;
        int o = C.group_tiles ? o0 : o0 + g;
        float2 v = make_float2(0.f, 0.f);
        if (r < C.n_in && t < P.NT && o < C.nouter) v = in[o * C.in_o + t * C.in_t + r * C.in_r + e];
        sm[i] = v;
    }
    __syncthreads();
    if (C.fwd) block_fft<true, SLOTS>(sm, C.P, W, W, 1, false, Bf.tw, P.twn);
    if (C.mult) {
        block_product(P, Bf, C, sm, W, t0, o0);
        __syncthreads();
    }
    if (C.inv) block_fft<true, SLOTS>(sm, C.P, W, W, 1, true, Bf.tw, P.twn);
    for (int i = threadIdx.x; i < C.n_out * W; i += blockDim.x) {
        int r = i / W, q = i - r * W;
        int g = q / rw, e = q - g * rw;
        int t = C.group_tiles ? t0 + g : t0;
        int o = C.group_tiles ? o0 : o0 + g;
        if (t < P.NT && o < C.nouter) out[o * C.out_o + t * C.out_t + r * C.out_r + e] = sm[i];
    }
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
bool fft_fits(int nlines, int L) { return (nlines * L + 3) / 4 <= MAX_SLOTS * MAX_THREADS; }

static int gen_threads(int nlines, int L, int* per) {
    int slots = (nlines * L + 3) / 4;
    *per = slots <= 2 * MAX_THREADS ? 2 : 4;
    int th = (slots + *per - 1) / *per;
    th = ((th + 31) / 32) * 32;
    return th < 32 ? 32 : (th > MAX_THREADS ? MAX_THREADS : th);
}

template <int P>
static cudaError_t launch_reg(const Plan& Pl, const Buffers& Bf, const StageArgs& A, const ColArgs& C, dim3 grid,
                              int W, cudaStream_t s) {
    constexpr int N1 = ColShape<P>::N1;
    const bool fixed = Pl.TX == 8 && C.ncomp == 3 && C.G == 1 && !C.mult && C.group_tiles && C.in_r == 24 &&
                       C.out_r == 24;
    if constexpr (col_fixed_len(P)) {
        if (fixed) {
            return launch_chain(k_col_reg<P, 24>, grid, W * N1, (size_t)P * W * sizeof(float2), s, Pl, Bf, A, C);
        }
    }
    (void)fixed;
    return launch_chain(k_col_reg<P, 0>, grid, W * N1, (size_t)P * W * sizeof(float2), s, Pl, Bf, A, C);
}

template <int P>
static cudaError_t launch_z(const Plan& Pl, const Buffers& Bf, const StageArgs& A, const ColArgs& C, int nb,
                            cudaStream_t s) {
    const int W = C.G * 3 * Pl.TX;
    dim3 grid((Pl.py + C.G - 1) / C.G, Pl.NT, nb);
    return launch_chain(k_zconv<P>, grid, W, (size_t)P * W * sizeof(float2), s, Pl, Bf, A, C);
}

// The fixed-shape z pass: tiles of 8 kx columns, 4 ky per block, all pz / 2 rows data.
static bool z2_fixed(const Plan& Pl, const ColArgs& C, int P) {
    return Pl.TX == 8 && C.G == 4 && C.n_in == P / 2 && C.n_out == P / 2 && (long long)C.in_r * P < (1LL << 31) &&
           (long long)C.out_r * P < (1LL << 31);
}

template <int P>
static cudaError_t launch_z2(const Plan& Pl, const Buffers& Bf, const StageArgs& A, const ColArgs& C, int nb,
                             cudaStream_t s) {
    const int W = C.G * 3 * Pl.TX;
    dim3 grid((Pl.py + C.G - 1) / C.G, Pl.NT, nb);
    if (z2_fixed(Pl, C, P))
        return launch_chain(k_zconv2<P, 8, 4>, grid, 2 * W, (size_t)P * W * sizeof(float2), s, Pl, Bf, A, C);
    return launch_chain(k_zconv2<P, 0, 0>, grid, 2 * W, (size_t)P * W * sizeof(float2), s, Pl, Bf, A, C);
}

// Whether a y pass of this plan runs the fixed three-factor split kernel
// (k_col_split<1024, true>), the one with the choice of a half per block.
static bool split_fixed(const Plan& Pl, const ColArgs& C) {
    return Pl.TX == 8 && C.ncomp == 1 && C.G == 1 && C.in_r == 24 && C.out_r == 24;
}

template <int PH>
static cudaError_t launch_split(const Plan& Pl, const Buffers& Bf, const StageArgs& A, const ColArgs& C, int nb,
                                cudaStream_t s, bool js) {
    constexpr int N1 = ColShape<PH>::N1;
    const int W = C.G * C.ncomp * Pl.TX;
    dim3 grid(((Pl.NT + C.G - 1) / C.G) * (C.ncomp == 3 ? 1 : 3), C.nouter, nb);
    const bool fixed = split_fixed(Pl, C);
    const size_t smem = ((size_t)PH * W + 2 * PH) * sizeof(float2);   // transform buffer + twiddle table
    if (fixed) {
        const int n1 = PH == 1024 ? ColShape3<PH>::N1 : N1;   // three-factor shape (see k_col_split)
        if constexpr (PH == 1024) {
            if (js) {
                // a half per block; the inverse's two blocks form a cluster
                dim3 g2(grid.x * 2, grid.y, grid.z);
                if (C.fwd) return launch_chain(k_col_split<PH, true, true>, g2, W * n1, smem, s, Pl, Bf, A, C);
                return launch_chain_cl(k_col_split<PH, true, true>, g2, dim3(W * n1), smem, s, 2, Pl, Bf, A, C);
            }
        }
        return launch_chain(k_col_split<PH, true>, grid, W * n1, smem, s, Pl, Bf, A, C);
    }
    return launch_chain(k_col_split<PH, false>, grid, W * N1, smem, s, Pl, Bf, A, C);
}

// z pass with one thread per column (pz <= 32); false if it does not apply.
static bool zconv_applies(const Plan& P) { return P.nz > 1 && P.pz <= 32 && 2 * P.nz <= P.pz; }

// k_zconv2: 2 W = 6 G TX threads, at most ZSPLIT_THREADS (its launch bound)
static const int ZSPLIT_THREADS = 192;
static int zsplit_groups(const Plan& P) {
    int G = 1;
    while (G * 2 <= P.py && 2 * G * 2 * 3 * P.TX <= ZSPLIT_THREADS) G *= 2;
    return G;
}

static int zconv_groups(const Plan& P) {
    int G = 1;
    while (G * 2 <= P.py && G * 2 * 3 * P.TX <= 256) G *= 2;
    return G;
}

static cudaError_t launch_col(const Plan& P, const Buffers& Bf, const StageArgs& A, const ColArgs& C, int nb,
                              cudaStream_t s) {
    const int W = C.G * C.ncomp * P.TX;
    dim3 grid;
    // one component per block: the three component blocks of a tile are
    // consecutive in x, so they run together and share the L2 lines of the
    // tile rows (each component is a third of a row)
    const int nc = C.ncomp == 3 ? 1 : 3;
    if (C.group_tiles) grid = dim3(((P.NT + C.G - 1) / C.G) * nc, C.nouter, nb);
    else grid = dim3(((C.nouter + C.G - 1) / C.G) * nc, P.NT, nb);
    switch (C.P) {
        case 1: return launch_reg<1>(P, Bf, A, C, grid, W, s);
        case 2: return launch_reg<2>(P, Bf, A, C, grid, W, s);
        case 4: return launch_reg<4>(P, Bf, A, C, grid, W, s);
        case 8: return launch_reg<8>(P, Bf, A, C, grid, W, s);
        case 16: return launch_reg<16>(P, Bf, A, C, grid, W, s);
        case 32: return launch_reg<32>(P, Bf, A, C, grid, W, s);
        case 64: return launch_reg<64>(P, Bf, A, C, grid, W, s);
        case 128: return launch_reg<128>(P, Bf, A, C, grid, W, s);
        case 256: return launch_reg<256>(P, Bf, A, C, grid, W, s);
        case 512: return launch_reg<512>(P, Bf, A, C, grid, W, s);
        case 1024: return launch_reg<1024>(P, Bf, A, C, grid, W, s);
        default: break;
    }
    int per;
    int th = gen_threads(W, C.P, &per);
    size_t sm = (size_t)C.P * W * sizeof(float2);
    if (per == 2) return launch_chain(k_col_gen<2>, grid, th, sm, s, P, Bf, A, C);
    return launch_chain(k_col_gen<4>, grid, th, sm, s, P, Bf, A, C);
}

// Threads of a register-path block: W columns x N1 threads each.
static int reg_threads(int P, int W) { return W * col_threads_per_column(P); }

// Group count (power of two, <= limit) for a column pass: as large as keeps
// the block within `max_threads` threads and `smem_cap` bytes.
static int pick_groups(int width, int P, int limit, int max_threads, size_t smem_cap) {
    int G = 1;
    while (G * 2 <= limit) {
        int W = G * 2 * width;
        size_t sm = (size_t)P * W * sizeof(float2);
        bool ok = sm <= smem_cap && (P > 1024 ? fft_fits(W, P) : reg_threads(P, W) <= max_threads);
        if (!ok) break;
        G *= 2;
    }
    return G;
}

// Layout strides of the tiled spectra.
static void spec_strides(const Plan& P, int rows, long long& sb, long long& sz, long long& st, long long& sr) {
    sr = 3LL * P.TX;                    // one row (ky or y) of a tile
    st = (long long)rows * sr;          // one tile
    sz = (long long)P.NT * st;          // one z plane
    sb = (long long)P.nz * sz;          // one instance
}

static const size_t COL_SMEM_CAP = 48 * 1024;
static const int COL_MAX_THREADS = 256;
// A half per block in the fixed split y passes (forward, inverse) by default.
static const bool Y_SPLIT_RULE[2] = {false, false};

// One launch of the demag convolution: part 0 = 2-D (fwd y, product, inv y);
// 3-D: part 1 = forward y, 2 = z forward / product / z inverse, 3 = inverse y.
// Groups per block of a column part as the tuning asks, within the rule's
// (largest feasible) count; a count of 0 keeps the rule.
static int tuned_groups(const Tune* T, int part, int rule) {
    if (!T || T->col_g[part] <= 0) return rule;
    int G = 1;
    while (G * 2 <= T->col_g[part] && G * 2 <= rule) G *= 2;
    return G;
}

cudaError_t launch_conv_part(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s, int part,
                             const Tune* T) {
    long long sb, sz, st, sr, tb, tz, tt, tr;
    spec_strides(P, P.ny, sb, sz, st, sr);
    spec_strides(P, P.py, tb, tz, tt, tr);
    ColArgs C{};
    if (part == 0) {
        C.in = Bf.spec; C.out = Bf.spec;
        C.in_b = C.out_b = sb; C.in_o = C.out_o = 0; C.in_t = C.out_t = st; C.in_r = C.out_r = sr;
        C.P = P.py; C.n_in = P.ny; C.n_out = P.ny;
        C.fwd = 1; C.mult = 1; C.inv = 1; C.ncomp = 3; C.ky_is_row = 1;
        C.group_tiles = 1; C.nouter = 1;
        C.G = tuned_groups(T, 0, pick_groups(3 * P.TX, P.py, P.NT, COL_MAX_THREADS, COL_SMEM_CAP));
    } else if (part == 1 || part == 3) {
        bool fwd = part == 1;
        C.in = fwd ? Bf.spec : Bf.spec2;
        C.out = fwd ? Bf.spec2 : Bf.spec;
        C.in_b = fwd ? sb : tb; C.in_o = fwd ? sz : tz; C.in_t = fwd ? st : tt; C.in_r = fwd ? sr : tr;
        C.out_b = fwd ? tb : sb; C.out_o = fwd ? tz : sz; C.out_t = fwd ? tt : st; C.out_r = fwd ? tr : sr;
        C.P = P.py; C.n_in = fwd ? P.ny : P.py; C.n_out = fwd ? P.py : P.ny;
        C.fwd = fwd; C.inv = !fwd;
        bool three = P.py <= 1024 ? reg_threads(P.py, 3 * P.TX) <= 512 && (size_t)P.py * 3 * P.TX * 8 <= COL_SMEM_CAP
                                  : fft_fits(3 * P.TX, P.py) && (size_t)P.py * 3 * P.TX * 8 <= COL_SMEM_CAP;
        C.ncomp = three ? 3 : 1;
        C.group_tiles = 1; C.nouter = P.nz;
        C.G = tuned_groups(T, part, pick_groups(C.ncomp * P.TX, P.py, P.NT, COL_MAX_THREADS, COL_SMEM_CAP));
        if (P.py == 2048 && 2 * P.ny <= P.py) {
            // two register transforms of 1024 per column (split of the padded length)
            const bool three = reg_threads(1024, 3 * P.TX) <= 512 && (size_t)1024 * 3 * P.TX * 8 <= 96 * 1024;
            C.ncomp = three ? 3 : 1;
            C.G = tuned_groups(T, part, pick_groups(C.ncomp * P.TX, 1024, P.NT, 512, 96 * 1024));
            const int ys = T ? T->y_split[part == 1 ? 0 : 1] : -1;
            return launch_split<1024>(P, Bf, A, C, nb, s, ys > 0 || (ys < 0 && Y_SPLIT_RULE[part == 1 ? 0 : 1]));
        }
    } else {
        C.in = Bf.spec2; C.out = Bf.spec2;
        C.in_b = C.out_b = tb; C.in_o = C.out_o = tr; C.in_t = C.out_t = tt; C.in_r = C.out_r = tz;
        C.P = P.pz; C.n_in = P.nz; C.n_out = P.nz; C.fwd = 1; C.mult = 1; C.inv = 1; C.ncomp = 3; C.ky_is_row = 0;
        C.group_tiles = 0; C.nouter = P.py;
        C.G = tuned_groups(T, 2, pick_groups(3 * P.TX, P.pz, P.py, COL_MAX_THREADS, COL_SMEM_CAP));
        if (zconv_applies(P)) {
            C.G = tuned_groups(T, 2, zconv_groups(P));
            // the split kernel: the rule for pz = 32, a tuning choice for pz = 16
            const bool split = P.pz == 32 ? (!T || T->z_split != 0) : (P.pz == 16 && T && T->z_split == 1);
            if (split) {
                // k_zconv2's halves are kept whole warps (W = 96 for every grid
                // with 32 or more kx x ky columns per block), so that no warp
                // diverges on the half; its barriers sit outside the per-half
                // branches either way
                const int G2 = tuned_groups(T, 2, zsplit_groups(P));
                if ((3 * G2 * P.TX) % 32 == 0) {
                    C.G = G2;
                    return P.pz == 32 ? launch_z2<32>(P, Bf, A, C, nb, s) : launch_z2<16>(P, Bf, A, C, nb, s);
                }
            }
            switch (P.pz) {
                case 2: return launch_z<2>(P, Bf, A, C, nb, s);
                case 4: return launch_z<4>(P, Bf, A, C, nb, s);
                case 8: return launch_z<8>(P, Bf, A, C, nb, s);
                case 16: return launch_z<16>(P, Bf, A, C, nb, s);
                case 32: return launch_z<32>(P, Bf, A, C, nb, s);
                default: break;
            }
        }
    }
    return launch_col(P, Bf, A, C, nb, s);
}

cudaError_t launch_convolution(const Plan& P, const Buffers& Bf, const StageArgs& A, int nb, cudaStream_t s,
                               const Tune* T) {
    if (P.nz == 1) return launch_conv_part(P, Bf, A, nb, s, 0, T);
    cudaError_t e;
    for (int part = 1; part <= 3; part++)
        if ((e = launch_conv_part(P, Bf, A, nb, s, part, T)) != cudaSuccess) return e;
    return cudaSuccess;
}

// The tunable choices of a plan's column passes: the rule's (largest) group
// count of each part present (0 where the part is not launched), and whether
// the split z kernel is an alternative.
void conv_tunables(const Plan& P, int gmax[4], int* z_split_choice, int* z_split_rule, int* y_split_choice,
                   int y_split_rule[2]) {
    for (int k = 0; k < 4; k++) gmax[k] = 0;
    *z_split_choice = 0;
    *z_split_rule = 0;
    *y_split_choice = 0;
    y_split_rule[0] = Y_SPLIT_RULE[0];
    y_split_rule[1] = Y_SPLIT_RULE[1];
    if (P.nz == 1) {
        gmax[0] = pick_groups(3 * P.TX, P.py, P.NT, COL_MAX_THREADS, COL_SMEM_CAP);
        return;
    }
    for (int part = 1; part <= 3; part += 2) {
        bool three = P.py <= 1024 ? reg_threads(P.py, 3 * P.TX) <= 512 && (size_t)P.py * 3 * P.TX * 8 <= COL_SMEM_CAP
                                  : fft_fits(3 * P.TX, P.py) && (size_t)P.py * 3 * P.TX * 8 <= COL_SMEM_CAP;
        int nc = three ? 3 : 1;
        gmax[part] = pick_groups(nc * P.TX, P.py, P.NT, COL_MAX_THREADS, COL_SMEM_CAP);
        if (P.py == 2048 && 2 * P.ny <= P.py) {
            const bool t3 = reg_threads(1024, 3 * P.TX) <= 512 && (size_t)1024 * 3 * P.TX * 8 <= 96 * 1024;
            gmax[part] = pick_groups((t3 ? 3 : 1) * P.TX, 1024, P.NT, 512, 96 * 1024);
            // the fixed split kernel (tiles of 8, one component per block)
            // runs at one group per block, the only count this shape allows
            if (P.TX == 8 && !t3 && gmax[part] == 1) *y_split_choice = 1;
        }
    }
    gmax[2] = pick_groups(3 * P.TX, P.pz, P.py, COL_MAX_THREADS, COL_SMEM_CAP);
    if (zconv_applies(P)) {
        gmax[2] = zconv_groups(P);
        if ((P.pz == 32 || P.pz == 16) && (3 * zsplit_groups(P) * P.TX) % 32 == 0) {
            *z_split_choice = 1;
            *z_split_rule = P.pz == 32 ? 1 : 0;
        }
    }
}

int convolution_launches(const Plan& P) { return P.nz == 1 ? 1 : 3; }

// Whether the column passes of a plan fit (at group count 1).
bool col_fits(const Plan& P) {
    const size_t cap = 200 * 1024;
    auto fits = [&](int ncomp, int L) {
        size_t sm = (size_t)L * ncomp * P.TX * 8;
        if (sm > cap) return false;
        return L <= 1024 ? reg_threads(L, ncomp * P.TX) <= 512 : fft_fits(ncomp * P.TX, L);
    };
    if (P.nz == 1) return fits(3, P.py);
    return fits(1, P.py) && fits(3, P.pz);
}

cudaError_t col_init() {
    cudaError_t e;
    if ((e = upload_tw32()) != cudaSuccess) return e;
    const int lim = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_col_gen<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_col_gen<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) return e;
#define MMCQ_SET(Pv, Wv)                                                                                 \
    if ((e = cudaFuncSetAttribute(k_col_reg<Pv, Wv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != \
        cudaSuccess)                                                                                        \
        return e;
    MMCQ_SET(1, 0) MMCQ_SET(2, 0) MMCQ_SET(4, 0) MMCQ_SET(8, 0) MMCQ_SET(16, 0) MMCQ_SET(32, 0) MMCQ_SET(64, 0)
    MMCQ_SET(128, 0) MMCQ_SET(256, 0) MMCQ_SET(512, 0) MMCQ_SET(1024, 0)
    MMCQ_SET(64, 24) MMCQ_SET(128, 24) MMCQ_SET(256, 24) MMCQ_SET(512, 24)
#undef MMCQ_SET
#define MMCQ_SET(Pv)                                                                                            \
    if ((e = cudaFuncSetAttribute(k_zconv<Pv>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) \
        return e;
    MMCQ_SET(2) MMCQ_SET(4) MMCQ_SET(8) MMCQ_SET(16) MMCQ_SET(32)
#undef MMCQ_SET
    if ((e = cudaFuncSetAttribute(k_zconv2<32, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_zconv2<32, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_col_split<1024, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_col_split<1024, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_col_split<1024, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  lim)) != cudaSuccess)
        return e;

    if ((e = cudaFuncSetAttribute(k_zconv2<16, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_zconv2<16, 8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_zconv2<32, 0, 0>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_zconv2<32, 8, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

}  // namespace mq
