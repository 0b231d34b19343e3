// Internal types shared by the host side and the kernels of the mmcq library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mq {

constexpr int MAX_STAGES = 7;
constexpr int MAX_MODES = 4;      // cavity modes (mode 0: the paper's single mode)
constexpr int MAX_SLOTS = 4;      // 4-value FFT slots held per thread per stage
constexpr int MAX_THREADS = 1024;
constexpr int XINV_THREADS = 768;  // register budget of the torque kernel (85 per thread)

enum Kind { KIND_RK4 = 0, KIND_DP45 = 1 };
enum CavMode { CAV_E = 0, CAV_P = 1 };
enum Flag { FLAG_NAN = 1, FLAG_DT_UNDERFLOW = 2, FLAG_HIST_FULL = 4, FLAG_TIMEOUT = 8 };

// A TMA tensor map (the driver's 128-byte CUtensorMap, opaque here), passed to
// kernels by value as a __grid_constant__ parameter.
struct alignas(64) TensorMap {
    unsigned long long v[16];
};

// The tensor map of a handle's x-half-spectrum (4-D: 3 TX values of a tile
// row, y, tile, plane), encoded on the host for the spectrum at `base`.
struct SpecMap {
    TensorMap map;
    const void* base;
    bool valid;
};

// x / d for 0 <= x < 2^31 by multiply-high (Granlund & Montgomery 1994):
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, q = (mulhi(x, m) + x) >> s.
struct FastDiv {
    unsigned d, m, s;
};

inline FastDiv make_fastdiv(unsigned d) {
    unsigned s = 0;
    while ((1ull << s) < d) s++;
    unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
    return FastDiv{d, (unsigned)m, s};
}

#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv& f) { return (__umulhi(x, f.m) + x) >> f.s; }
#endif

// Shape of one handle: grid, padding and the spectrum tiling.
struct Plan {
    int nx, ny, nz, B;
    long long N;      // cells per instance
    int px, py, pz;   // padded FFT sizes (px >= 2)
    int L;            // px / 2: length of the packed complex FFT along x
    int hx;           // px / 2 + 1 half-spectrum columns
    int TX;           // kx columns per tile
    int NT;           // tiles per row, NT * TX >= hx
    int hyk, hzk;     // stored kernel extent along ky, kz: py/2 + 1, pz/2 + 1
    int nrows;        // ny * nz rows per instance
    int R;            // x rows per block in the x passes
    int nblk;         // x-pass blocks per instance: ceil(nrows / R)
    int lt;           // log2(TX)
    FastDiv fd_nx, fd_ny, fd_nz, fd_L1, fd_half;   // divisions by nx, ny, nz, L + 1, L / 2 + 1
    int twn;          // twiddle table length (power of two >= every FFT length)
};

// Constants of the material shared by every instance.
struct Material {
    float exch[3];    // 2 A / d_a^2 for a = x, y, z (divided by Ms_i per cell)
    float two_ku;     // 2 Ku
    float u[3];       // anisotropy axis (unit)
    float pre;        // -gamma / (1 + alpha^2)
    float alpha;
    double vc;        // cell volume
    double hbar;
};

// Per-instance parameters (set from the host).
struct InstParams {
    double bext[3];
    double wc[MAX_MODES], kappa[MAX_MODES], x0[MAX_MODES], p0[MAX_MODES];
    double brms_scale[MAX_MODES];   // B_rms,k,i = brms_scale[k] * profile_k,i
    double drv_amp, drv_wcut, drv_t0;   // B_ext += drv_amp B_rms,0,i sinc(drv_wcut (t - drv_t0))
    double inv_nmag;     // 1 / number of magnetised cells (spatial average of m)
    int cav_on[MAX_MODES];
    int drv_on;
    int pad_;
};

// Per-instance integrator and cavity state (owned by the device).
struct InstState {
    double t, tcav, dt, t_end;
    double a_re[MAX_MODES], a_im[MAX_MODES];     // alpha_k at the start of the step (E-mode)
    double as_re[MAX_MODES], as_im[MAX_MODES];   // alpha_k of the stage about to be evaluated (E-mode)
    double S[MAX_MODES], C[MAX_MODES];           // P-mode accumulators
    double ka_re[MAX_MODES][MAX_STAGES], ka_im[MAX_MODES][MAX_STAGES];
    double X[MAX_MODES];    // last reduced coupling sums (include V_c)
    double err;             // last error estimate (DP45)
    long long nacc, nrej, nhist;
    long long nmh;          // recorded spatial averages of m
    int mcur;               // which m buffer holds the accepted state
    int k1slot;             // DP45: k buffer holding stage 1 (FSAL)
    int have_k1;            // DP45: stage 1 valid for the current state
    int done;               // reached t_end
    int poison;             // DP45: a stage of the current attempt was not finite
};

// Launch parameters the autotuner may override (0 / -1: the fixed rules).
// None of them changes a data layout, so every choice computes the same thing.
struct Tune {
    int col_g[4];   // groups per block of each column part (2-D, y forward, z, y inverse); 0 = rule
    int z_split;    // pz = 32: 1 the split z kernel, 0 one thread per column; -1 = rule
    int x_pipe;     // L = 1024: 1 the pipelined x inverse, 0 the per-row kernel; -1 = rule
    int y_split[2]; // fixed split y passes (forward, inverse): 1 a half per block, 0 both halves; -1 = rule
};

// Device buffers of one handle.
struct Buffers {
    float4* m[2];     // [B][N] (x, y, z, Ms); m[mcur] is the accepted state
    float4* ms;       // [B][N] stage input
    float4* k[MAX_STAGES];  // [B][N] stage torques (w unused)
    float4* e6;       // [B][N] DP45 partial error vector
    float2* spec;     // [B][nz][NT][ny][3][TX] x-half-spectrum
    float2* spec2;    // [B][nz][NT][py][3][TX] after the y transform (3-D only)
    float* kern;      // [hzk][hyk][NT*TX][6] demag kernel (real, scaled)
    float4* prof[MAX_MODES];  // [N] coupling-profile shape of each mode (or null: uniform +y)
    InstParams* ip;
    InstState* st;
    double* xpart;    // [MAX_MODES][B][x-pass blocks] FP64 partial coupling sums
    float* epart;     // [B][nrows] partial error maxima
    unsigned* counter;  // [B] blocks finished in the current kernel
    double* hist;     // [B][hcap] accepted step lengths
    int hcap;
    double* mpart;    // [B][nrows-blocks][3] FP64 partial sums of m (recording only)
    double* mhist;    // [B][hcap][4] t, <mx>, <my>, <mz> after accepted steps (recording only)
    int* flags;
    const float2* tw; // [twn] exp(-2 pi i k / twn)
    float4* fout;     // [N] field output of eval_field
    double* cpart;    // [B][cpart_n] FP64 block partials of the read-out coupling sum
    int cpart_n;      // blocks per instance of that sum
};

// What one launch of the stage kernels does.
struct StageArgs {
    int kind;      // KIND_RK4 / KIND_DP45
    int stage;     // 0-based stage index
    int mode;      // CAV_E / CAV_P
    int terms;     // field terms (eval_field) or 31
    int field_only;  // eval_field: write the field, no state change
    int inst0;     // first instance of this launch (eval_field: one instance)
    float tol;
    int record;    // record <m> every `record` accepted steps (0: off)
    int nmodes;    // cavity modes in use (highest enabled mode + 1)
};

}  // namespace mq
