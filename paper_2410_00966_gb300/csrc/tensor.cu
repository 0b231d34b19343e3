// Demag-kernel set-up on the device, in FP64.
//
// The paper lists B_demag among the effective-field terms (Sec. 2.1) but does
// not describe how Mumax3 builds its kernel.  Here the cell-pair tensor is the
// Newell, Williams & Dunlop (1993) cell-averaged tensor -- the 27-point
// second difference of their f (diagonal) and g (off-diagonal) functions --
// for centre distances up to 16 largest cell edges, and the point-dipole
// tensor V (delta_ab - 3 r_a r_b / r^2) / (4 pi r^3) beyond.  It is laid on the
// zero-padded grid with wrap-around offsets, transformed with an FP64 FFT
// along x, y and z, and stored as FP32 after folding in -mu0 / (px py pz).
// Its real spectrum has the parity of the tensor (xx, yy, zz even; xy odd in
// kx and ky, xz in kx and kz, yz in ky and kz), so only ky <= py/2 and
// kz <= pz/2 are kept; the convolution passes restore the signs.
#include <math.h>

#include "common.cuh"

namespace mq {

__device__ double nf(double x, double y, double z) {
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    if (x2 + z2 > 0.0) r += 0.5 * y * (z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (x2 + y2 > 0.0) r += 0.5 * z * (y2 - x2) * asinh(z / sqrt(x2 + y2));
    if (x > 0.0 && R > 0.0) r -= x * y * z * atan(y * z / (x * R));
    r += (2.0 * x2 - y2 - z2) * R / 6.0;
    return r;
}

__device__ double ng(double x, double y, double z) {
    double sg = 1.0;
    if (x < 0.0) { sg = -sg; x = -x; }
    if (y < 0.0) { sg = -sg; y = -y; }
    z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    if (x2 + y2 > 0.0) r += x * y * z * asinh(z / sqrt(x2 + y2));
    if (y2 + z2 > 0.0) r += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2));
    if (x2 + z2 > 0.0) r += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (z > 0.0 && R > 0.0) r -= z2 * z / 6.0 * atan(x * y / (z * R));
    if (y > 0.0 && R > 0.0) r -= z * y2 / 2.0 * atan(x * z / (y * R));
    if (x > 0.0 && R > 0.0) r -= z * x2 / 2.0 * atan(y * z / (x * R));
    r -= x * y * R / 3.0;
    return sg * r;
}

// Component c (0..5 = xx, yy, zz, xy, xz, yz) of the tensor at offset (X,Y,Z).
__device__ double tensor_component(int c, double X, double Y, double Z, double dx, double dy, double dz) {
    const double PI = 3.14159265358979323846;
    double h = fmax(dx, fmax(dy, dz));
    double r2 = X * X + Y * Y + Z * Z;
    if (r2 > 256.0 * h * h) {   // beyond 16 cell edges: point dipole
        double r = sqrt(r2);
        double pre = dx * dy * dz / (4.0 * PI * r2 * r);
        switch (c) {
            case 0: return pre * (1.0 - 3.0 * X * X / r2);
            case 1: return pre * (1.0 - 3.0 * Y * Y / r2);
            case 2: return pre * (1.0 - 3.0 * Z * Z / r2);
            case 3: return -pre * 3.0 * X * Y / r2;
            case 4: return -pre * 3.0 * X * Z / r2;
            default: return -pre * 3.0 * Y * Z / r2;
        }
    }
    double acc = 0.0;
    for (int i = -1; i <= 1; i++)
        for (int j = -1; j <= 1; j++)
            for (int k = -1; k <= 1; k++) {
                double w = (double)((i == 0 ? 2 : -1) * (j == 0 ? 2 : -1) * (k == 0 ? 2 : -1));
                double x = X + i * dx, y = Y + j * dy, z = Z + k * dz;
                double v;
                switch (c) {
                    case 0: v = nf(x, y, z); break;
                    case 1: v = nf(y, x, z); break;
                    case 2: v = nf(z, y, x); break;
                    case 3: v = ng(x, y, z); break;
                    case 4: v = ng(x, z, y); break;
                    default: v = ng(y, z, x); break;
                }
                acc += w * v;
            }
    return acc / (4.0 * PI * dx * dy * dz);
}

struct TensorGeom {
    int nx, ny, nz, px, py, pz;
    double dx, dy, dz;
};

// Fill the padded real-space tensor component c (complex FP64, imaginary 0).
__global__ void k_tensor_fill(double2* R, int c, TensorGeom g) {
    long long P = (long long)g.px * g.py * g.pz;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= P) return;
    int i = (int)(idx % g.px);
    int j = (int)((idx / g.px) % g.py);
    int k = (int)(idx / ((long long)g.px * g.py));
    // index -> offset of the cyclic convolution; unreachable indices stay 0
    int X = i < g.nx ? i : (i > g.px - g.nx ? i - g.px : INT_MIN);
    int Y = j < g.ny ? j : (j > g.py - g.ny ? j - g.py : INT_MIN);
    int Z = k < g.nz ? k : (k > g.pz - g.nz ? k - g.pz : INT_MIN);
    double v = 0.0;
    if (X != INT_MIN && Y != INT_MIN && Z != INT_MIN)
        v = tensor_component(c, X * g.dx, Y * g.dy, Z * g.dz, g.dx, g.dy, g.dz);
    R[idx] = make_double2(v, 0.0);
}

// FP64 radix-2 Stockham FFT of one line per block (length n <= 4096), lines
// of a [z][y][x] array selected by (axis); ping-pong in shared memory.
__global__ void k_fft64_line(double2* a, int axis, int px, int py, int pz, const double2* __restrict__ tw,
                             int twn) {
    extern __shared__ double2 sd[];
    int n = axis == 0 ? px : (axis == 1 ? py : pz);
    long long line = blockIdx.x;
    long long base, stride;
    if (axis == 0) { base = line * px; stride = 1; }
    else if (axis == 1) { long long i = line % px, k = line / px; base = k * (long long)px * py + i; stride = px; }
    else { base = line; stride = (long long)px * py; }
    double2* A = sd;
    double2* Bv = sd + n;
    for (int e = threadIdx.x; e < n; e += blockDim.x) A[e] = a[base + e * stride];
    __syncthreads();
    for (int Ns = 1; Ns < n; Ns *= 2) {
        for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
            int jm = j & (Ns - 1);
            double2 w = tw[jm * (twn / (2 * Ns))];
            double2 u = A[j], v = A[j + n / 2];
            double2 vw = make_double2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
            int d = (j - jm) * 2 + jm;
            Bv[d] = make_double2(u.x + vw.x, u.y + vw.y);
            Bv[d + Ns] = make_double2(u.x - vw.x, u.y - vw.y);
        }
        __syncthreads();
        double2* t = A; A = Bv; Bv = t;
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) a[base + e * stride] = A[e];
}

// Keep the real part on the mirror-reduced grid, scaled, as FP32.
__global__ void k_tensor_extract(const double2* R, float* kern, int c, int px, int py, int pz, int hx, int hyk,
                                 int hzk, int W, double scale) {
    long long total = (long long)hzk * hyk * W;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int kx = (int)(idx % W);
    int ky = (int)((idx / W) % hyk);
    int kz = (int)(idx / ((long long)W * hyk));
    float v = 0.f;
    if (kx < hx) v = (float)(scale * R[((long long)kz * py + ky) * px + kx].x);
    kern[idx * 6 + c] = v;
}

// Builds the demag kernel of a plan into `kern` ([hzk][hyk][NT*TX][6] floats).
// Needs a scratch of px*py*pz double2; returns the first CUDA error.
cudaError_t build_demag_kernel(const Plan& P, double dx, double dy, double dz, double mu0, float* kern,
                               double2* scratch, cudaStream_t s) {
    TensorGeom g{P.nx, P.ny, P.nz, P.px, P.py, P.pz, dx, dy, dz};
    long long Ptot = (long long)P.px * P.py * P.pz;
    int nmax = P.px > P.py ? P.px : P.py;
    if (P.pz > nmax) nmax = P.pz;
    // FP64 twiddles exp(-2 pi i k / nmax)
    double2* tw = nullptr;
    cudaError_t e = cudaMalloc(&tw, sizeof(double2) * nmax);
    if (e != cudaSuccess) return e;
    {
        double2* h = new double2[nmax];
        for (int k = 0; k < nmax; k++) {
            double ang = -2.0 * 3.14159265358979323846 * k / nmax;
            h[k] = make_double2(cos(ang), sin(ang));
        }
        e = cudaMemcpy(tw, h, sizeof(double2) * nmax, cudaMemcpyHostToDevice);
        delete[] h;
        if (e != cudaSuccess) { cudaFree(tw); return e; }
    }
    cudaFuncSetAttribute(k_fft64_line, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * (int)sizeof(double2));
    const double scale = -mu0 / (double)Ptot;
    const int W = P.NT * P.TX;
    for (int c = 0; c < 6; c++) {
        if (P.nz == 1 && (c == 4 || c == 5)) {   // xz, yz vanish in a single layer
            long long total = (long long)P.hzk * P.hyk * W;
            cudaMemsetAsync(scratch, 0, sizeof(double2) * Ptot, s);
            k_tensor_extract<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(scratch, kern, c, P.px, P.py, P.pz, P.hx,
                                                                          P.hyk, P.hzk, W, scale);
            continue;
        }
        k_tensor_fill<<<(unsigned)((Ptot + 255) / 256), 256, 0, s>>>(scratch, c, g);
        for (int axis = 0; axis < 3; axis++) {
            int n = axis == 0 ? P.px : (axis == 1 ? P.py : P.pz);
            if (n == 1) continue;
            long long nlines = Ptot / n;
            int th = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
            k_fft64_line<<<(unsigned)nlines, th, 2 * n * sizeof(double2), s>>>(scratch, axis, P.px, P.py, P.pz, tw, nmax);
        }
        long long total = (long long)P.hzk * P.hyk * W;
        k_tensor_extract<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(scratch, kern, c, P.px, P.py, P.pz, P.hx,
                                                                      P.hyk, P.hzk, W, scale);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(tw);
    return e != cudaSuccess ? e : e2;
}

}  // namespace mq
