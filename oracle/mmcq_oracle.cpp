// FP64 CPU oracle for the LLG + cavity-QED hot path of Mumax3-cQED
// (arXiv 2410.00966).
//
// TEST INFRASTRUCTURE ONLY.  Only tests, the package smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or constant generator with the CUDA library; every formula is
// written out here from the paper (and from the published demag-tensor and
// Runge-Kutta literature the paper relies on) in plain loops.
//
// What it computes, by paper section / equation:
//   * LLG right-hand side, Eq. (llg) of Sec. 2.1.
//   * Effective field terms listed in Sec. 2.1: Zeeman, demagnetisation,
//     exchange, uniaxial anisotropy (thermal and DMI are out of scope: all
//     runs are at T = 0 and none uses DMI).
//   * Cavity field B_cav = B_rms * Gamma(t), Eq. (bcav) / Eq. (gammafinal),
//     Sec. 2.2, in two forms:
//       E-mode: the photon amplitude alpha is integrated as an ODE state next
//               to m, using the classical equations of motion of Sec. 2.2
//               (Eq. eqmotionspinclasical, Eq. eqmotionaclasical) with the loss
//               substitution omega_c -> omega_c - i kappa.  Integrating alpha
//               out (Appendix A) gives exactly Eq. (gammafinal).
//       P-mode: the paper-literal recursive accumulators S_n, C_n of Sec. 3.1
//               (Eq. Sdiscrete, Eq. Cdiscrete) and Gamma from
//               Eq. (gammadiscretefinal).
//   * Demag tensor: Newell, Williams & Dunlop (1993) cell-averaged tensor,
//     point-dipole form beyond a switch radius (the paper does not describe
//     Mumax3's demag kernel; this is the reading used by both sides).
//   * Integrators: classic RK4 and Dormand-Prince 5(4) (the paper uses
//     Mumax3's unmodified ODE solver, Sec. 3.1).
//   * Appendix C: the excitation amp * B_rms * sinc(omega_cut t) added to
//     B_ext, the spatially averaged m after each accepted step, and the
//     numerical Fourier transform of that average (response spectra).
//
// Parity of this oracle against the real Mumax3-cQED program is unpinned
// (no program output is available); each function is pinned instead by the
// closed forms, invariants and brute-force checks in tests/test_oracle_*.py.
//
// Build: g++ -O2 -fopenmp -shared -fPIC -o liboracle.so mmcq_oracle.cpp

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

static const double OR_PI = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// Demag tensor (Newell et al. 1993).  The paper lists B_demag among the field
// terms (Sec. 2.1) without giving the method.
// ---------------------------------------------------------------------------

// Newell's f(x,y,z); even in every argument.  Written for a generic real type
// so that an extended-precision copy can pin the double one.
template <typename T>
static T newell_f_t(T x, T y, T z) {
    x = std::fabs(x); y = std::fabs(y); z = std::fabs(z);
    T x2 = x * x, y2 = y * y, z2 = z * z;
    T R = std::sqrt(x2 + y2 + z2);
    T r = 0;
    if (x2 + z2 > 0) r += T(0.5) * y * (z2 - x2) * std::asinh(y / std::sqrt(x2 + z2));
    if (x2 + y2 > 0) r += T(0.5) * z * (y2 - x2) * std::asinh(z / std::sqrt(x2 + y2));
    if (x > 0 && R > 0) r -= x * y * z * std::atan(y * z / (x * R));
    r += (T(2) * x2 - y2 - z2) * R / T(6);
    return r;
}

// Newell's g(x,y,z); odd in x and y, even in z.
template <typename T>
static T newell_g_t(T x, T y, T z) {
    T sgn = 1;
    if (x < 0) { sgn = -sgn; x = -x; }
    if (y < 0) { sgn = -sgn; y = -y; }
    z = std::fabs(z);
    T x2 = x * x, y2 = y * y, z2 = z * z;
    T R = std::sqrt(x2 + y2 + z2);
    T r = 0;
    if (x2 + y2 > 0) r += x * y * z * std::asinh(z / std::sqrt(x2 + y2));
    if (y2 + z2 > 0) r += y / T(6) * (T(3) * z2 - y2) * std::asinh(x / std::sqrt(y2 + z2));
    if (x2 + z2 > 0) r += x / T(6) * (T(3) * z2 - x2) * std::asinh(y / std::sqrt(x2 + z2));
    if (z > 0 && R > 0) r -= z2 * z / T(6) * std::atan(x * y / (z * R));
    if (y > 0 && R > 0) r -= z * y2 / T(2) * std::atan(x * z / (y * R));
    if (x > 0 && R > 0) r -= z * x2 / T(2) * std::atan(y * z / (x * R));
    r -= x * y * R / T(3);
    return sgn * r;
}

// Weight of offset e in {-1,0,1} in the 27-point second-difference stencil.
static inline int nw(int e) { return e == 0 ? 2 : -1; }

// Exact Newell tensor between two cells of size dx*dy*dz whose centres differ
// by (X,Y,Z).  out = {Nxx, Nyy, Nzz, Nxy, Nxz, Nyz}.  N is positive-definite
// in the self term (a cube gives 1/3 on the diagonal) and H = -N M.
template <typename T>
static void newell_t(T X, T Y, T Z, T dx, T dy, T dz, T out[6]) {
    T sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    for (int i = -1; i <= 1; i++)
        for (int j = -1; j <= 1; j++)
            for (int k = -1; k <= 1; k++) {
                T w = T(nw(i) * nw(j) * nw(k));
                T x = X + i * dx, y = Y + j * dy, z = Z + k * dz;
                sxx += w * newell_f_t<T>(x, y, z);
                syy += w * newell_f_t<T>(y, x, z);
                szz += w * newell_f_t<T>(z, y, x);
                sxy += w * newell_g_t<T>(x, y, z);
                sxz += w * newell_g_t<T>(x, z, y);
                syz += w * newell_g_t<T>(y, z, x);
            }
    T c = T(1) / (T(4) * T(OR_PI) * dx * dy * dz);
    out[0] = sxx * c; out[1] = syy * c; out[2] = szz * c;
    out[3] = sxy * c; out[4] = sxz * c; out[5] = syz * c;
}

// Point-dipole tensor of a source cell of volume V at offset r:
// N_ab = V/(4 pi r^3) (delta_ab - 3 r_a r_b / r^2).
static void dipole_tensor(double X, double Y, double Z, double V, double out[6]) {
    double r2 = X * X + Y * Y + Z * Z;
    double r = std::sqrt(r2);
    double c = V / (4.0 * OR_PI * r2 * r);
    out[0] = c * (1.0 - 3.0 * X * X / r2);
    out[1] = c * (1.0 - 3.0 * Y * Y / r2);
    out[2] = c * (1.0 - 3.0 * Z * Z / r2);
    out[3] = -c * 3.0 * X * Y / r2;
    out[4] = -c * 3.0 * X * Z / r2;
    out[5] = -c * 3.0 * Y * Z / r2;
}

// Switch radius, in units of the largest cell edge: Newell's closed form is
// used up to and including this distance, the point dipole beyond it.
static const double OR_R_SWITCH = 16.0;

// The demag tensor as the method defines it here.
static void demag_tensor(double X, double Y, double Z, double dx, double dy, double dz,
                         double out[6]) {
    double h = std::fmax(dx, std::fmax(dy, dz));
    double r2 = X * X + Y * Y + Z * Z;
    if (r2 <= (OR_R_SWITCH * h) * (OR_R_SWITCH * h))
        newell_t<double>(X, Y, Z, dx, dy, dz, out);
    else
        dipole_tensor(X, Y, Z, dx * dy * dz, out);
}

// Aharoni (1998) demagnetising factor D_z of a rectangular prism with full
// edges (2a, 2b, 2c) along (x, y, z); an independent closed form that the
// cell-averaged Newell tensor must reproduce.
static double aharoni_dz(double a, double b, double c) {
    double abc = std::sqrt(a * a + b * b + c * c);
    double ab = std::sqrt(a * a + b * b), bc = std::sqrt(b * b + c * c),
           ac = std::sqrt(a * a + c * c);
    double s = 0;
    s += (b * b - c * c) / (2 * b * c) * std::log((abc - a) / (abc + a));
    s += (a * a - c * c) / (2 * a * c) * std::log((abc - b) / (abc + b));
    s += b / (2 * c) * std::log((ab + a) / (ab - a));
    s += a / (2 * c) * std::log((ab + b) / (ab - b));
    s += c / (2 * a) * std::log((bc - b) / (bc + b));
    s += c / (2 * b) * std::log((ac - a) / (ac + a));
    s += 2 * std::atan(a * b / (c * abc));
    s += (a * a * a + b * b * b - 2 * c * c * c) / (3 * a * b * c);
    s += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * abc;
    s += c / (a * b) * (ac + bc);
    s -= (std::pow(ab, 3) + std::pow(bc, 3) + std::pow(ac, 3)) / (3 * a * b * c);
    return s / OR_PI;
}

// ---------------------------------------------------------------------------
// Plain radix-2 complex FFT (FP64), used for the oracle's own zero-padded
// convolution.  sign = -1 forward, +1 inverse (unnormalised).
// ---------------------------------------------------------------------------
// tw[k] = exp(sign * 2 pi i k / n) for k < n/2.
static void fft1d(cplx* a, int n, const cplx* tw) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        int step = n / len;
        for (int k = 0; k < len / 2; k++) {
            cplx w = tw[k * step];
            for (int i = 0; i < n; i += len) {
                cplx u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
        }
    }
}

static std::vector<cplx> twiddles(int n, int sign) {
    std::vector<cplx> tw(n / 2 + 1);
    for (int k = 0; k <= n / 2; k++) {
        double ang = sign * 2.0 * OR_PI * k / n;
        tw[k] = cplx(std::cos(ang), std::sin(ang));
    }
    return tw;
}

// 3-D FFT of an array laid out [z][y][x] with sizes (px, py, pz).
static void fft3d(cplx* a, int px, int py, int pz, int sign) {
    std::vector<cplx> twx = twiddles(px, sign), twy = twiddles(py, sign), twz = twiddles(pz, sign);
#pragma omp parallel if ((long)px * py * pz >= 32768)
    {
        std::vector<cplx> line(std::max(px, std::max(py, pz)));
#pragma omp for collapse(2)
        for (int z = 0; z < pz; z++)
            for (int y = 0; y < py; y++) fft1d(a + ((size_t)z * py + y) * px, px, twx.data());
#pragma omp for collapse(2)
        for (int z = 0; z < pz; z++)
            for (int x = 0; x < px; x++) {
                for (int y = 0; y < py; y++) line[y] = a[((size_t)z * py + y) * px + x];
                fft1d(line.data(), py, twy.data());
                for (int y = 0; y < py; y++) a[((size_t)z * py + y) * px + x] = line[y];
            }
#pragma omp for collapse(2)
        for (int y = 0; y < py; y++)
            for (int x = 0; x < px; x++) {
                for (int z = 0; z < pz; z++) line[z] = a[((size_t)z * py + y) * px + x];
                fft1d(line.data(), pz, twz.data());
                for (int z = 0; z < pz; z++) a[((size_t)z * py + y) * px + x] = line[z];
            }
    }
}

static int pow2_at_least(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// ---------------------------------------------------------------------------
// Simulation state.
// ---------------------------------------------------------------------------
enum { OR_DEMAG_NONE = 0, OR_DEMAG_DIRECT = 1, OR_DEMAG_FFT = 2 };
enum { OR_RK4 = 0, OR_DP45 = 1 };
enum { OR_CAV_E = 0, OR_CAV_P = 1 };
// Cavity modes: mode 0 is the paper's single mode (Sec. 2.2); the paper notes
// that more modes follow the same equations, each with its own B_rms map
// (Sec. 4, multimode remark).  Mode k has its own omega_c, kappa, x0, p0,
// alpha and S, C; the cavity time t_cav is shared.
static const int OR_MAX_MODES = 4;

struct oracle {
    int nx, ny, nz;
    long n;
    double dx, dy, dz, vc;
    double Aex, alpha, Ku, u[3];
    double gamma, mu0, hbar;
    std::vector<double> ms;    // [n]
    std::vector<double> m;     // [n*3]
    double bext[3];
    // cavity modes (Sec. 2.2 / 3.1)
    int cav_on[OR_MAX_MODES];
    double wc[OR_MAX_MODES], kappa[OR_MAX_MODES], x0[OR_MAX_MODES], p0[OR_MAX_MODES];
    std::vector<double> brms[OR_MAX_MODES];  // [n*3] in tesla
    int cav_mode;
    cplx a[OR_MAX_MODES];                    // E-mode photon amplitudes alpha_k
    double S[OR_MAX_MODES], C[OR_MAX_MODES]; // P-mode accumulators (include V_c)
    double t, tcav;
    // excitation of Appendix C: B_ext += amp B_rms,i sinc(omega_cut (t - t0))
    int drv_on;
    double drv_amp, drv_wcut, drv_t0;
    // spatially averaged m after each accepted step: (t, <mx>, <my>, <mz>)
    int record;
    std::vector<double> mavg;
    // integrator
    int kind; double tol, dt_next;
    long n_acc, n_rej;
    std::vector<double> dt_hist;
    // demag
    int demag;
    int px, py, pz;
    std::vector<double> Nreal;   // direct: [(2nz-1)(2ny-1)(2nx-1)][6]
    std::vector<cplx> Nhat;      // fft: [6][pz*py*px]
};

static inline long cidx(const oracle* o, int x, int y, int z) {
    return ((long)z * o->ny + y) * o->nx + x;
}

// Demag field B_demag,i = -mu0 sum_j N(r_i - r_j) Ms_j m_j  (Sec. 2.1 term
// list), by the plain O(N^2) sum.
static void demag_direct(const oracle* o, const double* m, double* B) {
    int nx = o->nx, ny = o->ny, nz = o->nz;
    int ox = 2 * nx - 1, oy = 2 * ny - 1;
#pragma omp parallel for collapse(3) schedule(static) if (o->n >= 256)
    for (int zi = 0; zi < nz; zi++)
        for (int yi = 0; yi < ny; yi++)
            for (int xi = 0; xi < nx; xi++) {
                double h[3] = {0, 0, 0};
                for (int zj = 0; zj < nz; zj++)
                    for (int yj = 0; yj < ny; yj++)
                        for (int xj = 0; xj < nx; xj++) {
                            long j = cidx(o, xj, yj, zj);
                            double M[3] = {o->ms[j] * m[3 * j], o->ms[j] * m[3 * j + 1],
                                           o->ms[j] * m[3 * j + 2]};
                            long t = (((long)(zi - zj + nz - 1) * oy + (yi - yj + ny - 1)) * ox +
                                      (xi - xj + nx - 1)) * 6;
                            const double* N = &o->Nreal[t];
                            h[0] += N[0] * M[0] + N[3] * M[1] + N[4] * M[2];
                            h[1] += N[3] * M[0] + N[1] * M[1] + N[5] * M[2];
                            h[2] += N[4] * M[0] + N[5] * M[1] + N[2] * M[2];
                        }
                long i = cidx(o, xi, yi, zi);
                B[3 * i] = -o->mu0 * h[0];
                B[3 * i + 1] = -o->mu0 * h[1];
                B[3 * i + 2] = -o->mu0 * h[2];
            }
}

// Same convolution through the oracle's own zero-padded FFT.
static void demag_fft(const oracle* o, const double* m, double* B) {
    int px = o->px, py = o->py, pz = o->pz;
    size_t P = (size_t)px * py * pz;
    std::vector<cplx> Mh(3 * P, cplx(0, 0));
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long i = cidx(o, x, y, z);
                size_t p = ((size_t)z * py + y) * px + x;
                for (int c = 0; c < 3; c++) Mh[c * P + p] = o->ms[i] * m[3 * i + c];
            }
    for (int c = 0; c < 3; c++) fft3d(&Mh[c * P], px, py, pz, -1);
    const cplx *Nxx = &o->Nhat[0], *Nyy = &o->Nhat[P], *Nzz = &o->Nhat[2 * P],
               *Nxy = &o->Nhat[3 * P], *Nxz = &o->Nhat[4 * P], *Nyz = &o->Nhat[5 * P];
    std::vector<cplx> Hh(3 * P);
#pragma omp parallel for if (P >= 32768)
    for (long p = 0; p < (long)P; p++) {
        cplx mx = Mh[p], my = Mh[P + p], mz = Mh[2 * P + p];
        Hh[p] = Nxx[p] * mx + Nxy[p] * my + Nxz[p] * mz;
        Hh[P + p] = Nxy[p] * mx + Nyy[p] * my + Nyz[p] * mz;
        Hh[2 * P + p] = Nxz[p] * mx + Nyz[p] * my + Nzz[p] * mz;
    }
    for (int c = 0; c < 3; c++) fft3d(&Hh[c * P], px, py, pz, +1);
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long i = cidx(o, x, y, z);
                size_t p = ((size_t)z * py + y) * px + x;
                for (int c = 0; c < 3; c++) B[3 * i + c] = -o->mu0 * Hh[c * P + p].real() / (double)P;
            }
}

static void demag_field(const oracle* o, const double* m, double* B) {
    if (o->demag == OR_DEMAG_DIRECT) demag_direct(o, m, B);
    else if (o->demag == OR_DEMAG_FFT) demag_fft(o, m, B);
    else std::memset(B, 0, sizeof(double) * 3 * o->n);
}

// Exchange field (Sec. 2.1 term list): B = 2A/Ms_i sum_j (m_j - m_i)/d_ij^2
// over the six face neighbours that exist and carry magnetisation (free,
// Neumann boundaries).
static void exchange_field(const oracle* o, const double* m, double* B) {
#pragma omp parallel for collapse(3) if (o->n >= 32768)
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long i = cidx(o, x, y, z);
                double h[3] = {0, 0, 0};
                if (o->ms[i] > 0) {
                    const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                                          {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};
                    const double d2[3] = {o->dx * o->dx, o->dy * o->dy, o->dz * o->dz};
                    for (int q = 0; q < 6; q++) {
                        int xn = x + nb[q][0], yn = y + nb[q][1], zn = z + nb[q][2];
                        if (xn < 0 || yn < 0 || zn < 0 || xn >= o->nx || yn >= o->ny || zn >= o->nz)
                            continue;
                        long j = cidx(o, xn, yn, zn);
                        if (o->ms[j] <= 0) continue;
                        for (int c = 0; c < 3; c++) h[c] += (m[3 * j + c] - m[3 * i + c]) / d2[q / 2];
                    }
                    double pre = 2.0 * o->Aex / o->ms[i];
                    for (int c = 0; c < 3; c++) h[c] *= pre;
                }
                for (int c = 0; c < 3; c++) B[3 * i + c] = h[c];
            }
}

// Uniaxial anisotropy (Sec. 2.1 term list): B = 2 Ku / Ms (m.u) u.
static void anis_field(const oracle* o, const double* m, double* B) {
    for (long i = 0; i < o->n; i++) {
        double mu = m[3 * i] * o->u[0] + m[3 * i + 1] * o->u[1] + m[3 * i + 2] * o->u[2];
        double pre = o->ms[i] > 0 ? 2.0 * o->Ku / o->ms[i] * mu : 0.0;
        for (int c = 0; c < 3; c++) B[3 * i + c] = pre * o->u[c];
    }
}

// X_k = V_c sum_i Ms_i m_i . B_rms,k,i  -- the coupling-weighted magnetisation
// that drives cavity mode k (Eq. gammafinal integrand times V_c).
static double cavity_X(const oracle* o, const double* m, int k = 0) {
    const double* b = o->brms[k].data();
    double s = 0;
    for (long i = 0; i < o->n; i++)
        s += o->ms[i] * (m[3 * i] * b[3 * i] + m[3 * i + 1] * b[3 * i + 1] + m[3 * i + 2] * b[3 * i + 2]);
    return o->vc * s;
}

// Gamma_k(t) from the P-mode accumulators, Eq. (gammadiscretefinal), with
// x0 = 2 Re alpha0, p0 = -2 Im alpha0 and S, C already carrying V_c.
static double gamma_P(const oracle* o, int k, double tc) {
    double e = std::exp(-o->kappa[k] * tc);
    return e * std::cos(o->wc[k] * tc) * (o->x0[k] - 2.0 * o->S[k] / o->hbar) -
           e * std::sin(o->wc[k] * tc) * (o->p0[k] - 2.0 * o->C[k] / o->hbar);
}

static bool any_cavity(const oracle* o) {
    for (int k = 0; k < OR_MAX_MODES; k++)
        if (o->cav_on[k]) return true;
    return false;
}

// Total effective field B_eff' = B_ext + B_demag + B_exch + B_anis + B_rms*Gamma
// (Sec. 2.1 term list and Eq. bcav).
static void total_field(const oracle* o, const double* m, const double* Gamma, double* B, double drive = 0.0) {
    std::vector<double> t1(3 * o->n), t2(3 * o->n);
    demag_field(o, m, B);
    exchange_field(o, m, t1.data());
    anis_field(o, m, t2.data());
    for (long i = 0; i < o->n; i++)
        for (int c = 0; c < 3; c++) {
            double b = B[3 * i + c] + t1[3 * i + c] + t2[3 * i + c] + o->bext[c];
            for (int k = 0; k < OR_MAX_MODES; k++)
                if (o->cav_on[k]) b += o->brms[k][3 * i + c] * Gamma[k];
            if (o->ms[i] > 0) b += drive * o->brms[0][3 * i + c];
            B[3 * i + c] = b;
        }
}

// The excitation of Appendix C (the example script adds amp B_rms sin(w t)/(w t)
// to B_ext, with the B_rms map of the cavity mode): the factor
// amp sinc(omega_cut (t - t0)) at simulation time t, with sinc(0) = 1; it
// multiplies the map of mode 0.
static double drive_factor(const oracle* o, double t) {
    if (!o->drv_on) return 0.0;
    double x = o->drv_wcut * (t - o->drv_t0);
    return o->drv_amp * (x == 0.0 ? 1.0 : std::sin(x) / x);
}

// LLG torque, Eq. (llg): dm/dt = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)].
static void llg_rhs(const oracle* o, const double* m, const double* B, double* dm) {
    double pre = -o->gamma / (1.0 + o->alpha * o->alpha);
    for (long i = 0; i < o->n; i++) {
        const double* v = m + 3 * i;
        const double* b = B + 3 * i;
        double mxb[3] = {v[1] * b[2] - v[2] * b[1], v[2] * b[0] - v[0] * b[2], v[0] * b[1] - v[1] * b[0]};
        double mxmxb[3] = {v[1] * mxb[2] - v[2] * mxb[1], v[2] * mxb[0] - v[0] * mxb[2],
                           v[0] * mxb[1] - v[1] * mxb[0]};
        for (int c = 0; c < 3; c++)
            dm[3 * i + c] = o->ms[i] > 0 ? pre * (mxb[c] + o->alpha * mxmxb[c]) : 0.0;
    }
}

// Full right-hand side at cavity time tc.  E-mode: Gamma = 2 Re(alpha) and
// d(alpha)/dt = -(kappa + i omega_c) alpha + i X / hbar (Eq. eqmotionaclasical
// with omega_c -> omega_c - i kappa; the spin operator is S = -Ms m V_c/gamma,
// Sec. 2.1).  P-mode: Gamma from the accumulators, alpha not integrated.
// a, da: one amplitude per mode (OR_MAX_MODES).
static void rhs(const oracle* o, const double* m, const cplx* a, double tc, double* dm, cplx* da,
                double* Xout, double ts = 0.0) {
    double Gamma[OR_MAX_MODES] = {0, 0, 0, 0};
    for (int k = 0; k < OR_MAX_MODES; k++)
        if (o->cav_on[k]) Gamma[k] = (o->cav_mode == OR_CAV_E) ? 2.0 * a[k].real() : gamma_P(o, k, tc);
    std::vector<double> B(3 * o->n);
    total_field(o, m, Gamma, B.data(), drive_factor(o, ts));
    llg_rhs(o, m, B.data(), dm);
    for (int k = 0; k < OR_MAX_MODES; k++) {
        double X = o->cav_on[k] ? cavity_X(o, m, k) : 0.0;
        if (Xout) Xout[k] = X;
        if (da) {
            if (o->cav_on[k] && o->cav_mode == OR_CAV_E)
                da[k] = -cplx(o->kappa[k], o->wc[k]) * a[k] + cplx(0.0, X / o->hbar);
            else
                da[k] = 0;
        }
    }
}

static void normalise(const oracle* o, double* m) {
    for (long i = 0; i < o->n; i++) {
        if (o->ms[i] <= 0) { m[3 * i] = m[3 * i + 1] = m[3 * i + 2] = 0; continue; }
        double r = std::sqrt(m[3 * i] * m[3 * i] + m[3 * i + 1] * m[3 * i + 1] + m[3 * i + 2] * m[3 * i + 2]);
        if (r > 0) for (int c = 0; c < 3; c++) m[3 * i + c] /= r;
    }
}

// P-mode: fold the newly accepted point t_n = t_{n-1} + dt into S and C
// (right-endpoint rectangle rule of Eq. Sdiscrete / Eq. Cdiscrete, S_0 = C_0 = 0,
// nothing is added at t_0).  X is taken at the accepted, renormalised m(t_n).
// Every stage of the following step then sees these S_n, C_n through
// Eq. (gammadiscretefinal) at its own stage time.
static void after_accept(oracle* o, double dt) {
    o->t += dt;
    o->tcav += dt;
    o->n_acc++;
    o->dt_hist.push_back(dt);
    if (o->record) {
        // <m> over the magnetised cells of the accepted, renormalised state
        double sm[3] = {0, 0, 0};
        long nm = 0;
        for (long i = 0; i < o->n; i++) {
            if (o->ms[i] <= 0) continue;
            nm++;
            for (int c = 0; c < 3; c++) sm[c] += o->m[3 * i + c];
        }
        o->mavg.push_back(o->t);
        for (int c = 0; c < 3; c++) o->mavg.push_back(nm ? sm[c] / nm : 0.0);
    }
    for (int k = 0; k < OR_MAX_MODES; k++) {
        if (!o->cav_on[k] || o->cav_mode != OR_CAV_P) continue;
        double X = cavity_X(o, o->m.data(), k);
        double tc = o->tcav;
        double e = std::exp(o->kappa[k] * tc);
        o->S[k] += e * std::sin(o->wc[k] * tc) * X * dt;
        o->C[k] += e * std::cos(o->wc[k] * tc) * X * dt;
    }
}

// Classic RK4 on (m, alpha); m renormalised at the end of the step only.
static void step_rk4(oracle* o, double dt) {
    long n3 = 3 * o->n;
    std::vector<double> k[4], tmp(n3);
    cplx ka[4][OR_MAX_MODES];
    for (int s = 0; s < 4; s++) k[s].resize(n3);
    const double c[4] = {0.0, 0.5, 0.5, 1.0};
    for (int s = 0; s < 4; s++) {
        cplx as[OR_MAX_MODES];
        for (int j = 0; j < OR_MAX_MODES; j++) as[j] = o->a[j];
        if (s == 0) {
            for (long q = 0; q < n3; q++) tmp[q] = o->m[q];
        } else {
            for (long q = 0; q < n3; q++) tmp[q] = o->m[q] + c[s] * dt * k[s - 1][q];
            for (int j = 0; j < OR_MAX_MODES; j++) as[j] = o->a[j] + c[s] * dt * ka[s - 1][j];
        }
        rhs(o, tmp.data(), as, o->tcav + c[s] * dt, k[s].data(), ka[s], nullptr, o->t + c[s] * dt);
    }
    for (long q = 0; q < n3; q++)
        o->m[q] += dt / 6.0 * (k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q]);
    for (int j = 0; j < OR_MAX_MODES; j++)
        o->a[j] += dt / 6.0 * (ka[0][j] + 2.0 * ka[1][j] + 2.0 * ka[2][j] + ka[3][j]);
    normalise(o, o->m.data());
    after_accept(o, dt);
}

// Dormand & Prince (1980) RK5(4) coefficients.
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

// One Dormand-Prince attempt of length dt.  The 5th-order solution is
// renormalised, the 7th stage is evaluated there, and the error is
// max_i |m5_i - m4_i| over cells (m5 before renormalisation).  If force is
// set the step is accepted regardless (replay of a recorded dt sequence).
static int step_dp45(oracle* o, double dt, int force, double* err_out) {
    long n3 = 3 * o->n;
    std::vector<double> k[7], tmp(n3), m5(n3), m4(n3);
    cplx ka[7][OR_MAX_MODES];
    for (int s = 0; s < 7; s++) k[s].resize(n3);
    cplx a5[OR_MAX_MODES];
    for (int j = 0; j < OR_MAX_MODES; j++) a5[j] = o->a[j];
    for (int s = 0; s < 7; s++) {
        cplx as[OR_MAX_MODES];
        for (int j = 0; j < OR_MAX_MODES; j++) as[j] = o->a[j];
        if (s < 6) {
            for (long q = 0; q < n3; q++) {
                double v = o->m[q];
                for (int j = 0; j < s; j++) v += dt * DP_A[s][j] * k[j][q];
                tmp[q] = v;
            }
            for (int j = 0; j < s; j++)
                for (int q = 0; q < OR_MAX_MODES; q++) as[q] += dt * DP_A[s][j] * ka[j][q];
        } else {
            for (long q = 0; q < n3; q++) {
                double v = o->m[q];
                for (int j = 0; j < 6; j++) v += dt * DP_B5[j] * k[j][q];
                m5[q] = v;
                tmp[q] = v;
            }
            normalise(o, tmp.data());
            for (int j = 0; j < 6; j++)
                for (int q = 0; q < OR_MAX_MODES; q++) as[q] += dt * DP_B5[j] * ka[j][q];
            for (int q = 0; q < OR_MAX_MODES; q++) a5[q] = as[q];
        }
        rhs(o, tmp.data(), as, o->tcav + DP_C[s] * dt, k[s].data(), ka[s], nullptr, o->t + DP_C[s] * dt);
    }
    double err = 0;
    for (long i = 0; i < o->n; i++) {
        double e2 = 0;
        for (int c = 0; c < 3; c++) {
            double v4 = o->m[3 * i + c];
            for (int j = 0; j < 7; j++) v4 += dt * DP_B4[j] * k[j][3 * i + c];
            double d = m5[3 * i + c] - v4;
            e2 += d * d;
        }
        err = std::fmax(err, std::sqrt(e2));
    }
    if (err_out) *err_out = err;
    int accept = force || err <= o->tol;
    if (accept) {
        std::vector<double> mn = m5;
        normalise(o, mn.data());
        o->m = mn;
        for (int q = 0; q < OR_MAX_MODES; q++) o->a[q] = a5[q];
        after_accept(o, dt);
    } else {
        o->n_rej++;
    }
    return accept;
}

// Step-size controller for the adaptive integrator.
static double dp_next_dt(double dt, double err, double tol) {
    double f = err > 0 ? 0.9 * std::pow(tol / err, 0.2) : 5.0;
    if (f > 5.0) f = 5.0;
    if (f < 0.2) f = 0.2;
    return dt * f;
}

extern "C" {

// ---- tensor entry points ---------------------------------------------------
void or_newell(double X, double Y, double Z, double dx, double dy, double dz, double* out) {
    newell_t<double>(X, Y, Z, dx, dy, dz, out);
}
void or_newell_ld(double X, double Y, double Z, double dx, double dy, double dz, double* out) {
    long double o[6];
    newell_t<long double>(X, Y, Z, dx, dy, dz, o);
    for (int i = 0; i < 6; i++) out[i] = (double)o[i];
}
void or_dipole(double X, double Y, double Z, double V, double* out) { dipole_tensor(X, Y, Z, V, out); }
void or_demag_tensor(double X, double Y, double Z, double dx, double dy, double dz, double* out) {
    demag_tensor(X, Y, Z, dx, dy, dz, out);
}
double or_r_switch(void) { return OR_R_SWITCH; }
double or_aharoni_dz(double a, double b, double c) { return aharoni_dz(a, b, c); }
void or_fft3d(double* re_im, int px, int py, int pz, int sign) {
    fft3d(reinterpret_cast<cplx*>(re_im), px, py, pz, sign);
}

// ---- simulation handle -----------------------------------------------------
oracle* or_create(int nx, int ny, int nz, double dx, double dy, double dz, double Ms, double Aex,
                  double alpha, double Ku, const double* u, double gamma, double mu0, double hbar,
                  int demag) {
    if (nx < 1 || ny < 1 || nz < 1) return nullptr;
    oracle* o = new oracle();
    o->nx = nx; o->ny = ny; o->nz = nz;
    o->n = (long)nx * ny * nz;
    o->dx = dx; o->dy = dy; o->dz = dz; o->vc = dx * dy * dz;
    o->Aex = Aex; o->alpha = alpha; o->Ku = Ku;
    double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int c = 0; c < 3; c++) o->u[c] = un > 0 ? u[c] / un : 0.0;
    o->gamma = gamma; o->mu0 = mu0; o->hbar = hbar;
    o->ms.assign(o->n, Ms);
    o->m.assign(3 * o->n, 0.0);
    for (long i = 0; i < o->n; i++) o->m[3 * i] = 1.0;
    o->bext[0] = o->bext[1] = o->bext[2] = 0;
    for (int k = 0; k < OR_MAX_MODES; k++) {
        o->cav_on[k] = 0; o->wc[k] = o->kappa[k] = o->x0[k] = o->p0[k] = 0;
        o->brms[k].assign(3 * o->n, 0.0);
        o->a[k] = 0; o->S[k] = o->C[k] = 0;
    }
    o->cav_mode = OR_CAV_E;
    o->t = o->tcav = 0;
    o->drv_on = 0; o->drv_amp = o->drv_wcut = o->drv_t0 = 0;
    o->record = 0;
    o->kind = OR_RK4; o->tol = 1e-6; o->dt_next = 0;
    o->n_acc = o->n_rej = 0;
    o->demag = demag;
    if (demag == OR_DEMAG_DIRECT) {
        int ox = 2 * nx - 1, oy = 2 * ny - 1, oz = 2 * nz - 1;
        o->Nreal.resize((size_t)ox * oy * oz * 6);
#pragma omp parallel for collapse(3) schedule(dynamic)
        for (int k = 0; k < oz; k++)
            for (int j = 0; j < oy; j++)
                for (int i = 0; i < ox; i++)
                    demag_tensor((i - nx + 1) * dx, (j - ny + 1) * dy, (k - nz + 1) * dz, dx, dy, dz,
                                 &o->Nreal[(((size_t)k * oy + j) * ox + i) * 6]);
    } else if (demag == OR_DEMAG_FFT) {
        o->px = pow2_at_least(2 * nx - 1);
        o->py = pow2_at_least(2 * ny - 1);
        o->pz = pow2_at_least(2 * nz - 1);
        size_t P = (size_t)o->px * o->py * o->pz;
        o->Nhat.assign(6 * P, cplx(0, 0));
        // Real-space tensor on the padded grid; index i maps to offset i for
        // i < n and to i - p for i > p - n (wrap-around of the cyclic
        // convolution); other indices are never reached and stay zero.
#pragma omp parallel for collapse(3) schedule(dynamic)
        for (int k = 0; k < o->pz; k++)
            for (int j = 0; j < o->py; j++)
                for (int i = 0; i < o->px; i++) {
                    int X = i < nx ? i : (i > o->px - nx ? i - o->px : 1 << 30);
                    int Y = j < ny ? j : (j > o->py - ny ? j - o->py : 1 << 30);
                    int Z = k < nz ? k : (k > o->pz - nz ? k - o->pz : 1 << 30);
                    if (X == 1 << 30 || Y == 1 << 30 || Z == 1 << 30) continue;
                    double N[6];
                    demag_tensor(X * dx, Y * dy, Z * dz, dx, dy, dz, N);
                    size_t p = ((size_t)k * o->py + j) * o->px + i;
                    for (int c = 0; c < 6; c++) o->Nhat[c * P + p] = N[c];
                }
        for (int c = 0; c < 6; c++) fft3d(&o->Nhat[c * P], o->px, o->py, o->pz, -1);
    }
    return o;
}

void or_destroy(oracle* o) { delete o; }
long or_ncells(const oracle* o) { return o->n; }
void or_pad_sizes(const oracle* o, int* out) { out[0] = o->px; out[1] = o->py; out[2] = o->pz; }

void or_set_ms(oracle* o, const double* ms) {
    for (long i = 0; i < o->n; i++) o->ms[i] = ms[i] > 0 ? ms[i] : 0.0;
    normalise(o, o->m.data());
}
void or_set_m(oracle* o, const double* m) {
    std::memcpy(o->m.data(), m, sizeof(double) * 3 * o->n);
    normalise(o, o->m.data());
}
void or_get_m(const oracle* o, double* m) { std::memcpy(m, o->m.data(), sizeof(double) * 3 * o->n); }
void or_set_bias(oracle* o, const double* B) { for (int c = 0; c < 3; c++) o->bext[c] = B[c]; }

// Every mode starts from alpha_k(0) = (x0_k - i p0_k)/2 with empty
// accumulators at t_cav = 0 (ResetMemoryTerm, Sec. 3.2).
static void reset_memory(oracle* o) {
    o->tcav = 0;
    for (int k = 0; k < OR_MAX_MODES; k++) {
        o->S[k] = o->C[k] = 0;
        o->a[k] = cplx(0.5 * o->x0[k], -0.5 * o->p0[k]);
    }
}

// Cavity mode k set-up (Sec. 3.2 built-ins B_rms, Wc, Kappa; mode 0 is the
// paper's single mode).  With profile_is_brms the profile is B_rms in tesla.
// Otherwise B_rms,i = s * profile_i with s = g sqrt(2 hbar / (gamma V_c sum_i Ms_i)),
// the macrospin relation g = B_rms sqrt(gamma Ms V / (2 hbar)) obtained by
// matching the linearised equations of motion to the normal-phase polariton
// formula (Eq. dickepolaritons with the Dicke mapping of Sec. 4).  A null
// profile means a uniform unit vector along +y.  Configuring a mode restarts
// the cavity memory of every mode.
void or_set_cavity_mode(oracle* o, int k, double wc, double kappa, double g, const double* profile,
                        int profile_is_brms) {
    if (k < 0 || k >= OR_MAX_MODES) return;
    o->cav_on[k] = 1; o->wc[k] = wc; o->kappa[k] = kappa;
    double s = 1.0;
    if (!profile_is_brms) {
        double sm = 0;
        for (long i = 0; i < o->n; i++) sm += o->ms[i];
        s = sm > 0 ? g * std::sqrt(2.0 * o->hbar / (o->gamma * o->vc * sm)) : 0.0;
    }
    for (long i = 0; i < o->n; i++)
        for (int c = 0; c < 3; c++) {
            double p = profile ? profile[3 * i + c] : (c == 1 ? 1.0 : 0.0);
            o->brms[k][3 * i + c] = s * p;
        }
    reset_memory(o);
}
void or_set_cavity(oracle* o, double wc, double kappa, double g, const double* profile, int profile_is_brms) {
    or_set_cavity_mode(o, 0, wc, kappa, g, profile, profile_is_brms);
}
void or_get_brms_mode(const oracle* o, int k, double* out) {
    std::memcpy(out, o->brms[k].data(), sizeof(double) * 3 * o->n);
}
void or_get_brms(const oracle* o, double* out) { or_get_brms_mode(o, 0, out); }
// x0 = 2 Re alpha0, p0 = -2 Im alpha0 (Sec. 3.2 built-ins X0, P0).
void or_set_cavity_init_mode(oracle* o, int k, double x0, double p0) {
    o->x0[k] = x0; o->p0[k] = p0;
    o->a[k] = cplx(0.5 * x0, -0.5 * p0);
}
void or_set_cavity_init(oracle* o, double x0, double p0) { or_set_cavity_init_mode(o, 0, x0, p0); }
// ResetMemoryTerm(): the current state becomes the cavity's t = 0.
void or_reset_cavity(oracle* o) { reset_memory(o); }
void or_disable_cavity(oracle* o) {
    for (int k = 0; k < OR_MAX_MODES; k++) o->cav_on[k] = 0;
}
void or_set_integrator(oracle* o, int kind, double tol, int mode) {
    o->kind = kind; o->tol = tol; o->cav_mode = mode;
}

// RK4: n steps of dt.  DP45: n attempts; dt > 0 sets the next trial step.
long or_step(oracle* o, long n, double dt) {
    long acc = 0;
    if (o->kind == OR_RK4) {
        for (long s = 0; s < n; s++) { step_rk4(o, dt); acc++; }
        return acc;
    }
    if (dt > 0) o->dt_next = dt;
    for (long s = 0; s < n; s++) {
        double err;
        double h = o->dt_next;
        int ok = step_dp45(o, h, 0, &err);
        acc += ok;
        o->dt_next = dp_next_dt(h, err, o->tol);
    }
    return acc;
}
// DP45 replay: accept each given step length in turn (no controller).
void or_replay(oracle* o, const double* dts, long n) {
    for (long s = 0; s < n; s++) step_dp45(o, dts[s], 1, nullptr);
}
double or_last_error(oracle* o, double dt) {
    // error estimate of an attempt of length dt from the current state,
    // without changing the state
    oracle copy = *o;
    double err;
    step_dp45(&copy, dt, 0, &err);
    return err;
}
long or_dt_history(const oracle* o, double* out, long max) {
    long n = (long)o->dt_hist.size();
    if (out) for (long i = 0; i < n && i < max; i++) out[i] = o->dt_hist[i];
    return n;
}

// out = {t, t_cav, Re alpha, Im alpha, |alpha|^2, Gamma, S, C, X, dt_next,
//        n_accepted, n_rejected} of mode k.  In P-mode alpha is reconstructed
// from the accumulators: alpha(t) = e^{-(kappa + i omega_c) t}[alpha0 - S/hbar + i C/hbar]
// (Sec. 2.2, a-posteriori photon amplitude).
void or_get_cavity_mode(const oracle* o, int k, double* out) {
    double X = o->cav_on[k] ? cavity_X(o, o->m.data(), k) : 0.0;
    cplx a = o->a[k];
    double G = 2.0 * a.real();
    if (o->cav_on[k] && o->cav_mode == OR_CAV_P) {
        cplx a0(0.5 * o->x0[k], -0.5 * o->p0[k]);
        a = std::exp(-cplx(o->kappa[k], o->wc[k]) * o->tcav) * (a0 + cplx(-o->S[k] / o->hbar, o->C[k] / o->hbar));
        G = gamma_P(o, k, o->tcav);
    }
    out[6] = o->S[k]; out[7] = o->C[k];
    out[0] = o->t; out[1] = o->tcav; out[2] = a.real(); out[3] = a.imag(); out[4] = std::norm(a);
    out[5] = o->cav_on[k] ? G : 0.0; out[8] = X; out[9] = o->dt_next;
    out[10] = (double)o->n_acc; out[11] = (double)o->n_rej;
}
void or_get_cavity(const oracle* o, double* out) { or_get_cavity_mode(o, 0, out); }

void or_set_alpha(oracle* o, double re, double im) { o->a[0] = cplx(re, im); }
void or_set_alpha_mode(oracle* o, int k, double re, double im) { o->a[k] = cplx(re, im); }

// ---- single evaluations for pins and sampled parity --------------------------
void or_demag(const oracle* o, const double* m, double* B) { demag_field(o, m, B); }
void or_exchange(const oracle* o, const double* m, double* B) { exchange_field(o, m, B); }
void or_anis(const oracle* o, const double* m, double* B) { anis_field(o, m, B); }
// Total field at the current simulation time (the drive, if on, at o->t),
// with Gamma for mode 0 and no field from the other modes.
void or_field(const oracle* o, const double* m, double Gamma, double* B) {
    double G[OR_MAX_MODES] = {Gamma, 0, 0, 0};
    total_field(o, m, G, B, drive_factor(o, o->t));
}
// Same with one Gamma per mode.
void or_field_modes(const oracle* o, const double* m, const double* Gamma, double* B) {
    total_field(o, m, Gamma, B, drive_factor(o, o->t));
}

// Appendix C excitation: B_ext += amp B_rms,i sinc(omega_cut (t - t0)); amp = 0 turns it off.
void or_set_drive(oracle* o, double amp, double wcut, double t0) {
    o->drv_on = amp != 0.0;
    o->drv_amp = amp; o->drv_wcut = wcut; o->drv_t0 = t0;
}
double or_drive_factor(const oracle* o, double t) { return drive_factor(o, t); }

// Record <m> over the magnetised cells after every accepted step.
void or_set_recording(oracle* o, int on) { o->record = on != 0; }
long or_mavg_history(const oracle* o, double* out, long max) {
    long n = (long)(o->mavg.size() / 4);
    long c = n < max ? n : max;
    if (out && c > 0) std::memcpy(out, o->mavg.data(), sizeof(double) * 4 * c);
    return n;
}

// Numerical Fourier transform of a sampled signal y(t_n) (Appendix C: the
// broadband response is the Fourier transform of the spatially averaged m):
//   S(w) = sum_n c_n (y_n - ybar) exp(-i w t_n),
// trapezoid weights c_1 = (t_2 - t_1)/2, c_n = (t_{n+1} - t_{n-1})/2,
// c_N = (t_N - t_{N-1})/2 (any sample spacing), and ybar = sum c_n y_n / sum c_n,
// the time average.  out[2k], out[2k+1] = Re, Im S(w_k).
void or_spectrum(const double* t, const double* y, long n, const double* w, long nw, double* out) {
    std::vector<double> c(n > 0 ? n : 1, 0.0);
    if (n >= 2) {
        c[0] = 0.5 * (t[1] - t[0]);
        c[n - 1] = 0.5 * (t[n - 1] - t[n - 2]);
        for (long q = 1; q + 1 < n; q++) c[q] = 0.5 * (t[q + 1] - t[q - 1]);
    }
    double cs = 0, cy = 0;
    for (long q = 0; q < n; q++) { cs += c[q]; cy += c[q] * y[q]; }
    double ybar = cs > 0 ? cy / cs : 0.0;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nw; k++) {
        double re = 0, im = 0;
        for (long q = 0; q < n; q++) {
            double v = c[q] * (y[q] - ybar);
            re += v * std::cos(w[k] * t[q]);
            im -= v * std::sin(w[k] * t[q]);
        }
        out[2 * k] = re;
        out[2 * k + 1] = im;
    }
}
void or_rhs(const oracle* o, const double* m, double are, double aim, double tc, double* dm,
            double* da) {
    cplx a[OR_MAX_MODES] = {cplx(are, aim), 0, 0, 0}, d[OR_MAX_MODES];
    rhs(o, m, a, tc, dm, d, nullptr);
    da[0] = d[0].real(); da[1] = d[0].imag();
}
// Right-hand side with every mode's amplitude: a, da = OR_MAX_MODES (re, im) pairs.
void or_rhs_modes(const oracle* o, const double* m, const double* a, double tc, double* dm, double* da) {
    cplx aa[OR_MAX_MODES], d[OR_MAX_MODES];
    for (int k = 0; k < OR_MAX_MODES; k++) aa[k] = cplx(a[2 * k], a[2 * k + 1]);
    rhs(o, m, aa, tc, dm, d, nullptr);
    for (int k = 0; k < OR_MAX_MODES; k++) { da[2 * k] = d[k].real(); da[2 * k + 1] = d[k].imag(); }
}
double or_cavity_X(const oracle* o, const double* m) { return cavity_X(o, m, 0); }
double or_cavity_X_mode(const oracle* o, const double* m, int k) { return cavity_X(o, m, k); }
int or_max_modes(void) { return OR_MAX_MODES; }
// Threads of the OpenMP loops (n < 1: all cores); returns the number in use.
int or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

// Demag field at a list of cells by the direct sum, with the tensor evaluated
// on the fly (no table): usable on grids far too large for the O(N^2) table.
void or_demag_at(const oracle* o, const double* m, const long* cells, long nc, double* B) {
#pragma omp parallel for schedule(dynamic)
    for (long q = 0; q < nc; q++) {
        long i = cells[q];
        int xi = (int)(i % o->nx), yi = (int)((i / o->nx) % o->ny), zi = (int)(i / ((long)o->nx * o->ny));
        double h[3] = {0, 0, 0};
        for (int zj = 0; zj < o->nz; zj++)
            for (int yj = 0; yj < o->ny; yj++)
                for (int xj = 0; xj < o->nx; xj++) {
                    long j = cidx(o, xj, yj, zj);
                    if (o->ms[j] <= 0) continue;
                    double N[6];
                    demag_tensor((xi - xj) * o->dx, (yi - yj) * o->dy, (zi - zj) * o->dz, o->dx, o->dy,
                                 o->dz, N);
                    double M[3] = {o->ms[j] * m[3 * j], o->ms[j] * m[3 * j + 1], o->ms[j] * m[3 * j + 2]};
                    h[0] += N[0] * M[0] + N[3] * M[1] + N[4] * M[2];
                    h[1] += N[3] * M[0] + N[1] * M[1] + N[5] * M[2];
                    h[2] += N[4] * M[0] + N[5] * M[1] + N[2] * M[2];
                }
        for (int c = 0; c < 3; c++) B[3 * q + c] = -o->mu0 * h[c];
    }
}

// ---- discrete adjoint of the RK4 path (gradients) -------------------------------
// Vector-Jacobian product of the right-hand side at (m, alpha) of mode 0
// (E-mode): given cotangents u (of dm/dt, per cell) and nu (of d alpha/dt, as
// (re, im)), returns the cotangent of m (gm), of alpha (ga) and the parameter
// cotangents dp = (B_ext x, y, z; eta; omega_c; kappa), eta the scale of the
// B_rms map (B_rms -> eta B_rms, at eta = 1).  Written from Eq. (llg), the
// field terms of Sec. 2.1, Eq. (bcav) and the amplitude equation of Sec. 2.2.
static void rhs_vjp(const oracle* o, const double* m, cplx a, const double* u, const double* nu, double* gm,
                    double* ga, double* dp, double* gms) {
    const long n = o->n;
    const double G = 2.0 * a.real();
    double Gam[OR_MAX_MODES] = {G, 0, 0, 0};
    std::vector<double> B(3 * n), lb(3 * n, 0.0), v(3 * n, 0.0), D(3 * n);
    total_field(o, m, Gam, B.data(), 0.0);
    const double pre = -o->gamma / (1.0 + o->alpha * o->alpha), al = o->alpha;
    const double* br = o->brms[0].data();
    const double lX = nu[1] / o->hbar;      // cotangent of X (f_i = ... + X / hbar)
    double X = 0;
    for (long i = 0; i < n; i++) {
        if (o->ms[i] <= 0) { for (int c = 0; c < 3; c++) gm[3 * i + c] = 0; continue; }
        const double* mi = m + 3 * i;
        const double* bi = &B[3 * i];
        const double* ui = u + 3 * i;
        double mb = mi[0] * bi[0] + mi[1] * bi[1] + mi[2] * bi[2];
        double um = ui[0] * mi[0] + ui[1] * mi[1] + ui[2] * mi[2];
        double ub = ui[0] * bi[0] + ui[1] * bi[1] + ui[2] * bi[2];
        double mm = mi[0] * mi[0] + mi[1] * mi[1] + mi[2] * mi[2];
        double bxu[3] = {bi[1] * ui[2] - bi[2] * ui[1], bi[2] * ui[0] - bi[0] * ui[2], bi[0] * ui[1] - bi[1] * ui[0]};
        double uxm[3] = {ui[1] * mi[2] - ui[2] * mi[1], ui[2] * mi[0] - ui[0] * mi[2], ui[0] * mi[1] - ui[1] * mi[0]};
        for (int c = 0; c < 3; c++) {
            // d/dm of u . [m x B + al m x (m x B)] at fixed B
            gm[3 * i + c] = pre * (bxu[c] + al * (mb * ui[c] + um * bi[c] - 2.0 * ub * mi[c]));
            // d/dB of the same
            lb[3 * i + c] = pre * (uxm[c] + al * (um * mi[c] - mm * ui[c]));
            // X = V_c sum Ms m . B_rms
            gm[3 * i + c] += lX * o->vc * o->ms[i] * br[3 * i + c];
            v[3 * i + c] = lb[3 * i + c] / o->ms[i];
        }
        X += o->vc * o->ms[i] * (mi[0] * br[3 * i] + mi[1] * br[3 * i + 1] + mi[2] * br[3 * i + 2]);
    }
    // field terms are linear in m: demag (symmetric kernel, B = D(Ms m), so the
    // transpose is Ms D(lb)); exchange (B_i = c_i sum_j w_ij (m_j - m_i), c = 2A/Ms,
    // transpose sum_j w_ij (c_j lb_j - c_i lb_i)); anisotropy (symmetric per cell)
    demag_field(o, v.data(), D.data());       // D(Ms * (lb / Ms)) = D(lb)
    const double d2[3] = {o->dx * o->dx, o->dy * o->dy, o->dz * o->dz};
    const int nb6[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int z = 0; z < o->nz; z++)
        for (int y = 0; y < o->ny; y++)
            for (int x = 0; x < o->nx; x++) {
                long i = cidx(o, x, y, z);
                if (o->ms[i] <= 0) continue;
                double ci = 2.0 * o->Aex / o->ms[i];
                for (int q = 0; q < 6; q++) {
                    int xn = x + nb6[q][0], yn = y + nb6[q][1], zn = z + nb6[q][2];
                    if (xn < 0 || yn < 0 || zn < 0 || xn >= o->nx || yn >= o->ny || zn >= o->nz) continue;
                    long j = cidx(o, xn, yn, zn);
                    if (o->ms[j] <= 0) continue;
                    double cj = 2.0 * o->Aex / o->ms[j];
                    for (int c = 0; c < 3; c++) gm[3 * i + c] += (cj * lb[3 * j + c] - ci * lb[3 * i + c]) / d2[q / 2];
                }
                double lu = lb[3 * i] * o->u[0] + lb[3 * i + 1] * o->u[1] + lb[3 * i + 2] * o->u[2];
                for (int c = 0; c < 3; c++)
                    gm[3 * i + c] += o->ms[i] * D[3 * i + c] + 2.0 * o->Ku / o->ms[i] * lu * o->u[c];
            }
    double pb = 0, sb[3] = {0, 0, 0};
    for (long i = 0; i < n; i++)
        for (int c = 0; c < 3; c++) { pb += br[3 * i + c] * lb[3 * i + c]; sb[c] += lb[3 * i + c]; }
    // Ms_i (mask fixed, B_rms map fixed) enters through the demag input Ms m,
    // the 1/Ms_i of exchange and anisotropy, and X:
    // dJ/dMs_i += m_i . D(lb)_i - lb_i . (B_exch,i + B_anis,i) / Ms_i + lX V_c m_i . B_rms,i
    if (gms) {
        std::vector<double> Bx(3 * n), Ba(3 * n);
        exchange_field(o, m, Bx.data());
        anis_field(o, m, Ba.data());
        for (long i = 0; i < n; i++) {
            if (o->ms[i] <= 0) continue;
            double v = 0;
            for (int c = 0; c < 3; c++)
                v += m[3 * i + c] * D[3 * i + c] - lb[3 * i + c] * (Bx[3 * i + c] + Ba[3 * i + c]) / o->ms[i] +
                     lX * o->vc * m[3 * i + c] * br[3 * i + c];
            gms[i] += v;
        }
    }
    const double kap = o->kappa[0], w = o->wc[0];
    // d alpha/dt = -(kappa + i omega) alpha + i X / hbar as a real pair; B_cav = B_rms 2 Re alpha
    ga[0] = -kap * nu[0] - w * nu[1] + 2.0 * pb;
    ga[1] = w * nu[0] - kap * nu[1];
    for (int c = 0; c < 3; c++) dp[c] = sb[c];
    dp[3] = G * pb + lX * X;
    dp[4] = nu[0] * a.imag() - nu[1] * a.real();
    dp[5] = -nu[0] * a.real() - nu[1] * a.imag();
}

// Objective after nsteps RK4 steps of dt from the current state (E-mode,
// cavity mode 0 only, no drive):
//   J = w . <m>(T) + wn |alpha(T)|^2 + wavg (1/W) sum_{n = N-W+1}^{N} |alpha_n|^2,
// the last term the photon number averaged over the last W steps.  Gradient
// by the discrete adjoint of the RK4 map with the per-step renormalisation:
// grad = dJ/d(B_ext x, y, z; eta; omega_c; kappa); if gm0 is given dJ/dm0 (per
// cell), if gms is given dJ/dMs (per cell, mask and B_rms map held fixed).
// The state is left at step nsteps.  Returns J.
double or_adjoint_rk4(oracle* o, long nsteps, double dt, const double* wv, double wn, double wavg, long window,
                      double* grad, double* gm0, double* gms) {
    const long n3 = 3 * o->n;
    std::vector<std::vector<double>> ms_ck((size_t)nsteps + 1);
    std::vector<cplx> a_ck((size_t)nsteps + 1);
    for (long q = 0; q <= nsteps; q++) {
        ms_ck[q] = o->m;
        a_ck[q] = o->a[0];
        if (q < nsteps) step_rk4(o, dt);
    }
    if (window < 1) window = 1;
    if (window > nsteps) window = nsteps;
    long nm = 0;
    double avg[3] = {0, 0, 0};
    for (long i = 0; i < o->n; i++)
        if (o->ms[i] > 0) { nm++; for (int c = 0; c < 3; c++) avg[c] += o->m[3 * i + c]; }
    double J = wn * std::norm(o->a[0]);
    for (int c = 0; c < 3; c++) J += wv[c] * (nm ? avg[c] / nm : 0.0);
    for (long q = nsteps - window + 1; q <= nsteps; q++) J += wavg / window * std::norm(a_ck[q]);
    // terminal cotangents
    std::vector<double> lm(n3, 0.0);
    for (long i = 0; i < o->n; i++)
        if (o->ms[i] > 0) for (int c = 0; c < 3; c++) lm[3 * i + c] = wv[c] / nm;
    double la[2] = {2.0 * wn * o->a[0].real(), 2.0 * wn * o->a[0].imag()};
    for (int c = 0; c < 6; c++) grad[c] = 0;
    if (gms) for (long i = 0; i < o->n; i++) gms[i] = 0;
    const double cc[4] = {0.0, 0.5, 0.5, 1.0}, bb[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    std::vector<double> Y[4], K[4], lk[4], g(n3), mp(n3), lp(n3);
    cplx Ya[4], Ka[4];
    double lka[4][2];
    for (int s = 0; s < 4; s++) { Y[s].resize(n3); K[s].resize(n3); lk[s].resize(n3); }
    for (long q = nsteps - 1; q >= 0; q--) {
        // the averaged photon number sees alpha at step q + 1
        if (q + 1 >= nsteps - window + 1) {
            la[0] += 2.0 * wavg / window * a_ck[q + 1].real();
            la[1] += 2.0 * wavg / window * a_ck[q + 1].imag();
        }
        // recompute the stages of step q from its checkpoint
        const std::vector<double>& m0 = ms_ck[q];
        const cplx a0 = a_ck[q];
        for (int s = 0; s < 4; s++) {
            Ya[s] = a0;
            for (long e = 0; e < n3; e++) Y[s][e] = m0[e];
            if (s > 0) {
                for (long e = 0; e < n3; e++) Y[s][e] += cc[s] * dt * K[s - 1][e];
                Ya[s] += cc[s] * dt * Ka[s - 1];
            }
            cplx aa[OR_MAX_MODES] = {Ya[s], 0, 0, 0}, da[OR_MAX_MODES];
            rhs(o, Y[s].data(), aa, 0.0, K[s].data(), da, nullptr, 0.0);
            Ka[s] = da[0];
        }
        for (long e = 0; e < n3; e++) mp[e] = m0[e] + dt * (bb[0] * K[0][e] + bb[1] * K[1][e] + bb[2] * K[2][e] + bb[3] * K[3][e]);
        // renormalisation m = m'/|m'|: cotangent (lm - (lm.mh) mh) / |m'|
        for (long i = 0; i < o->n; i++) {
            double r = std::sqrt(mp[3 * i] * mp[3 * i] + mp[3 * i + 1] * mp[3 * i + 1] + mp[3 * i + 2] * mp[3 * i + 2]);
            if (o->ms[i] <= 0 || r <= 0) { for (int c = 0; c < 3; c++) lp[3 * i + c] = 0; continue; }
            double h[3] = {mp[3 * i] / r, mp[3 * i + 1] / r, mp[3 * i + 2] / r};
            double d = lm[3 * i] * h[0] + lm[3 * i + 1] * h[1] + lm[3 * i + 2] * h[2];
            for (int c = 0; c < 3; c++) lp[3 * i + c] = (lm[3 * i + c] - d * h[c]) / r;
        }
        // y' = y + dt sum b_s k_s
        for (int s = 0; s < 4; s++) {
            for (long e = 0; e < n3; e++) lk[s][e] = dt * bb[s] * lp[e];
            lka[s][0] = dt * bb[s] * la[0];
            lka[s][1] = dt * bb[s] * la[1];
        }
        std::vector<double> nl(lp);
        double nla[2] = {la[0], la[1]};
        for (int s = 3; s >= 0; s--) {
            double ga[2], dp[6];
            rhs_vjp(o, Y[s].data(), Ya[s], lk[s].data(), lka[s], g.data(), ga, dp, gms);
            for (long e = 0; e < n3; e++) nl[e] += g[e];
            nla[0] += ga[0];
            nla[1] += ga[1];
            if (s > 0) {
                // Y_s = y + c_s dt k_{s-1}
                for (long e = 0; e < n3; e++) lk[s - 1][e] += cc[s] * dt * g[e];
                lka[s - 1][0] += cc[s] * dt * ga[0];
                lka[s - 1][1] += cc[s] * dt * ga[1];
            }
            for (int c = 0; c < 6; c++) grad[c] += dp[c];
        }
        lm.swap(nl);
        la[0] = nla[0];
        la[1] = nla[1];
    }
    if (gm0) std::memcpy(gm0, lm.data(), sizeof(double) * n3);
    return J;
}

// Energy terms (J): {Zeeman, demag, exchange, anisotropy, cavity coupling,
// photon, total}.  The cavity pair is -X_k * 2Re(alpha_k) and
// hbar omega_c,k |alpha_k|^2 summed over the modes, from the Hamiltonian
// Eq. (startH) with S = -Ms m V_c / gamma.
void or_energy(const oracle* o, double* out) {
    long n = o->n;
    std::vector<double> Bd(3 * n), Bx(3 * n);
    demag_field(o, o->m.data(), Bd.data());
    exchange_field(o, o->m.data(), Bx.data());
    double ez = 0, ed = 0, ex = 0, ea = 0;
    for (long i = 0; i < n; i++) {
        const double* v = &o->m[3 * i];
        double w = o->ms[i] * o->vc;
        ez -= w * (v[0] * o->bext[0] + v[1] * o->bext[1] + v[2] * o->bext[2]);
        ed -= 0.5 * w * (v[0] * Bd[3 * i] + v[1] * Bd[3 * i + 1] + v[2] * Bd[3 * i + 2]);
        ex -= 0.5 * w * (v[0] * Bx[3 * i] + v[1] * Bx[3 * i + 1] + v[2] * Bx[3 * i + 2]);
        if (o->ms[i] > 0) {
            double mu = v[0] * o->u[0] + v[1] * o->u[1] + v[2] * o->u[2];
            ea -= o->Ku * o->vc * mu * mu;
        }
    }
    double ec = 0, ep = 0;
    for (int k = 0; k < OR_MAX_MODES; k++) {
        if (!o->cav_on[k]) continue;
        double X = cavity_X(o, o->m.data(), k);
        ec -= X * 2.0 * o->a[k].real();
        ep += o->hbar * o->wc[k] * std::norm(o->a[k]);
    }
    out[0] = ez; out[1] = ed; out[2] = ex; out[3] = ea; out[4] = ec; out[5] = ep;
    out[6] = ez + ed + ex + ea + ec + ep;
}

}  // extern "C"
