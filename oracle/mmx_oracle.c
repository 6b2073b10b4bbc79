/*
 * mmx_oracle.c -- plain, slow, CPU FP64 oracle for the demag-extrapolated
 * explicit LLG integrator of Lepadatu, "Speeding up explicit numerical
 * evaluation methods for micromagnetic simulations using demagnetizing field
 * polynomial extrapolation" (arXiv 2107.06729).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference legs of bench.py may load this library.  The product
 * path (libmmx) shares no code, header, table or helper with this file.
 *
 * Every routine follows a definition written out literally:
 *   - Newell demag tensor (Sec. II, Eq. 2, tensor formulas of ref. [24],
 *     Newell, Williams & Dunlop, J. Geophys. Res. 98, 9551 (1993)):
 *     27-term second-difference sums of the auxiliary functions f and g,
 *     evaluated in IEEE binary128 and rounded to double once per entry.
 *   - Demag field, Eq. 2: H(r0) = -sum_r N(r - r0) M(r), both as the literal
 *     O(N^2) sum and through the convolution theorem with a textbook
 *     radix-2 complex FFT on a zero-padded grid.
 *   - Effective field (Sec. II: applied, demag, exchange, anisotropy) with
 *     textbook finite-difference micromagnetics (6-point Laplacian with free
 *     (Neumann) boundaries, uniaxial anisotropy, mu0 = 4 pi 1e-7).
 *   - LLG right-hand side, Eq. 1, in its explicit Landau-Lifshitz form.
 *   - Explicit embedded Runge-Kutta step, Eq. 3-4, with Butcher tableaux from
 *     the cited publications (refs. [26]-[31]).
 *   - Step-size controller, Eq. 5, with the paper's constants.
 *   - Demag polynomial extrapolation, Eq. 6, with the explicit self term and
 *     the priming of the first p iterations.
 *   - Normalised mean absolute error, Eq. 7.
 *
 * Readings where the paper is silent or garbled (each also listed in the
 * design notes of the repository):
 *   R1 Eq. 6 sign: the stored field is the non-self part G_i = H_i + N00 M_i
 *      and H(t) = sum_i L_i(t) G_i - N00 M(t), so that the self term -N00 M of
 *      Eq. 2 is what is added back exactly at every sub-step.
 *   R2 Eq. 4 index range: F_1 = F(t0, M0), F_k = F(t0 + a_k h,
 *      M0 + h sum_{l<k} b_kl F_l).
 *   R3 Eq. 5 exponent read as 1/(n+1), n the order of the propagated
 *      solution.
 *   R4 Error norm e: maximum over cells of |m - m_hat| (m = M/Ms).
 *   R5 Renormalisation m <- m/|m| of every cell after each accepted step.
 *   R6 FSAL methods reuse F_s of the previous accepted step as F_1 only
 *      when no extrapolation is used (p < 0); with extrapolation (and while
 *      priming) F_1 is recomputed with the exact stage-1 demag field, which
 *      is also the field stored in the history.
 *   R7 Rejected attempts keep t0, M0 and the exact stage-1 field; the
 *      history of exact fields is not modified.
 *   R8 The last step is clipped to land on t_end; an accepted clipped step
 *      does not change the controller's proposed step.
 *   R9 e > e_max is accepted, and counted as a forced accept, when the step
 *      cannot be reduced: the attempted h or the controller's proposal (the
 *      attempt may be the clipped last step) is at h_min.
 *   R10 The second-order Adams-Bashforth-Moulton method (Sec. II, ref. [32];
 *      the paper gives only its name, order and two evaluations per step) is
 *      read as the variable-step AB2 predictor
 *        P = M_n + h [(1 + w/2) F_n - (w/2) F_{n-1}],  w = h / h_{n-1},
 *      the trapezoidal (AM2) corrector M_{n+1} = M_n + h/2 [F_n + F(t+h, P)],
 *      and e = |M_{n+1} - P| (R4 norm), controller order 2.  The two
 *      evaluations are F_n (stage 1, exact demag) and F(t+h, P) (stage 2,
 *      Eq. 6 at t + h).  The first step after a start uses w = 0 (Euler
 *      predictor); a rejection keeps F_n and F_{n-1}.
 *
 * The integrator works on the unit magnetisation m = M/Ms; fields are A/m.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_ASINH asinhq
#define Q_ATAN atanq
#define Q_SQRT sqrtq
#define Q_PI M_PIq
#else
/* On aarch64 Linux, long double is IEEE binary128. */
_Static_assert(LDBL_MANT_DIG == 113, "oracle needs binary128 long double");
typedef long double qreal;
#define Q_ASINH asinhl
#define Q_ATAN atanl
#define Q_SQRT sqrtl
#define Q_PI 3.141592653589793238462643383279502884L
#endif

#define OM_MU0 (4.0e-7 * M_PI)

/* ------------------------------------------------------------------------ */
/* Newell auxiliary functions (ref. [24]).                                   */
/* Terms whose transcendental argument has a vanishing denominator also     */
/* have a vanishing polynomial prefactor; they are dropped (limit value 0). */
/* ------------------------------------------------------------------------ */
static qreal newell_f(qreal x, qreal y, qreal z)
{
    qreal x2 = x * x, y2 = y * y, z2 = z * z;
    qreal R = Q_SQRT(x2 + y2 + z2);
    if (R == 0) return 0;
    qreal res = (2 * x2 - y2 - z2) * R / 6;
    qreal rxz = Q_SQRT(x2 + z2);
    qreal rxy = Q_SQRT(x2 + y2);
    if (rxz > 0) res += y / 2 * (z2 - x2) * Q_ASINH(y / rxz);
    if (rxy > 0) res += z / 2 * (y2 - x2) * Q_ASINH(z / rxy);
    if (x != 0) res -= x * y * z * Q_ATAN(y * z / (x * R));
    return res;
}

static qreal newell_g(qreal x, qreal y, qreal z)
{
    qreal x2 = x * x, y2 = y * y, z2 = z * z;
    qreal R = Q_SQRT(x2 + y2 + z2);
    if (R == 0) return 0;
    qreal res = -x * y * R / 3;
    qreal rxy = Q_SQRT(x2 + y2);
    qreal ryz = Q_SQRT(y2 + z2);
    qreal rxz = Q_SQRT(x2 + z2);
    if (rxy > 0) res += x * y * z * Q_ASINH(z / rxy);
    if (ryz > 0) res += y / 6 * (3 * z2 - y2) * Q_ASINH(x / ryz);
    if (rxz > 0) res += x / 6 * (3 * z2 - x2) * Q_ASINH(y / rxz);
    if (z != 0) res -= z2 * z / 6 * Q_ATAN(x * y / (z * R));
    if (y != 0) res -= z * y2 / 2 * Q_ATAN(x * z / (y * R));
    if (x != 0) res -= z * x2 / 2 * Q_ATAN(y * z / (x * R));
    return res;
}

/* 27-term second-difference combination: weight (1,-2,1) per axis at
 * offsets (-d, 0, +d), overall -1/(4 pi dx dy dz).  Lengths are scaled by
 * the largest cell edge; the tensor is dimensionless and f, g are
 * homogeneous of degree 3, so the scaling is exact. */
static double newell_combine(qreal (*fn)(qreal, qreal, qreal),
                             qreal X, qreal Y, qreal Z,
                             qreal dx, qreal dy, qreal dz)
{
    static const int w[3] = {1, -2, 1};
    qreal acc = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                qreal v = fn(X + (i - 1) * dx, Y + (j - 1) * dy, Z + (k - 1) * dz);
                acc += (qreal)(w[i] * w[j] * w[k]) * v;
            }
    return (double)(-acc / (4 * Q_PI * dx * dy * dz));
}

/* Newell tensor for the integer cell offset (X, Y, Z) (target minus source,
 * in cells), any sign.  out = {Nxx, Nyy, Nzz, Nxy, Nxz, Nyz}. */
void om_newell_entry(int X, int Y, int Z, double dx_, double dy_, double dz_, double out[6])
{
    double L = dx_;
    if (dy_ > L) L = dy_;
    if (dz_ > L) L = dz_;
    qreal dx = (qreal)dx_ / L, dy = (qreal)dy_ / L, dz = (qreal)dz_ / L;
    qreal x = X * dx, y = Y * dy, z = Z * dz;
    out[0] = newell_combine(newell_f, x, y, z, dx, dy, dz);      /* Nxx */
    out[1] = newell_combine(newell_f, y, x, z, dy, dx, dz);      /* Nyy */
    out[2] = newell_combine(newell_f, z, y, x, dz, dy, dx);      /* Nzz */
    out[3] = newell_combine(newell_g, x, y, z, dx, dy, dz);      /* Nxy */
    out[4] = newell_combine(newell_g, x, z, y, dx, dz, dy);      /* Nxz */
    out[5] = newell_combine(newell_g, y, z, x, dy, dz, dx);      /* Nyz */
}

/* Tensor for all non-negative offsets 0 <= X < nx etc.
 * Layout N6[c][Z][Y][X], c in {xx, yy, zz, xy, xz, yz}. */
void om_newell_octant(int nx, int ny, int nz, double dx, double dy, double dz, double *N6)
{
    long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (long idx = 0; idx < n; idx++) {
        int X = (int)(idx % nx), Y = (int)((idx / nx) % ny), Z = (int)(idx / ((long)nx * ny));
        double e[6];
        om_newell_entry(X, Y, Z, dx, dy, dz, e);
        for (int c = 0; c < 6; c++) N6[c * n + idx] = e[c];
    }
}

/* Signed-offset lookup from the octant table.  Diagonal components are even
 * in every axis; xy is odd in X and Y, xz odd in X and Z, yz odd in Y and Z
 * (the parity of f and g; checked against om_newell_entry in the tests). */
static void tensor_at(const double *N6, int nx, int ny, int nz, int X, int Y, int Z, double T[3][3])
{
    long n = (long)nx * ny * nz;
    int ax = X < 0 ? -X : X, ay = Y < 0 ? -Y : Y, az = Z < 0 ? -Z : Z;
    long i = ((long)az * ny + ay) * nx + ax;
    double sx = X < 0 ? -1.0 : 1.0, sy = Y < 0 ? -1.0 : 1.0, sz = Z < 0 ? -1.0 : 1.0;
    T[0][0] = N6[0 * n + i];
    T[1][1] = N6[1 * n + i];
    T[2][2] = N6[2 * n + i];
    T[0][1] = T[1][0] = sx * sy * N6[3 * n + i];
    T[0][2] = T[2][0] = sx * sz * N6[4 * n + i];
    T[1][2] = T[2][1] = sy * sz * N6[5 * n + i];
}

/* ------------------------------------------------------------------------ */
/* Eq. 2, literal sum.  m is SoA [3][nz][ny][nx] unit vectors, H in A/m.     */
/* ------------------------------------------------------------------------ */
void om_demag_direct(int nx, int ny, int nz, const double *N6, double Ms,
                     const double *m, double *H)
{
    long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long i0 = 0; i0 < n; i0++) {
        int x0 = (int)(i0 % nx), y0 = (int)((i0 / nx) % ny), z0 = (int)(i0 / ((long)nx * ny));
        double h[3] = {0, 0, 0};
        for (long i = 0; i < n; i++) {
            int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
            double T[3][3];
            tensor_at(N6, nx, ny, nz, x - x0, y - y0, z - z0, T);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++)
                    h[a] -= T[a][b] * Ms * m[b * n + i];
        }
        for (int a = 0; a < 3; a++) H[a * n + i0] = h[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Textbook iterative radix-2 Cooley-Tukey complex FFT (bit reversal, then  */
/* log2(L) butterfly passes).  sign = -1 forward, +1 inverse (unscaled).    */
/* ------------------------------------------------------------------------ */
static void fft1d(double *re, double *im, int L, int sign)
{
    for (int i = 1, j = 0; i < L; i++) {
        int bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= L; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; k++) {
            double ang = sign * 2.0 * M_PI * k / len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < L; s += len) {
                int a = s + k, b = s + k + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] += tr; im[a] += ti;
            }
        }
    }
}

/* 3D transform of a [Pz][Py][Px] complex array, along each axis in turn. */
static void fft3d(double *re, double *im, int Px, int Py, int Pz, int sign)
{
    int Lmax = Px > Py ? Px : Py;
    if (Pz > Lmax) Lmax = Pz;
    long P = (long)Px * Py * Pz;
    (void)P;
#pragma omp parallel
    {
        double *br = malloc(sizeof(double) * Lmax), *bi = malloc(sizeof(double) * Lmax);
#pragma omp for schedule(static)
        for (long r = 0; r < (long)Py * Pz; r++) {
            for (int x = 0; x < Px; x++) { br[x] = re[r * Px + x]; bi[x] = im[r * Px + x]; }
            fft1d(br, bi, Px, sign);
            for (int x = 0; x < Px; x++) { re[r * Px + x] = br[x]; im[r * Px + x] = bi[x]; }
        }
#pragma omp for schedule(static)
        for (long r = 0; r < (long)Px * Pz; r++) {
            long x = r % Px, z = r / Px;
            for (int y = 0; y < Py; y++) { long i = (z * Py + y) * Px + x; br[y] = re[i]; bi[y] = im[i]; }
            fft1d(br, bi, Py, sign);
            for (int y = 0; y < Py; y++) { long i = (z * Py + y) * Px + x; re[i] = br[y]; im[i] = bi[y]; }
        }
#pragma omp for schedule(static)
        for (long r = 0; r < (long)Px * Py; r++) {
            for (int z = 0; z < Pz; z++) { long i = (long)z * Px * Py + r; br[z] = re[i]; bi[z] = im[i]; }
            fft1d(br, bi, Pz, sign);
            for (int z = 0; z < Pz; z++) { long i = (long)z * Px * Py + r; re[i] = br[z]; im[i] = bi[z]; }
        }
        free(br); free(bi);
    }
}

static int pad_pow2(int n)
{
    /* smallest power of two >= 2n - 1: a circular convolution of that size
     * equals the linear one for offsets in [-(n-1), n-1]. */
    int need = 2 * n - 1, P = 1;
    while (P < need) P <<= 1;
    return P;
}

/* Spectrum of the full tensor (self term included) on the padded grid:
 * Kre/Kim[6][P], entries placed circularly at (X mod Px, ...). */
typedef struct {
    int nx, ny, nz, Px, Py, Pz;
    double *Kre, *Kim; /* [6][P] */
} om_kernel;

static void kernel_build(om_kernel *K, int nx, int ny, int nz, const double *N6)
{
    K->nx = nx; K->ny = ny; K->nz = nz;
    K->Px = pad_pow2(nx); K->Py = pad_pow2(ny); K->Pz = pad_pow2(nz);
    long P = (long)K->Px * K->Py * K->Pz;
    K->Kre = calloc(6 * P, sizeof(double));
    K->Kim = calloc(6 * P, sizeof(double));
    for (int Z = -(nz - 1); Z <= nz - 1; Z++)
        for (int Y = -(ny - 1); Y <= ny - 1; Y++)
            for (int X = -(nx - 1); X <= nx - 1; X++) {
                double T[3][3];
                tensor_at(N6, nx, ny, nz, X, Y, Z, T);
                long ix = (X + K->Px) % K->Px, iy = (Y + K->Py) % K->Py, iz = (Z + K->Pz) % K->Pz;
                long i = (iz * K->Py + iy) * K->Px + ix;
                K->Kre[0 * P + i] = T[0][0];
                K->Kre[1 * P + i] = T[1][1];
                K->Kre[2 * P + i] = T[2][2];
                K->Kre[3 * P + i] = T[0][1];
                K->Kre[4 * P + i] = T[0][2];
                K->Kre[5 * P + i] = T[1][2];
            }
    for (int c = 0; c < 6; c++) fft3d(K->Kre + c * P, K->Kim + c * P, K->Px, K->Py, K->Pz, -1);
}

static void kernel_free(om_kernel *K)
{
    free(K->Kre); free(K->Kim);
    K->Kre = K->Kim = NULL;
}

/* Eq. 2 through the convolution theorem.  Convolution sum H(r0) = -sum_r
 * N(r0 - r) M(r); N is even under r -> -r, so this is Eq. 2 as printed. */
static void demag_fft_k(const om_kernel *K, double Ms, const double *m, double *H)
{
    int nx = K->nx, ny = K->ny, nz = K->nz, Px = K->Px, Py = K->Py, Pz = K->Pz;
    long n = (long)nx * ny * nz, P = (long)Px * Py * Pz;
    double *Mre = calloc(3 * P, sizeof(double)), *Mim = calloc(3 * P, sizeof(double));
    double *Hre = calloc(3 * P, sizeof(double)), *Him = calloc(3 * P, sizeof(double));
    for (int c = 0; c < 3; c++)
        for (long i = 0; i < n; i++) {
            long x = i % nx, y = (i / nx) % ny, z = i / ((long)nx * ny);
            Mre[c * P + (z * Py + y) * Px + x] = Ms * m[c * n + i];
        }
    for (int c = 0; c < 3; c++) fft3d(Mre + c * P, Mim + c * P, Px, Py, Pz, -1);
    static const int comp[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    for (long k = 0; k < P; k++)
        for (int a = 0; a < 3; a++) {
            double hr = 0, hi = 0;
            for (int b = 0; b < 3; b++) {
                double kr = K->Kre[comp[a][b] * P + k], ki = K->Kim[comp[a][b] * P + k];
                double mr = Mre[b * P + k], mi = Mim[b * P + k];
                hr -= kr * mr - ki * mi;
                hi -= kr * mi + ki * mr;
            }
            Hre[a * P + k] = hr; Him[a * P + k] = hi;
        }
    for (int c = 0; c < 3; c++) fft3d(Hre + c * P, Him + c * P, Px, Py, Pz, +1);
    for (int c = 0; c < 3; c++)
        for (long i = 0; i < n; i++) {
            long x = i % nx, y = (i / nx) % ny, z = i / ((long)nx * ny);
            H[c * n + i] = Hre[c * P + (z * Py + y) * Px + x] / (double)P;
        }
    free(Mre); free(Mim); free(Hre); free(Him);
}

void om_demag_fft(int nx, int ny, int nz, const double *N6, double Ms, const double *m, double *H)
{
    om_kernel K;
    kernel_build(&K, nx, ny, nz, N6);
    demag_fft_k(&K, Ms, m, H);
    kernel_free(&K);
}

/* ------------------------------------------------------------------------ */
/* Effective-field terms other than demag (Sec. II, textbook forms).        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double Ms, A, K, ku[3], alpha, gamma;
    double H0[3], pulse[3], t_on, t_off;
} om_problem;

void om_applied_field(const om_problem *p, double t, double Ha[3])
{
    int on = (t >= p->t_on && t < p->t_off);
    for (int a = 0; a < 3; a++) Ha[a] = p->H0[a] + (on ? p->pulse[a] : 0.0);
}

/* Exchange: H_ex = 2A/(mu0 Ms) * sum_axes (m+ - 2m + m-)/d^2, a missing
 * neighbour replaced by the cell itself (free boundary).  Anisotropy:
 * H_an = 2K/(mu0 Ms) (m.u) u. */
void om_exchange_anisotropy(const om_problem *p, const double *m, double *H)
{
    int nx = p->nx, ny = p->ny, nz = p->nz;
    long n = (long)nx * ny * nz;
    double cex = 2.0 * p->A / (OM_MU0 * p->Ms);
    double can = 2.0 * p->K / (OM_MU0 * p->Ms);
    for (long i = 0; i < n; i++) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        long xm = x > 0 ? i - 1 : i, xp = x < nx - 1 ? i + 1 : i;
        long ym = y > 0 ? i - nx : i, yp = y < ny - 1 ? i + nx : i;
        long zm = z > 0 ? i - (long)nx * ny : i, zp = z < nz - 1 ? i + (long)nx * ny : i;
        double mu = 0;
        for (int a = 0; a < 3; a++) mu += m[a * n + i] * p->ku[a];
        for (int a = 0; a < 3; a++) {
            const double *c = m + a * n;
            double lap = (c[xp] - 2 * c[i] + c[xm]) / (p->dx * p->dx)
                       + (c[yp] - 2 * c[i] + c[ym]) / (p->dy * p->dy)
                       + (c[zp] - 2 * c[i] + c[zm]) / (p->dz * p->dz);
            H[a * n + i] = cex * lap + can * mu * p->ku[a];
        }
    }
}

/* Eq. 1 solved for dM/dt (Landau-Lifshitz form), written for m = M/Ms:
 * dm/dt = -gamma/(1+alpha^2) [ m x H + alpha m x (m x H) ]. */
void om_llg_rhs(long n, double gamma, double alpha, const double *m, const double *H, double *F)
{
    double g = gamma / (1.0 + alpha * alpha);
    for (long i = 0; i < n; i++) {
        double mx = m[i], my = m[n + i], mz = m[2 * n + i];
        double hx = H[i], hy = H[n + i], hz = H[2 * n + i];
        double cx = my * hz - mz * hy, cy = mz * hx - mx * hz, cz = mx * hy - my * hx;
        double dx = my * cz - mz * cy, dy = mz * cx - mx * cz, dz = mx * cy - my * cx;
        F[i] = -g * (cx + alpha * dx);
        F[n + i] = -g * (cy + alpha * dy);
        F[2 * n + i] = -g * (cz + alpha * dz);
    }
}

/* ------------------------------------------------------------------------ */
/* Butcher tableaux (Eq. 3-4) from the cited publications.                  */
/* ------------------------------------------------------------------------ */
#define OM_MAXS 8
typedef struct {
    int s, order, adaptive, fsal;
    double a[OM_MAXS], b[OM_MAXS][OM_MAXS], c[OM_MAXS], chat[OM_MAXS];
} om_tableau;

enum { OM_RK4 = 0, OM_HEUN12, OM_RK23, OM_RKF45, OM_RKCK45, OM_RKDP54, OM_RKF56, OM_ABM2, OM_NMETHODS };

static void set_row(double *dst, int n, const double *src)
{
    for (int i = 0; i < n; i++) dst[i] = src[i];
}

int om_get_tableau(int method, om_tableau *T)
{
    memset(T, 0, sizeof(*T));
    switch (method) {
    case OM_RK4: { /* classical fourth-order Runge-Kutta, ref. [26] */
        T->s = 4; T->order = 4; T->adaptive = 0;
        double a[] = {0, 0.5, 0.5, 1};
        set_row(T->a, 4, a);
        T->b[1][0] = 0.5;
        T->b[2][1] = 0.5;
        T->b[3][2] = 1.0;
        double c[] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
        set_row(T->c, 4, c);
        set_row(T->chat, 4, c);
        return 0; }
    case OM_HEUN12: { /* Heun (order 2) with the Euler (order 1) estimate */
        T->s = 2; T->order = 2; T->adaptive = 1;
        T->a[1] = 1;
        T->b[1][0] = 1;
        T->c[0] = 0.5; T->c[1] = 0.5;
        T->chat[0] = 1; T->chat[1] = 0;
        return 0; }
    case OM_RK23: { /* Bogacki-Shampine 3(2), FSAL, ref. [27] */
        T->s = 4; T->order = 3; T->adaptive = 1; T->fsal = 1;
        double a[] = {0, 0.5, 0.75, 1};
        set_row(T->a, 4, a);
        T->b[1][0] = 0.5;
        T->b[2][1] = 0.75;
        T->b[3][0] = 2.0 / 9; T->b[3][1] = 1.0 / 3; T->b[3][2] = 4.0 / 9;
        double c[] = {2.0 / 9, 1.0 / 3, 4.0 / 9, 0};
        double ch[] = {7.0 / 24, 0.25, 1.0 / 3, 0.125};
        set_row(T->c, 4, c);
        set_row(T->chat, 4, ch);
        return 0; }
    case OM_RKF45: { /* Runge-Kutta-Fehlberg 4(5), ref. [28]; propagates order 4 */
        T->s = 6; T->order = 4; T->adaptive = 1;
        double a[] = {0, 0.25, 3.0 / 8, 12.0 / 13, 1, 0.5};
        set_row(T->a, 6, a);
        T->b[1][0] = 0.25;
        T->b[2][0] = 3.0 / 32; T->b[2][1] = 9.0 / 32;
        T->b[3][0] = 1932.0 / 2197; T->b[3][1] = -7200.0 / 2197; T->b[3][2] = 7296.0 / 2197;
        T->b[4][0] = 439.0 / 216; T->b[4][1] = -8; T->b[4][2] = 3680.0 / 513; T->b[4][3] = -845.0 / 4104;
        T->b[5][0] = -8.0 / 27; T->b[5][1] = 2; T->b[5][2] = -3544.0 / 2565; T->b[5][3] = 1859.0 / 4104;
        T->b[5][4] = -11.0 / 40;
        double c[] = {25.0 / 216, 0, 1408.0 / 2565, 2197.0 / 4104, -0.2, 0};
        double ch[] = {16.0 / 135, 0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55};
        set_row(T->c, 6, c);
        set_row(T->chat, 6, ch);
        return 0; }
    case OM_RKCK45: { /* Cash-Karp, ref. [30]; propagates order 4 */
        T->s = 6; T->order = 4; T->adaptive = 1;
        double a[] = {0, 0.2, 0.3, 0.6, 1, 7.0 / 8};
        set_row(T->a, 6, a);
        T->b[1][0] = 0.2;
        T->b[2][0] = 3.0 / 40; T->b[2][1] = 9.0 / 40;
        T->b[3][0] = 0.3; T->b[3][1] = -0.9; T->b[3][2] = 1.2;
        T->b[4][0] = -11.0 / 54; T->b[4][1] = 2.5; T->b[4][2] = -70.0 / 27; T->b[4][3] = 35.0 / 27;
        T->b[5][0] = 1631.0 / 55296; T->b[5][1] = 175.0 / 512; T->b[5][2] = 575.0 / 13824;
        T->b[5][3] = 44275.0 / 110592; T->b[5][4] = 253.0 / 4096;
        double c[] = {2825.0 / 27648, 0, 18575.0 / 48384, 13525.0 / 55296, 277.0 / 14336, 0.25};
        double ch[] = {37.0 / 378, 0, 250.0 / 621, 125.0 / 594, 0, 512.0 / 1771};
        set_row(T->c, 6, c);
        set_row(T->chat, 6, ch);
        return 0; }
    case OM_RKDP54: { /* Dormand-Prince 5(4), FSAL, ref. [31]; propagates order 5 */
        T->s = 7; T->order = 5; T->adaptive = 1; T->fsal = 1;
        double a[] = {0, 0.2, 0.3, 0.8, 8.0 / 9, 1, 1};
        set_row(T->a, 7, a);
        T->b[1][0] = 0.2;
        T->b[2][0] = 3.0 / 40; T->b[2][1] = 9.0 / 40;
        T->b[3][0] = 44.0 / 45; T->b[3][1] = -56.0 / 15; T->b[3][2] = 32.0 / 9;
        T->b[4][0] = 19372.0 / 6561; T->b[4][1] = -25360.0 / 2187; T->b[4][2] = 64448.0 / 6561;
        T->b[4][3] = -212.0 / 729;
        T->b[5][0] = 9017.0 / 3168; T->b[5][1] = -355.0 / 33; T->b[5][2] = 46732.0 / 5247;
        T->b[5][3] = 49.0 / 176; T->b[5][4] = -5103.0 / 18656;
        T->b[6][0] = 35.0 / 384; T->b[6][1] = 0; T->b[6][2] = 500.0 / 1113; T->b[6][3] = 125.0 / 192;
        T->b[6][4] = -2187.0 / 6784; T->b[6][5] = 11.0 / 84;
        double c[] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
        double ch[] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                       187.0 / 2100, 1.0 / 40};
        set_row(T->c, 7, c);
        set_row(T->chat, 7, ch);
        return 0; }
    case OM_ABM2: { /* Adams-Bashforth-Moulton 2 (R10): not a Runge-Kutta
                     * tableau; only the evaluation times (t0, t0 + h) and the
                     * order are given here, the step is in attempt_step */
        T->s = 2; T->order = 2; T->adaptive = 1;
        T->a[1] = 1;
        return 0; }
    case OM_RKF56: { /* Runge-Kutta-Fehlberg 5(6), ref. [29]; propagates order 5 */
        T->s = 8; T->order = 5; T->adaptive = 1;
        double a[] = {0, 1.0 / 6, 4.0 / 15, 2.0 / 3, 0.8, 1, 0, 1};
        set_row(T->a, 8, a);
        T->b[1][0] = 1.0 / 6;
        T->b[2][0] = 4.0 / 75; T->b[2][1] = 16.0 / 75;
        T->b[3][0] = 5.0 / 6; T->b[3][1] = -8.0 / 3; T->b[3][2] = 2.5;
        T->b[4][0] = -8.0 / 5; T->b[4][1] = 144.0 / 25; T->b[4][2] = -4; T->b[4][3] = 16.0 / 25;
        T->b[5][0] = 361.0 / 320; T->b[5][1] = -18.0 / 5; T->b[5][2] = 407.0 / 128;
        T->b[5][3] = -11.0 / 80; T->b[5][4] = 55.0 / 128;
        T->b[6][0] = -11.0 / 640; T->b[6][1] = 0; T->b[6][2] = 11.0 / 256; T->b[6][3] = -11.0 / 160;
        T->b[6][4] = 11.0 / 256; T->b[6][5] = 0;
        T->b[7][0] = 93.0 / 640; T->b[7][1] = -18.0 / 5; T->b[7][2] = 803.0 / 256;
        T->b[7][3] = -11.0 / 160; T->b[7][4] = 99.0 / 256; T->b[7][5] = 0; T->b[7][6] = 1;
        double c[] = {31.0 / 384, 0, 1125.0 / 2816, 9.0 / 32, 125.0 / 768, 5.0 / 66, 0, 0};
        double ch[] = {7.0 / 1408, 0, 1125.0 / 2816, 9.0 / 32, 125.0 / 768, 0, 5.0 / 66, 5.0 / 66};
        set_row(T->c, 8, c);
        set_row(T->chat, 8, ch);
        return 0; }
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Eq. 6: Lagrange basis at tau over nodes tau_i (times relative to t0).    */
/* ------------------------------------------------------------------------ */
void om_lagrange_weights(int p, const double *tau_nodes, double tau, double *w)
{
    for (int i = 0; i <= p; i++) {
        double L = 1.0;
        for (int j = 0; j <= p; j++)
            if (j != i) L *= (tau - tau_nodes[j]) / (tau_nodes[i] - tau_nodes[j]);
        w[i] = L;
    }
}

/* Eq. 5. */
double om_controller_factor(double e, double e_max, int order, double cmin, double cmax)
{
    if (!(e > 0)) return cmax;
    double c = pow(0.8 * e_max / e, 1.0 / (order + 1));
    if (c < cmin) c = cmin;
    if (c > cmax) c = cmax;
    return c;
}

/* Eq. 7: (1/N) sum_i |m_i - m~_i|  (m = M/Ms). */
double om_epsilon(long n, const double *m, const double *mref)
{
    double s = 0;
    for (long i = 0; i < n; i++) {
        double d0 = m[i] - mref[i], d1 = m[n + i] - mref[n + i], d2 = m[2 * n + i] - mref[2 * n + i];
        s += sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    return s / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Integrator: Eq. 3-6 with the readings R1-R10.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int method;
    int extrap_order; /* p; -1 = full demag at every sub-step */
    int adaptive;     /* 0: fixed h (controller disabled) */
    double h, tol, hmin, hmax, cmin, cmax;
} om_integrator;

typedef struct {
    double t, h;
    long accepted, rejected, exact_evals, extrap_evals, forced;
    double last_err;
} om_stats;

#define OM_MAXP 8

typedef struct {
    om_problem prob;
    om_integrator integ;
    om_tableau T;
    om_kernel K;
    double N00[3];
    long n;
    double *m;           /* current m0 [3n] */
    double *F[OM_MAXS];  /* stage derivatives */
    double *Y, *H, *Hd, *M1, *G;
    double *hist[OM_MAXP + 1];
    double hist_t[OM_MAXP + 1];
    int hist_n;          /* number of stored exact fields (<= p+1) */
    int f1_valid;        /* F[0] already holds F_1 for the current t0 */
    double *Fprev;       /* ABM2: F at the previous accepted step start */
    double h_prev;       /* ABM2: previous accepted step, 0 after a start */
    double t, h_ctrl;
    om_stats st;
} om_sim;

/* Total field for stage input Y at time t with the given demag field. */
static void stage_rhs(om_sim *S, double t, const double *Y, const double *Hdem, double *Fout)
{
    long n = S->n;
    double Ha[3];
    om_applied_field(&S->prob, t, Ha);
    om_exchange_anisotropy(&S->prob, Y, S->H);
    for (int a = 0; a < 3; a++)
        for (long i = 0; i < n; i++) S->H[a * n + i] += Ha[a] + Hdem[a * n + i];
    om_llg_rhs(n, S->prob.gamma, S->prob.alpha, Y, S->H, Fout);
}

void *om_sim_create(const om_problem *prob, const om_integrator *integ, const double *N6, const double *m0)
{
    om_sim *S = calloc(1, sizeof(om_sim));
    S->prob = *prob;
    S->integ = *integ;
    if (om_get_tableau(integ->method, &S->T) != 0) { free(S); return NULL; }
    if (integ->extrap_order > OM_MAXP) { free(S); return NULL; }
    S->n = (long)prob->nx * prob->ny * prob->nz;
    long n = S->n;
    kernel_build(&S->K, prob->nx, prob->ny, prob->nz, N6);
    S->N00[0] = N6[0]; S->N00[1] = N6[n]; S->N00[2] = N6[2 * n];
    S->m = malloc(sizeof(double) * 3 * n);
    memcpy(S->m, m0, sizeof(double) * 3 * n);
    for (int k = 0; k < S->T.s; k++) S->F[k] = calloc(3 * n, sizeof(double));
    S->Y = calloc(3 * n, sizeof(double));
    S->H = calloc(3 * n, sizeof(double));
    S->Hd = calloc(3 * n, sizeof(double));
    S->M1 = calloc(3 * n, sizeof(double));
    S->G = calloc(3 * n, sizeof(double));
    S->Fprev = calloc(3 * n, sizeof(double));
    S->h_prev = 0;
    for (int i = 0; i <= OM_MAXP; i++) S->hist[i] = calloc(3 * n, sizeof(double));
    S->t = 0;
    S->h_ctrl = integ->h;
    return S;
}

void om_sim_destroy(void *handle)
{
    om_sim *S = handle;
    if (!S) return;
    kernel_free(&S->K);
    free(S->m);
    for (int k = 0; k < S->T.s; k++) free(S->F[k]);
    free(S->Y); free(S->H); free(S->Hd); free(S->M1); free(S->G); free(S->Fprev);
    for (int i = 0; i <= OM_MAXP; i++) free(S->hist[i]);
    free(S);
}

void om_sim_get_m(void *handle, double *m) { om_sim *S = handle; memcpy(m, S->m, sizeof(double) * 3 * S->n); }
void om_sim_set_time(void *handle, double t) { ((om_sim *)handle)->t = t; }

void om_sim_get_stats(void *handle, om_stats *st)
{
    om_sim *S = handle;
    *st = S->st;
    st->t = S->t;
    st->h = S->h_ctrl;
}

/* One attempted step of size h from (t, m).  Returns 1 if accepted. */
static int attempt_step(om_sim *S, double h, int *stop_err)
{
    om_tableau *T = &S->T;
    long n = S->n;
    int p = S->integ.extrap_order;
    int s = T->s;
    int extrap = (p >= 0 && S->st.accepted >= p); /* priming: first p accepted steps in full mode */
    double t0 = S->t;
    int k0 = 0;

    /* Stage 1: F_1 = F(t0, m0) with the exact demag field. */
    if (S->f1_valid) {
        k0 = 1;
    } else {
        demag_fft_k(&S->K, S->prob.Ms, S->m, S->Hd);
        S->st.exact_evals++;
        stage_rhs(S, t0, S->m, S->Hd, S->F[0]);
        k0 = 1;
        if (p >= 0) {
            /* push G(t0) = H + N00 M into the history (newest first) */
            for (int i = (S->hist_n < p + 1 ? S->hist_n : p); i > 0; i--) {
                double *tmp = S->hist[i];
                S->hist[i] = S->hist[i - 1];
                S->hist[i - 1] = tmp;
                S->hist_t[i] = S->hist_t[i - 1];
            }
            for (int a = 0; a < 3; a++)
                for (long i = 0; i < n; i++)
                    S->hist[0][a * n + i] = S->Hd[a * n + i] + S->N00[a] * S->prob.Ms * S->m[a * n + i];
            S->hist_t[0] = t0;
            if (S->hist_n < p + 1) S->hist_n++;
        }
        /* F_1 at this t0 stays valid through rejections (R7) */
        S->f1_valid = 1;
    }

    const int abm = (S->integ.method == OM_ABM2);
    for (int k = k0; k < s; k++) {
        if (abm) {
            /* R10: AB2 predictor P = M_n + h [(1 + w/2) F_n - (w/2) F_{n-1}] */
            double w = S->h_prev > 0 ? h / S->h_prev : 0.0;
            for (long i = 0; i < 3 * n; i++)
                S->Y[i] = S->m[i] + h * ((1.0 + 0.5 * w) * S->F[0][i] - 0.5 * w * S->Fprev[i]);
        } else {
            /* Y_k = m0 + h sum_{l<k} b_kl F_l  (Eq. 4, reading R2) */
            for (long i = 0; i < 3 * n; i++) {
                double acc = S->m[i];
                for (int l = 0; l < k; l++) acc += h * T->b[k][l] * S->F[l][i];
                S->Y[i] = acc;
            }
        }
        double tk = t0 + T->a[k] * h;
        if (!extrap) {
            demag_fft_k(&S->K, S->prob.Ms, S->Y, S->Hd);
            S->st.exact_evals++;
        } else {
            /* Eq. 6 with reading R1 */
            double tau_nodes[OM_MAXP + 1], w[OM_MAXP + 1];
            for (int i = 0; i <= p; i++) tau_nodes[i] = S->hist_t[i] - t0;
            om_lagrange_weights(p, tau_nodes, T->a[k] * h, w);
            for (int a = 0; a < 3; a++)
                for (long i = 0; i < n; i++) {
                    double g = 0;
                    for (int j = 0; j <= p; j++) g += w[j] * S->hist[j][a * n + i];
                    S->Hd[a * n + i] = g - S->N00[a] * S->prob.Ms * S->Y[a * n + i];
                }
            S->st.extrap_evals++;
        }
        stage_rhs(S, tk, S->Y, S->Hd, S->F[k]);
    }

    /* Eq. 3: propagated solution and embedded estimate; error norm R4. */
    double e = 0;
    for (long i = 0; i < n; i++) {
        double d2 = 0;
        for (int a = 0; a < 3; a++) {
            double acc = S->m[a * n + i], dd = 0;
            if (abm) {
                /* R10: trapezoidal corrector; e from corrector - predictor */
                long j = a * n + i;
                acc = S->m[j] + 0.5 * h * (S->F[0][j] + S->F[1][j]);
                dd = acc - S->Y[j];
            } else {
                for (int l = 0; l < s; l++) {
                    acc += h * T->c[l] * S->F[l][a * n + i];
                    dd += h * (T->c[l] - T->chat[l]) * S->F[l][a * n + i];
                }
            }
            S->M1[a * n + i] = acc;
            d2 += dd * dd;
        }
        double ei = sqrt(d2);
        if (!(ei <= e)) e = ei; /* NaN propagates */
    }
    S->st.last_err = e;
    if (e != e) { *stop_err = 1; return 0; }

    int accept = 1;
    if (S->integ.adaptive && T->adaptive) {
        if (e > S->integ.tol) {
            /* R9: the step cannot be reduced further */
            if (h <= S->integ.hmin || S->h_ctrl <= S->integ.hmin) S->st.forced++;
            else accept = 0;
        }
    }
    if (!accept) {
        S->st.rejected++;
        return 0;
    }
    /* accept: renormalise (R5); a cell without material (m = 0, reading R11:
     * the vacuum between the particles of an array) has no torque and stays 0 */
    for (long i = 0; i < n; i++) {
        double mx = S->M1[i], my = S->M1[n + i], mz = S->M1[2 * n + i];
        double r = sqrt(mx * mx + my * my + mz * mz);
        if (r == 0.0) {
            S->m[i] = S->m[n + i] = S->m[2 * n + i] = 0.0;
            continue;
        }
        S->m[i] = mx / r; S->m[n + i] = my / r; S->m[2 * n + i] = mz / r;
    }
    S->st.accepted++;
    /* FSAL reuse (R6): only without extrapolation (p < 0), where no exact
     * stage-1 field has to be stored for the history. */
    if (abm) {
        /* R10: F_n becomes F_{n-1} of the next step */
        double *tmp = S->Fprev;
        S->Fprev = S->F[0];
        S->F[0] = tmp;
        S->h_prev = h;
        S->f1_valid = 0;
    } else if (T->fsal && p < 0) {
        double *tmp = S->F[0];
        S->F[0] = S->F[s - 1];
        S->F[s - 1] = tmp;
        S->f1_valid = 1;
    } else {
        S->f1_valid = 0;
    }
    return 1;
}

/* Integrate to t_end.  Returns 0, or -1 on a non-finite error estimate.
 * max_attempts bounds the number of attempted steps (<= 0: unbounded). */
int om_sim_run(void *handle, double t_end, long max_attempts)
{
    om_sim *S = handle;
    long attempts = 0;
    int adaptive = S->integ.adaptive && S->T.adaptive;
    while (S->t < t_end) {
        if (max_attempts > 0 && attempts >= max_attempts) return 1;
        double remaining = t_end - S->t;
        int clipped = 0;
        double h = S->h_ctrl;
        /* R8; a relative slack of 1e-9 absorbs the rounding of t */
        if (h * (1.0 + 1e-9) >= remaining) { h = remaining; clipped = 1; }
        int err = 0;
        int acc = attempt_step(S, h, &err);
        attempts++;
        if (err) return -1;
        double hnew = S->h_ctrl;
        if (adaptive) {
            double c = om_controller_factor(S->st.last_err, S->integ.tol, S->T.order,
                                            S->integ.cmin, S->integ.cmax);
            hnew = h * c;
            if (hnew < S->integ.hmin) hnew = S->integ.hmin;
            if (hnew > S->integ.hmax) hnew = S->integ.hmax;
        }
        if (acc) {
            S->t = clipped ? t_end : S->t + h;
            if (!clipped) S->h_ctrl = hnew; /* R8 */
        } else {
            S->h_ctrl = hnew;
        }
    }
    return 0;
}
