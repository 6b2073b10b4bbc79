// tensor_host.cpp -- host set-up of the demagnetising kernel for Eq. 2
// (Sec. II): the Newell tensor of a cell-centred mesh (ref. [24]) and its
// spectrum on the zero-padded FFT grid.
//
// The tensor of two uniformly magnetised cuboid cells at offset (X, Y, Z) is
// -1/(4 pi dx dy dz) times the threefold central second difference (steps
// dx, dy, dz) of Newell's auxiliary function f (diagonal components) or g
// (off-diagonal components), with the arguments permuted per component.
// The second differences cancel catastrophically at large offsets, so f and
// g are tabulated on the node grid in binary128 and differenced separably in
// binary128 before rounding to double once.
//
// The spectrum is real because every component is even or odd along each
// axis: even axes transform with a cosine sum, odd axes with a sine sum and
// a factor -i each (two odd axes give -1).  Only kx in [0, nx], ky in
// [0, Py/2], kz in [0, Pz/2] are stored; the device folds the rest.
#include <cmath>
#include <cstring>
#include <cstdio>
#include <thread>
#include <vector>
#include <algorithm>
#include <functional>

#include "tensor_host.h"

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 quad;
static inline quad q_sqrt(quad v) { return sqrtq(v); }
static inline quad q_asinh(quad v) { return asinhq(v); }
static inline quad q_atan(quad v) { return atanq(v); }
static const quad Q_PI_ = M_PIq;
#else
#include <cfloat>
static_assert(LDBL_MANT_DIG == 113, "binary128 long double required");
typedef long double quad;
static inline quad q_sqrt(quad v) { return sqrtl(v); }
static inline quad q_asinh(quad v) { return asinhl(v); }
static inline quad q_atan(quad v) { return atanl(v); }
static const quad Q_PI_ = 3.141592653589793238462643383279502884L;
#endif

namespace {

// Newell's f(x, y, z): the diagonal-component auxiliary function.
quad aux_f(quad x, quad y, quad z)
{
    const quad xx = x * x, yy = y * y, zz = z * z;
    const quad r2 = xx + yy + zz;
    if (r2 == 0) return 0;
    const quad r = q_sqrt(r2);
    quad acc = r * (2 * xx - yy - zz) / 6;
    const quad sxz = xx + zz, sxy = xx + yy;
    if (sxz != 0) acc += (zz - xx) * y * q_asinh(y / q_sqrt(sxz)) / 2;
    if (sxy != 0) acc += (yy - xx) * z * q_asinh(z / q_sqrt(sxy)) / 2;
    if (x != 0) acc -= x * y * z * q_atan((y * z) / (x * r));
    return acc;
}

// Newell's g(x, y, z): the off-diagonal (xy) auxiliary function.
quad aux_g(quad x, quad y, quad z)
{
    const quad xx = x * x, yy = y * y, zz = z * z;
    const quad r2 = xx + yy + zz;
    if (r2 == 0) return 0;
    const quad r = q_sqrt(r2);
    quad acc = -(x * y * r) / 3;
    if (xx + yy != 0) acc += x * y * z * q_asinh(z / q_sqrt(xx + yy));
    if (yy + zz != 0) acc += y * (3 * zz - yy) * q_asinh(x / q_sqrt(yy + zz)) / 6;
    if (xx + zz != 0) acc += x * (3 * zz - xx) * q_asinh(y / q_sqrt(xx + zz)) / 6;
    if (z != 0) acc -= zz * z * q_atan((x * y) / (z * r)) / 6;
    if (y != 0) acc -= z * yy * q_atan((x * z) / (y * r)) / 2;
    if (x != 0) acc -= z * xx * q_atan((y * z) / (x * r)) / 2;
    return acc;
}

void parallel_for(long n, const std::function<void(long, long)> &body)
{
    unsigned hw = std::thread::hardware_concurrency();
    long nt = std::max(1L, std::min<long>(hw ? hw : 4, 64));
    if (n < 64) nt = 1;
    std::vector<std::thread> th;
    long chunk = (n + nt - 1) / nt;
    for (long t = 0; t < nt; ++t) {
        long lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back(body, lo, hi);
    }
    for (auto &x : th) x.join();
}

// One tensor component for offsets [0,nx) x [0,ny) x [0,nz), layout
// out[(Z*ny + Y)*nx + X].  node(i, j, k) evaluates the auxiliary function at
// the node (i dx, j dy, k dz) with the component's argument permutation;
// par[] = +1/-1 is the parity of that function along each axis.
void component(int nx, int ny, int nz, const int par[3],
               const std::function<quad(int, int, int)> &node, quad scale, double *out)
{
    const long Nx1 = nx + 1, Ny1 = ny + 1, Nz1 = nz + 1;
    std::vector<quad> F((size_t)Nx1 * Ny1 * Nz1);
    parallel_for((long)F.size(), [&](long lo, long hi) {
        for (long t = lo; t < hi; ++t) {
            int i = (int)(t % Nx1), j = (int)((t / Nx1) % Ny1), k = (int)(t / (Nx1 * Ny1));
            F[t] = node(i, j, k);
        }
    });
    // D_x: [X][j][k] for X in [0,nx)
    std::vector<quad> A((size_t)nx * Ny1 * Nz1);
    for (long k = 0; k < Nz1; ++k)
        for (long j = 0; j < Ny1; ++j) {
            const quad *f = &F[(k * Ny1 + j) * Nx1];
            quad *a = &A[(k * Ny1 + j) * nx];
            for (int X = 0; X < nx; ++X) {
                quad lo = X == 0 ? par[0] * f[1] : f[X - 1];
                a[X] = lo - 2 * f[X] + f[X + 1];
            }
        }
    F.clear();
    F.shrink_to_fit();
    // D_y: [X][Y][k] for Y in [0,ny)
    std::vector<quad> B((size_t)nx * ny * Nz1);
    for (long k = 0; k < Nz1; ++k)
        for (int Y = 0; Y < ny; ++Y) {
            const quad *am = Y == 0 ? &A[(k * Ny1 + 1) * nx] : &A[(k * Ny1 + Y - 1) * nx];
            const quad *a0 = &A[(k * Ny1 + Y) * nx];
            const quad *ap = &A[(k * Ny1 + Y + 1) * nx];
            const quad sm = Y == 0 ? (quad)par[1] : (quad)1;
            quad *b = &B[(k * ny + Y) * nx];
            for (int X = 0; X < nx; ++X) b[X] = sm * am[X] - 2 * a0[X] + ap[X];
        }
    A.clear();
    A.shrink_to_fit();
    // D_z and scale
    for (int Z = 0; Z < nz; ++Z) {
        const quad *bm = Z == 0 ? &B[(size_t)1 * ny * nx] : &B[(size_t)(Z - 1) * ny * nx];
        const quad *b0 = &B[(size_t)Z * ny * nx];
        const quad *bp = &B[(size_t)(Z + 1) * ny * nx];
        const quad sm = Z == 0 ? (quad)par[2] : (quad)1;
        double *o = out + (size_t)Z * ny * nx;
        for (long t = 0; t < (long)ny * nx; ++t) o[t] = (double)(scale * (sm * bm[t] - 2 * b0[t] + bp[t]));
    }
}

// cos / sin of 2 pi m / P with exact values at multiples of pi/2.
void trig_table(int P, std::vector<double> &c, std::vector<double> &s)
{
    c.assign(P, 0.0);
    s.assign(P, 0.0);
    for (int m = 0; m < P; ++m) {
        int q4 = 4 * m;
        if (q4 % P == 0) {
            int q = (q4 / P) & 3;
            static const double cq[4] = {1, 0, -1, 0}, sq[4] = {0, 1, 0, -1};
            c[m] = cq[q];
            s[m] = sq[q];
        } else {
            long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)m / (long double)P;
            c[m] = (double)cosl(ang);
            s[m] = (double)sinl(ang);
        }
    }
}

// Real transform along one axis of a [outer][n][inner] array:
// even:  y(k) = x(0) + 2 sum_{X>=1} x(X) cos(2 pi k X / P)
// odd:   y(k) = 2 sum_{X>=1} x(X) sin(2 pi k X / P)
// for k in [0, H).
void axis_transform(const std::vector<double> &in, std::vector<double> &out, long outer, int n, long inner,
                    int H, int P, bool odd)
{
    std::vector<double> c, s;
    trig_table(P, c, s);
    out.assign((size_t)outer * H * inner, 0.0);
    parallel_for(outer, [&](long lo, long hi) {
        for (long o = lo; o < hi; ++o)
            for (int k = 0; k < H; ++k) {
                double *y = &out[((size_t)o * H + k) * inner];
                const double *x0 = &in[(size_t)o * n * inner];
                if (!odd)
                    for (long t = 0; t < inner; ++t) y[t] = x0[t];
                for (int X = 1; X < n; ++X) {
                    int m = (int)(((long)k * X) % P);
                    double w = 2.0 * (odd ? s[m] : c[m]);
                    const double *x = x0 + (size_t)X * inner;
                    for (long t = 0; t < inner; ++t) y[t] += w * x[t];
                }
            }
    });
}

} // namespace

extern "C" int mmx_host_tensor(const mmx_host_tensor_args *a, double *N6_out)
{
    const int nx = a->nx, ny = a->ny, nz = a->nz;
    double L = std::max(a->dx, std::max(a->dy, a->dz));
    const quad dx = (quad)a->dx / L, dy = (quad)a->dy / L, dz = (quad)a->dz / L;
    const quad scale = -1 / (4 * Q_PI_ * dx * dy * dz);
    const long n = (long)nx * ny * nz;
    const int even[3] = {1, 1, 1};
    const int pxy[3] = {-1, -1, 1}, pxz[3] = {-1, 1, -1}, pyz[3] = {1, -1, -1};
    component(nx, ny, nz, even, [&](int i, int j, int k) { return aux_f(i * dx, j * dy, k * dz); }, scale, N6_out + 0 * n);
    component(nx, ny, nz, even, [&](int i, int j, int k) { return aux_f(j * dy, i * dx, k * dz); }, scale, N6_out + 1 * n);
    component(nx, ny, nz, even, [&](int i, int j, int k) { return aux_f(k * dz, j * dy, i * dx); }, scale, N6_out + 2 * n);
    component(nx, ny, nz, pxy, [&](int i, int j, int k) { return aux_g(i * dx, j * dy, k * dz); }, scale, N6_out + 3 * n);
    component(nx, ny, nz, pxz, [&](int i, int j, int k) { return aux_g(i * dx, k * dz, j * dy); }, scale, N6_out + 4 * n);
    component(nx, ny, nz, pyz, [&](int i, int j, int k) { return aux_g(j * dy, k * dz, i * dx); }, scale, N6_out + 5 * n);
    return 0;
}

extern "C" int mmx_host_spectrum(const mmx_host_tensor_args *a, const double *N6, double *N00,
                                 double *K_out)
{
    const int nx = a->nx, ny = a->ny, nz = a->nz;
    const int Px = 2 * nx, Py = ny > 1 ? 2 * ny : 1, Pz = nz > 1 ? 2 * nz : 1;
    const int Hx = nx + 1, Hy = Py / 2 + 1, Hz = Pz / 2 + 1;
    const long n = (long)nx * ny * nz;
    const double norm = -a->Ms / ((double)Px * Py * Pz);
    for (int c = 0; c < 3; ++c) N00[c] = N6[c * n];
    // parity per component along (x, y, z): false = even, true = odd
    static const bool odd[6][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int comp = 0; comp < 6; ++comp) {
        std::vector<double> t0(N6 + comp * n, N6 + (comp + 1) * n), t1, t2, t3;
        if (comp < 3) t0[0] = 0.0;  // the self term is added back exactly on the device
        // layout [z][y][x]: x-axis has outer = nz*ny, inner = 1
        axis_transform(t0, t1, (long)nz * ny, nx, 1, Hx, Px, odd[comp][0]);   // -> [z][y][Hx]
        axis_transform(t1, t2, nz, ny, Hx, Hy, Py, odd[comp][1]);             // -> [z][Hy][Hx]
        axis_transform(t2, t3, 1, nz, (long)Hy * Hx, Hz, Pz, odd[comp][2]);   // -> [Hz][Hy][Hx]
        int nodd = odd[comp][0] + odd[comp][1] + odd[comp][2];
        double sgn = nodd == 2 ? -1.0 : 1.0;  // (-i)^2 from two sine transforms
        for (int kz = 0; kz < Hz; ++kz)
            for (int ky = 0; ky < Hy; ++ky)
                for (int kx = 0; kx < Hx; ++kx) {
                    double v = sgn * norm * t3[((size_t)kz * Hy + ky) * Hx + kx];
                    K_out[(((size_t)kx * Hz + kz) * Hy + ky) * 6 + comp] = v;
                }
    }
    return 0;
}
