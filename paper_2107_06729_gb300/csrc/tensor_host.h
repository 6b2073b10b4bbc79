// tensor_host.h -- host-side set-up of the demag kernel (Eq. 2, Sec. II).
#pragma once

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double Ms;
} mmx_host_tensor_args;

// Newell tensor at offsets [0,nx) x [0,ny) x [0,nz); N6_out[6][nz][ny][nx],
// components {xx, yy, zz, xy, xz, yz}.
int mmx_host_tensor(const mmx_host_tensor_args *a, double *N6_out);

// Spectrum of -Ms N / (Px Py Pz) with the self term N(0) removed, over
// kx in [0, nx], kz in [0, Pz/2], ky in [0, Py/2]:
// K_out[(kx*Hz + kz)*Hy + ky][6].  N00[3] receives the diagonal of N(0).
int mmx_host_spectrum(const mmx_host_tensor_args *a, const double *N6, double *N00, double *K_out);

#ifdef __cplusplus
}
#endif
