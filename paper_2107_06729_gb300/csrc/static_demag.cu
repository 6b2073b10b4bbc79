// static_demag.cu -- mmx_demag_static: one exact demag evaluation (the same
// three FFT kernels as mmx_demag) for callers that cannot allocate device
// memory, for instance code that runs while its stream is being captured
// into a CUDA graph (cudaMalloc is not allowed there) or code inside a
// process whose device memory is owned by another allocator.  It needs no
// context: the tensor spectrum, the twiddle tables and the spectrum scratch
// of the FFT passes live in one file-scope device array of fixed size.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tensor_host.h"

void mmx_set_thread_error(const char *msg);
size_t mmxk_yz_smem_bytes(const mmx_ctx *c);
size_t mmxk_x_smem_bytes(const mmx_ctx *c);

namespace {

// Shared by every call on a device; every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[MMX_STATIC_SCRATCH_BYTES];

struct DeviceSlot {
    unsigned char *base = nullptr;  // device address of g_static_scratch on this device
    bool cached = false;            // tensor spectrum of `key` is resident
    mmx_mesh key{};
    double Ms = 0;
    int prec = -1;
    double N00[3] = {0, 0, 0};
};

constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }

int fail(int code, const char *msg)
{
    mmx_set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" int mmx_demag_static(const mmx_mesh *mesh, double Ms, int precision, const void *m_dev, void *H_dev,
                                void *cuda_stream)
{
    if (!mesh || !m_dev || !H_dev) return fail(MMX_ERR_ARG, "null argument");
    if (!pow2(mesh->nx) || !pow2(mesh->ny) || !pow2(mesh->nz) || mesh->nx < 2)
        return fail(MMX_ERR_ARG, "mesh sizes must be powers of two with nx >= 2");
    if (!(mesh->dx > 0 && mesh->dy > 0 && mesh->dz > 0 && std::isfinite(mesh->dx) && std::isfinite(mesh->dy) &&
          std::isfinite(mesh->dz)))
        return fail(MMX_ERR_ARG, "cell sizes must be > 0");
    if (!(Ms > 0) || !std::isfinite(Ms)) return fail(MMX_ERR_ARG, "Ms must be > 0");
    if (precision != MMX_FP64 && precision != MMX_FP32_MIXED) return fail(MMX_ERR_ARG, "unknown precision");

    // a throw-away description that points into the static array
    mmx_ctx c;
    c.prec = precision;
    c.esz = precision == MMX_FP64 ? 8 : 4;
    c.stream = (cudaStream_t)cuda_stream;
    c.nx = mesh->nx;
    c.ny = mesh->ny;
    c.nz = mesh->nz;
    c.n = (long long)c.nx * c.ny * c.nz;
    c.Px = 2 * c.nx;
    c.Py = c.ny > 1 ? 2 * c.ny : 1;
    c.Pz = c.nz > 1 ? 2 * c.nz : 1;
    c.Hy = c.Py / 2 + 1;
    c.Hz = c.Pz / 2 + 1;
    c.rows = 3LL * c.ny * c.nz;
    c.profiling = false;
    c.launches = 0;
    c.split = false;  // the fused y-z pass only: no room for a second spectrum
    c.nd = 3;
    c.allow_tma = false;  // no device state word to report a bounded wait in
    c.stall_test = false;
    c.xi_tma = c.xi_tma_ok = false;
    c.st = nullptr;
    c.trows = mmxk_default_trows(&c);
    c.Tb = nullptr;
    if (mmxk_yz_smem_bytes(&c) > 227 * 1024 || mmxk_x_smem_bytes(&c) > 227 * 1024 || c.Pz > mmxk_yz_max_pz(&c))
        return fail(MMX_ERR_ARG, "mesh too large for the single-CTA FFT passes");
    const size_t kbytes = align256((size_t)(c.nx + 1) * c.Hz * c.Hy * 6 * c.esz);
    const size_t txb = align256((size_t)c.Px * 2 * c.esz), tyb = align256((size_t)c.Py * 2 * c.esz),
                 tzb = align256((size_t)c.Pz * 2 * c.esz);
    const size_t sbytes = align256((size_t)c.rows * c.nx * 2 * c.esz);
    if (kbytes + txb + tyb + tzb + sbytes > MMX_STATIC_SCRATCH_BYTES)
        return fail(MMX_ERR_ARG, "mesh too large for the 16 MiB static scratch of mmx_demag_static");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(MMX_ERR_CUDA, "cudaGetDevice failed");
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSlot &slot = g_slots[dev];
    if (!slot.base) {
        // once per device, with that device current: the host-side name of the
        // array is not a device address
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(MMX_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        slot.base = (unsigned char *)p;
    }
    c.K = slot.base;
    c.twx = slot.base + kbytes;
    c.twy = slot.base + kbytes + txb;
    c.twz = slot.base + kbytes + txb + tyb;
    c.S = slot.base + kbytes + txb + tyb + tzb;
    // field by field: the struct has padding after nz that callers need not clear
    const bool same = slot.cached && slot.prec == precision && slot.Ms == Ms && slot.key.nx == mesh->nx &&
                      slot.key.ny == mesh->ny && slot.key.nz == mesh->nz && slot.key.dx == mesh->dx &&
                      slot.key.dy == mesh->dy && slot.key.dz == mesh->dz;
    if (!same) {
        // a new description needs a stream synchronisation and a blocking copy,
        // neither of which is allowed while the stream is being captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (c.stream && cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess) {
            cudaGetLastError();
            return fail(MMX_ERR_CUDA, "cudaStreamIsCapturing failed");
        }
        if (cs != cudaStreamCaptureStatusNone)
            return fail(MMX_ERR_ARG, "mmx_demag_static: first call for this mesh, Ms and precision made during "
                                     "stream capture; make it before the capture");
        // tensor spectrum for this mesh (host set-up, then a copy into the array)
        slot.cached = false;
        mmx_host_tensor_args ta{c.nx, c.ny, c.nz, mesh->dx, mesh->dy, mesh->dz, Ms};
        std::vector<double> N6((size_t)6 * c.n);
        mmx_host_tensor(&ta, N6.data());
        std::vector<double> Kspec((size_t)(c.nx + 1) * c.Hz * c.Hy * 6);
        mmx_host_spectrum(&ta, N6.data(), slot.N00, Kspec.data());
        if (c.stream) cudaStreamSynchronize(c.stream);  // earlier calls may still read the array
        if (mmxk_setup_buffers(&c, Kspec.data()) != 0) {
            cudaGetLastError();
            return fail(MMX_ERR_CUDA, "copy of the tensor spectrum into the static scratch failed");
        }
        slot.key = *mesh;
        slot.Ms = Ms;
        slot.prec = precision;
        slot.cached = true;
    }
    for (int i = 0; i < 3; ++i) c.ph.msN00[i] = Ms * slot.N00[i];
    mmxk_demag(&c, c.stream, nullptr, 0, 0, m_dev, 0, H_dev, m_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MMX_ERR_CUDA, cudaGetErrorString(e));
    return MMX_OK;
}
