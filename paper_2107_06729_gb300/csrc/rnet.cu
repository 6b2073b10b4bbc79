// Learned residual correction of the extrapolated demag field (declared in
// include/mmx_residual.h).  The paper's extrapolation (Sec. II, Eq. 6) has
// no learned part; this net predicts its error from the stage state.
//
// Forward: each 3x3x3 layer is an implicit GEMM, M = cells, N = output
// channels, K = 27 taps x input channels (k_rnet_conv_tc): tcgen05.mma
// 128 x N x 16 on the 5th-generation tensor cores with FP32 accumulators in
// TMEM; the input halo sits in shared memory in the canonical K-major layout
// so that every tap's A operand is the same layout at a shifted start
// address; each k-chunk plane of the halo is one 5-D tensor-memory-access
// copy (zero-filled outside the mesh) and the weights arrive by one bulk
// copy per CTA.  Bias, ReLU and the BF16 rounding of the output are fused.
// Backward (training only), also on the tensor cores: the input gradient is
// the same kernel with tap-flipped, transposed weights (the output gradient
// rounded to BF16 where it enters), the weight gradient a GEMM over cells
// (k_rnet_wgrad_tc, below).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/mmx_residual.h"
#include "internal.h"

namespace {

constexpr int RN_TY = 4;  // tile rows per CTA (4 warps, one y row each)
constexpr int NLAYER = 4;
constexpr int CIN[NLAYER] = {6, 32, 32, 32}, COUT[NLAYER] = {32, 32, 32, 3};
constexpr int CINP[NLAYER] = {16, 32, 32, 32};

constexpr long long p_off(int l)
{
    return l == 0 ? 0 : p_off(l - 1) + 27LL * COUT[l - 1] * CIN[l - 1] + COUT[l - 1];
}
static_assert(p_off(NLAYER) == MMX_RNET_PARAMS, "parameter count");
// the same offsets as scalars, for device code
constexpr long long PO1 = 5216, PO2 = 32896, PO3 = 60576;
static_assert(p_off(1) == PO1 && p_off(2) == PO2 && p_off(3) == PO3, "parameter offsets");

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// x (FP32, [6][cells]) -> layer-0 input (BF16, [cells][16], channels 6..15 zero)
__global__ void k_rnet_pack(const float *__restrict__ x, long long n, __nv_bfloat16 *__restrict__ a0)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(c < 6 ? x[c * n + i] : 0.0f);
    uint4 *dst = (uint4 *)(a0 + i * 16);
    dst[0] = ((const uint4 *)v)[0];
    dst[1] = ((const uint4 *)v)[1];
}

// ---- tcgen05 version of the layer ------------------------------------------
// The CTA computes D[128][N] = sum over taps and k-steps of A_t[128][16] B_t[16][N]
// on the 5th-generation tensor cores: row j = oy*32 + ox of the tile is the
// cell (x0 + ox - 1, y0 + oy, z) for ox = 1..30 (ox = 0 and 31 are computed
// and dropped).  The input halo is kept in shared memory as 16-byte rows
// [k-chunk][cell] with cells (hz, hy, hx), hx = 0..31, in row-major order
// after TC_PAD pad rows, i.e. in the canonical K-major layout without
// swizzle (8-row core matrices of 16-byte rows); the A operand of tap
// (tz, ty, tx) is then the same layout starting TC_PAD - 1 + (tz*6 + ty)*32
// + tx rows in.  Each k-chunk plane of a tile's halo is one tensor-memory-
// access copy: a 5-D view (8 channels, k-chunk, x, y, z) of the channels-last
// activations, box (8, 1, 32, 6, 3) at (0, kc, x0 - 1, y0 - 1, z - 1), which
// lands in exactly this row order and is zero-filled outside the mesh.  The
// weights are [tap][k-chunk][n] 16-byte rows (the same layout for B) and
// arrive by one bulk copy per CTA.  One lane issues the MMAs into TMEM
// accumulators (FP32) and commits them to an mbarrier.  Every wait is
// bounded in time; on expiry the kernel sets *fault, waits once more
// (bounded) for its own operations in flight and frees its TMEM.
constexpr int TC_HY = RN_TY + 2, TC_ROWS = 3 * TC_HY * 32;  // halo cells
constexpr int TC_PAD = 8;    // leading pad rows: the halo copy lands 128-byte aligned
constexpr int TC_NE = 592;   // rows per k-chunk plane (>= TC_PAD + the last tap's overrun = 585); 74 x 128 B
constexpr int TC_TX = 30;    // valid cells per tile row
constexpr uint32_t TC_PLANE_BYTES = (uint32_t)TC_ROWS * 16;  // one halo copy
// weights in the shared-memory layout of the tensor-core layers, per layer
// [27][Cin/8][N][8] BF16 (N = 32, or 16 for the last layer): one bulk copy each
constexpr long long TCO1 = 13824, TCO2 = 41472, TCO3 = 69120, TC_TOTAL = 82944;
constexpr unsigned long long TC_WAIT_NS = 1000000000ULL;
// independent accumulators (32 TMEM columns apart): consecutive MMAs of a tile
// go to different ones, so that they do not wait on each other's results
constexpr int TC_NACC = 4;

__host__ __device__ constexpr size_t tc_smem(int cinp, int n)
{
    // 128 bytes of alignment slack, halo planes, weights, 4 mbarriers + TMEM slot
    return 128 + (size_t)(cinp / 8) * TC_NE * 16 + (size_t)27 * (cinp / 8) * n * 16 + 64;
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes)
{
    // start address, leading and stride byte offsets in 16-byte units; version 1; no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <int N_>
__host__ __device__ constexpr uint32_t umma_idesc_bf16()
{
    // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both K-major,
    // N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mbar_init(uint32_t m)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(m) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ bool tc_mbar_wait(uint32_t m, unsigned parity, unsigned long long limit_ns)
{
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(m), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255) == 0) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
}

// the halo planes of one tile (KC copies) into the buffer at hb, counted on mbar
template <int KC>
__device__ __forceinline__ void tc_load_halo(const CUtensorMap *tm, uint32_t hb, uint32_t mbar, int x0, int y0, int z)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(KC * TC_PLANE_BYTES)
                 : "memory");
#pragma unroll
    for (int v = 0; v < KC; ++v)
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
            "%5, %6}], [%7];\n" ::"r"(hb + (uint32_t)(v * TC_NE + TC_PAD) * 16u),
            "l"(tm), "r"(0), "r"(v), "r"(x0 - 1), "r"(y0 - 1), "r"(z - 1), "r"(mbar)
            : "memory");
}

// MODE 0: hidden layer (bias, ReLU, BF16 [cells][32] out); 1: last layer (bias,
// FP32 [3][cells] out); 2: input gradient of a layer (tap-flipped, transposed
// weights; FP32 [cells][32] out, masked by ReLU' of the layer input `mask`,
// and its BF16 copy in out2)
template <int CINP_, int N_, int MODE>
__global__ void __launch_bounds__(128) k_rnet_conv_tc(const __grid_constant__ CUtensorMap tmap,
                                                      const __nv_bfloat16 *__restrict__ Wtc,
                                                      const float *__restrict__ bias, int cout, void *out, int nx,
                                                      int ny, int nz, int *fault,
                                                      const __nv_bfloat16 *__restrict__ mask, void *out2)
{
    constexpr int KC = CINP_ / 8;  // 16-byte k-chunks per cell
    extern __shared__ __align__(128) unsigned char tc_smem_raw[];
    unsigned char *base = tc_smem_raw + ((128u - (smem_u32(tc_smem_raw) & 127u)) & 127u);
    uint4 *hal2 = (uint4 *)base;                       // halo planes [KC][TC_NE], 128-byte aligned
    uint4 *wsm = hal2 + KC * TC_NE;                    // [27][KC][N_]
    uint64_t *mbar = (uint64_t *)(wsm + 27 * KC * N_); // [0] MMAs done, [1] weights, [2 + b] halo buffer b
    uint32_t *tmem_slot = (uint32_t *)(mbar + 4);
    constexpr uint32_t WBYTES = 27u * KC * N_ * 16u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int txc = (nx + TC_TX - 1) / TC_TX, tyc = (ny + RN_TY - 1) / RN_TY;
    const int ntiles = txc * tyc * nz;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(32 * TC_NACC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 32)
        for (int i = 0; i < 4; ++i) tc_mbar_init(smem_u32(mbar + i));
    // pad rows (never written by the copies): zero in every plane
    for (int e = threadIdx.x; e < KC * (TC_NE - TC_ROWS); e += blockDim.x) {
        const int v = e / (TC_NE - TC_ROWS), r = e % (TC_NE - TC_ROWS);
        hal2[v * TC_NE + (r < TC_PAD ? r : TC_ROWS + r)] = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t mb = smem_u32(mbar), mw = smem_u32(mbar + 1);
    const uint32_t hal_s = smem_u32(hal2), w_s = smem_u32(wsm);
    auto tile_xyz = [&](int tl, int &x0, int &y0, int &z) {
        x0 = (tl % txc) * TC_TX;
        y0 = ((tl / txc) % tyc) * RN_TY;
        z = tl / (txc * tyc);
    };
    // lane 0 of warp 0: weights and the first tile's halo in flight
    bool wok = true;
    int uses[2] = {0, 0};  // completed uses of each halo buffer's barrier (its parity)
    bool pending = false;  // a halo copy issued and not yet waited for
    bool inok = true;      // thread 0: the weights and this tile's halo arrived
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mw), "r"(WBYTES) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(w_s),
            "l"(Wtc), "r"(WBYTES), "r"(mw)
            : "memory");
        if ((int)blockIdx.x < ntiles) {
            int x0, y0, z;
            tile_xyz(blockIdx.x, x0, y0, z);
            tc_load_halo<KC>(&tmap, hal_s, smem_u32(mbar + 2), x0, y0, z);
            pending = true;
        }
    }
    // persistent loop over tiles; the weights stay in shared memory and the
    // next tile's halo is copied in while this tile's MMAs or epilogue run
    for (int tile = blockIdx.x, it = 0; tile < ntiles; tile += gridDim.x, ++it) {
        int x0, y0, z;
        tile_xyz(tile, x0, y0, z);
        const int b = 0;
        const int next = tile + (int)gridDim.x;
        // this tile's MMAs overwrite the accumulators the previous tile's TMEM
        // loads read before the barrier that ended that iteration
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (warp == 0) {
            if (lane == 0) {
                if (it == 0) {
                    wok = tc_mbar_wait(mw, 0, TC_WAIT_NS);
                    if (!wok) {
                        atomicExch(fault, 1);
                        (void)tc_mbar_wait(mw, 0, TC_WAIT_NS);  // the copy in flight
                    }
                }
                bool hok = tc_mbar_wait(smem_u32(mbar + 2 + b), uses[b] & 1, TC_WAIT_NS);
                if (!hok) {
                    atomicExch(fault, 1);
                    hok = tc_mbar_wait(smem_u32(mbar + 2 + b), uses[b] & 1, TC_WAIT_NS);
                }
                uses[b]++;
                pending = !hok;
                inok = wok && hok;
                if (wok && hok) {
                    constexpr uint32_t idesc = umma_idesc_bf16<N_>();
                    const uint32_t hb = hal_s + (uint32_t)(b * KC * TC_NE) * 16u;
                    for (int t = 0; t < 27; ++t) {
                        const int tz = t / 9, ty = (t / 3) % 3, tx = t % 3;
                        const uint32_t row0 = (uint32_t)(TC_PAD - 1 + (tz * TC_HY + ty) * 32 + tx);
#pragma unroll
                        for (int ks = 0; ks < KC / 2; ++ks) {
                            const uint64_t ad = umma_desc(hb + ((uint32_t)(2 * ks * TC_NE) + row0) * 16u, TC_NE * 16u, 128u);
                            const uint64_t bd = umma_desc(w_s + (uint32_t)((t * KC + 2 * ks) * N_) * 16u, N_ * 16u, 128u);
                            const int i = t * (KC / 2) + ks;
                            const uint32_t acc = (i >= TC_NACC) ? 1u : 0u;  // the first MMA of each accumulator overwrites it
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                    tmem + 32u * (i % TC_NACC)),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                                : "memory");
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                             : "memory");
            }
            __syncwarp();  // the other lanes of the issuing warp do not spin beside it
        }
        bool ok = tc_mbar_wait(mb, it & 1, TC_WAIT_NS);
        if (!ok) {
            if (lane == 0) atomicExch(fault, 1);
            ok = tc_mbar_wait(mb, it & 1, TC_WAIT_NS);  // let the MMAs in flight finish before TMEM is freed
        }
        // this tile's MMAs are done with the buffer, so the next tile's halo can come in now
        if (threadIdx.x == 0 && ok && next < ntiles) {
            int nx0, ny0, nz0;
            tile_xyz(next, nx0, ny0, nz0);
            tc_load_halo<KC>(&tmap, hal_s, smem_u32(mbar + 2), nx0, ny0, nz0);
            pending = true;
        }
        // one decision for the whole CTA (the TMEM loads below are warp-collective);
        // a weight or halo copy that never arrived also ends the loop, so that a
        // fault costs a bounded number of waits whatever the number of tiles
        ok = __syncthreads_and(ok && inok) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;  // a barrier phase or a copy is lost: stop, free TMEM below
        {
            // warp w reads TMEM lanes 32w..32w+31 = tile rows oy = w, ox = lane; the
            // accumulators are summed in FP32
            float v[N_];
#pragma unroll
            for (int c = 0; c < N_; ++c) v[c] = 0.0f;
#pragma unroll
            for (int a = 0; a < TC_NACC; ++a) {
                uint32_t u[N_];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + 32u * a;
                if constexpr (N_ == 32) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                          "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]),
                          "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]),
                          "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
                        : "r"(taddr));
                } else {
                    static_assert(N_ == 16, "N is 16 or 32");
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];\n"
                        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
                          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
                          "=r"(u[14]), "=r"(u[15])
                        : "r"(taddr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int c = 0; c < N_; ++c) v[c] += __uint_as_float(u[c]);
            }
            const int x = x0 + lane - 1, y = y0 + warp;
            if (lane >= 1 && lane <= TC_TX && x < nx && y < ny) {
                const size_t ncell = (size_t)nx * ny * nz;
                const size_t cell = ((size_t)z * ny + y) * nx + x;
                if constexpr (MODE == 0) {
                    __align__(16) __nv_bfloat162 h[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        h[c] = __floats2bfloat162_rn(fmaxf(v[2 * c] + bias[2 * c], 0.0f),
                                                     fmaxf(v[2 * c + 1] + bias[2 * c + 1], 0.0f));
                    uint4 *dst = (uint4 *)((__nv_bfloat16 *)out + cell * 32);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dst[q] = ((const uint4 *)h)[q];
                } else if constexpr (MODE == 2) {
                    __align__(16) __nv_bfloat16 mk[32];
                    __align__(16) float g[32];
                    __align__(16) __nv_bfloat162 h[16];
#pragma unroll
                    for (int q = 0; q < 4; ++q) ((uint4 *)mk)[q] = ((const uint4 *)(mask + cell * 32))[q];
#pragma unroll
                    for (int c = 0; c < 32; ++c) g[c] = (__bfloat162float(mk[c]) > 0.0f) ? v[c] : 0.0f;
#pragma unroll
                    for (int c = 0; c < 16; ++c) h[c] = __floats2bfloat162_rn(g[2 * c], g[2 * c + 1]);
                    uint4 *df = (uint4 *)((float *)out + cell * 32);
#pragma unroll
                    for (int q = 0; q < 8; ++q) df[q] = ((const uint4 *)g)[q];
                    uint4 *db = (uint4 *)((__nv_bfloat16 *)out2 + cell * 32);
#pragma unroll
                    for (int q = 0; q < 4; ++q) db[q] = ((const uint4 *)h)[q];
                } else {
                    float *r = (float *)out;
                    for (int c = 0; c < cout; ++c) r[c * ncell + cell] = v[c] + bias[c];
                }
            }
        }
        // TMEM reads of this tile done before the next tile's MMAs overwrite the accumulators
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
    }
    // a halo copy still in flight (only after a lost barrier phase): let it land first
    if (threadIdx.x == 0 && pending) {
        (void)tc_mbar_wait(smem_u32(mbar + 2), uses[0] & 1, TC_WAIT_NS);
    }
    if (threadIdx.x == 0 && (int)blockIdx.x >= ntiles) (void)tc_mbar_wait(mw, 0, TC_WAIT_NS);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(32 * TC_NACC)
                     : "memory");
}

// loss terms: dz3 [cells][8] = 2 (r - target) / (3 cells), sum of squares into *loss
__global__ void k_rnet_loss(const float *__restrict__ r, const float *__restrict__ tgt, long long n,
                            float *__restrict__ dz3, __nv_bfloat16 *__restrict__ dz3b, double *loss)
{
    __shared__ double s_sum[8];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (i < n) {
        const float k = (float)(2.0 / (3.0 * (double)n));
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float d = 0.0f;
            if (c < 3) {
                d = r[c * n + i] - tgt[c * n + i];
                sq += (double)d * d;
            }
            dz3[i * 8 + c] = k * d;
            dz3b[i * 16 + c] = __float2bfloat16_rn(k * d);
            dz3b[i * 16 + 8 + c] = __float2bfloat16_rn(0.0f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_sum[w];
        atomicAdd(loss, s);
    }
}

// N consecutive FP32 accumulator columns of this warp's 32 TMEM lanes
template <int N>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float *v)
{
    uint32_t u[N];
    if constexpr (N == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
              "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
              "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]),
              "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]),
              "=r"(u[30]), "=r"(u[31])
            : "r"(taddr));
    } else {
        static_assert(N == 16, "N is 16 or 32");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
              "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = __uint_as_float(u[c]);
}

// ---- weight and bias gradients -------------------------------------------
// gW[t][o][c] = sum_p dz[p][o] A[p + d_t][c] (d_t the offset of tap t) is,
// with q = p + d_t, sum_q dz[q - d_t][o] A[q][c]: per CTA a GEMM on the
// tensor cores, D[(tx, o)][c] += sum_q dzs[(tx, o)][q] A[c][q] over tiles of
// WG_TC cells q along x, one accumulator per (tz, ty) tap "slab" of the CTA's
// slab group (grid.y = tz: ty = 0..2).  The 3 x COUTP rows (tx, o) of a slab
// are dz shifted by the x-tap; the other rows of its 128-row MMA are the
// next slab's rows (or zero) and are never read back.  dz (FP32) enters as a
// BF16 pair hi + lo, two MMAs into the same accumulator (about 16 bits), so
// the gradient keeps FP32-like accuracy; the activations are BF16 already.
// Both operands are built by the threads in shared memory in the canonical
// K-major layout without swizzle (8-row core matrices of 16-byte rows): a
// 16-byte row holds 8 consecutive cells of one (tx, o) or of one c.  The
// accumulators stay in TMEM over all tiles of the CTA; at the end the CTA
// writes its partial sums to scratch [cta][27][COUTP][CINP], which a second
// kernel adds up.  Every wait is bounded; on expiry the kernel sets *fault,
// waits once more for its own MMAs and frees its TMEM.
constexpr int WG_TKC = 2;          // 16-byte k-chunks (8 cells each) per tile: one MMA k-step
constexpr int WG_TC = 8 * WG_TKC;  // cells per tile
template <int COUTP_> __host__ __device__ constexpr int wg_gs() { return 3 * COUTP_ / 8; }  // row groups per slab
// row groups per k-chunk: three slabs, plus the rows the last slab's MMA reads beyond its own
template <int COUTP_> __host__ __device__ constexpr int wg_groups() { return 2 * wg_gs<COUTP_>() + 16; }
// dynamic shared memory of one CTA: the operands need about 22 KB, but the
// launch asks for 56 KB so that at most four CTAs share an SM and their
// TMEM allocations (at most 128 of the 512 columns each) always fit: no CTA
// ever waits in tcgen05.alloc
template <int CINP_, int COUTP_> __host__ __device__ constexpr size_t wg_smem()
{
    constexpr size_t need = 128 + (size_t)2 * WG_TKC * wg_groups<COUTP_>() * 128 + (size_t)WG_TKC * (CINP_ / 8) * 128 + 64;
    return need > 56 * 1024 ? need : 56 * 1024;
}

template <int CINP_, int COUTP_>
__global__ void __launch_bounds__(128) k_rnet_wgrad_tc(const float *__restrict__ dz,
                                                       const __nv_bfloat16 *__restrict__ A, float *__restrict__ part,
                                                       int nx, int ny, int nz, int *fault)
{
    constexpr int GS = wg_gs<COUTP_>(), NG = wg_groups<COUTP_>(), KCB = CINP_ / 8;
    constexpr uint32_t NCOL = 3 * CINP_;  // accumulator columns: three slabs of N = CINP
    constexpr uint32_t NALLOC = NCOL <= 32 ? 32 : (NCOL <= 64 ? 64 : (NCOL <= 128 ? 128 : 256));
    extern __shared__ __align__(128) unsigned char wg_raw[];
    unsigned char *base = wg_raw + ((128u - (smem_u32(wg_raw) & 127u)) & 127u);
    uint4 *dzs = (uint4 *)base;                     // [hi / lo][WG_TKC][NG][8] 16-byte rows
    uint4 *as = dzs + 2 * WG_TKC * NG * 8;          // [WG_TKC][KCB][8]
    uint64_t *mbar = (uint64_t *)(as + WG_TKC * KCB * 8);
    uint32_t *tmem_slot = (uint32_t *)(mbar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tz = blockIdx.y;
    const int txc = (nx + WG_TC - 1) / WG_TC;
    const long long ntiles = (long long)txc * ny * nz;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(NALLOC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 32) tc_mbar_init(smem_u32(mbar));
    // rows never written (beyond the last slab) stay zero
    for (int e = threadIdx.x; e < 2 * WG_TKC * NG * 8 + WG_TKC * KCB * 8; e += blockDim.x)
        dzs[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t mb = smem_u32(mbar), dz_s = smem_u32(dzs), a_s = smem_u32(as);
    bool ok = true;
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int xt = (int)(tile % txc);
        const long long rest = tile / txc;
        const int y = (int)(rest % ny), z = (int)(rest / ny), x0 = xt * WG_TC;
        // dz rows: slab s (ty), x-tap tx, channel o, k-chunk kc; cell q = x0 + 8 kc + e
        // takes dz at q - d: (x - (tx - 1), y - (s - 1), z - (tz - 1)), zero outside the mesh.
        // Consecutive threads take consecutive o: each load of a warp reads one 128-byte run.
        for (int r = threadIdx.x; r < 9 * COUTP_ * WG_TKC; r += blockDim.x) {
            const int o = r % COUTP_;
            int rr = r / COUTP_;
            const int tx = rr % 3;
            rr /= 3;
            const int sl = rr % 3, kc = rr / 3;
            const int yy = y - (sl - 1), zz = z - (tz - 1);
            const bool rowok = yy >= 0 && yy < ny && zz >= 0 && zz < nz;
            const float *src = dz + (((long long)(rowok ? zz : 0) * ny + (rowok ? yy : 0)) * nx) * COUTP_ + o;
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int xx = x0 + 8 * kc + e - (tx - 1);
                const float v = (rowok && xx >= 0 && xx < nx) ? src[(long long)xx * COUTP_] : 0.0f;
                hi[e] = __float2bfloat16_rn(v);
                lo[e] = __float2bfloat16_rn(v - __bfloat162float(hi[e]));
            }
            const int m = tx * COUTP_ + o, g = sl * GS + (m >> 3);
            dzs[((0 * WG_TKC + kc) * NG + g) * 8 + (m & 7)] = *(const uint4 *)hi;
            dzs[((1 * WG_TKC + kc) * NG + g) * 8 + (m & 7)] = *(const uint4 *)lo;
        }
        // activations: row c, k-chunk kc, unshifted; cells beyond nx zero
        for (int r = threadIdx.x; r < CINP_ * WG_TKC; r += blockDim.x) {
            const int c = r % CINP_, kc = r / CINP_;
            const __nv_bfloat16 *src = A + (((long long)z * ny + y) * nx) * CINP_ + c;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int xx = x0 + 8 * kc + e;
                v[e] = xx < nx ? src[(long long)xx * CINP_] : __float2bfloat16_rn(0.0f);
            }
            as[(kc * KCB + (c >> 3)) * 8 + (c & 7)] = *(const uint4 *)v;
        }
        // the operands written by the threads become visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (threadIdx.x == 0) {
            constexpr uint32_t idesc = umma_idesc_bf16<CINP_>();
#pragma unroll
            for (int sl = 0; sl < 3; ++sl)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < WG_TKC / 2; ++ks) {
                        const uint64_t ad = umma_desc(
                            dz_s + (uint32_t)(((h * WG_TKC + 2 * ks) * NG + sl * GS) * 8) * 16u, NG * 128u, 128u);
                        const uint64_t bd = umma_desc(a_s + (uint32_t)(2 * ks * KCB * 8) * 16u, KCB * 128u, 128u);
                        // the first MMA into each slab's accumulator overwrites it
                        const uint32_t acc = (it > 0 || h > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                tmem + (uint32_t)(sl * CINP_)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                            : "memory");
                    }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                         : "memory");
        }
        __syncwarp();
        // the MMAs read the operands: the next tile may only overwrite them afterwards
        bool done = tc_mbar_wait(mb, it & 1, TC_WAIT_NS);
        if (!done) {
            if (lane == 0) atomicExch(fault, 1);
            done = tc_mbar_wait(mb, it & 1, TC_WAIT_NS);  // let the MMAs in flight finish before TMEM is freed
        }
        ok = __syncthreads_and(ok && done) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;
    }
    // partial sums of this CTA: warp w reads TMEM lanes 32w..32w+31 (MMA rows m)
    if (ok) {
        const int m = warp * 32 + lane;
        const bool mine = m < 3 * COUTP_;
        const int tx = m / COUTP_, o = m % COUTP_;
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            float v[CINP_];
            tmem_load<CINP_>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * CINP_), v);
            if (mine) {
                const int t = tz * 9 + sl * 3 + tx;
                float4 *dst = (float4 *)(part + (((size_t)blockIdx.x * 27 + t) * COUTP_ + o) * CINP_);
#pragma unroll
                for (int q = 0; q < CINP_ / 4; ++q)
                    dst[q] = it > 0 ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NALLOC) : "memory");
}

// gW[t][o][c] (o < cout, c < cin) = sum over the CTAs' partial sums
template <int CINP_, int COUTP_>
__global__ void k_rnet_wgrad_sum(const float *__restrict__ part, int nparts, int cin, int cout, float *__restrict__ gW)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 27 * cout * cin) return;
    const int c = i % cin, o = (i / cin) % cout, t = i / (cin * cout);
    const float *p = part + ((size_t)t * COUTP_ + o) * CINP_ + c;
    float sum = 0.0f;
    for (int b = 0; b < nparts; ++b) sum += p[(size_t)b * 27 * COUTP_ * CINP_];
    gW[i] = sum;
}

// gb[o] = sum_p dz[p][o]: per CTA a shared sum over a range of cells, then
// one atomic per channel
template <int COUTP_>
__global__ void __launch_bounds__(256) k_rnet_bgrad(const float *__restrict__ dz, long long n, int cout,
                                                    float *__restrict__ gb)
{
    __shared__ float s[COUTP_];
    if (threadIdx.x < COUTP_) s[threadIdx.x] = 0.0f;
    __syncthreads();
    constexpr int PER = 256 / COUTP_;  // cells per pass of the CTA
    const int o = threadIdx.x % COUTP_;
    float acc = 0.0f;
    for (long long p = (long long)blockIdx.x * PER + threadIdx.x / COUTP_; p < n; p += (long long)gridDim.x * PER)
        acc += dz[p * COUTP_ + o];
    atomicAdd(&s[o], acc);
    __syncthreads();
    if (threadIdx.x < cout) atomicAdd(&gb[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_rnet_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ Vv,
                            const float *__restrict__ G, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = 0.9f * M[i] + 0.1f * g;
    const float v = 0.999f * Vv[i] + 0.001f * g * g;
    M[i] = m;
    Vv[i] = v;
    P[i] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
}

// the same weights in the tensor-core layers' shared-memory layout:
// per layer [27][Cin_pad/8][N][8], N = 32 (16 for the last layer), zero padded
__global__ void k_rnet_cast_tc(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Wtc)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TC_TOTAL) return;
    long long j, po;
    int cin, cout, kcn, nn;
    if (i < TCO1) {
        j = i, po = 0, cin = 6, cout = 32, kcn = 2, nn = 32;
    } else if (i < TCO2) {
        j = i - TCO1, po = PO1, cin = 32, cout = 32, kcn = 4, nn = 32;
    } else if (i < TCO3) {
        j = i - TCO2, po = PO2, cin = 32, cout = 32, kcn = 4, nn = 32;
    } else {
        j = i - TCO3, po = PO3, cin = 32, cout = 3, kcn = 4, nn = 16;
    }
    const int e = (int)(j % 8);
    const long long row = j / 8;
    const int n = (int)(row % nn), kc = (int)((row / nn) % kcn), t = (int)(row / ((long long)nn * kcn));
    const int k = kc * 8 + e;
    float v = 0.0f;
    if (n < cout && k < cin) v = P[po + ((long long)t * cout + n) * cin + k];
    Wtc[i] = __float2bfloat16_rn(v);
}

// input-gradient weights in the tensor-core layout: for layer l = 3, 2, 1,
// [27][Cout_pad/8][32][8] with W'[t'][n = ci][k = co] = W[26 - t'][co][ci]
// (taps flipped: the gradient reads dz at p - offset); Cout_pad = 16 for the
// last layer, 32 otherwise
constexpr long long TT2 = 13824, TT1 = 41472, TT_TOTAL = 69120;
__global__ void k_rnet_cast_tc_t(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Wt)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TT_TOTAL) return;
    long long j, po;
    int cout, kcn;
    if (i < TT2) {
        j = i, po = PO3, cout = 3, kcn = 2;
    } else if (i < TT1) {
        j = i - TT2, po = PO2, cout = 32, kcn = 4;
    } else {
        j = i - TT1, po = PO1, cout = 32, kcn = 4;
    }
    const int e = (int)(j % 8);
    const long long row = j / 8;
    const int n = (int)(row % 32), kc = (int)((row / 32) % kcn), tp = (int)(row / (32LL * kcn));
    const int k = kc * 8 + e;
    float v = 0.0f;
    if (k < cout) v = P[po + ((long long)(26 - tp) * cout + k) * 32 + n];
    Wt[i] = __float2bfloat16_rn(v);
}

// stage k of an extrapolated attempt with the learned residual: Eq. 6 with
// the attempt's weights (the same sum, in the same order, as the stage
// kernel's) into G, and the net's packed input (Y_k, G_ext / Ms)
__global__ void k_res_stage_in(DevState *st, int k, int np1, const float *__restrict__ hist,
                               const float *__restrict__ Y, long long n, float inv_Ms, float *__restrict__ G,
                               __nv_bfloat16 *__restrict__ a0, int count)
{
    if (st->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (count && blockIdx.x == 0 && threadIdx.x == 0) st->extrap_evals++;
    if (i >= n) return;
    const float *wf = st->coef[k].wf;
    float g[3] = {0.0f, 0.0f, 0.0f};
    for (int j = 0; j < np1; ++j) {
        const float w = wf[j];
        const float *Gj = hist + (size_t)j * 3 * n;
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] += w * Gj[c * n + i];
    }
    __align__(16) __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        G[c * n + i] = g[c];
        v[c] = __float2bfloat16_rn(Y[c * n + i]);
        v[3 + c] = __float2bfloat16_rn(g[c] * inv_Ms);
    }
#pragma unroll
    for (int c = 6; c < 16; ++c) v[c] = __float2bfloat16_rn(0.0f);
    uint4 *dst = (uint4 *)(a0 + i * 16);
    dst[0] = ((const uint4 *)v)[0];
    dst[1] = ((const uint4 *)v)[1];
}

// G += Ms r (the net's output, [3][cells])
__global__ void k_res_stage_out(const DevState *st, const float *__restrict__ r, long long n3, float Ms,
                                float *__restrict__ G)
{
    if (st->done) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) G[i] += Ms * r[i];
}

// periodic check: the net-corrected field Gc + Ms r against the exact field
// G of the same stage; the maxima of |difference| and |G| into the state
// (non-negative FP32 values compare as their bit patterns)
__global__ void k_res_check_cmp(DevState *st, const float *__restrict__ r, const float *__restrict__ Gc,
                                const float *__restrict__ G, long long n3, float Ms)
{
    __shared__ unsigned int s_num, s_den;
    if (threadIdx.x == 0) {
        s_num = 0u;
        s_den = 0u;
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) {
        const float g = G[i];
        const float d = fabsf(Gc[i] + Ms * r[i] - g);
        atomicMax(&s_num, __float_as_uint(d == d ? d : INFINITY));
        atomicMax(&s_den, __float_as_uint(fabsf(g)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&st->check_num_bits, s_num);
        atomicMax(&st->check_den_bits, s_den);
    }
}

// training pairs: xg (T, [3][cells]) = sum_j w_j G_j
template <typename T>
__global__ void k_res_accum(const T *__restrict__ G, double w, T *__restrict__ acc, long long n3, int first)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const T v = (T)w * G[i];
    acc[i] = first ? v : acc[i] + v;
}

template <typename T>
__global__ void k_res_finish(const T *__restrict__ m, const T *__restrict__ G, const T *__restrict__ Gext,
                             double inv_Ms, long long n, float *__restrict__ x, float *__restrict__ target)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    x[i] = (float)m[i];
    x[3 * n + i] = (float)(Gext[i] * (T)inv_Ms);
    target[i] = (float)((G[i] - Gext[i]) * (T)inv_Ms);
}

}  // namespace

struct mmx_rnet {
    cudaStream_t s = nullptr;
    long long max_cells = 0;
    float *P = nullptr, *Pm = nullptr, *Pv = nullptr, *grad = nullptr;
    __nv_bfloat16 *Wtc = nullptr, *Wtt = nullptr;
    __nv_bfloat16 *dz3b = nullptr, *dzAb = nullptr, *dzBb = nullptr;  // BF16 copies of the output gradients
    __nv_bfloat16 *a[NLAYER] = {nullptr, nullptr, nullptr, nullptr};
    float *r = nullptr, *dz3 = nullptr, *dzA = nullptr, *dzB = nullptr;
    double *loss_d = nullptr;
    int *fault = nullptr;  // set by a tensor-core layer whose bounded wait ran out
    int nsm = 1;
    float *part = nullptr;   // weight gradient: partial sums [nsm][27][32][32] of the CTAs
    CUtensorMap tm[NLAYER];  // 5-D views of the layer inputs for the halo copies
    CUtensorMap tmg[3];      // the same for the gradients dz3b, dzAb, dzBb
    int tm_nx = 0, tm_ny = 0, tm_nz = 0;
    bool tm_ok = false;
    int grid_cap = 0;         // MMX_RNET_GRID_CAP=n: at most n persistent CTAs (0: two per SM)
    int step = 0;
    int nx = 0, ny = 0, nz = 0;
    std::string err;
};

namespace {

int rfail(mmx_rnet *net, int code, const std::string &msg)
{
    if (net) net->err = msg;
    return code;
}

#define RCK(call)                                                                                      \
    do {                                                                                               \
        cudaError_t e__ = (call);                                                                      \
        if (e__ != cudaSuccess) return rfail(net, MMX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

std::once_flag smem_once;
cudaError_t smem_status = cudaSuccess;

cudaError_t set_tc_smem()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_rnet_conv_tc<16, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem(16, 32))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_conv_tc<32, 32, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem(32, 32))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_conv_tc<16, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem(16, 32))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_conv_tc<32, 32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem(32, 32))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_wgrad_tc<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wg_smem<32, 8>())) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_wgrad_tc<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wg_smem<32, 32>())) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_rnet_wgrad_tc<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wg_smem<16, 32>())) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_rnet_conv_tc<32, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tc_smem(32, 16));
}

// the four layers on the tensor-core kernels (two persistent CTAs per SM
// overlap each other's halo copies)
void forward_tc(mmx_rnet *net, int nx, int ny, int nz);

// 5-D view (8 channels, k-chunk, x, y, z) of channels-last BF16 activations
// with cinp channels per cell; box (8, 1, 32, 6, 3), zero fill outside
PFN_cuTensorMapEncodeTiled_v12000 lookup_encoder()
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

bool encode_halo_map(CUtensorMap *tm, const void *base, int cinp, int nx, int ny, int nz)
{
    static const PFN_cuTensorMapEncodeTiled_v12000 enc = lookup_encoder();  // once, thread-safe
    if (!enc) return false;
    const cuuint64_t dims[5] = {8, (cuuint64_t)(cinp / 8), (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t row = (cuuint64_t)cinp * 2;
    const cuuint64_t strides[4] = {16, row, row * nx, row * nx * ny};
    const cuuint32_t box[5] = {8, 1, 32, (cuuint32_t)TC_HY, 3};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool halo_maps(mmx_rnet *net, int nx, int ny, int nz)
{
    if (net->tm_nx == nx && net->tm_ny == ny && net->tm_nz == nz) return net->tm_ok;
    bool ok = true;
    for (int l = 0; l < NLAYER && ok; ++l) ok = encode_halo_map(&net->tm[l], net->a[l], CINP[l], nx, ny, nz);
    ok = ok && encode_halo_map(&net->tmg[0], net->dz3b, 16, nx, ny, nz) &&
         encode_halo_map(&net->tmg[1], net->dzAb, 32, nx, ny, nz) &&
         encode_halo_map(&net->tmg[2], net->dzBb, 32, nx, ny, nz);
    net->tm_nx = nx;
    net->tm_ny = ny;
    net->tm_nz = nz;
    net->tm_ok = ok;
    return ok;
}

cudaError_t raise_conv_smem_once() { return set_tc_smem(); }

// the shared-memory limits of every layer kernel, raised once per process
cudaError_t raise_conv_smem()
{
    std::call_once(smem_once, [] { smem_status = raise_conv_smem_once(); });
    return smem_status;
}

// after a stream synchronisation: the fault word of the tensor-core layers
int check_fault(mmx_rnet *net)
{
    int f = 0;
    RCK(cudaMemcpy(&f, net->fault, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) return rfail(net, MMX_ERR_CUDA, "a bounded tensor-core wait gave up (MMA not completed)");
    return MMX_OK;
}

int check_mesh(mmx_rnet *net, int nx, int ny, int nz)
{
    if (nx < 1 || ny < 1 || nz < 1 || nz > 65535 || (long long)nx * ny * nz > net->max_cells)
        return rfail(net, MMX_ERR_ARG, "mesh size out of range for this net");
    return MMX_OK;
}

// forward through all layers from the packed input a[0]; output in net->r.
// MMX_ERR_CUDA when the tensor maps of the halo copies cannot be encoded.
int forward_layers(mmx_rnet *net, int nx, int ny, int nz)
{
    if (!halo_maps(net, nx, ny, nz))
        return rfail(net, MMX_ERR_CUDA, "the tensor maps of the layer inputs could not be encoded");
    forward_tc(net, nx, ny, nz);
    return MMX_OK;
}

void forward_tc(mmx_rnet *net, int nx, int ny, int nz)
{
    const long long tiles = (long long)((nx + TC_TX - 1) / TC_TX) * ((ny + RN_TY - 1) / RN_TY) * nz;
    long long cap = (long long)net->nsm * 2;
    if (net->grid_cap > 0 && net->grid_cap < cap) cap = net->grid_cap;
    const dim3 g((unsigned)(tiles < cap ? tiles : cap));
    k_rnet_conv_tc<16, 32, 0><<<g, 128, tc_smem(16, 32), net->s>>>(
        net->tm[0], net->Wtc, net->P + p_off(0) + 27 * 32 * 6, 32, net->a[1], nx, ny, nz, net->fault, nullptr, nullptr);
    k_rnet_conv_tc<32, 32, 0><<<g, 128, tc_smem(32, 32), net->s>>>(
        net->tm[1], net->Wtc + TCO1, net->P + p_off(1) + 27 * 32 * 32, 32, net->a[2], nx, ny, nz, net->fault, nullptr, nullptr);
    k_rnet_conv_tc<32, 32, 0><<<g, 128, tc_smem(32, 32), net->s>>>(
        net->tm[2], net->Wtc + TCO2, net->P + p_off(2) + 27 * 32 * 32, 32, net->a[3], nx, ny, nz, net->fault, nullptr, nullptr);
    k_rnet_conv_tc<32, 16, 1><<<g, 128, tc_smem(32, 16), net->s>>>(
        net->tm[3], net->Wtc + TCO3, net->P + p_off(3) + 27 * 3 * 32, 3, net->r, nx, ny, nz, net->fault, nullptr, nullptr);
}

// weight and bias gradients of one layer into gW ([27][cout][cin], then
// b[cout]): the tensor-core partial sums per CTA, their sum, the bias sum
template <int CINP_, int COUTP_>
void wgrad_layer(mmx_rnet *net, const float *dz, const __nv_bfloat16 *A, int cin, int cout, float *gW, int nx, int ny,
                 int nz)
{
    const long long n = (long long)nx * ny * nz;
    const long long tiles = (long long)((nx + WG_TC - 1) / WG_TC) * ny * nz;
    long long g = net->nsm;
    if (net->grid_cap > 0 && net->grid_cap < g) g = net->grid_cap;
    if (tiles < g) g = tiles;
    k_rnet_wgrad_tc<CINP_, COUTP_><<<dim3((unsigned)g, 3), 128, wg_smem<CINP_, COUTP_>(), net->s>>>(
        dz, A, net->part, nx, ny, nz, net->fault);
    const int nw = 27 * cout * cin;
    k_rnet_wgrad_sum<CINP_, COUTP_><<<(unsigned)((nw + 255) / 256), 256, 0, net->s>>>(net->part, (int)g, cin, cout,
                                                                                      gW);
    const long long nb = (n + 1023) / 1024;
    k_rnet_bgrad<COUTP_><<<(unsigned)(nb < 1024 ? nb : 1024), 256, 0, net->s>>>(dz, n, cout, gW + nw);
}

int refresh_weights(mmx_rnet *net)
{
    k_rnet_cast_tc<<<(unsigned)((TC_TOTAL + 255) / 256), 256, 0, net->s>>>(net->P, net->Wtc);
    k_rnet_cast_tc_t<<<(unsigned)((TT_TOTAL + 255) / 256), 256, 0, net->s>>>(net->P, net->Wtt);
    RCK(cudaGetLastError());
    return MMX_OK;
}

void lagrange(int p, const double *tau_nodes, double tau, double *w)
{
    for (int i = 0; i <= p; ++i) {
        double L = 1.0;
        for (int j = 0; j <= p; ++j)
            if (j != i) L *= (tau - tau_nodes[j]) / (tau_nodes[i] - tau_nodes[j]);
        w[i] = L;
    }
}

template <typename T>
int sample_t(mmx_ctx *c, int p, const void *m_nodes, const double *t_nodes, const void *m, double t, float *x,
             float *target)
{
    const long long n = c->n, n3 = 3 * n;
    double tau[6], w[6];
    for (int i = 0; i <= p; ++i) tau[i] = t_nodes[i] - t_nodes[p];
    lagrange(p, tau, t - t_nodes[p], w);
    T *Gext = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&Gext, n3 * sizeof(T), c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("cudaMallocAsync: ") + cudaGetErrorString(e);
        return MMX_ERR_OOM;
    }
    const unsigned nb3 = (unsigned)((n3 + 255) / 256);
    for (int j = 0; j <= p; ++j) {
        mmxk_demag(c, c->stream, nullptr, 0, 0, (const T *)m_nodes + (size_t)j * n3, 0, c->G, nullptr);
        k_res_accum<T><<<nb3, 256, 0, c->stream>>>((const T *)c->G, w[j], Gext, n3, j == 0);
    }
    mmxk_demag(c, c->stream, nullptr, 0, 0, m, 0, c->G, nullptr);
    k_res_finish<T><<<nb3, 256, 0, c->stream>>>((const T *)m, (const T *)c->G, Gext, 1.0 / c->mat.Ms, n, x, target);
    e = cudaGetLastError();
    cudaFreeAsync(Gext, c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("mmx_residual_sample launch: ") + cudaGetErrorString(e);
        return MMX_ERR_CUDA;
    }
    return MMX_OK;
}

}  // namespace

extern "C" int mmx_rnet_create(long long max_cells, void *cuda_stream, mmx_rnet **out)
{
    if (!out || max_cells < 1 || max_cells > (1LL << 26)) return MMX_ERR_ARG;
    *out = nullptr;
    mmx_rnet *net = new mmx_rnet();
    net->s = (cudaStream_t)cuda_stream;
    net->max_cells = max_cells;
    const size_t P = MMX_RNET_PARAMS * sizeof(float);
    bool ok = cudaMalloc(&net->P, P) == cudaSuccess && cudaMalloc(&net->Pm, P) == cudaSuccess &&
              cudaMalloc(&net->Pv, P) == cudaSuccess && cudaMalloc(&net->grad, P) == cudaSuccess &&
              cudaMalloc(&net->Wtc, TC_TOTAL * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->Wtt, TT_TOTAL * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->dz3b, max_cells * 16 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->dzAb, max_cells * 32 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->dzBb, max_cells * 32 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->a[0], max_cells * 16 * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&net->r, max_cells * 3 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&net->dz3, max_cells * 8 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&net->dzA, max_cells * 32 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&net->dzB, max_cells * 32 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&net->loss_d, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&net->fault, sizeof(int)) == cudaSuccess;
    for (int l = 1; l < NLAYER && ok; ++l)
        ok = cudaMalloc(&net->a[l], max_cells * 32 * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mmx_rnet_destroy(net);
        return MMX_ERR_OOM;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&net->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || net->nsm < 1)
        net->nsm = 1;
    if (cudaMalloc(&net->part, (size_t)net->nsm * 27 * 32 * 32 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        mmx_rnet_destroy(net);
        return MMX_ERR_OOM;
    }
    const char *gcap = getenv("MMX_RNET_GRID_CAP");
    net->grid_cap = gcap ? atoi(gcap) : 0;
    if (raise_conv_smem() != cudaSuccess || cudaMemsetAsync(net->fault, 0, sizeof(int), net->s) != cudaSuccess ||
        cudaMemsetAsync(net->P, 0, P, net->s) != cudaSuccess ||
        cudaMemsetAsync(net->Pm, 0, P, net->s) != cudaSuccess ||
        cudaMemsetAsync(net->Pv, 0, P, net->s) != cudaSuccess ||
        cudaMemsetAsync(net->grad, 0, P, net->s) != cudaSuccess || refresh_weights(net) != MMX_OK) {
        cudaGetLastError();
        mmx_rnet_destroy(net);
        return MMX_ERR_CUDA;
    }
    *out = net;
    return MMX_OK;
}

extern "C" int mmx_rnet_set_params(mmx_rnet *net, const float *params_host)
{
    if (!net || !params_host) return rfail(net, MMX_ERR_ARG, "NULL argument");
    const size_t P = MMX_RNET_PARAMS * sizeof(float);
    RCK(cudaMemcpyAsync(net->P, params_host, P, cudaMemcpyHostToDevice, net->s));
    RCK(cudaMemsetAsync(net->Pm, 0, P, net->s));
    RCK(cudaMemsetAsync(net->Pv, 0, P, net->s));
    net->step = 0;
    if (int rc = refresh_weights(net)) return rc;
    RCK(cudaStreamSynchronize(net->s));
    return MMX_OK;
}

extern "C" int mmx_rnet_get_params(mmx_rnet *net, float *params_host)
{
    if (!net || !params_host) return rfail(net, MMX_ERR_ARG, "NULL argument");
    RCK(cudaMemcpyAsync(params_host, net->P, MMX_RNET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, net->s));
    RCK(cudaStreamSynchronize(net->s));
    return check_fault(net);
}

extern "C" int mmx_rnet_forward(mmx_rnet *net, int nx, int ny, int nz, const float *x_dev, float *r_dev)
{
    if (!net || !x_dev) return rfail(net, MMX_ERR_ARG, "NULL argument");
    if (int rc = check_mesh(net, nx, ny, nz)) return rc;
    const long long n = (long long)nx * ny * nz;
    k_rnet_pack<<<(unsigned)((n + 255) / 256), 256, 0, net->s>>>(x_dev, n, net->a[0]);
    if (int rc = forward_layers(net, nx, ny, nz)) return rc;
    if (r_dev) RCK(cudaMemcpyAsync(r_dev, net->r, n * 3 * sizeof(float), cudaMemcpyDeviceToDevice, net->s));
    RCK(cudaGetLastError());
    net->nx = nx;
    net->ny = ny;
    net->nz = nz;
    return MMX_OK;
}

extern "C" int mmx_rnet_train_step(mmx_rnet *net, int nx, int ny, int nz, const float *x_dev,
                                   const float *target_dev, float lr, double *loss_out)
{
    if (!net || !x_dev || !target_dev) return rfail(net, MMX_ERR_ARG, "NULL argument");
    if (!(lr > 0.0f)) return rfail(net, MMX_ERR_ARG, "learning rate must be positive");
    if (int rc = mmx_rnet_forward(net, nx, ny, nz, x_dev, nullptr)) return rc;
    const long long n = (long long)nx * ny * nz;
    cudaStream_t s = net->s;
    RCK(cudaMemsetAsync(net->loss_d, 0, sizeof(double), s));
    RCK(cudaMemsetAsync(net->grad, 0, MMX_RNET_PARAMS * sizeof(float), s));
    k_rnet_loss<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(net->r, target_dev, n, net->dz3, net->dz3b,
                                                           net->loss_d);
    // input gradients on the tensor cores (dz rounded to BF16 where it enters);
    // weight gradients on the tensor cores (dz as a BF16 pair hi + lo)
    if (!halo_maps(net, nx, ny, nz))
        return rfail(net, MMX_ERR_CUDA, "the tensor maps of the layer inputs could not be encoded");
    const long long tiles = (long long)((nx + TC_TX - 1) / TC_TX) * ((ny + RN_TY - 1) / RN_TY) * nz;
    long long gcap_bwd = 2LL * net->nsm;
    if (net->grid_cap > 0 && net->grid_cap < gcap_bwd) gcap_bwd = net->grid_cap;
    const dim3 gt((unsigned)(tiles < gcap_bwd ? tiles : gcap_bwd));
    float *G = net->grad;
    // layer 3 (32 -> 3)
    wgrad_layer<32, 8>(net, net->dz3, net->a[3], 32, 3, G + p_off(3), nx, ny, nz);
    k_rnet_conv_tc<16, 32, 2><<<gt, 128, tc_smem(16, 32), s>>>(net->tmg[0], net->Wtt, nullptr, 32, net->dzA, nx, ny,
                                                               nz, net->fault, net->a[3], net->dzAb);
    // layer 2
    wgrad_layer<32, 32>(net, net->dzA, net->a[2], 32, 32, G + p_off(2), nx, ny, nz);
    k_rnet_conv_tc<32, 32, 2><<<gt, 128, tc_smem(32, 32), s>>>(net->tmg[1], net->Wtt + TT2, nullptr, 32, net->dzB,
                                                               nx, ny, nz, net->fault, net->a[2], net->dzBb);
    // layer 1
    wgrad_layer<32, 32>(net, net->dzB, net->a[1], 32, 32, G + p_off(1), nx, ny, nz);
    k_rnet_conv_tc<32, 32, 2><<<gt, 128, tc_smem(32, 32), s>>>(net->tmg[2], net->Wtt + TT1, nullptr, 32, net->dzA,
                                                               nx, ny, nz, net->fault, net->a[1], net->dzAb);
    // layer 0 (6 -> 32; input padded to 16 channels)
    wgrad_layer<16, 32>(net, net->dzA, net->a[0], 6, 32, G + p_off(0), nx, ny, nz);
    net->step++;
    const double c1 = 1.0 / (1.0 - pow(0.9, net->step)), c2 = 1.0 / (1.0 - pow(0.999, net->step));
    k_rnet_adam<<<(MMX_RNET_PARAMS + 255) / 256, 256, 0, s>>>(net->P, net->Pm, net->Pv, G, MMX_RNET_PARAMS, lr,
                                                               (float)c1, (float)c2);
    if (int rc = refresh_weights(net)) return rc;
    RCK(cudaGetLastError());
    if (loss_out) {
        double l = 0.0;
        RCK(cudaMemcpyAsync(&l, net->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
        RCK(cudaStreamSynchronize(s));
        if (int rc = check_fault(net)) return rc;
        *loss_out = l / (3.0 * (double)n);
    }
    return MMX_OK;
}

extern "C" int mmx_rnet_get_grads(mmx_rnet *net, float *grads_host)
{
    if (!net || !grads_host) return rfail(net, MMX_ERR_ARG, "NULL argument");
    RCK(cudaMemcpyAsync(grads_host, net->grad, MMX_RNET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, net->s));
    RCK(cudaStreamSynchronize(net->s));
    return check_fault(net);
}

extern "C" int mmx_rnet_get_activation(mmx_rnet *net, int layer, void *dst_host, size_t bytes)
{
    if (!net || !dst_host || layer < 0 || layer > NLAYER) return rfail(net, MMX_ERR_ARG, "invalid argument");
    const size_t n = (size_t)net->nx * net->ny * net->nz;
    if (n == 0) return rfail(net, MMX_ERR_STATE, "no forward pass yet");
    const size_t want = layer == NLAYER ? n * 3 * sizeof(float) : n * (layer == 0 ? 16 : 32) * 2;
    if (bytes != want) return rfail(net, MMX_ERR_ARG, "size does not match the last forward pass");
    const void *src = layer == NLAYER ? (const void *)net->r : (const void *)net->a[layer];
    RCK(cudaMemcpyAsync(dst_host, src, bytes, cudaMemcpyDeviceToHost, net->s));
    RCK(cudaStreamSynchronize(net->s));
    return check_fault(net);
}

extern "C" const char *mmx_rnet_last_error(const mmx_rnet *net)
{
    return net ? net->err.c_str() : "";
}

extern "C" void mmx_rnet_destroy(mmx_rnet *net)
{
    if (!net) return;
    if (net->s) cudaStreamSynchronize(net->s);
    void *bufs[] = {net->P,   net->Pm,  net->Pv,  net->grad, net->part, net->a[0],  net->a[1], net->a[2],
                    net->a[3], net->r, net->dz3, net->dzA,  net->dzB, net->loss_d, net->fault, net->Wtc,
                    net->Wtt,  net->dz3b, net->dzAb, net->dzBb};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete net;
}

extern "C" int mmx_residual_sample(mmx_ctx *c, int p, const void *m_nodes_dev, const double *t_nodes,
                                   const void *m_dev, double t, float *x_dev, float *target_dev)
{
    if (!c) return MMX_ERR_ARG;
    if (p < 0 || p > 5 || !m_nodes_dev || !t_nodes || !m_dev || !x_dev || !target_dev) {
        c->err = "mmx_residual_sample: invalid argument";
        return MMX_ERR_ARG;
    }
    const size_t field_bytes = (size_t)3 * c->n * c->esz;
    for (int i = 0; i <= p; ++i)
        if (((uintptr_t)m_nodes_dev + i * field_bytes) % 16 != 0) {
            c->err = "mmx_residual_sample: every node field must start on a 16-byte boundary";
            return MMX_ERR_ARG;
        }
    if ((uintptr_t)m_dev % 16 != 0 || (uintptr_t)x_dev % 16 != 0 || (uintptr_t)target_dev % 16 != 0) {
        c->err = "mmx_residual_sample: arrays must start on a 16-byte boundary";
        return MMX_ERR_ARG;
    }
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j < i; ++j)
            if (!(t_nodes[i] != t_nodes[j])) {
                c->err = "mmx_residual_sample: node times must be distinct";
                return MMX_ERR_ARG;
            }
    return c->prec == MMX_FP64 ? sample_t<double>(c, p, m_nodes_dev, t_nodes, m_dev, t, x_dev, target_dev)
                               : sample_t<float>(c, p, m_nodes_dev, t_nodes, m_dev, t, x_dev, target_dev);
}

int mmxk_rnet_stage(mmx_rnet *net, mmx_ctx *c, cudaStream_t s, int k)
{
    const long long n = c->n;
    cudaStream_t keep = net->s;
    int *keep_fault = net->fault;
    net->s = s;  // the context's stream, possibly being captured
    // the layers report an expired bounded wait through the context's fault
    // word, which the controller and every state read of the context check
    net->fault = &c->st->fault;
    k_res_stage_in<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->st, k, c->ctl.p + 1, (const float *)c->hist,
                                                             (const float *)c->Y[k & 1], n, (float)(1.0 / c->mat.Ms),
                                                             (float *)c->G, net->a[0], 1);
    (void)forward_layers(net, c->nx, c->ny, c->nz);  // cannot fail: the maps were encoded at attach time
    k_res_stage_out<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(c->st, net->r, 3 * n, (float)c->mat.Ms,
                                                                  (float *)c->G);
    net->s = keep;
    net->fault = keep_fault;
    net->nx = c->nx;
    net->ny = c->ny;
    net->nz = c->nz;
    return 6;
}

int mmxk_rnet_check(mmx_rnet *net, mmx_ctx *c, cudaStream_t s, int k)
{
    const long long n = c->n;
    cudaStream_t keep = net->s;
    int *keep_fault = net->fault;
    net->s = s;
    net->fault = &c->st->fault;
    k_res_stage_in<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->st, k, c->ctl.p + 1, (const float *)c->hist,
                                                             (const float *)c->Y[k & 1], n, (float)(1.0 / c->mat.Ms),
                                                             (float *)c->Gc, net->a[0], 0);
    (void)forward_layers(net, c->nx, c->ny, c->nz);  // cannot fail: the maps were encoded at attach time
    k_res_check_cmp<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(c->st, net->r, (const float *)c->Gc,
                                                                  (const float *)c->G, 3 * n, (float)c->mat.Ms);
    net->s = keep;
    net->fault = keep_fault;
    net->nx = c->nx;
    net->ny = c->ny;
    net->nz = c->nz;
    return 6;
}

extern "C" int mmx_set_residual(mmx_ctx *c, mmx_rnet *net)
{
    if (!c) return MMX_ERR_ARG;
    if (net) {
        if (c->prec != MMX_FP32_MIXED) {
            c->err = "mmx_set_residual: the learned residual runs with FP32 fields only";
            return MMX_ERR_ARG;
        }
        if (c->ctl.p < 0) {
            c->err = "mmx_set_residual: the context does not extrapolate (extrap_order < 0)";
            return MMX_ERR_ARG;
        }
        if (c->n > net->max_cells) {
            c->err = "mmx_set_residual: the mesh has more cells than the net was created for";
            return MMX_ERR_ARG;
        }
        if (!halo_maps(net, c->nx, c->ny, c->nz)) {
            c->err = "mmx_set_residual: the tensor maps of the net's layer inputs could not be encoded";
            return MMX_ERR_CUDA;
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("mmx_set_residual: ") + cudaGetErrorString(e);
        return MMX_ERR_CUDA;
    }
    if (net && !c->Gc && cudaMalloc(&c->Gc, (size_t)3 * c->n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        c->Gc = nullptr;
        c->err = "mmx_set_residual: device allocation failed";
        return MMX_ERR_OOM;
    }
    // the captured attempt graphs hold the old stage sequence
    mmx_drop_graphs(c);
    c->rnet = net;
    c->ctl.has_net = net ? 1 : 0;
    // the next attempt uses the net; the periodic check starts afresh
    if (int rc = mmx_state_edit(c, [](DevState &st) {
            st.mode_next = 0;
            st.att_mode = 0;
            st.since_check = 0;
            st.net_ok = 1;
            st.check_num_bits = 0u;
            st.check_den_bits = 0u;
        }))
        return rc;
    return MMX_OK;
}

extern "C" int mmx_set_residual_check(mmx_ctx *c, int every, double tol)
{
    if (!c) return MMX_ERR_ARG;
    if (every < 0 || !(tol >= 0) || !std::isfinite(tol)) {
        c->err = "mmx_set_residual_check: need every >= 0 and a finite tol >= 0";
        return MMX_ERR_ARG;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("mmx_set_residual_check: ") + cudaGetErrorString(e);
        return MMX_ERR_CUDA;
    }
    mmx_drop_graphs(c);
    c->ctl.check_every = every;
    c->ctl.check_tol = tol;
    return MMX_OK;
}

extern "C" int mmx_residual_stats(mmx_ctx *c, long long *out4)
{
    if (!c || !out4) return MMX_ERR_ARG;
    DevState st;
    if (int rc = mmx_state_read(c, &st)) return rc;
    out4[0] = st.fallbacks;
    out4[1] = st.checks;
    out4[2] = st.check_fails;
    out4[3] = st.net_ok;
    return MMX_OK;
}
