// kernels.cu -- host entry points of the kernel layer of libmmx: precision
// dispatch, the kernel-pointer table over the translation units that hold the
// FFT kernel families, and the stage kernels (instantiated here).
#include "kernels_impl.cuh"

const void *mmxk_tab_fused(int kind, bool f64, int L);  // fft_fused_f32.cu / fft_fused_f64.cu
const void *mmxk_tab_split(int kind, bool f64, int L);  // fft_split.cu
const void *mmxk_tab_pipe(int kind, bool f64, int L);   // fft_pipe.cu

const void *mmxk_stage_tab_f32(int nf, int nh, bool last, bool stage0);  // stage_f32.cu
const void *mmxk_stage_tab_f64(int nf, int nh, bool last, bool stage0);  // stage_f64.cu
const void *mmxk_control_f32();
const void *mmxk_control_f64();

const void *mmxk_stage_kernel(bool f64, int nf, int nh, bool last, bool stage0)
{
    return f64 ? mmxk_stage_tab_f64(nf, nh, last, stage0) : mmxk_stage_tab_f32(nf, nh, last, stage0);
}

const void *mmxk_control_kernel(bool f64) { return f64 ? mmxk_control_f64() : mmxk_control_f32(); }

const void *mmxk_kernel(int kind, bool f64, int L)
{
    switch (kind) {
    case K_XF:
    case K_XI:
    case K_YZ: return mmxk_tab_fused(kind, f64, L);
    case K_YF:
    case K_YI:
    case K_ZM:
    case K_ZMR: return mmxk_tab_split(kind, f64, L);
    default: return mmxk_tab_pipe(kind, f64, L);
    }
}


bool mmxk_early_solution(const mmx_ctx *c)
{
    // FSAL: the last Eq. 4 row equals the Eq. 3 weights and c_S = 0.  Only
    // where the passes are latency-bound (the fused y-z pass: the column fits
    // one CTA): on meshes with the split passes the stage kernels and the
    // passes are HBM-bound, and running the passes beside the last stage
    // measured slower (512 x 512 x 16, RK23 p = 2: 0.645 -> 0.682 ms per step)
    const TabArgs &t = c->tab;
    const int S = t.s;
    if (c->split || t.abm || !t.fsal || S < 2 || t.c[S - 1] != 0.0) return false;
    for (int l = 0; l < S - 1; ++l)
        if (t.b[S - 1][l] != t.c[l]) return false;
    return true;
}

void mmxk_prepare(mmx_ctx *c, cudaStream_t s)
{
    k_prepare<<<1, 256, 0, s>>>(c->st, c->tab, c->ph, c->ctl.p);
    c->launches++;
}

// Top of an attempt body with the learned residual: the body the controller
// chose becomes the current one, and exactly one body's condition is set.
__global__ void k_mode_gate(DevState *st, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1,
                            cudaGraphConditionalHandle h2, int use)
{
    const int mode = st->done ? -1 : st->mode_next;
    if (mode >= 0) st->att_mode = mode;
    if (use) {
        cudaGraphSetConditional(h0, mode == 0 ? 1u : 0u);
        cudaGraphSetConditional(h1, mode == 1 ? 1u : 0u);
        cudaGraphSetConditional(h2, mode == 2 ? 1u : 0u);
    }
}

void mmxk_mode_gate(mmx_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1,
                    cudaGraphConditionalHandle h2, int use)
{
    k_mode_gate<<<1, 1, 0, s>>>(c->st, h0, h1, h2, use);
    c->launches++;
}

// Sets the while condition of one loop of a batched run from the device state
// before the loop starts: a member that is done, or (priming loop) already
// primed, skips the loop.  Batched graphs do not reset conditions at launch.
__global__ void k_gate(const DevState *st, int p, int prime_loop, cudaGraphConditionalHandle h)
{
    const bool run = !st->done && (!prime_loop || st->hist_n < p + 1);
    cudaGraphSetConditional(h, run ? 1u : 0u);
}

static int add_kernel_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, const void *fn, dim3 grid,
                           dim3 block, void **args, cudaGraphNode_t *out)
{
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(fn);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, nd, &kp) == cudaSuccess ? 0 : MMX_ERR_CUDA;
}

int mmxk_add_prepare_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, mmx_ctx *c, cudaGraphNode_t *out)
{
    DevState *st = c->st;
    TabArgs tab = c->tab;
    PhysArgs ph = c->ph;
    int p = c->ctl.p;
    void *args[] = {&st, &tab, &ph, &p};
    return add_kernel_node(g, deps, nd, (const void *)k_prepare, dim3(1), dim3(256), args, out);
}

int mmxk_add_gate_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, mmx_ctx *c,
                       cudaGraphConditionalHandle h, int prime_loop, cudaGraphNode_t *out)
{
    const DevState *st = c->st;
    int p = c->ctl.p;
    void *args[] = {&st, &p, &prime_loop, &h};
    return add_kernel_node(g, deps, nd, (const void *)k_gate, dim3(1), dim3(1), args, out);
}

int mmxk_default_trows(const mmx_ctx *c) { return pick_trows(c); }

int mmxk_set_trows(mmx_ctx *c, int tr)
{
    const bool f64 = c->prec == MMX_FP64;
    const size_t xs = f64 ? x_smem<double>(c, tr) : x_smem<float>(c, tr);
    if (tr < 1 || tr > 16 || xs > 200 * 1024) return MMX_ERR_ARG;
    if (xs > 48 * 1024)
        for (int kind : {(int)K_XF, (int)K_XI})
            if (!raise_smem_limit(mmxk_kernel(kind, f64, c->Px), xs)) return MMX_ERR_CUDA;
    c->trows = tr;
    return 0;
}

size_t mmxk_split_smem_bytes(const mmx_ctx *c)
{
    if (c->prec == MMX_FP64) return std::max(yf_smem<double>(c, split_rows<double>(c)), zm_smem<double>(c));
    return std::max(yf_smem<float>(c, split_rows<float>(c)), zm_smem<float>(c));
}

int mmxk_yz_max_pz(const mmx_ctx *c) { return c->prec == MMX_FP64 ? reg_max_len<double>() : reg_max_len<float>(); }

size_t mmxk_yz_smem_bytes(const mmx_ctx *c)
{
    return c->prec == MMX_FP64 ? yz_smem<double>(c) : yz_smem<float>(c);
}
size_t mmxk_x_smem_bytes(const mmx_ctx *c)
{
    const int tr = c->trows ? c->trows : pick_trows(c);
    return c->prec == MMX_FP64 ? x_smem<double>(c, tr) : x_smem<float>(c, tr);
}

int mmxk_setup_buffers(mmx_ctx *c, const double *Kspec_host)
{
    return c->prec == MMX_FP64 ? setup_t<double>(c, Kspec_host) : setup_t<float>(c, Kspec_host);
}

void mmxk_demag_parts(mmx_ctx *c, cudaStream_t s, const DevState *st, int stage0, int src_mode, const void *src,
                      int dst_mode, void *dst, const void *self_src, int parts)
{
    if (c->prec == MMX_FP64)
        demag_t<double>(c, s, st, stage0, src_mode, src, dst_mode, dst, self_src, parts);
    else
        demag_t<float>(c, s, st, stage0, src_mode, src, dst_mode, dst, self_src, parts);
}

void mmxk_demag(mmx_ctx *c, cudaStream_t s, const DevState *st, int stage0, int src_mode, const void *src,
                int dst_mode, void *dst, const void *self_src)
{
    mmxk_demag_parts(c, s, st, stage0, src_mode, src, dst_mode, dst, self_src, 7);
}

void mmxk_control(mmx_ctx *c, cudaStream_t s, int prime_graph, cudaGraphConditionalHandle cond, int use_cond)
{
    if (c->prec == MMX_FP64)
        control_t<double>(c, s, prime_graph, cond, use_cond);
    else
        control_t<float>(c, s, prime_graph, cond, use_cond);
}

void mmxk_stage(mmx_ctx *c, cudaStream_t s, int k, int extrap, int prime_graph, cudaGraphConditionalHandle cond,
                int use_cond)
{
    if (c->prec == MMX_FP64)
        stage_t<double>(c, s, k, extrap, prime_graph, cond, use_cond);
    else
        stage_t<float>(c, s, k, extrap, prime_graph, cond, use_cond);
}
