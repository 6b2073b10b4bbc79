// internal.h -- definitions shared by the host and device parts of libmmx.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/mmx.h"

#define MMX_MAXS 8
#define MMX_MAXP 6
#define MMX_NHIST (MMX_MAXP + 1)

// Coefficients of one stage for the current attempt, prepared by one CTA
// (at the end of the previous attempt, or before the first one) so that the
// stage kernels do no FP64 arithmetic.  `state` republishes the words of the
// attempt's state that the stage kernels need, beside their coefficients, so
// that one uniform load brings both.
struct StageCoef {
    double cb[MMX_MAXS];       // h b_{k+1,l}; at the last stage h c_l
    double ce[MMX_MAXS];       // at the last stage h (c_l - c_hat_l)
    double w[MMX_NHIST + 1];   // Eq. 6 Lagrange weights at t0 + a_k h (one pad word)
    double H[4];               // applied field at t0 + a_k h (one pad word)
    float cbf[MMX_MAXS], cef[MMX_MAXS];
    float wf[MMX_NHIST + 1], Hf[4];
    float pad_[8];
    int state[8];              // done, cur, fbase, head, f1_valid (copies; see publish_state)
};

// Integrator state kept in device memory; kernels read it at launch and the
// controller kernel that ends each attempt updates it.  Everything the host
// needs to resume a run lives here.
struct DevState {
    double t;        // start time t0 of the current attempt
    double h;        // step of the current attempt (possibly clipped)
    double h_ctrl;   // step proposed by the controller (Eq. 5)
    double t_end;
    double last_err;
    double h_prev;   // ABM2: last accepted step (0 after a (re)start)
    double hist_t[MMX_NHIST];   // times of the stored exact fields (Eq. 6)
    int cur;         // which magnetisation buffer holds m0
    int fbase;       // slot of F_1 in the stage-derivative ring (FSAL rotation)
    int f1_valid;    // F_1 for this t0 already computed
    int hist_n;      // history slots assigned (<= p+1), incl. the current t0
    int head;        // slot of the current t0
    int done;
    int status;
    int clipped;     // current attempt lands exactly on t_end
    int loop_more;   // last value handed to the graph's while condition
    // learned residual attached: which attempt body runs (0 the net at the
    // extrapolated stages, 1 exact demag at every stage, 2 exact with the
    // net checked at stage 2), chosen by the controller for the next attempt
    int att_mode;    // body of the current attempt (set by the gate kernel)
    int mode_next;
    int since_check; // accepted steps since the last periodic check
    int net_ok;      // the last check was within tolerance
    unsigned int check_num_bits, check_den_bits;  // check: max |G_net - G|, max |G| (FP32 bits)
    long long fallbacks, checks, check_fails;
    long long accepted, rejected, exact_evals, extrap_evals, forced, attempts;
    long long acc_target;     // stop when accepted reaches this
    long long attempt_limit;  // attempts allowed in the current run
    long long run_attempts;
    long long prime_attempts;  // attempts made by priming loops (launch accounting)
    unsigned long long t_start_ns, time_limit_ns;
    StageCoef coef[MMX_MAXS];  // everything before coef is the "head" the controller copies
    // outside the head (the controller never writes these back):
    int spec_src;  // m buffer the attempt's new state went to (the speculative demag passes read it)
    int fault;     // a bounded device wait gave up (the context is unusable); sticky
    int pad_[2];
};

static_assert(sizeof(DevState) % 8 == 0, "DevState is copied as 8-byte words");
static_assert(offsetof(DevState, coef) % 16 == 0 && sizeof(StageCoef) % 16 == 0,
              "stage coefficients are read with 16-byte loads");

struct TabArgs {
    int s, order, adaptive, fsal;
    int abm;  // Adams-Bashforth-Moulton 2: coefficients per attempt, F_{n-1} in slot s
    double a[MMX_MAXS];
    double b[MMX_MAXS][MMX_MAXS];
    double c[MMX_MAXS];
    double e[MMX_MAXS];  // c - c_hat
};

struct PhysArgs {
    int nx, ny, nz;
    long long n;
    double wx, wy, wz;   // 2A/(mu0 Ms d^2) per axis
    double can;          // 2K/(mu0 Ms)
    double ku[3];
    double gp;           // gamma / (1 + alpha^2)
    double alpha;
    double msN00[3];     // Ms * N00 (self demag)
    double H0[3], pulse[3], t_on, t_off;
};

struct CtlArgs {
    int p;         // extrapolation order, -1 = full
    int adaptive;  // controller enabled (integrator flag and tableau)
    int nslots;    // stage-derivative slots
    int prime;     // this graph primes the history: stop once primed
    double tol, hmin, hmax, cmin, cmax, safety;
    double cmin_pow, cmax_pow;  // cmin^(n+1), cmax^(n+1): clamp limits of Eq. 5
    int has_net;       // a learned residual is attached: choose the next attempt's body
    int check_every;   // periodic exact check every this many accepted steps (0: none)
    double check_tol;  // check: max |G_net - G| <= check_tol max |G|
};

struct mmx_ctx {
    mmx_mesh mesh;
    mmx_material mat;
    mmx_field field;
    mmx_integrator integ;
    int prec;  // mmx_precision
    size_t esz;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    cudaStream_t cap_stream2;       // second capture stream: the speculative demag passes
    cudaStream_t cap_stream3;       // capture of the conditional attempt bodies (learned residual)
    void *Gc;                       // learned residual's check: the net-corrected field at stage 2
    cudaEvent_t ev_fork, ev_join;   // fork and join of the two capture streams
    int nx, ny, nz;
    long long n;
    int Px, Py, Pz, Hy, Hz;
    long long rows;  // 3 * ny * nz
    double N00[3];
    TabArgs tab;
    PhysArgs ph;
    CtlArgs ctl;
    // device buffers (element type per precision)
    void *m[2], *Y[2], *F, *G, *hist, *S, *K, *twx, *twy, *twz;
    void *mlo;   // FP32: low words of the compensated state of m[0] and m[1] ([2][3][n]); null in FP64
    void *errpart;  // largest error norm of each CTA of the last stage
    void *Tb;    // split y/z path: y spectrum [kx][c nz + z][Py] (complex)
    void *tw4 = nullptr;  // FP32 split path with a 1024-point axis: four-step twiddles [k2][n1] = w1024^(n1 k2)
    bool r4 = false;      // the 1024-point y passes run as four-step register transforms
    bool r4x = false;     // ... and the 1024-point x passes
    void *tw512 = nullptr;  // FP32 with a 512-point x axis: four-step twiddles [k2][n1] = w512^(n1 k2), k2 < 16
    bool r4xh = false;      // the 512-point x-forward pass runs as a four-step register transform
    bool r4xih = false;     // ... and the 512-point x-inverse pass
    void *tw4y = nullptr;   // FP32 fused y-z pass with Py = 256: four-step twiddles [k2][n1] = w256^(n1 k2)
    bool split;  // the y-z column does not fit one CTA: YF, ZM, YI instead of YZ
    int nd;           // kernels per exact demag evaluation
    bool allow_tma;   // TMA passes allowed (the context owns a fault word)
    bool stall_test;  // MMX_TEST_STALL_TMA: the TMA XI's waits run out (failure-path test)
    bool xi_tma_ok;   // the TMA XI is set up for this mesh
    bool xi_tma;      // XI runs with TMA tile loads
    int trows;        // rows per CTA of the plain x passes
    bool tuned;       // pass configuration chosen by timing (autotuner)
    double demag_us;  // timed exact evaluation of the chosen configuration
    CUtensorMap xi_tmap;  // the x spectrum S as [nx][rows] 8-byte words
    DevState *st;
    DevState *h_st;  // pinned host mirror
    // graphs: [0] main loop, [1] priming loop
    cudaGraphExec_t gexec[2];
    cudaGraph_t graph[2];
    bool graph_ok[2];
    struct mmx_rnet *rnet = nullptr;  // learned residual at the extrapolated stages (mmx_set_residual)
    bool use_graphs;
    // profiling: an event pair around every timed launch.  Outside a graph
    // the pair is synchronised at once; runs capture each attempt once more
    // as a graph with event-record nodes around every kernel (pgexec, per
    // loop kind) and read the pairs after each launch, so that the times are
    // those of kernels running back to back on the device.
    bool profiling;
    // mode 2: the stage kernels of an extrapolated attempt that run back to
    // back (every stage but the last, no demag pass between them) share one
    // event pair, which then counts all of their launches
    bool prof_group = false;
    double prof_ms[MMX_NPROF];
    long long prof_n[MMX_NPROF];
    cudaEvent_t ev_a, ev_b;
    int prof_cap = -1;                 // loop kind whose profiled graph is being captured, else -1
    std::vector<cudaEvent_t> pev[2];   // event pairs of the profiled graphs
    std::vector<int> pcls[2];          // profile class of each pair
    std::vector<int> pcnt[2];          // launches each pair spans
    cudaGraphExec_t pgexec[2];
    cudaGraph_t pgraph[2];
    bool pgraph_ok[2] = {false, false};
    long long launches;
    long long launches_dev_at_sync;
    std::string err;
};

// mmx_api.cu: profiling event pairs (see mmx_ctx::prof_cap) and dropping
// the captured graphs (after the stage sequence changed, and at destroy)
void mmx_prof_begin(mmx_ctx *c, cudaStream_t s);
void mmx_prof_end(mmx_ctx *c, cudaStream_t s, int cls, int count = 1);
void mmx_drop_graphs(mmx_ctx *c);
// kernels.cu: stage S-2 writes the new state (and the speculative demag
// passes fork after it): an FSAL tableau, whose last-stage input Y_S is the
// Eq. 3 solution, on a mesh with the fused y-z pass
bool mmxk_early_solution(const mmx_ctx *c);
// synchronises the context and applies f to its device state (read, edit,
// write back); a copy of the state for reading only
#include <functional>
int mmx_state_edit(mmx_ctx *c, const std::function<void(DevState &)> &f);
int mmx_state_read(mmx_ctx *c, DevState *out);

// kernels.cu
int mmxk_setup_buffers(mmx_ctx *c, const double *Kspec_host);
// one exact Eq. 2 evaluation: XF -> YZ -> XI
//   stage0: skip when F_1 is still valid (rejected retry / FSAL)
//   src_mode 0: src, 1: m[cur];  dst_mode 0: dst, 1: history slot head
//   self_src != NULL: subtract Ms N00 self_src (full field, as in mmx_demag)
void mmxk_demag(mmx_ctx *c, cudaStream_t s, const DevState *st, int stage0, int src_mode,
                const void *src, int dst_mode, void *dst, const void *self_src);
// the same passes, a subset of them: parts = 1 (x forward) | 2 (y-z, tensor
// multiply) | 4 (x inverse); src_mode 2 reads m[spec_src]
void mmxk_demag_parts(mmx_ctx *c, cudaStream_t s, const DevState *st, int stage0, int src_mode, const void *src,
                      int dst_mode, void *dst, const void *self_src, int parts);
// the controller kernel that ends every attempt
void mmxk_control(mmx_ctx *c, cudaStream_t s, int prime_graph, cudaGraphConditionalHandle cond, int use_cond);
void mmxk_stage(mmx_ctx *c, cudaStream_t s, int k, int extrap, int prime_graph,
                cudaGraphConditionalHandle cond, int use_cond);
// stage_f32.cu / stage_f64.cu: the stage kernel instance for nf stage
// derivatives and nh demag sources read, and the controller kernel
const void *mmxk_stage_kernel(bool f64, int nf, int nh, bool last, bool stage0);
const void *mmxk_control_kernel(bool f64);
// rows per CTA of the plain x passes: the default, and setting a candidate
// (raises the kernels' shared-memory limit; MMX_ERR_ARG if it does not fit)
int mmxk_default_trows(const mmx_ctx *c);
// longest z transform of the fused y-z pass (its z columns are held in
// registers); taller meshes take the split passes
int mmxk_yz_max_pz(const mmx_ctx *c);
int mmxk_set_trows(mmx_ctx *c, int trows);
// fills DevState::coef for the attempt described by the device state
void mmxk_prepare(mmx_ctx *c, cudaStream_t s);
// batched runs: the same preparation as an explicit graph node, and a node
// that sets a loop's while condition from the device state
// the learned residual at stage k of an extrapolated attempt: G = G_ext + Ms r
// into c->G (launched on s); returns the number of kernels launched
int mmxk_rnet_stage(struct mmx_rnet *net, mmx_ctx *c, cudaStream_t s, int k);
// the periodic check at stage k of an exact attempt: the net's corrected
// field G_ext + Ms r against the exact G (maxima into the state); kernels launched
int mmxk_rnet_check(struct mmx_rnet *net, mmx_ctx *c, cudaStream_t s, int k);
// the gate at the top of an attempt body with the learned residual: makes
// the chosen body current and sets the three bodies' conditions
void mmxk_mode_gate(mmx_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1,
                    cudaGraphConditionalHandle h2, int use);
int mmxk_add_prepare_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, mmx_ctx *c, cudaGraphNode_t *out);
int mmxk_add_gate_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, mmx_ctx *c,
                       cudaGraphConditionalHandle h, int prime_loop, cudaGraphNode_t *out);
