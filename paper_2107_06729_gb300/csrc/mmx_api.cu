// mmx_api.cu -- C ABI of libmmx (declared in include/mmx.h).
//
// The integration loop runs on the device: one CUDA graph holds a
// conditional WHILE node whose body is one attempted step (Eq. 3-4 stages,
// demag FFTs where the schedule needs them); the controller kernel of Eq. 5
// that ends each attempt decides acceptance, the next step and whether the
// loop continues.  A second graph with full demag at every stage primes the
// extrapolation history (the first p steps, Sec. II after Eq. 6).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "tensor_host.h"

size_t mmxk_yz_smem_bytes(const mmx_ctx *c);
size_t mmxk_x_smem_bytes(const mmx_ctx *c);
size_t mmxk_split_smem_bytes(const mmx_ctx *c);

namespace {

thread_local std::string g_create_err;

// Butcher tableaux of the methods of Sec. II (refs. [26]-[31]) as exact
// fractions: rows of (numerator, denominator).
struct Frac {
    double n, d;
};

struct MethodDef {
    int s, order, adaptive, fsal;
    std::vector<Frac> a;
    std::vector<std::vector<Frac>> b;
    std::vector<Frac> c, chat;
};

MethodDef method_def(int m)
{
    MethodDef d{};
    switch (m) {
    case MMX_RK4:
        d = {4, 4, 0, 0, {{0, 1}, {1, 2}, {1, 2}, {1, 1}},
             {{}, {{1, 2}}, {{0, 1}, {1, 2}}, {{0, 1}, {0, 1}, {1, 1}}},
             {{1, 6}, {1, 3}, {1, 3}, {1, 6}},
             {{1, 6}, {1, 3}, {1, 3}, {1, 6}}};
        break;
    case MMX_HEUN12:
        d = {2, 2, 1, 0, {{0, 1}, {1, 1}}, {{}, {{1, 1}}}, {{1, 2}, {1, 2}}, {{1, 1}, {0, 1}}};
        break;
    case MMX_RK23_BS:
        d = {4, 3, 1, 1, {{0, 1}, {1, 2}, {3, 4}, {1, 1}},
             {{}, {{1, 2}}, {{0, 1}, {3, 4}}, {{2, 9}, {1, 3}, {4, 9}}},
             {{2, 9}, {1, 3}, {4, 9}, {0, 1}},
             {{7, 24}, {1, 4}, {1, 3}, {1, 8}}};
        break;
    case MMX_RKF45:
        d = {6, 4, 1, 0, {{0, 1}, {1, 4}, {3, 8}, {12, 13}, {1, 1}, {1, 2}},
             {{},
              {{1, 4}},
              {{3, 32}, {9, 32}},
              {{1932, 2197}, {-7200, 2197}, {7296, 2197}},
              {{439, 216}, {-8, 1}, {3680, 513}, {-845, 4104}},
              {{-8, 27}, {2, 1}, {-3544, 2565}, {1859, 4104}, {-11, 40}}},
             {{25, 216}, {0, 1}, {1408, 2565}, {2197, 4104}, {-1, 5}, {0, 1}},
             {{16, 135}, {0, 1}, {6656, 12825}, {28561, 56430}, {-9, 50}, {2, 55}}};
        break;
    case MMX_RKCK45:
        d = {6, 4, 1, 0, {{0, 1}, {1, 5}, {3, 10}, {3, 5}, {1, 1}, {7, 8}},
             {{},
              {{1, 5}},
              {{3, 40}, {9, 40}},
              {{3, 10}, {-9, 10}, {6, 5}},
              {{-11, 54}, {5, 2}, {-70, 27}, {35, 27}},
              {{1631, 55296}, {175, 512}, {575, 13824}, {44275, 110592}, {253, 4096}}},
             {{2825, 27648}, {0, 1}, {18575, 48384}, {13525, 55296}, {277, 14336}, {1, 4}},
             {{37, 378}, {0, 1}, {250, 621}, {125, 594}, {0, 1}, {512, 1771}}};
        break;
    case MMX_RKDP54:
        d = {7, 5, 1, 1, {{0, 1}, {1, 5}, {3, 10}, {4, 5}, {8, 9}, {1, 1}, {1, 1}},
             {{},
              {{1, 5}},
              {{3, 40}, {9, 40}},
              {{44, 45}, {-56, 15}, {32, 9}},
              {{19372, 6561}, {-25360, 2187}, {64448, 6561}, {-212, 729}},
              {{9017, 3168}, {-355, 33}, {46732, 5247}, {49, 176}, {-5103, 18656}},
              {{35, 384}, {0, 1}, {500, 1113}, {125, 192}, {-2187, 6784}, {11, 84}}},
             {{35, 384}, {0, 1}, {500, 1113}, {125, 192}, {-2187, 6784}, {11, 84}, {0, 1}},
             {{5179, 57600}, {0, 1}, {7571, 16695}, {393, 640}, {-92097, 339200}, {187, 2100}, {1, 40}}};
        break;
    case MMX_RKF56:
        d = {8, 5, 1, 0, {{0, 1}, {1, 6}, {4, 15}, {2, 3}, {4, 5}, {1, 1}, {0, 1}, {1, 1}},
             {{},
              {{1, 6}},
              {{4, 75}, {16, 75}},
              {{5, 6}, {-8, 3}, {5, 2}},
              {{-8, 5}, {144, 25}, {-4, 1}, {16, 25}},
              {{361, 320}, {-18, 5}, {407, 128}, {-11, 80}, {55, 128}},
              {{-11, 640}, {0, 1}, {11, 256}, {-11, 160}, {11, 256}, {0, 1}},
              {{93, 640}, {-18, 5}, {803, 256}, {-11, 160}, {99, 256}, {0, 1}, {1, 1}}},
             {{31, 384}, {0, 1}, {1125, 2816}, {9, 32}, {125, 768}, {5, 66}, {0, 1}, {0, 1}},
             {{7, 1408}, {0, 1}, {1125, 2816}, {9, 32}, {125, 768}, {0, 1}, {5, 66}, {5, 66}}};
        break;
    case MMX_ABM2:
        // stage times and order only: the predictor and error coefficients
        // depend on the step ratio and are set per attempt on the device
        d = {2, 2, 1, 0, {{0, 1}, {1, 1}}, {{}, {{1, 1}}}, {{1, 2}, {1, 2}}, {{1, 1}, {0, 1}}};
        break;
    default:
        d.s = 0;
    }
    return d;
}

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }
bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

int fail(mmx_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(mmx_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, MMX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e__ = (call);                                       \
        if (e__ != cudaSuccess) return cuda_fail(c, e__, #call);        \
    } while (0)

std::string validate(const mmx_mesh *mesh, const mmx_material *mat, const mmx_field *field,
                     const mmx_integrator *in, int precision)
{
    if (!mesh || !mat || !field || !in) return "null argument";
    if (!pow2(mesh->nx) || !pow2(mesh->ny) || !pow2(mesh->nz))
        return "mesh sizes must be powers of two";
    if (mesh->nx < 2) return "nx must be at least 2";
    if (mesh->nx > 2048 || mesh->ny > 2048 || mesh->nz > 2048) return "mesh side above 2048 cells";
    if (3.0 * mesh->nx * mesh->ny * mesh->nz >= 2147483647.0) return "mesh above 2^31/3 cells";
    if (!finite_pos(mesh->dx) || !finite_pos(mesh->dy) || !finite_pos(mesh->dz)) return "cell sizes must be > 0";
    if (!finite_pos(mat->Ms) || !finite_pos(mat->gamma)) return "Ms and gamma must be > 0";
    if (!std::isfinite(mat->A) || mat->A < 0 || !std::isfinite(mat->alpha) || mat->alpha < 0 || !std::isfinite(mat->K))
        return "A, alpha must be >= 0 and K finite";
    double ku2 = mat->ku[0] * mat->ku[0] + mat->ku[1] * mat->ku[1] + mat->ku[2] * mat->ku[2];
    if (mat->K != 0 && std::fabs(ku2 - 1.0) > 1e-9) return "anisotropy axis ku must be a unit vector";
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(field->H0[i]) || !std::isfinite(field->pulse_H[i])) return "field must be finite";
    if (std::isnan(field->t_on) || std::isnan(field->t_off)) return "pulse window must not be NaN";
    if (in->method < MMX_RK4 || in->method > MMX_ABM2) return "unknown method";
    if (in->extrap_order < -1 || in->extrap_order > MMX_MAXP) return "extrap_order must be in [-1, 6]";
    if (!finite_pos(in->h)) return "h must be > 0";
    if (in->adaptive) {
        if (!finite_pos(in->tol) || !finite_pos(in->hmin) || !finite_pos(in->hmax) || in->hmin > in->hmax)
            return "adaptive: need tol > 0 and 0 < hmin <= hmax";
        if (!finite_pos(in->cmin) || !(in->cmin <= 1.0) || !(in->cmax >= 1.0) || !std::isfinite(in->cmax))
            return "adaptive: need 0 < cmin <= 1 <= cmax";
        if (!(in->safety > 0 && in->safety <= 1)) return "adaptive: safety must be in (0, 1]";
    }
    if (precision != MMX_FP64 && precision != MMX_FP32_MIXED) return "unknown precision";
    return "";
}

int read_state(mmx_ctx *c)
{
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(c->h_st, c->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    if (c->h_st->fault) return fail(c, MMX_ERR_CUDA, "a bounded device wait gave up (a tensor copy or tensor-core operation did not complete)");
    return 0;
}

int write_state(mmx_ctx *c)
{
    CK(cudaMemcpyAsync(c->st, c->h_st, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return 0;
}

void reset_history(DevState *s)
{
    s->hist_n = 1;
    s->head = 0;
    for (int i = 0; i < MMX_NHIST; ++i) s->hist_t[i] = 0;
    s->hist_t[0] = s->t;
    s->f1_valid = 0;
    s->fbase = 0;
    s->h_prev = 0;  // ABM2 restarts with the Euler predictor
}

// Extrapolated attempts captured into a graph run speculatively: while the
// controller decides on an attempt, the x and y-z demag passes of the next
// attempt already transform the new m on a second stream (for an FSAL
// tableau on a fused-pass mesh, whose new state stage S-2 writes, already
// while the last stage runs; a rejected attempt needs no new demag: its exact
// field and F_1 are kept, and the x-inverse pass of the retry skips).  Such a body starts at
// the x-inverse pass; the
// first attempt of a loop gets its x and y-z passes from front_kernels.
bool speculative(const mmx_ctx *c, int prime) { return c->ctl.p >= 0 && !prime; }

// x and y-z demag passes of m[cur] before a speculative attempt loop (they
// skip, like the x-inverse pass, when F_1 of this t0 is still valid)
void front_kernels(mmx_ctx *c, cudaStream_t s) { mmxk_demag_parts(c, s, c->st, 1, 1, nullptr, 1, c->G, nullptr, 3); }

// One attempted step, launched on stream s.  prime: full demag at every
// stage (priming or extrap_order < 0).  s2: second capture stream of a
// speculative body (null: the whole attempt on s).
int body_kernels(mmx_ctx *c, cudaStream_t s, int prime, cudaGraphConditionalHandle cond, int use_cond,
                 cudaStream_t s2 = nullptr)
{
    const int p = c->ctl.p;
    const int extrap = (p >= 0 && !prime);
    const bool spec = s2 && speculative(c, prime);
    // stage S-2 writes the new state (FSAL tableau, fused y-z pass): the next
    // attempt's x and y-z passes then start beside the last stage, not after it
    const bool early = spec && !c->rnet && mmxk_early_solution(c);
    auto fork = [&] {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(s2, c->ev_fork, 0);
        mmxk_demag_parts(c, s2, c->st, 0, 2, nullptr, 1, c->G, nullptr, 3);
    };
    if (spec)
        mmxk_demag_parts(c, s, c->st, 1, 1, nullptr, 1, c->G, nullptr, 4);
    else
        mmxk_demag(c, s, c->st, 1, 1, nullptr, p >= 0 ? 1 : 0, c->G, nullptr);
    mmxk_stage(c, s, 0, extrap, prime && p >= 0, cond, use_cond);
    if (early && c->tab.s == 2) fork();
    for (int k = 1; k < c->tab.s; ++k) {
        if (!extrap) mmxk_demag(c, s, c->st, 0, 0, c->Y[k & 1], 0, c->G, nullptr);
        // learned residual: its kernels leave G = G_ext + Ms r in c->G, which the
        // stage then reads like an exact evaluation
        const bool res = extrap && c->rnet;
        if (res) c->launches += mmxk_rnet_stage(c->rnet, c, s, k);
        mmxk_stage(c, s, k, res ? 0 : extrap, prime && p >= 0, cond, use_cond);
        if (early && k == c->tab.s - 2) fork();
    }
    if (!spec) {
        mmxk_control(c, s, prime && p >= 0, cond, use_cond);
        return 0;
    }
    if (!early) {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(s2, c->ev_fork, 0);
    }
    mmxk_control(c, s, 0, cond, use_cond);
    if (!early) mmxk_demag_parts(c, s2, c->st, 0, 2, nullptr, 1, c->G, nullptr, 3);
    cudaEventRecord(c->ev_join, s2);
    cudaStreamWaitEvent(s, c->ev_join, 0);
    return 0;
}

// One attempt of a context with the learned residual attached, in body
// `mode`: 0 the net's correction G_ext + Ms r at the extrapolated stages,
// 1 exact demag at every stage (the fallback), 2 exact demag with the net's
// correction checked against it at stage 2 (the periodic check).  With s2
// the body is speculative (it starts at the x-inverse pass and ends with the
// controller beside the next attempt's x and y-z passes), else whole.
int res_body(mmx_ctx *c, cudaStream_t s, int mode, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s2)
{
    if (s2)
        mmxk_demag_parts(c, s, c->st, 1, 1, nullptr, 1, c->G, nullptr, 4);
    else
        mmxk_demag(c, s, c->st, 1, 1, nullptr, 1, c->G, nullptr);
    mmxk_stage(c, s, 0, 0, 0, cond, use_cond);
    for (int k = 1; k < c->tab.s; ++k) {
        if (mode == 0) {
            c->launches += mmxk_rnet_stage(c->rnet, c, s, k);
        } else {
            mmxk_demag(c, s, c->st, 0, 0, c->Y[k & 1], 0, c->G, nullptr);
            if (mode == 2 && k == 1) c->launches += mmxk_rnet_check(c->rnet, c, s, k);
        }
        mmxk_stage(c, s, k, 0, 0, cond, use_cond);
    }
    if (!s2) {
        mmxk_control(c, s, 0, cond, use_cond);
        return 0;
    }
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(s2, c->ev_fork, 0);
    mmxk_control(c, s, 0, cond, use_cond);
    mmxk_demag_parts(c, s2, c->st, 0, 2, nullptr, 1, c->G, nullptr, 3);
    cudaEventRecord(c->ev_join, s2);
    cudaStreamWaitEvent(s, c->ev_join, 0);
    return 0;
}

// The attempt body of a while loop (handle hw) of a context with the
// learned residual, built into `body`: a gate kernel, then one conditional
// IF node per body mode (exactly one of which runs), each captured from
// res_body.
int build_res_body(mmx_ctx *c, cudaGraph_t body, cudaGraphConditionalHandle hw)
{
    cudaGraphConditionalHandle hm[3];
    for (int i = 0; i < 3; ++i) CK(cudaGraphConditionalHandleCreate(&hm[i], body, 0, 0));
    CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    mmxk_mode_gate(c, c->cap_stream, hm[0], hm[1], hm[2], 1);
    cudaError_t e = cudaSuccess;
    for (int mode = 0; mode < 3 && e == cudaSuccess; ++mode) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *ed = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(c->cap_stream, &cs, nullptr, &g, &deps, &ed, &nd);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hm[mode];
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, ed, nd, &cp);
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(c->cap_stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(c->cap_stream3, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            res_body(c, c->cap_stream3, mode, hw, 1, c->cap_stream2);
            cudaGraph_t sub;
            e = cudaStreamEndCapture(c->cap_stream3, &sub);
        }
    }
    cudaGraph_t outer;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &outer);
    if (e != cudaSuccess) return cuda_fail(c, e, "attempt bodies of the learned residual");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "attempt bodies of the learned residual");
    return 0;
}

int kernels_per_attempt(const mmx_ctx *c, int prime)
{
    const int p = c->ctl.p;
    const int extrap = (p >= 0 && !prime);
    const int nd = c->nd;  // kernels per demag evaluation
    // + 1: the controller kernel after the last stage
    return extrap ? nd + c->tab.s + 1 + (c->rnet ? 6 * (c->tab.s - 1) : 0) : (nd + 1) * c->tab.s + 1;
}

int build_graph(mmx_ctx *c, int which)
{
    if (c->graph_ok[which]) return 0;
    const bool prof = c->profiling;
    c->profiling = false;
    const long long launches = c->launches;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (c->rnet && which == 0) {
        const int rc = build_res_body(c, body, h);
        if (rc) return rc;
    } else {
        CK(cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        body_kernels(c, c->cap_stream, which == 1 || c->ctl.p < 0, h, 1, c->cap_stream2);
        cudaGraph_t captured;
        CK(cudaStreamEndCapture(c->cap_stream, &captured));
    }
    c->launches = launches;
    c->profiling = prof;
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, g, 0));
    c->graph[which] = g;
    c->gexec[which] = ex;
    c->graph_ok[which] = true;
    return 0;
}

// Profiled attempt graph of loop kind `which`: the body with an event pair
// around every timed launch (no conditional node: the host reads the loop
// flag after each attempt).
int build_prof_graph(mmx_ctx *c, int which)
{
    if (c->pgraph_ok[which]) return 0;
    const long long launches = c->launches;
    c->pcls[which].clear();
    c->pcnt[which].clear();
    c->prof_cap = which;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        body_kernels(c, c->cap_stream, which == 1 || c->ctl.p < 0, 0, 0, c->cap_stream2);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->cap_stream, &g);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&c->pgexec[which], g, 0);
            if (e == cudaSuccess) c->pgraph[which] = g;
            else cudaGraphDestroy(g);
        }
    }
    c->prof_cap = -1;
    c->launches = launches;
    if (e != cudaSuccess) return cuda_fail(c, e, "profiled attempt graph");
    c->pgraph_ok[which] = true;
    return 0;
}

// Runs attempts until the device says stop (done, or primed for which = 1).
int run_loop(mmx_ctx *c, int which)
{
    const int prime = (which == 1 || c->ctl.p < 0);
    if (c->use_graphs && speculative(c, prime) && !(c->rnet && c->profiling)) {
        front_kernels(c, c->stream);
        c->launches += c->nd - 1;
    }
    if (c->rnet && which == 0 && (c->profiling || !c->use_graphs)) {
        // one attempt at a time, the body chosen on the host from the state
        for (;;) {
            mmxk_mode_gate(c, c->stream, 0, 0, 0, 0);
            res_body(c, c->stream, c->h_st->mode_next, 0, 0, nullptr);
            int rc = read_state(c);
            if (rc) return rc;
            if (!c->h_st->loop_more) return 0;
        }
    }
    if (c->use_graphs && c->profiling) {
        int rc = build_prof_graph(c, which);
        if (rc) return rc;
        for (;;) {
            CK(cudaGraphLaunch(c->pgexec[which], c->stream));
            CK(cudaStreamSynchronize(c->stream));
            const std::vector<int> &cls = c->pcls[which];
            for (size_t i = 0; i < cls.size(); ++i) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, c->pev[which][2 * i], c->pev[which][2 * i + 1]));
                c->prof_ms[cls[i]] += ms;
                c->prof_n[cls[i]] += c->pcnt[which][i];
            }
            rc = read_state(c);
            if (rc) return rc;
            c->launches += kernels_per_attempt(c, prime);
            if (!c->h_st->loop_more) return 0;
        }
    }
    if (c->use_graphs && !c->profiling) {
        int rc = build_graph(c, which);
        if (rc) return rc;
        const long long before = c->h_st->run_attempts;
        CK(cudaGraphLaunch(c->gexec[which], c->stream));
        rc = read_state(c);
        if (rc) return rc;
        c->launches += (c->h_st->run_attempts - before) * kernels_per_attempt(c, prime);
        return 0;
    }
    // one attempt at a time, synchronising to read the loop flag
    for (;;) {
        body_kernels(c, c->stream, prime, 0, 0);
        int rc = read_state(c);
        if (rc) return rc;
        if (!c->h_st->loop_more) return 0;
    }
}

// Process-wide cache of Newell tensors by mesh (the tensor does not depend on
// Ms): contexts of an ensemble that share a mesh compute it once.  Entries
// are dropped oldest first above kTensorCacheBytes.
const size_t kTensorCacheBytes = (size_t)512 << 20;

struct TensorEntry {
    int nx, ny, nz;
    double dx, dy, dz;
    std::shared_ptr<const std::vector<double>> N6;
};

std::mutex g_tensor_mu;
std::deque<TensorEntry> g_tensors;

std::shared_ptr<const std::vector<double>> tensor_for(const mmx_host_tensor_args &ta)
{
    {
        std::lock_guard<std::mutex> lk(g_tensor_mu);
        for (const TensorEntry &e : g_tensors)
            if (e.nx == ta.nx && e.ny == ta.ny && e.nz == ta.nz && e.dx == ta.dx && e.dy == ta.dy && e.dz == ta.dz)
                return e.N6;
    }
    auto N6 = std::make_shared<std::vector<double>>((size_t)6 * ta.nx * ta.ny * ta.nz);
    mmx_host_tensor(&ta, N6->data());
    const size_t bytes = N6->size() * sizeof(double);
    if (bytes <= kTensorCacheBytes / 4) {
        std::lock_guard<std::mutex> lk(g_tensor_mu);
        size_t total = bytes;
        for (const TensorEntry &e : g_tensors) total += e.N6->size() * sizeof(double);
        while (!g_tensors.empty() && total > kTensorCacheBytes) {
            total -= g_tensors.front().N6->size() * sizeof(double);
            g_tensors.pop_front();
        }
        g_tensors.push_back({ta.nx, ta.ny, ta.nz, ta.dx, ta.dy, ta.dz, N6});
    }
    return N6;
}

// ------------------------------------------------------------ autotuner
// Pass configurations of one exact demag evaluation: rows per CTA of the
// plain x passes and XI with TMA tile loads or plain.  After about 20 ms of
// warm-up evaluations, each candidate is timed twice, round robin (CUDA
// events, one warm-up and three evaluations of a seeded pseudo-random field
// on the context's own buffers), and the fastest minimum kept; results are
// cached per mesh and precision for the process.
struct Plan {
    int trows;
    bool xi_tma;
    double us;
};
struct PlanKey {
    int nx, ny, nz, prec;
    bool operator==(const PlanKey &o) const { return nx == o.nx && ny == o.ny && nz == o.nz && prec == o.prec; }
};
std::mutex g_plan_mu;
std::vector<std::pair<PlanKey, Plan>> g_plans;

double time_demag(mmx_ctx *c)
{
    mmxk_demag(c, c->stream, nullptr, 0, 0, c->m[0], 0, c->G, nullptr);
    cudaEventRecord(c->ev_a, c->stream);
    for (int i = 0; i < 3; ++i) mmxk_demag(c, c->stream, nullptr, 0, 0, c->m[0], 0, c->G, nullptr);
    cudaEventRecord(c->ev_b, c->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(c->ev_b) != cudaSuccess || cudaEventElapsedTime(&ms, c->ev_a, c->ev_b) != cudaSuccess) {
        cudaGetLastError();
        return 1e30;
    }
    if (cudaGetLastError() != cudaSuccess) return 1e30;
    return 1e3 * ms / 3.0;
}

void apply_plan(mmx_ctx *c, const Plan &p)
{
    mmxk_set_trows(c, p.trows);
    c->xi_tma = p.xi_tma && c->xi_tma_ok;
    c->nd = c->split ? 5 : 3;
    c->demag_us = p.us;
}

int autotune(mmx_ctx *c)
{
    const PlanKey key{c->nx, c->ny, c->nz, c->prec};
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const auto &e : g_plans)
            if (e.first == key) {
                apply_plan(c, e.second);
                c->tuned = true;
                return 0;
            }
    }
    const long long launches = c->launches;
    // time on a seeded pseudo-random field (not zeros) in m[0]; cleared after
    {
        const size_t cnt = (size_t)3 * c->n;
        std::vector<unsigned char> host(cnt * c->esz);
        uint64_t x = 0x9E3779B97F4A7C15ULL;
        for (size_t i = 0; i < cnt; ++i) {
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            const double v = (double)(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
            if (c->esz == 8)
                memcpy(&host[i * 8], &v, 8);
            else {
                const float f = (float)v;
                memcpy(&host[i * 4], &f, 4);
            }
        }
        if (cudaMemcpy(c->m[0], host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return MMX_ERR_CUDA;
        }
    }
    std::vector<int> rows;
    for (int tr = 2; tr <= 16; tr *= 2)
        if (mmxk_set_trows(c, tr) == 0) rows.push_back(tr);
    const int tr0 = mmxk_default_trows(c);
    if (std::find(rows.begin(), rows.end(), tr0) == rows.end()) rows.push_back(tr0);
    std::vector<Plan> cand;
    for (int xt = 0; xt <= (c->xi_tma_ok ? 1 : 0); ++xt)
        for (int tr : rows) cand.push_back(Plan{tr, xt == 1, 1e30});
    // bring the clocks up first (about 20 ms of evaluations), then two
    // round-robin passes over the candidates, keeping each one's minimum
    apply_plan(c, cand[0]);
    double spent = 0;
    for (int i = 0; i < 200 && spent < 20000; ++i) spent += 4 * time_demag(c);
    for (int round = 0; round < 2; ++round)
        for (Plan &p : cand) {
            apply_plan(c, p);
            p.us = std::min(p.us, time_demag(c));
        }
    Plan best = cand[0];
    for (const Plan &p : cand)
        if (p.us < best.us) best = p;
    if (getenv("MMX_AUTOTUNE_LOG"))
        for (const Plan &p : cand)
            fprintf(stderr, "mmx autotune %dx%dx%d %s: x_rows %d xi_tma %d -> %.1f us%s\n", c->nx, c->ny, c->nz,
                    c->prec == MMX_FP64 ? "fp64" : "fp32", p.trows, (int)p.xi_tma, p.us,
                    (&p == &best || (p.trows == best.trows && p.xi_tma == best.xi_tma))
                        ? "  (kept)"
                        : "");
    apply_plan(c, best);
    cudaMemset(c->m[0], 0, (size_t)3 * c->n * c->esz);
    c->launches = launches;
    c->tuned = true;
    if (best.us >= 1e30) return MMX_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.push_back({key, best});
    return 0;
}

}  // namespace

void mmx_set_thread_error(const char *msg) { g_create_err = msg ? msg : ""; }

// Event pair around one timed launch; see mmx_ctx::prof_cap.
void mmx_prof_begin(mmx_ctx *c, cudaStream_t s)
{
    if (c->prof_cap >= 0) {
        const int w = c->prof_cap;
        const size_t i = c->pcls[w].size();
        while (c->pev[w].size() < 2 * i + 2) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            c->pev[w].push_back(e);
        }
        // an external record: a real event-record node in the captured graph
        cudaEventRecordWithFlags(c->pev[w][2 * i], s, cudaEventRecordExternal);
        return;
    }
    cudaEventRecord(c->ev_a, s);
}

void mmx_prof_end(mmx_ctx *c, cudaStream_t s, int cls, int count)
{
    if (c->prof_cap >= 0) {
        const int w = c->prof_cap;
        const size_t i = c->pcls[w].size();
        if (c->pev[w].size() < 2 * i + 2) return;  // no event could be made: this launch is not timed
        cudaEventRecordWithFlags(c->pev[w][2 * i + 1], s, cudaEventRecordExternal);
        c->pcls[w].push_back(cls);
        c->pcnt[w].push_back(count);
        return;
    }
    cudaEventRecord(c->ev_b, s);
    cudaEventSynchronize(c->ev_b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_a, c->ev_b);
    c->prof_ms[cls] += ms;
    c->prof_n[cls] += count;
}

int mmx_state_edit(mmx_ctx *c, const std::function<void(DevState &)> &f)
{
    int rc = read_state(c);
    if (rc) return rc;
    f(*c->h_st);
    return write_state(c);
}

int mmx_state_read(mmx_ctx *c, DevState *out)
{
    int rc = read_state(c);
    if (rc) return rc;
    *out = *c->h_st;
    return 0;
}

void mmx_drop_graphs(mmx_ctx *c)
{
    for (int i = 0; i < 2; ++i) {
        if (c->graph_ok[i]) {
            cudaGraphExecDestroy(c->gexec[i]);
            cudaGraphDestroy(c->graph[i]);
            c->graph_ok[i] = false;
        }
        if (c->pgraph_ok[i]) {
            cudaGraphExecDestroy(c->pgexec[i]);
            cudaGraphDestroy(c->pgraph[i]);
            c->pgraph_ok[i] = false;
        }
    }
}

extern "C" {

int mmx_create(const mmx_mesh *mesh, const mmx_material *mat, const mmx_field *field, const mmx_integrator *integ,
               int precision, void *cuda_stream, mmx_ctx **out)
{
    if (!out) return MMX_ERR_ARG;
    *out = nullptr;
    std::string why = validate(mesh, mat, field, integ, precision);
    if (!why.empty()) {
        g_create_err = why;
        return MMX_ERR_ARG;
    }
    mmx_ctx *c = new (std::nothrow) mmx_ctx();
    if (!c) return MMX_ERR_OOM;
    c->mesh = *mesh;
    c->mat = *mat;
    c->field = *field;
    c->integ = *integ;
    c->prec = precision;
    c->esz = precision == MMX_FP64 ? 8 : 4;
    c->stream = (cudaStream_t)cuda_stream;
    c->nx = mesh->nx;
    c->ny = mesh->ny;
    c->nz = mesh->nz;
    c->n = (long long)c->nx * c->ny * c->nz;
    c->Px = 2 * c->nx;
    c->Py = c->ny > 1 ? 2 * c->ny : 1;
    c->Pz = c->nz > 1 ? 2 * c->nz : 1;
    c->Hy = c->Py / 2 + 1;
    c->Hz = c->Pz / 2 + 1;
    c->rows = 3LL * c->ny * c->nz;
    c->use_graphs = getenv("MMX_NO_GRAPH") == nullptr;
    // fused y-z pass while one column fits comfortably in one CTA, else the
    // split passes; MMX_FORCE_SPLIT forces the split passes
    const bool big = mmxk_yz_smem_bytes(c) > 160 * 1024 || c->Pz > mmxk_yz_max_pz(c);
    if (c->Pz > mmxk_yz_max_pz(c) && c->Py < 2) {
        g_create_err = "ny = 1 with nz above 8 (FP32) or 4 (FP64) is not supported";
        delete c;
        return MMX_ERR_ARG;
    }
    const bool force_split = getenv("MMX_FORCE_SPLIT") != nullptr;
    c->split = (big || force_split) && c->Py >= 2;
    c->nd = c->split ? 5 : 3;
    c->allow_tma = true;
    c->stall_test = getenv("MMX_TEST_STALL_TMA") != nullptr;
    c->trows = mmxk_default_trows(c);
    if (mmxk_x_smem_bytes(c) > 227 * 1024 || (c->split && mmxk_split_smem_bytes(c) > 227 * 1024) ||
        (!c->split && mmxk_yz_smem_bytes(c) > 227 * 1024)) {
        g_create_err = "mesh too large for the FFT passes";
        delete c;
        return MMX_ERR_ARG;
    }

    // tableau
    MethodDef md = method_def(integ->method);
    TabArgs &T = c->tab;
    memset(&T, 0, sizeof(T));
    T.s = md.s;
    T.order = md.order;
    T.adaptive = md.adaptive;
    T.fsal = md.fsal;
    T.abm = integ->method == MMX_ABM2 ? 1 : 0;
    for (int i = 0; i < md.s; ++i) {
        T.a[i] = md.a[i].n / md.a[i].d;
        T.c[i] = md.c[i].n / md.c[i].d;
        T.e[i] = md.c[i].n / md.c[i].d - md.chat[i].n / md.chat[i].d;
        for (size_t j = 0; j < md.b[i].size(); ++j) T.b[i][j] = md.b[i][j].n / md.b[i][j].d;
    }
    // physics
    const double mu0 = 4e-7 * M_PI;
    PhysArgs &P = c->ph;
    P.nx = c->nx;
    P.ny = c->ny;
    P.nz = c->nz;
    P.n = c->n;
    const double cex = 2.0 * mat->A / (mu0 * mat->Ms);
    P.wx = cex / (mesh->dx * mesh->dx);
    P.wy = cex / (mesh->dy * mesh->dy);
    P.wz = cex / (mesh->dz * mesh->dz);
    P.can = 2.0 * mat->K / (mu0 * mat->Ms);
    for (int i = 0; i < 3; ++i) {
        P.ku[i] = mat->ku[i];
        P.H0[i] = field->H0[i];
        P.pulse[i] = field->pulse_H[i];
    }
    P.t_on = field->t_on;
    P.t_off = field->t_off;
    P.gp = mat->gamma / (1.0 + mat->alpha * mat->alpha);
    P.alpha = mat->alpha;
    CtlArgs &C = c->ctl;
    C.p = integ->extrap_order;
    C.adaptive = (integ->adaptive && md.adaptive) ? 1 : 0;
    C.nslots = md.s + T.abm;  // ABM2 keeps F_{n-1} in one more slot
    C.prime = 0;
    C.tol = integ->tol;
    C.hmin = integ->hmin;
    C.hmax = integ->hmax;
    C.cmin = integ->cmin;
    C.cmax = integ->cmax;
    C.safety = integ->safety;
    C.cmin_pow = std::pow(integ->cmin, md.order + 1);
    C.cmax_pow = std::pow(integ->cmax, md.order + 1);

    // tensor (host, binary128; shared by contexts of the same mesh) and spectrum
    mmx_host_tensor_args ta{c->nx, c->ny, c->nz, mesh->dx, mesh->dy, mesh->dz, mat->Ms};
    std::shared_ptr<const std::vector<double>> N6 = tensor_for(ta);
    std::vector<double> Kspec((size_t)(c->nx + 1) * c->Hz * c->Hy * 6);
    mmx_host_spectrum(&ta, N6->data(), c->N00, Kspec.data());
    for (int i = 0; i < 3; ++i) P.msN00[i] = mat->Ms * c->N00[i];

    // device buffers
    auto alloc = [&](void **p, size_t bytes) -> bool {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        return cudaMalloc(p, bytes) == cudaSuccess;
    };
    const size_t fb = (size_t)3 * c->n * c->esz;
    const int nh = std::max(1, C.p + 1);
    bool ok = true;
    ok = ok && alloc(&c->m[0], fb) && alloc(&c->m[1], fb) && alloc(&c->Y[0], fb) && alloc(&c->Y[1], fb);
    c->mlo = nullptr;
    c->errpart = nullptr;
    if (c->prec == MMX_FP32_MIXED) ok = ok && alloc(&c->mlo, 2 * fb);
    ok = ok && alloc(&c->F, fb * C.nslots) && alloc(&c->G, fb) && alloc(&c->hist, fb * nh);
    ok = ok && alloc(&c->errpart, (size_t)((c->n + 127) / 128) * c->esz);
    ok = ok && alloc(&c->S, (size_t)c->rows * c->nx * 2 * c->esz);
    if (c->split) ok = ok && alloc(&c->Tb, (size_t)c->nx * 3 * c->nz * c->Py * 2 * c->esz);
    ok = ok && alloc(&c->K, Kspec.size() * c->esz);
    ok = ok && alloc(&c->twx, (size_t)c->Px * 2 * c->esz) && alloc(&c->twy, (size_t)c->Py * 2 * c->esz) &&
         alloc(&c->twz, (size_t)c->Pz * 2 * c->esz);
    if (c->prec == MMX_FP32_MIXED && c->split && (c->Px == 1024 || c->Py == 1024))
        ok = ok && alloc(&c->tw4, (size_t)1024 * 2 * c->esz);
    if (c->prec == MMX_FP32_MIXED && c->Px == 512) ok = ok && alloc(&c->tw512, (size_t)512 * 2 * c->esz);
    if (c->prec == MMX_FP32_MIXED && !c->split && c->Py == 256 && getenv("MMX_NO_R4") == nullptr)
        ok = ok && alloc(&c->tw4y, (size_t)256 * 2 * c->esz);
    ok = ok && alloc((void **)&c->st, sizeof(DevState));
    ok = ok && cudaMallocHost((void **)&c->h_st, sizeof(DevState)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->cap_stream3, cudaStreamNonBlocking) == cudaSuccess;
    c->Gc = nullptr;
    ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreate(&c->ev_a) == cudaSuccess && cudaEventCreate(&c->ev_b) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        g_create_err = "device allocation failed";
        mmx_destroy(c);
        return MMX_ERR_OOM;
    }
    int rc = mmxk_setup_buffers(c, Kspec.data());
    if (rc) {
        g_create_err = "kernel set-up failed";
        mmx_destroy(c);
        return rc;
    }
    cudaMemset(c->m[0], 0, fb);
    cudaMemset(c->m[1], 0, fb);
    if (c->mlo) cudaMemset(c->mlo, 0, 2 * fb);
    cudaMemset(c->F, 0, fb * C.nslots);
    cudaMemset(c->hist, 0, fb * nh);
    // pass configuration by timing, unless forced or switched off
    {
        const char *at = getenv("MMX_AUTOTUNE");
        const char *trs = getenv("MMX_TROWS");
        const bool forced = force_split || getenv("MMX_NO_TMA") != nullptr || trs != nullptr;
        if (trs) mmxk_set_trows(c, atoi(trs));
        if (!forced && !(at && at[0] == '0') && autotune(c) != 0) {
            g_create_err = "autotuning the demag passes failed";
            mmx_destroy(c);
            return MMX_ERR_CUDA;
        }
    }
    DevState &s = *c->h_st;
    memset(&s, 0, sizeof(s));
    s.t = 0;
    s.h_ctrl = integ->h;
    s.h = integ->h;
    s.t_end = 0;
    s.done = 1;
    s.net_ok = 1;  // a learned residual, once attached, starts as passing its check
    reset_history(&s);
    if (cudaMemcpy(c->st, c->h_st, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        g_create_err = "state upload failed";
        mmx_destroy(c);
        return MMX_ERR_CUDA;
    }
    *out = c;
    return MMX_OK;
}

int mmx_set_m(mmx_ctx *c, const void *m)
{
    if (!c || !m) return MMX_ERR_ARG;
    int rc = read_state(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->m[0], m, (size_t)3 * c->n * c->esz, cudaMemcpyDefault, c->stream));
    if (c->mlo) CK(cudaMemsetAsync(c->mlo, 0, (size_t)3 * c->n * c->esz, c->stream));  // low words of m[0]
    c->h_st->cur = 0;
    reset_history(c->h_st);
    return write_state(c);
}

int mmx_get_m(mmx_ctx *c, void *m)
{
    if (!c || !m) return MMX_ERR_ARG;
    int rc = read_state(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(m, c->m[c->h_st->cur], (size_t)3 * c->n * c->esz, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MMX_OK;
}

int mmx_set_time(mmx_ctx *c, double t)
{
    if (!c || !std::isfinite(t)) return MMX_ERR_ARG;
    int rc = read_state(c);
    if (rc) return rc;
    c->h_st->t = t;
    reset_history(c->h_st);
    return write_state(c);
}

int mmx_demag(mmx_ctx *c, const void *m_dev, void *H_dev)
{
    if (!c || !m_dev || !H_dev) return MMX_ERR_ARG;
    mmxk_demag(c, c->stream, nullptr, 0, 0, m_dev, 0, H_dev, m_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "mmx_demag launch");
    return MMX_OK;
}

// Host-side set-up, on the mirror c->h_st, of a run to t_end or of acc_more
// more accepted steps; false when there is nothing to do.  The caller holds
// a fresh copy of the device state and uploads it afterwards.
static bool begin_run(mmx_ctx *c, double t_end, long long acc_more)
{
    DevState &s = *c->h_st;
    if (acc_more <= 0 && !(t_end > s.t)) return false;
    s.t_end = t_end;
    s.acc_target = acc_more > 0 ? s.accepted + acc_more : LLONG_MAX;
    s.done = 0;
    s.status = 0;
    s.run_attempts = 0;
    s.attempt_limit = 50000000LL;
    s.t_start_ns = 0;
    const char *tl = getenv("MMX_TIME_LIMIT_S");
    s.time_limit_ns = (unsigned long long)((tl ? atof(tl) : 300.0) * 1e9);
    const double rem = s.t_end - s.t;
    const int cl = (s.h_ctrl * (1.0 + 1e-9) >= rem) ? 1 : 0;
    s.h = cl ? rem : s.h_ctrl;
    s.clipped = cl;
    s.loop_more = 1;
    return true;
}

// What the run that began with forced0 forced accepts returns (device
// status and the h_min warning), from the mirror read after the run.
static int end_status(mmx_ctx *c, long long forced0)
{
    const DevState &s = *c->h_st;
    if (s.status) {
        if (s.status == MMX_ERR_NONFINITE) return fail(c, s.status, "error estimate became non-finite");
        if (s.status == MMX_ERR_TIMEOUT) return fail(c, s.status, "attempt or time limit of the run reached");
        return fail(c, s.status, "device reported an error");
    }
    return s.forced > forced0 ? MMX_WARN_HMIN : MMX_OK;
}

static int run_common(mmx_ctx *c, double t_end, long long acc_more)
{
    int rc = read_state(c);
    if (rc) return rc;
    DevState &s = *c->h_st;
    const long long forced0 = s.forced;
    if (!begin_run(c, t_end, acc_more)) return MMX_OK;
    rc = write_state(c);
    if (rc) return rc;
    mmxk_prepare(c, c->stream);
    for (int guard = 0; guard < 1000; ++guard) {
        const int p = c->ctl.p;
        const int which = (p >= 0 && s.hist_n < p + 1) ? 1 : 0;
        rc = run_loop(c, which);
        if (rc) return rc;
        if (s.done) break;
        if (which == 0) return fail(c, MMX_ERR_STATE, "device loop stopped before the run finished");
    }
    return end_status(c, forced0);
}

int mmx_run(mmx_ctx *c, double t_end)
{
    if (!c || !std::isfinite(t_end)) return MMX_ERR_ARG;
    return run_common(c, t_end, 0);
}

int mmx_step(mmx_ctx *c, int n_accepted)
{
    if (!c || n_accepted < 1) return MMX_ERR_ARG;
    return run_common(c, DBL_MAX, n_accepted);
}

int mmx_get_stats(mmx_ctx *c, mmx_stats *o)
{
    if (!c || !o) return MMX_ERR_ARG;
    int rc = read_state(c);
    if (rc) return rc;
    const DevState &s = *c->h_st;
    o->t = s.t;
    o->h = s.h_ctrl;
    o->last_err = s.last_err;
    o->accepted = s.accepted;
    o->rejected = s.rejected;
    o->exact_evals = s.exact_evals;
    o->extrap_evals = s.extrap_evals;
    o->forced_accepts = s.forced;
    o->attempts = s.attempts;
    o->kernel_launches = c->launches;
    return MMX_OK;
}

struct BlobHeader {
    uint64_t magic;
    int32_t nx, ny, nz, prec, method, p, s;
    int32_t pad;
};
static const uint64_t kMagic = 0x31305854534d4d58ULL;  // "XMMSTX01"

int mmx_save_state(mmx_ctx *c, void *buf, size_t *len)
{
    if (!c || !len) return MMX_ERR_ARG;
    const size_t fb = (size_t)3 * c->n * c->esz;
    const int nh = std::max(1, c->ctl.p + 1);
    const size_t need = sizeof(BlobHeader) + sizeof(DevState) + fb * (2 + c->ctl.nslots + nh) + (c->mlo ? 2 * fb : 0);
    if (!buf) {
        *len = need;
        return MMX_OK;
    }
    if (*len < need) return fail(c, MMX_ERR_ARG, "buffer too small");
    int rc = read_state(c);
    if (rc) return rc;
    char *p = (char *)buf;
    BlobHeader hd{kMagic, c->nx, c->ny, c->nz, c->prec, c->integ.method, c->ctl.p, c->tab.s, 0};
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    memcpy(p, c->h_st, sizeof(DevState));
    p += sizeof(DevState);
    CK(cudaMemcpy(p, c->m[0], fb, cudaMemcpyDeviceToHost));
    p += fb;
    CK(cudaMemcpy(p, c->m[1], fb, cudaMemcpyDeviceToHost));
    p += fb;
    CK(cudaMemcpy(p, c->F, fb * c->ctl.nslots, cudaMemcpyDeviceToHost));
    p += fb * c->ctl.nslots;
    CK(cudaMemcpy(p, c->hist, fb * nh, cudaMemcpyDeviceToHost));
    p += fb * nh;
    if (c->mlo) CK(cudaMemcpy(p, c->mlo, 2 * fb, cudaMemcpyDeviceToHost));
    *len = need;
    return MMX_OK;
}

int mmx_load_state(mmx_ctx *c, const void *buf, size_t len)
{
    if (!c || !buf) return MMX_ERR_ARG;
    const size_t fb = (size_t)3 * c->n * c->esz;
    const int nh = std::max(1, c->ctl.p + 1);
    const size_t need = sizeof(BlobHeader) + sizeof(DevState) + fb * (2 + c->ctl.nslots + nh) + (c->mlo ? 2 * fb : 0);
    if (len < need) return fail(c, MMX_ERR_ARG, "state blob too short");
    BlobHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kMagic || hd.nx != c->nx || hd.ny != c->ny || hd.nz != c->nz || hd.prec != c->prec ||
        hd.method != c->integ.method || hd.p != c->ctl.p)
        return fail(c, MMX_ERR_ARG, "state blob does not match this context");
    const char *p = (const char *)buf + sizeof(hd);
    CK(cudaStreamSynchronize(c->stream));
    memcpy(c->h_st, p, sizeof(DevState));
    p += sizeof(DevState);
    CK(cudaMemcpy(c->m[0], p, fb, cudaMemcpyHostToDevice));
    p += fb;
    CK(cudaMemcpy(c->m[1], p, fb, cudaMemcpyHostToDevice));
    p += fb;
    CK(cudaMemcpy(c->F, p, fb * c->ctl.nslots, cudaMemcpyHostToDevice));
    p += fb * c->ctl.nslots;
    CK(cudaMemcpy(c->hist, p, fb * nh, cudaMemcpyHostToDevice));
    p += fb * nh;
    if (c->mlo) CK(cudaMemcpy(c->mlo, p, 2 * fb, cudaMemcpyHostToDevice));
    c->h_st->done = 1;
    return write_state(c);
}

int mmx_set_profiling(mmx_ctx *c, int enable)
{
    if (!c || enable < 0 || enable > 2) return MMX_ERR_ARG;
    const bool group = enable == 2;
    if (group != c->prof_group) {
        // the profiled attempt graphs hold the other mode's event pairs
        for (int i = 0; i < 2; ++i)
            if (c->pgraph_ok[i]) {
                cudaGraphExecDestroy(c->pgexec[i]);
                cudaGraphDestroy(c->pgraph[i]);
                c->pgraph_ok[i] = false;
            }
        c->prof_group = group;
    }
    c->profiling = enable != 0;
    for (int i = 0; i < MMX_NPROF; ++i) {
        c->prof_ms[i] = 0;
        c->prof_n[i] = 0;
    }
    return MMX_OK;
}

int mmx_get_profile(mmx_ctx *c, double *ms, long long *launches)
{
    if (!c || !ms || !launches) return MMX_ERR_ARG;
    for (int i = 0; i < MMX_NPROF; ++i) {
        ms[i] = c->prof_ms[i];
        launches[i] = c->prof_n[i];
    }
    return MMX_OK;
}

int mmx_get_plan(const mmx_ctx *c, mmx_plan *out)
{
    if (!c || !out) return MMX_ERR_ARG;
    out->yz_pass = c->split ? 1 : 0;
    out->x_rows = c->trows;
    out->xi_tma = c->xi_tma ? 1 : 0;
    out->tuned = c->tuned ? 1 : 0;
    out->demag_us = c->tuned ? c->demag_us : 0.0;
    out->kernels_per_demag = c->nd;
    return MMX_OK;
}

const char *mmx_last_error(const mmx_ctx *c)
{
    if (!c) return g_create_err.c_str();
    return c->err.c_str();
}

void mmx_destroy(mmx_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    mmx_drop_graphs(c);
    for (int i = 0; i < 2; ++i)
        for (cudaEvent_t e : c->pev[i]) cudaEventDestroy(e);
    void *bufs[] = {c->m[0], c->m[1], c->mlo, c->errpart, c->Y[0], c->Y[1], c->F, c->G, c->hist, c->S, c->K, c->twx, c->twy, c->twz, c->Tb,
                    c->tw4, c->tw512, c->tw4y, c->st};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->cap_stream3) cudaStreamDestroy(c->cap_stream3);
    if (c->Gc) cudaFree(c->Gc);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_a) cudaEventDestroy(c->ev_a);
    if (c->ev_b) cudaEventDestroy(c->ev_b);
    delete c;
}

}  // extern "C"

// ------------------------------------------------------------ batched runs

struct mmx_batch {
    std::vector<mmx_ctx *> c;
    std::vector<cudaStream_t> member_streams;  // distinct streams of the members
    std::vector<cudaEvent_t> ev;               // one per distinct member stream
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    std::vector<long long> forced0, prime0;
    std::vector<char> active;
    std::string err;
};

namespace {

int bfail(mmx_batch *b, int code, const std::string &msg)
{
    b->err = msg;
    return code;
}

#define BK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e__ = (call);                                                                 \
        if (e__ != cudaSuccess) return bfail(b, MMX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

// One parent graph; per member a chain  prepare -> gate -> while(priming
// attempt) -> gate -> while(extrapolated attempt)  (the priming pair only
// when p >= 0), the members' chains independent of one another.  The while
// bodies are the members' own attempts, captured as in build_graph, and
// each member's controller drives its own condition handles.
int build_batch_graph(mmx_batch *b)
{
    if (b->graph_ok) return 0;
    cudaGraph_t g;
    BK(cudaGraphCreate(&g, 0));
    for (mmx_ctx *c : b->c) {
        const long long launches = c->launches;
        cudaGraphNode_t prev;
        if (mmxk_add_prepare_node(g, nullptr, 0, c, &prev)) {
            cudaGraphDestroy(g);
            return bfail(b, MMX_ERR_CUDA, "adding a preparation node failed");
        }
        const int first = c->ctl.p >= 0 ? 1 : 0;
        for (int which = first; which >= 0; --which) {
            cudaGraphConditionalHandle h;
            cudaGraphNode_t gate, node;
            cudaGraphNodeParams cp{};
            cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
            if (e == cudaSuccess && speculative(c, which == 1 || c->ctl.p < 0)) {
                // the first attempt's x and y-z passes, as a child graph
                cudaGraph_t fg = nullptr;
                cudaGraphNode_t fn;
                e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    front_kernels(c, c->cap_stream);
                    e = cudaStreamEndCapture(c->cap_stream, &fg);
                }
                if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&fn, g, &prev, 1, fg);
                if (fg) cudaGraphDestroy(fg);
                if (e == cudaSuccess) prev = fn;
            }
            if (e == cudaSuccess && mmxk_add_gate_node(g, &prev, 1, c, h, which, &gate)) e = cudaErrorUnknown;
            if (e == cudaSuccess) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&node, g, &gate, nullptr, 1, &cp);
            }
            if (e == cudaSuccess && c->rnet && which == 0) {
                if (build_res_body(c, cp.conditional.phGraph_out[0], h)) e = cudaErrorUnknown;
            } else {
                if (e == cudaSuccess)
                    e = cudaStreamBeginCaptureToGraph(c->cap_stream, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                                      0, cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    body_kernels(c, c->cap_stream, which == 1 || c->ctl.p < 0, h, 1, c->cap_stream2);
                    cudaGraph_t captured;
                    e = cudaStreamEndCapture(c->cap_stream, &captured);
                }
            }
            if (e != cudaSuccess) {
                c->launches = launches;
                cudaGraphDestroy(g);
                return bfail(b, MMX_ERR_CUDA, std::string("building the batch graph: ") + cudaGetErrorString(e));
            }
            prev = node;
        }
        c->launches = launches;
    }
    cudaGraphExec_t ex;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return bfail(b, MMX_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    b->graph = g;
    b->gexec = ex;
    b->graph_ok = true;
    return 0;
}

// severity order of member results: errors, then the h_min warning
int combine(int acc, int rc)
{
    if (acc < 0) return acc;
    if (rc < 0) return rc;
    return std::max(acc, rc);
}

}  // namespace

extern "C" {

int mmx_batch_create(int n, mmx_ctx *const *members, void *cuda_stream, mmx_batch **out)
{
    if (!out) return MMX_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > 4096 || !members) {
        g_create_err = "batch: need 1 <= n <= 4096 members";
        return MMX_ERR_ARG;
    }
    std::vector<mmx_ctx *> v(members, members + n);
    for (int i = 0; i < n; ++i) {
        if (!v[i]) {
            g_create_err = "batch: NULL member";
            return MMX_ERR_ARG;
        }
    }
    std::vector<mmx_ctx *> sorted = v;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
        g_create_err = "batch: a context appears twice";
        return MMX_ERR_ARG;
    }
    mmx_batch *b = new (std::nothrow) mmx_batch();
    if (!b) return MMX_ERR_OOM;
    b->c = v;
    b->stream = (cudaStream_t)cuda_stream;
    for (mmx_ctx *c : v)
        if (std::find(b->member_streams.begin(), b->member_streams.end(), c->stream) == b->member_streams.end())
            b->member_streams.push_back(c->stream);
    bool ok = true;
    for (size_t i = 0; ok && i < b->member_streams.size(); ++i) {
        cudaEvent_t e;
        ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) b->ev.push_back(e);
    }
    if (!ok) {
        cudaGetLastError();
        g_create_err = "batch: event creation failed";
        mmx_batch_destroy(b);
        return MMX_ERR_CUDA;
    }
    b->forced0.assign(n, 0);
    b->prime0.assign(n, 0);
    b->active.assign(n, 0);
    *out = b;
    return MMX_OK;
}

int mmx_batch_run(mmx_batch *b, const double *t_end, int *status)
{
    if (!b || !t_end) return MMX_ERR_ARG;
    b->err.clear();
    const int n = (int)b->c.size();
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(t_end[i])) return bfail(b, MMX_ERR_ARG, "batch: t_end must be finite");
    bool graphs = true;
    for (mmx_ctx *c : b->c) graphs = graphs && c->use_graphs && !c->profiling;
    int rc_all = MMX_OK;
    if (!graphs) {
        // graphs disabled or a member is being profiled: the members' own runs
        for (int i = 0; i < n; ++i) {
            const int rc = run_common(b->c[i], t_end[i], 0);
            if (status) status[i] = rc;
            rc_all = combine(rc_all, rc);
        }
        return rc_all;
    }
    int rc = build_batch_graph(b);
    if (rc) return rc;
    // after the members' pending work
    for (size_t j = 0; j < b->member_streams.size(); ++j) {
        BK(cudaEventRecord(b->ev[j], b->member_streams[j]));
        BK(cudaStreamWaitEvent(b->stream, b->ev[j], 0));
    }
    for (mmx_ctx *c : b->c) BK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; ++i) {
        mmx_ctx *c = b->c[i];
        b->forced0[i] = c->h_st->forced;
        b->prime0[i] = c->h_st->prime_attempts;
        b->active[i] = begin_run(c, t_end[i], 0) ? 1 : 0;
        if (!b->active[i]) c->h_st->done = 1;
        BK(cudaMemcpyAsync(c->st, c->h_st, sizeof(DevState), cudaMemcpyHostToDevice, b->stream));
    }
    BK(cudaGraphLaunch(b->gexec, b->stream));
    for (mmx_ctx *c : b->c) BK(cudaMemcpyAsync(c->h_st, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; ++i) {
        mmx_ctx *c = b->c[i];
        const DevState &s = *c->h_st;
        const long long pa = s.prime_attempts - b->prime0[i];
        const int gates = c->ctl.p >= 0 ? 2 : 1;
        c->launches += 1 + gates + (speculative(c, c->ctl.p < 0) ? c->nd - 1 : 0);
        int r = MMX_OK;
        if (b->active[i]) {
            c->launches += pa * kernels_per_attempt(c, 1) + (s.run_attempts - pa) * kernels_per_attempt(c, c->ctl.p < 0);
            if (s.fault)
                r = fail(c, MMX_ERR_CUDA, "a bounded device wait gave up (a tensor copy or tensor-core operation did not complete)");
            else
                r = s.done ? end_status(c, b->forced0[i])
                           : fail(c, MMX_ERR_STATE, "batched loops stopped before the run finished");
        }
        if (status) status[i] = r;
        rc_all = combine(rc_all, r);
    }
    return rc_all;
}

const char *mmx_batch_last_error(const mmx_batch *b)
{
    if (!b) return g_create_err.c_str();
    return b->err.c_str();
}

void mmx_batch_destroy(mmx_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph_ok) {
        cudaGraphExecDestroy(b->gexec);
        cudaGraphDestroy(b->graph);
    }
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
