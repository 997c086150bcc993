// C ABI of the VOLDOR library (declared in include/voldor.h): context
// lifetime, argument checking, the Table 1 iteration as a sequence of kernel
// launches, CUDA-graph capture of voldor_em_step, and host readout.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "voldor_internal.cuh"

using namespace vd;

struct voldor_ctx {
    int W = 0, H = 0, T = 0, N = 0, flow_dtype = 0;
    voldor_params params{};
    voldor_intrinsics K{};
    DevParams dp{};
    DevState ds{};
    cudaStream_t stream = nullptr;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    size_t flows_bytes = 0;
    int* flag_dev = nullptr;          // inside the arena: counter of rejected flow blocks
    bool bootstrapped = false;
    bool poisoned = false;
    bool timing = false;
    std::map<long long, cudaGraphExec_t> graphs;
    std::map<long long, cudaGraph_t> raw_graphs;   // the captured graphs, for embedding in batches
    std::vector<cudaEvent_t> events;  // start/stop pairs of the timed graph
    int last_pairs = 0;
    int graph_pairs = 0;
    std::map<long long, long long> graph_kernels;   // kernel nodes per cached graph
    long long launches = 0;                          // kernels enqueued so far
    cudaError_t first_error = cudaSuccess;           // the error that poisoned the context
    cudaStream_t aux = nullptr;                      // second stream: P3P beside the pose preparation
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;   // hypothesis logarithms beside the scoring
    void* epi_base = nullptr;                        // epipolar bootstrap scratch
    int epi_cap = 0;                                 // samples it holds
    int epi_M = 0;                                   // samples of the last epipolar bootstrap
    void* ground_base = nullptr;                     // ground-plane scale scratch
};

namespace {

const voldor_status kCuda = VOLDOR_ERR_CUDA;

bool cuda_ok(voldor_ctx* c, cudaError_t e)
{
    if (e == cudaSuccess) return true;
    if (c) {
        if (c->first_error == cudaSuccess) c->first_error = e;
        c->poisoned = true;
    }
    return false;
}

bool launched(voldor_ctx* c) { return cuda_ok(c, cudaGetLastError()); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

bool params_ok(const voldor_params& p)
{
    if (!finite_pos(p.a1) || !std::isfinite(p.a2) || !std::isfinite(p.b1) || !std::isfinite(p.b2)) return false;
    if (!std::isfinite(p.lambda_) || p.lambda_ < 0.0) return false;
    if (!(p.gamma > 0.0 && p.gamma < 1.0)) return false;
    if (!finite_pos(p.sigma_t) || !finite_pos(p.sigma_r)) return false;
    if (!finite_pos(p.inv_depth_min) || !finite_pos(p.inv_depth_max) || !(p.inv_depth_max > p.inv_depth_min)) return false;
    if (!finite_pos(p.x_min) || !finite_pos(p.x_max) || !(p.x_max > p.x_min)) return false;
    if (!finite_pos(p.beta_min) || !(p.ms_tol >= 0.0) || !std::isfinite(p.ms_tol)) return false;
    if (p.hyps_per_frame < 1 || p.hyps_per_frame > 65536) return false;
    if (p.groups_per_frame < 1 || p.groups_per_frame > 262144) return false;
    if (p.ms_max_iter < 1 || p.ms_max_iter > 100000) return false;
    if (p.criterion != VOLDOR_CRITERION_MIE && p.criterion != VOLDOR_CRITERION_MLE) return false;
    if (p.residual != VOLDOR_RESIDUAL_FISK && p.residual != VOLDOR_RESIDUAL_GAUSSIAN) return false;
    return true;
}

DevParams make_dev_params(const voldor_ctx& c)
{
    const voldor_params& p = c.params;
    DevParams d{};
    d.W = c.W; d.H = c.H; d.T = c.T; d.N = c.N;
    d.S = p.hyps_per_frame; d.G = p.groups_per_frame; d.ms_max_iter = p.ms_max_iter;
    d.criterion = p.criterion;
    d.residual = p.residual;
    d.flow_f16 = c.flow_dtype == VOLDOR_FLOW_F16;
    d.fx = (float)c.K.fx; d.fy = (float)c.K.fy; d.cx = (float)c.K.cx; d.cy = (float)c.K.cy;
    d.inv_fx = (float)(1.0 / c.K.fx); d.inv_fy = (float)(1.0 / c.K.fy);
    d.fy_over_fx = (float)(c.K.fy / c.K.fx);
    d.log2_a1 = (float)std::log2(p.a1);
    d.a2_log2e = (float)(p.a2 / std::log(2.0));
    d.b1 = (float)p.b1; d.b2 = (float)p.b2; d.beta_min = (float)p.beta_min;
    d.lambda2 = (float)(p.lambda_ * p.lambda_);
    d.x_min = (float)p.x_min; d.x_max = (float)p.x_max;
    d.xs_min = (float)(p.x_min / (c.K.fx * c.K.fx));
    d.xs_max = (float)(p.x_max / (c.K.fx * c.K.fx));
    d.log2_fx2 = (float)std::log2(c.K.fx * c.K.fx);
    d.inv_depth_min = (float)p.inv_depth_min; d.inv_depth_max = (float)p.inv_depth_max;
    d.gamma = (float)p.gamma;
    d.fxd = c.K.fx; d.fyd = c.K.fy; d.cxd = c.K.cx; d.cyd = c.K.cy;
    d.inv_fxd = 1.0 / c.K.fx; d.inv_fyd = 1.0 / c.K.fy; d.fy_over_fx_d = c.K.fy / c.K.fx;
    d.sigma_t = p.sigma_t; d.sigma_r = p.sigma_r; d.ms_tol = p.ms_tol;
    d.seed = p.seed; d.window_id = p.window_id;
    d.w_magic = (unsigned)((1ull << 32) / (unsigned long long)c.W);
    const double kv[6] = {c.K.fx, c.K.fy, c.K.cx, c.K.cy, 1.0 / c.K.fx, 1.0 / c.K.fy};
    for (int i = 0; i < 6; ++i) {
        const float h = (float)kv[i];
        d.kdf[2 * i] = h;
        d.kdf[2 * i + 1] = (float)(kv[i] - (double)h);
    }
    return d;
}

// Carves every device buffer out of one allocation (or sizes it when base is
// null). Returns the total size.
size_t layout(voldor_ctx& c, char* base)
{
    const size_t N = (size_t)c.N, T = (size_t)c.T;
    const size_t S = (size_t)c.params.hyps_per_frame, G = (size_t)c.params.groups_per_frame;
    const int chunks = score_chunks((int)S, c.N);
    const int chunks_max = score_chunks_max((int)S, c.N);
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    DevState& s = c.ds;
    c.flows_bytes = T * N * (c.flow_dtype == VOLDOR_FLOW_F16 ? 4 : 8);
    s.flows = take(c.flows_bytes);
    s.theta = (float*)take(N * 4);
    s.wmap = (float*)take(T * N * 4);
    s.qs = (float*)take(T * N * 4);
    s.poses = (double*)take(T * 12 * 8);
    s.cum = (double*)take(T * 12 * 8);
    s.frames32 = (float*)take(T * 24 * 4);
    s.cum_df = (float*)take(T * 24 * 4);
    s.poses_df = (float*)take(T * 24 * 4);
    s.iter = (int*)take(4);
    s.status = (int*)take(16);
    c.flag_dev = (int*)take(4);
    s.pix = (PixRec*)take(N * sizeof(PixRec));
    s.pix_block_count = (int*)take(((N + kPixThreads - 1) / kPixThreads) * 4);
    s.prep_done = (unsigned*)take(4);
    s.pix_count = (int*)take(4);
    s.pix_vmask = (unsigned*)take(((N + kPixThreads - 1) / kPixThreads) * (kPixThreads / 32) * 4);
    s.p3p_claims = (int*)take(4);
    s.p3p_done = (unsigned long long*)take(8);
    s.grp_sols = (double*)take(G * kMaxSols * 12 * 8);
    s.grp_weight = (double*)take(G * 8);
    s.grp_count = (int*)take(G * 4);
    s.grp_offset = (int*)take(G * 4);
    s.n_hyp = (int*)take(4);
    s.hyp_Rt = (double*)take(S * 12 * 8);
    s.hyp_f32 = (float*)take(S * 12 * 4);
    s.hyp_pw = (float*)take(S * 16 * 4);
    s.hyp_w = (double*)take(S * 8);
    s.hyp_dp = (float*)take(S * 8 * 4);
    s.hyp_info = (long long*)take(S * 2 * 8);
    s.partial = (double*)take((size_t)chunks_max * S * 8);
    s.scores = (double*)take(S * 8);
    s.mie_prev_score = (float*)take(N * 4);
    s.mie_smp = (float*)take(N * 4);
    s.mie_smp_score = (float*)take(N * 4);
    s.mie_next = (int*)take(N * 4);
    s.labels = (unsigned char*)take(N);
    s.fb_fwd = (float*)take(T * N * 8);
    s.score_log = (long long*)take((size_t)kScoreLogMax * 2 * 8);
    s.n_chunks = chunks;
    s.score_hpt = kScoreDefaultHpt;
    return off;
}

// Longest flow vector a window may hold: four times the largest image side
// (a longer flow sends its pixel far outside every image the library
// accepts). Up to this length the Fisk constants of a pixel stay inside FP32:
// alpha = a1 e^{a2 |v|} reaches 2^2120 (kept as log2), mu / beta falls to
// ~4e-39, just below the normal range with 22 significant bits left; near
// 19,600 px the exponentials of the likelihood overflow and a pixel's
// likelihood would become inf or NaN.
constexpr float kMaxFlowPx = 16384.f;

// Counts the blocks that saw a non-finite flow or one longer than kMaxFlowPx.
__global__ void k_count_bad_flows(const void* flows, int f16, size_t n, int* out)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0;
    for (; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 v = f16 ? __half22float2(reinterpret_cast<const __half2*>(flows)[i]) : reinterpret_cast<const float2*>(flows)[i];
        bad |= !(isfinite(v.x) && isfinite(v.y) && fmaf(v.x, v.x, v.y * v.y) <= kMaxFlowPx * kMaxFlowPx);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAdd(out, 1);
}

voldor_status upload_flows(voldor_ctx* c, const void* flows, int on_device)
{
    if (!cuda_ok(c, cudaMemcpyAsync((void*)c->ds.flows, flows, c->flows_bytes,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream)))
        return kCuda;
    if (!cuda_ok(c, cudaMemsetAsync(c->flag_dev, 0, 4, c->stream))) return kCuda;
    const size_t n = (size_t)c->T * c->N;
    k_count_bad_flows<<<304, 256, 0, c->stream>>>(c->ds.flows, c->flow_dtype == VOLDOR_FLOW_F16, n, c->flag_dev);
    c->launches += 1;
    if (!launched(c)) return kCuda;
    int bad = 0;
    if (!cuda_ok(c, cudaMemcpyAsync(&bad, c->flag_dev, 4, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    if (bad) {
        // the context keeps no flow it rejects: zero flows, and the state must
        // be bootstrapped again before the next iteration
        if (!cuda_ok(c, cudaMemsetAsync((void*)c->ds.flows, 0, c->flows_bytes, c->stream))) return kCuda;
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
        c->bootstrapped = false;
        return VOLDOR_ERR_INVALID_ARG;
    }
    return VOLDOR_OK;
}

// One pose update of frame t (iteration counter already set on the device).
bool enqueue_pose_update(voldor_ctx* c, int t, cudaEvent_t ev0, cudaEvent_t ev1, int log_idx)
{
    const DevParams& p = c->dp;
    const DevState& s = c->ds;
    cudaStream_t st = c->stream;
    launch_frame_setup(p, s, st);
    launch_prep_count(p, s, t, st);
    // the minimal groups (drawn from the valid pixels the count pass listed)
    // and their P3P (FP64) run beside the write of the pixel records
    if (!cuda_ok(c, cudaEventRecord(c->ev_fork, st))) return false;
    if (!cuda_ok(c, cudaStreamWaitEvent(c->aux, c->ev_fork, 0))) return false;
    launch_p3p_groups(p, s, t, c->aux);
    if (!cuda_ok(c, cudaEventRecord(c->ev_join, c->aux))) return false;
    launch_prep_write(p, s, t, st);
    if (!cuda_ok(c, cudaStreamWaitEvent(st, c->ev_join, 0))) return false;
    launch_hyp_collect(p, s, st);
    // the meanshift's form of the hypotheses (FP64 se(3) logarithms) is
    // computed beside the dense scoring
    if (!cuda_ok(c, cudaEventRecord(c->ev_fork2, st))) return false;
    if (!cuda_ok(c, cudaStreamWaitEvent(c->aux, c->ev_fork2, 0))) return false;
    launch_hyp_log(p, s, c->aux);
    if (!cuda_ok(c, cudaEventRecord(c->ev_join2, c->aux))) return false;
    // External records become event-record nodes when the stream is captured
    if (ev0 && !cuda_ok(c, cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal))) return false;
    launch_score(p, s, log_idx, st);
    if (ev1 && !cuda_ok(c, cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal))) return false;
    launch_score_reduce(p, s, st);
    if (!cuda_ok(c, cudaStreamWaitEvent(st, c->ev_join2, 0))) return false;
    launch_meanshift(p, s, t, st);
    return launched(c);
}

bool enqueue_smooth(voldor_ctx* c)
{
    launch_frame_setup(c->dp, c->ds, c->stream);
    launch_emissions(c->dp, c->ds, c->ds.qs, c->stream);
    launch_forward_backward(c->dp, c->ds, c->stream);
    return launched(c);
}

bool enqueue_depth(voldor_ctx* c)
{
    launch_frame_setup(c->dp, c->ds, c->stream);
    launch_mie(c->dp, c->ds, c->stream);
    return launched(c);
}

bool enqueue_rigidness(voldor_ctx* c)
{
    launch_frame_setup(c->dp, c->ds, c->stream);
    launch_emissions(c->dp, c->ds, c->ds.wmap, c->stream);
    return launched(c);
}

// Table 1, one iteration, reading k from the device counter and advancing it.
bool enqueue_iteration(voldor_ctx* c, int pair_base)
{
    for (int t = 1; t <= c->T; ++t) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int log_idx = -1;
        if (c->timing) {
            const int idx = pair_base + t - 1;
            e0 = c->events[2 * idx];
            e1 = c->events[2 * idx + 1];
            log_idx = idx;
        }
        if (!enqueue_pose_update(c, t, e0, e1, log_idx)) return false;
    }
    if (!enqueue_smooth(c) || !enqueue_depth(c) || !enqueue_rigidness(c)) return false;
    launch_advance_iteration(c->ds, c->stream);
    return launched(c);
}

bool ensure_events(voldor_ctx* c, int pairs)
{
    while ((int)c->events.size() < 2 * pairs) {
        cudaEvent_t e;
        if (!cuda_ok(c, cudaEventCreate(&e))) return false;
        c->events.push_back(e);
    }
    return true;
}

// Captures n iterations of the VOLDOR loop (with timing events if asked) as a
// CUDA graph, instantiates it and keeps both forms on the context.
bool ensure_graph(voldor_ctx* c, int n_iters, bool timing)
{
    const long long key = (long long)n_iters * 2 + (timing ? 1 : 0);
    if (c->graphs.count(key)) return true;
    const bool saved_timing = c->timing;
    c->timing = timing;
    if (timing && !ensure_events(c, n_iters * c->T)) { c->timing = saved_timing; return false; }
    cudaStream_t cap = c->stream;
    bool own = false;
    if (cap == nullptr) {   // the legacy stream cannot be captured
        if (!cuda_ok(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) { c->timing = saved_timing; return false; }
        own = true;
    }
    cudaStream_t saved = c->stream;
    c->stream = cap;
    cudaGraph_t g = nullptr;
    bool ok = cuda_ok(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    if (ok) {
        for (int i = 0; i < n_iters && ok; ++i) ok = enqueue_iteration(c, i * c->T);
        cudaError_t ee = cudaStreamEndCapture(cap, &g);
        ok = ok && cuda_ok(c, ee);
    }
    c->stream = saved;
    c->timing = saved_timing;
    if (own) cudaStreamDestroy(cap);
    if (!ok) { if (g) cudaGraphDestroy(g); c->poisoned = true; return false; }
    size_t n_nodes = 0;
    long long n_kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (cudaGraphGetNodes(g, nodes.data(), &n_nodes) == cudaSuccess)
            for (size_t q = 0; q < n_nodes; ++q) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++n_kernels;
            }
    }
    cudaGraphExec_t ge = nullptr;
    if (!cuda_ok(c, cudaGraphInstantiate(&ge, g, 0))) { cudaGraphDestroy(g); return false; }
    c->graphs[key] = ge;
    c->raw_graphs[key] = g;
    c->graph_kernels[key] = n_kernels;
    if (timing) c->graph_pairs = n_iters * c->T;
    return true;
}

void drop_graphs(voldor_ctx* c)
{
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : c->raw_graphs) cudaGraphDestroy(kv.second);
    c->graphs.clear();
    c->raw_graphs.clear();
    c->graph_kernels.clear();
}

// Status of a window's status word 3: a bounded wait that gave up outranks
// degenerate frames.
voldor_status status_of_word(int w)
{
    if (w & kStatusTimeout) return VOLDOR_ERR_TIMEOUT;
    return w ? VOLDOR_ERR_DEGENERATE : VOLDOR_OK;
}

voldor_status read_status_word(voldor_ctx* c, int* host4)
{
    if (!cuda_ok(c, cudaMemcpyAsync(host4, c->ds.status, 16, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    return VOLDOR_OK;
}

}  // namespace

extern "C" {

void voldor_default_params(voldor_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->a1 = 0.01; p->a2 = 0.09; p->b1 = -0.0022; p->b2 = 1.0;
    p->lambda_ = 0.15; p->gamma = 0.9;
    p->sigma_t = 0.1; p->sigma_r = 0.004;
    p->inv_depth_min = 1.0 / 40.0; p->inv_depth_max = 1.0;
    p->x_min = 1e-6; p->x_max = 1e12; p->beta_min = 0.05;
    p->ms_tol = 1e-10;
    p->hyps_per_frame = 256; p->groups_per_frame = 1024; p->ms_max_iter = 100;
    p->criterion = VOLDOR_CRITERION_MIE;
    p->residual = VOLDOR_RESIDUAL_FISK;
    p->seed = 0; p->window_id = 0;
}

const char* voldor_status_string(voldor_status s)
{
    switch (s) {
        case VOLDOR_OK: return "ok";
        case VOLDOR_ERR_INVALID_ARG: return "invalid argument";
        case VOLDOR_ERR_CUDA: return "CUDA error (context poisoned)";
        case VOLDOR_ERR_OOM: return "device out of memory";
        case VOLDOR_ERR_NOT_BOOTSTRAPPED: return "context not bootstrapped";
        case VOLDOR_ERR_DEGENERATE: return "a frame had no weighted pose hypothesis";
        case VOLDOR_ERR_TIMEOUT: return "device-side wait timed out";
        case VOLDOR_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

voldor_status voldor_init_window(voldor_ctx** out, int width, int height, int T, const voldor_intrinsics* K,
                                 const voldor_params* params, const void* flows, int flow_dtype, int flows_on_device,
                                 void* cuda_stream)
{
    if (!out) return VOLDOR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!K || !flows || width < 2 || height < 2 || T < 1 || T > kMaxT) return VOLDOR_ERR_INVALID_ARG;
    if (width > kMaxImageSide || height > kMaxImageSide) return VOLDOR_ERR_INVALID_ARG;
    if ((long long)width * height > 0x7fffffffLL) return VOLDOR_ERR_INVALID_ARG;
    if (!finite_pos(K->fx) || !finite_pos(K->fy) || !std::isfinite(K->cx) || !std::isfinite(K->cy))
        return VOLDOR_ERR_INVALID_ARG;
    if (flow_dtype != VOLDOR_FLOW_F32 && flow_dtype != VOLDOR_FLOW_F16) return VOLDOR_ERR_INVALID_ARG;
    voldor_params p;
    if (params) p = *params; else voldor_default_params(&p);
    if (!params_ok(p)) return VOLDOR_ERR_INVALID_ARG;

    voldor_ctx* c = new (std::nothrow) voldor_ctx();
    if (!c) return VOLDOR_ERR_OOM;
    c->W = width; c->H = height; c->T = T; c->N = width * height;
    c->flow_dtype = flow_dtype; c->params = p; c->K = *K;
    c->stream = (cudaStream_t)cuda_stream;
    c->dp = make_dev_params(*c);
    const size_t bytes = layout(*c, nullptr);
    cudaError_t e = cudaMalloc(&c->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return e == cudaErrorMemoryAllocation ? VOLDOR_ERR_OOM : VOLDOR_ERR_CUDA;
    }
    c->arena_bytes = bytes;
    layout(*c, (char*)c->arena);
    if (!cuda_ok(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking)) ||
        !cuda_ok(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) ||
        !cuda_ok(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) ||
        !cuda_ok(c, cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming)) ||
        !cuda_ok(c, cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming))) {
        voldor_destroy(c);
        return kCuda;
    }
    if (!cuda_ok(c, cudaMemsetAsync(c->arena, 0, bytes, c->stream))) { voldor_destroy(c); return kCuda; }
    voldor_status st = upload_flows(c, flows, flows_on_device);
    if (st != VOLDOR_OK) { voldor_destroy(c); return st; }
    *out = c;
    return VOLDOR_OK;
}

voldor_status voldor_set_flows(voldor_ctx* c, const void* flows, int flows_on_device)
{
    if (!c || !flows) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    return upload_flows(c, flows, flows_on_device);
}

voldor_status voldor_bootstrap(voldor_ctx* c, int mode, const double* T1)
{
    if (!c) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (mode == VOLDOR_BOOT_EPIPOLAR) return voldor_bootstrap_epipolar(c, 512, 1.0, nullptr);
    if (mode != VOLDOR_BOOT_GIVEN_POSE || !T1) return VOLDOR_ERR_INVALID_ARG;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T1[i])) return VOLDOR_ERR_INVALID_ARG;
    launch_bootstrap(c->dp, c->ds, T1, c->stream);
    c->launches += 1;
    if (!cuda_ok(c, cudaMemsetAsync(c->ds.status, 0, 16, c->stream))) return kCuda;
    if (!launched(c)) return kCuda;
    c->bootstrapped = true;
    return VOLDOR_OK;
}

voldor_status voldor_bootstrap_epipolar(voldor_ctx* c, int n_samples, double baseline, double* T1_out)
{
    if (!c || n_samples < 1 || n_samples > VOLDOR_EPI_MAX_SAMPLES || !finite_pos(baseline)) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (n_samples > c->epi_cap) {
        if (c->epi_base && !cuda_ok(c, cudaFree(c->epi_base))) return kCuda;
        c->epi_base = nullptr;
        c->epi_cap = 0;
        if (cudaMalloc(&c->epi_base, epi_scratch_bytes(n_samples)) != cudaSuccess) {
            cudaGetLastError();
            c->epi_base = nullptr;
            return VOLDOR_ERR_OOM;
        }
        c->epi_cap = n_samples;
    }
    EpiState e;
    epi_layout(c->epi_base, n_samples, reinterpret_cast<float4*>(c->ds.pix), &e);
    c->launches += launch_epipolar(c->dp, c->ds, e, baseline, c->stream);
    if (!launched(c)) return kCuda;
    c->epi_M = n_samples;
    double T1d[12];
    long long info[8];
    if (!cuda_ok(c, cudaMemcpyAsync(T1d, e.T1, sizeof(T1d), cudaMemcpyDeviceToHost, c->stream)) ||
        !cuda_ok(c, cudaMemcpyAsync(info, e.info, sizeof(info), cudaMemcpyDeviceToHost, c->stream)) ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream)))
        return kCuda;
    if (info[0] < 0) return VOLDOR_ERR_DEGENERATE;
    double T1[16] = {0};
    for (int q = 0; q < 12; ++q) T1[q] = T1d[q];
    T1[15] = 1.0;
    for (int q = 0; q < 12; ++q)
        if (!std::isfinite(T1[q])) return VOLDOR_ERR_DEGENERATE;
    launch_bootstrap(c->dp, c->ds, T1, c->stream);
    c->launches += 1;
    if (!cuda_ok(c, cudaMemsetAsync(c->ds.status, 0, 16, c->stream))) return kCuda;
    if (!launched(c)) return kCuda;
    c->bootstrapped = true;
    if (T1_out) std::memcpy(T1_out, T1, sizeof(T1));
    return VOLDOR_OK;
}

voldor_status voldor_ground_scale(voldor_ctx* c, double camera_height, double max_tilt_rad, int apply,
                                 double* scale_out)
{
    if (!c || !finite_pos(camera_height) || !(max_tilt_rad > 0.0 && max_tilt_rad < 1.5707963267948966))
        return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    if (!c->ground_base) {
        if (cudaMalloc(&c->ground_base, kGroundScratchBytes) != cudaSuccess) {
            cudaGetLastError();
            c->ground_base = nullptr;
            return VOLDOR_ERR_OOM;
        }
    }
    unsigned* hist = static_cast<unsigned*>(c->ground_base);
    double* out = reinterpret_cast<double*>(static_cast<char*>(c->ground_base) + 4096 * 4);
    c->launches += launch_ground_scale(c->dp, c->ds, camera_height, std::cos(max_tilt_rad),
                                       1.0 / c->params.inv_depth_max, 1.0 / c->params.inv_depth_min, apply, hist,
                                       out, c->stream);
    if (!launched(c)) return kCuda;
    double h[3];
    if (!cuda_ok(c, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) ||
        !cuda_ok(c, cudaStreamSynchronize(c->stream)))
        return kCuda;
    if (!(h[2] > 0.0)) return VOLDOR_ERR_DEGENERATE;
    if (scale_out) *scale_out = h[0];
    return VOLDOR_OK;
}

voldor_status voldor_bootstrap_learned(voldor_ctx* c, const double* T1, voldor_net* net, int flags)
{
    if (!c || !net || !T1 || (flags & ~(VOLDOR_LEARNED_DEPTH | VOLDOR_LEARNED_RIGIDNESS))) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(T1[i])) return VOLDOR_ERR_INVALID_ARG;
    launch_bootstrap(c->dp, c->ds, T1, c->stream);          // poses, k, W, and a triangulated depth
    c->launches += 1;
    if (!launched(c)) return kCuda;
    int kernels = 0;
    voldor_status s = net_bootstrap(net, c->ds.flows, c->flow_dtype == VOLDOR_FLOW_F16, c->W, c->H, c->T,
                                    (float)(1.0 / c->params.inv_depth_max), (float)(1.0 / c->params.inv_depth_min),
                                    flags, c->ds.theta, c->ds.wmap, c->stream, &kernels);
    c->launches += kernels;
    if (s != VOLDOR_OK) return s == VOLDOR_ERR_CUDA ? (c->poisoned = true, kCuda) : s;
    if (!cuda_ok(c, cudaMemsetAsync(c->ds.status, 0, 16, c->stream))) return kCuda;
    c->bootstrapped = true;
    return VOLDOR_OK;
}

voldor_status voldor_em_step(voldor_ctx* c, int n_iters)
{
    if (!c || n_iters < 0) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    if (n_iters == 0) return VOLDOR_OK;
    const long long key = (long long)n_iters * 2 + (c->timing ? 1 : 0);
    if (!ensure_graph(c, n_iters, c->timing)) return kCuda;
    auto it = c->graphs.find(key);
    if (!cuda_ok(c, cudaMemsetAsync(c->ds.status + 3, 0, 4, c->stream))) return kCuda;
    if (c->timing && !cuda_ok(c, cudaMemsetAsync(c->ds.score_log, 0, (size_t)kScoreLogMax * 16, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaGraphLaunch(it->second, c->stream))) return kCuda;
    c->launches += c->graph_kernels[key];
    c->last_pairs = c->timing ? n_iters * c->T : 0;
    int st4[4];
    voldor_status rs = read_status_word(c, st4);
    if (rs != VOLDOR_OK) return rs;
    return status_of_word(st4[3]);
}

voldor_status voldor_get_pose_depth_rigidness(voldor_ctx* c, double* poses, float* depth, float* rigidness)
{
    if (!c) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    std::vector<double> p12;
    if (poses) {
        p12.resize((size_t)c->T * 12);
        if (!cuda_ok(c, cudaMemcpyAsync(p12.data(), c->ds.poses, p12.size() * 8, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    }
    if (depth && !cuda_ok(c, cudaMemcpyAsync(depth, c->ds.theta, (size_t)c->N * 4, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (rigidness && !cuda_ok(c, cudaMemcpyAsync(rigidness, c->ds.wmap, (size_t)c->T * c->N * 4, cudaMemcpyDeviceToHost, c->stream)))
        return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    if (poses) {
        for (int t = 0; t < c->T; ++t) {
            for (int q = 0; q < 12; ++q) poses[16 * t + q] = p12[12 * t + q];
            poses[16 * t + 12] = 0; poses[16 * t + 13] = 0; poses[16 * t + 14] = 0; poses[16 * t + 15] = 1;
        }
    }
    return VOLDOR_OK;
}

void voldor_destroy(voldor_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graphs(c);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->aux) { cudaStreamSynchronize(c->aux); cudaStreamDestroy(c->aux); }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_fork2) cudaEventDestroy(c->ev_fork2);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    if (c->arena) cudaFree(c->arena);
    if (c->epi_base) cudaFree(c->epi_base);
    if (c->ground_base) cudaFree(c->ground_base);
    cudaGetLastError();
    delete c;
}

voldor_status voldor_set_state(voldor_ctx* c, const double* poses, const float* depth, const float* rigidness, int iteration)
{
    if (!c || iteration < 0) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (poses) {
        std::vector<double> p12((size_t)c->T * 12);
        for (int t = 0; t < c->T; ++t)
            for (int q = 0; q < 12; ++q) {
                p12[12 * t + q] = poses[16 * t + q];
                if (!std::isfinite(p12[12 * t + q])) return VOLDOR_ERR_INVALID_ARG;
            }
        if (!cuda_ok(c, cudaMemcpyAsync(c->ds.poses, p12.data(), p12.size() * 8, cudaMemcpyHostToDevice, c->stream))) return kCuda;
        if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    }
    if (depth && !cuda_ok(c, cudaMemcpyAsync(c->ds.theta, depth, (size_t)c->N * 4, cudaMemcpyHostToDevice, c->stream))) return kCuda;
    if (rigidness && !cuda_ok(c, cudaMemcpyAsync(c->ds.wmap, rigidness, (size_t)c->T * c->N * 4, cudaMemcpyHostToDevice, c->stream)))
        return kCuda;
    launch_set_iteration(c->ds, iteration, c->stream);
    if (!launched(c)) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    c->bootstrapped = true;
    return VOLDOR_OK;
}

voldor_status voldor_pose_update(voldor_ctx* c, int k, int t)
{
    if (!c || k < 0 || t < 1) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (t > c->T) return VOLDOR_ERR_INVALID_ARG;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    if (!cuda_ok(c, cudaMemsetAsync(c->ds.status, 0, 16, c->stream))) return kCuda;
    launch_set_iteration(c->ds, k, c->stream);
    if (!enqueue_pose_update(c, t, nullptr, nullptr, -1)) return kCuda;
    int st4[4];
    voldor_status rs = read_status_word(c, st4);
    if (rs != VOLDOR_OK) return rs;
    return status_of_word(st4[3]);
}

voldor_status voldor_score_hypotheses(voldor_ctx* c, int t, int n, const double* R, const double* tv, double* L)
{
    if (!c || t < 1 || n < 1 || !R || !tv || !L) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (t > c->T || n > c->params.hyps_per_frame) return VOLDOR_ERR_INVALID_ARG;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    std::vector<double> h((size_t)n * 12);
    for (int i = 0; i < n; ++i) {
        for (int q = 0; q < 9; ++q) h[12 * i + q] = R[9 * i + q];
        for (int q = 0; q < 3; ++q) h[12 * i + 9 + q] = tv[3 * i + q];
        for (int q = 0; q < 12; ++q)
            if (!std::isfinite(h[12 * i + q])) return VOLDOR_ERR_INVALID_ARG;
    }
    if (!cuda_ok(c, cudaMemcpyAsync(c->ds.hyp_Rt, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream))) return kCuda;
    launch_frame_setup(c->dp, c->ds, c->stream);
    launch_pose_prep(c->dp, c->ds, t, c->stream);
    score_hyps_from_host(c->dp, c->ds, n, c->stream);
    launch_score(c->dp, c->ds, -1, c->stream);
    launch_score_reduce(c->dp, c->ds, c->stream);
    c->launches += 6;
    if (!launched(c)) return kCuda;
    if (!cuda_ok(c, cudaMemcpyAsync(L, c->ds.scores, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    return VOLDOR_OK;
}

voldor_status voldor_rigidness_smooth(voldor_ctx* c, int k)
{
    if (!c || k < 0) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    launch_set_iteration(c->ds, k, c->stream);
    return enqueue_smooth(c) ? VOLDOR_OK : kCuda;
}

voldor_status voldor_depth_update(voldor_ctx* c, int k)
{
    if (!c || k < 0) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    launch_set_iteration(c->ds, k, c->stream);
    return enqueue_depth(c) ? VOLDOR_OK : kCuda;
}

voldor_status voldor_rigidness_update(voldor_ctx* c)
{
    if (!c) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    return enqueue_rigidness(c) ? VOLDOR_OK : kCuda;
}

static bool buffer_of(voldor_ctx* c, int which, void** dev, size_t* bytes, bool* writable)
{
    const size_t N = (size_t)c->N, T = (size_t)c->T, S = (size_t)c->params.hyps_per_frame;
    *writable = false;
    switch (which) {
        case VOLDOR_BUF_SMOOTHED: *dev = c->ds.qs; *bytes = T * N * 4; *writable = true; return true;
        case VOLDOR_BUF_LABELS: *dev = c->ds.labels; *bytes = N; return true;
        case VOLDOR_BUF_HYPS: *dev = c->ds.hyp_Rt; *bytes = S * 12 * 8; return true;
        case VOLDOR_BUF_HYP_INFO: *dev = c->ds.hyp_info; *bytes = S * 2 * 8; return true;
        case VOLDOR_BUF_HYP_WEIGHT: *dev = c->ds.hyp_w; *bytes = S * 8; return true;
        case VOLDOR_BUF_SCORES: *dev = c->ds.scores; *bytes = S * 8; return true;
        case VOLDOR_BUF_POSE_INFO: *dev = c->ds.status; *bytes = 16; return true;
        case VOLDOR_BUF_DEPTH_SAMPLES: *dev = c->ds.mie_smp; *bytes = N * 4; return true;
        case VOLDOR_BUF_HYPS_F32: *dev = c->ds.hyp_f32; *bytes = S * 12 * 4; return true;
        case VOLDOR_BUF_EPI_E:
        case VOLDOR_BUF_EPI_MEDIANS:
        case VOLDOR_BUF_EPI_VALID:
        case VOLDOR_BUF_EPI_INFO:
        case VOLDOR_BUF_EPI_REFINED: {
            if (!c->epi_base || c->epi_M < 1) return false;
            EpiState e;
            epi_layout(c->epi_base, c->epi_M, reinterpret_cast<float4*>(c->ds.pix), &e);
            const size_t M = (size_t)c->epi_M;
            if (which == VOLDOR_BUF_EPI_E) { *dev = e.E; *bytes = M * 9 * 8; }
            else if (which == VOLDOR_BUF_EPI_MEDIANS) { *dev = e.median; *bytes = M * 4; }
            else if (which == VOLDOR_BUF_EPI_VALID) { *dev = e.valid; *bytes = M * 4; }
            else if (which == VOLDOR_BUF_EPI_INFO) { *dev = e.info; *bytes = 8 * 8; }
            else { *dev = e.refined; *bytes = 27 * 8; }
            return true;
        }
    }
    return false;
}

voldor_status voldor_get_buffer(voldor_ctx* c, int which, void* host, size_t bytes)
{
    if (!c || !host) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    void* dev;
    size_t size;
    bool w;
    if (!buffer_of(c, which, &dev, &size, &w) || bytes > size) return VOLDOR_ERR_INVALID_ARG;
    if (!cuda_ok(c, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    return VOLDOR_OK;
}

voldor_status voldor_set_buffer(voldor_ctx* c, int which, const void* host, size_t bytes)
{
    if (!c || !host) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    void* dev;
    size_t size;
    bool w;
    if (!buffer_of(c, which, &dev, &size, &w) || !w || bytes > size) return VOLDOR_ERR_INVALID_ARG;
    if (!cuda_ok(c, cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    return VOLDOR_OK;
}

voldor_status voldor_enable_timing(voldor_ctx* c, int on)
{
    if (!c) return VOLDOR_ERR_INVALID_ARG;
    c->timing = on != 0;
    return VOLDOR_OK;
}

voldor_status voldor_get_score_times(voldor_ctx* c, float* ms, long long* pairs, long long* hyps, int max, int* count)
{
    if (!c || !count || (max > 0 && !ms)) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    *count = c->last_pairs;
    for (int i = 0; i < c->last_pairs && i < max; ++i)
        if (!cuda_ok(c, cudaEventElapsedTime(&ms[i], c->events[2 * i], c->events[2 * i + 1]))) return kCuda;
    if (pairs || hyps) {
        const int n = std::min(std::min(c->last_pairs, max), kScoreLogMax);
        std::vector<long long> log((size_t)2 * (n > 0 ? n : 1));
        if (n > 0) {
            if (!cuda_ok(c, cudaMemcpy(log.data(), c->ds.score_log, (size_t)n * 16, cudaMemcpyDeviceToHost))) return kCuda;
            for (int i = 0; i < n; ++i) {
                if (pairs) pairs[i] = log[2 * i] * log[2 * i + 1];
                if (hyps) hyps[i] = log[2 * i];
            }
        }
    }
    return VOLDOR_OK;
}

long long voldor_kernel_launches(const voldor_ctx* c) { return c ? c->launches : 0; }

const char* voldor_last_error_string(const voldor_ctx* c)
{
    if (!c || c->first_error == cudaSuccess) return "no CUDA error";
    return cudaGetErrorString(c->first_error);
}

size_t voldor_device_bytes(const voldor_ctx* c) { return c ? c->arena_bytes : 0; }

voldor_status voldor_autotune(voldor_ctx* c, int* hpt_out, int* chunks_out, float* best_ms_out)
{
    if (!c) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (!c->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    // hypotheses and pixel records of frame 1 on the current state
    int k_saved = 0;
    if (!cuda_ok(c, cudaMemcpyAsync(&k_saved, c->ds.iter, 4, cudaMemcpyDeviceToHost, c->stream))) return kCuda;
    if (!cuda_ok(c, cudaStreamSynchronize(c->stream))) return kCuda;
    launch_frame_setup(c->dp, c->ds, c->stream);
    launch_pose_prep(c->dp, c->ds, 1, c->stream);
    launch_p3p_groups(c->dp, c->ds, 1, c->stream);
    launch_hyp_collect(c->dp, c->ds, c->stream);
    if (!launched(c)) return kCuda;
    cudaEvent_t e0, e1;
    if (!cuda_ok(c, cudaEventCreate(&e0)) || !cuda_ok(c, cudaEventCreate(&e1))) return kCuda;
    const int saved_hpt = c->ds.score_hpt, saved_chunks = c->ds.n_chunks;
    int best_hpt = saved_hpt, best_chunks = saved_chunks;
    float best = 1e30f;
    bool ok = true;
    const int hpts[3] = {8, 4, 2};
    const int waves[4] = {1, 2, 4, kTuneMaxWaves};
    for (int hi = 0; hi < 3 && ok; ++hi) {
        for (int wi = 0; wi < 4 && ok; ++wi) {
            c->ds.score_hpt = hpts[hi];
            c->ds.n_chunks = score_chunks_for(c->params.hyps_per_frame, c->N, hpts[hi], waves[wi]);
            launch_score(c->dp, c->ds, -1, c->stream);            // warm-up
            float ms[3];
            for (int r = 0; r < 3 && ok; ++r) {
                ok = cuda_ok(c, cudaEventRecord(e0, c->stream));
                launch_score(c->dp, c->ds, -1, c->stream);
                ok = ok && cuda_ok(c, cudaEventRecord(e1, c->stream)) && cuda_ok(c, cudaEventSynchronize(e1)) &&
                     cuda_ok(c, cudaEventElapsedTime(&ms[r], e0, e1)) && launched(c);
            }
            if (!ok) break;
            std::sort(ms, ms + 3);
            if (ms[1] < best) { best = ms[1]; best_hpt = hpts[hi]; best_chunks = c->ds.n_chunks; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return kCuda;
    c->ds.score_hpt = best_hpt;
    c->ds.n_chunks = best_chunks;
    if (best_hpt != saved_hpt || best_chunks != saved_chunks) drop_graphs(c);   // they captured the old shape
    launch_set_iteration(c->ds, k_saved, c->stream);
    if (!launched(c)) return kCuda;
    if (hpt_out) *hpt_out = best_hpt;
    if (chunks_out) *chunks_out = best_chunks;
    if (best_ms_out) *best_ms_out = best;
    return VOLDOR_OK;
}

voldor_status voldor_set_score_shape(voldor_ctx* c, int hpt, int chunks)
{
    if (!c || (hpt != 2 && hpt != 4 && hpt != 8) || chunks < 1) return VOLDOR_ERR_INVALID_ARG;
    if (chunks > score_chunks_max(c->params.hyps_per_frame, c->N)) return VOLDOR_ERR_INVALID_ARG;
    if (c->poisoned) return kCuda;
    if (hpt != c->ds.score_hpt || chunks != c->ds.n_chunks) {
        c->ds.score_hpt = hpt;
        c->ds.n_chunks = chunks;
        drop_graphs(c);
    }
    return VOLDOR_OK;
}

struct voldor_batch {
    std::vector<voldor_ctx*> ctxs;
    int n_iters = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t start = nullptr;
    std::vector<cudaEvent_t> done;
};

void voldor_batch_destroy(voldor_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->start) cudaEventDestroy(b->start);
    for (cudaEvent_t e : b->done) cudaEventDestroy(e);
    cudaGetLastError();
    delete b;
}

voldor_status voldor_batch_create(voldor_ctx* const* ctxs, int n, int n_iters, voldor_batch** out)
{
    if (!out) return VOLDOR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctxs || n < 1 || n_iters < 1) return VOLDOR_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return VOLDOR_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return VOLDOR_ERR_INVALID_ARG;     // a window may appear once
        if (ctxs[i]->poisoned) return kCuda;
        if (!ctxs[i]->bootstrapped) return VOLDOR_ERR_NOT_BOOTSTRAPPED;
    }
    voldor_batch* b = new (std::nothrow) voldor_batch();
    if (!b) return VOLDOR_ERR_OOM;
    b->ctxs.assign(ctxs, ctxs + n);
    b->n_iters = n_iters;
    auto fail = [&](voldor_status st) { voldor_batch_destroy(b); return st; };
    for (int i = 0; i < n; ++i)
        if (!ensure_graph(ctxs[i], n_iters, false)) return fail(kCuda);
    if (cudaEventCreate(&b->start) != cudaSuccess) return fail(kCuda);
    b->done.resize(n, nullptr);
    for (int i = 0; i < n; ++i)
        if (cudaEventCreate(&b->done[i]) != cudaSuccess) return fail(kCuda);
    if (cudaGraphCreate(&b->graph, 0) != cudaSuccess) return fail(kCuda);
    cudaGraphNode_t start_node;
    if (cudaGraphAddEventRecordNode(&start_node, b->graph, nullptr, 0, b->start) != cudaSuccess) return fail(kCuda);
    const long long key = (long long)n_iters * 2;
    for (int i = 0; i < n; ++i) {
        voldor_ctx* c = ctxs[i];
        cudaGraphNode_t reset, child, fin;
        cudaMemsetParams mp{};
        mp.dst = c->ds.status + 3;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = 1;
        mp.height = 1;
        if (cudaGraphAddMemsetNode(&reset, b->graph, &start_node, 1, &mp) != cudaSuccess) return fail(kCuda);
        if (cudaGraphAddChildGraphNode(&child, b->graph, &reset, 1, c->raw_graphs[key]) != cudaSuccess) return fail(kCuda);
        if (cudaGraphAddEventRecordNode(&fin, b->graph, &child, 1, b->done[i]) != cudaSuccess) return fail(kCuda);
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(kCuda);
    *out = b;
    return VOLDOR_OK;
}

voldor_status voldor_batch_run(voldor_batch* b, void* cuda_stream, float* latency_ms)
{
    if (!b) return VOLDOR_ERR_INVALID_ARG;
    for (voldor_ctx* c : b->ctxs)
        if (c->poisoned) return kCuda;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) {
        for (voldor_ctx* c : b->ctxs) c->poisoned = true;
        return kCuda;
    }
    for (voldor_ctx* c : b->ctxs) c->launches += c->graph_kernels[(long long)b->n_iters * 2];
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        for (voldor_ctx* c : b->ctxs) c->poisoned = true;
        return kCuda;
    }
    voldor_status result = VOLDOR_OK;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        voldor_ctx* c = b->ctxs[i];
        if (latency_ms && cudaEventElapsedTime(&latency_ms[i], b->start, b->done[i]) != cudaSuccess) return kCuda;
        int deg = 0;
        if (cudaMemcpy(&deg, c->ds.status + 3, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return kCuda;
        const voldor_status ws = status_of_word(deg);
        if (ws == VOLDOR_ERR_TIMEOUT || (ws == VOLDOR_ERR_DEGENERATE && result == VOLDOR_OK)) result = ws;
    }
    return result;
}

voldor_status voldor_em_batch(voldor_ctx* const* ctxs, int n, int n_iters)
{
    voldor_batch* b = nullptr;
    voldor_status st = voldor_batch_create(ctxs, n, n_iters, &b);
    if (st != VOLDOR_OK) return st;
    st = voldor_batch_run(b, nullptr, nullptr);
    voldor_batch_destroy(b);
    return st;
}

}  // extern "C"
