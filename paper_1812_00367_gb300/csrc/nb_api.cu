// nb_api.cu -- host runtime behind the C ABI of include/nb.h.
//
// The context owns the device scratch (packed predicted j-arrays, active
// lists, plans, partial sums, counters) and the CUDA graphs that replay one
// block step (select -> plan -> predict -> evaluate+correct) without host
// round trips.  Kernel launches go to the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nb_internal.cuh"

namespace nb {
cudaError_t launch_eval_fp64(const Dev &, int, const EvalLaunch &, int, cudaStream_t);
cudaError_t launch_eval_ex(const Dev &, int, const EvalLaunch &, int, cudaStream_t);
cudaError_t launch_eval_fp32(const Dev &, int, const EvalLaunch &, int, cudaStream_t);
cudaError_t launch_eval_fp32x(const Dev &, int, const EvalLaunch &, int, cudaStream_t);
int occupancy_fp64(int);
int occupancy_ex(int);
int occupancy_fp32(int);
int occupancy_fp32x(int);
cudaError_t launch_unpack64(const Dev &d, double *out, cudaStream_t st);
cudaError_t launch_plan_ex(const Dev &d, int mode_init, int count, cudaStream_t st);

cudaError_t launch_eval(const Dev &d, int mode, const EvalLaunch &L, int grid, cudaStream_t st) {
    if (grid <= 0) return cudaSuccess;
    if (mode == kModePot) return launch_eval_fp64(d, mode, L, grid, st);
    switch (d.precision) {
    case NB_FP64: return launch_eval_fp64(d, mode, L, grid, st);
    case NB_EX: return launch_eval_ex(d, mode, L, grid, st);
    case NB_FP32: return launch_eval_fp32(d, mode, L, grid, st);
    case NB_FP32X: return launch_eval_fp32x(d, mode, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}
int eval_occupancy(int precision, int mode) {
    if (mode == kModePot) return occupancy_fp64(mode);
    switch (precision) {
    case NB_FP64: return occupancy_fp64(mode);
    case NB_EX: return occupancy_ex(mode);
    case NB_FP32X: return occupancy_fp32x(mode);
    default: return occupancy_fp32(mode);
    }
}
}  // namespace nb

using namespace nb;

struct nb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;      // caller's stream (launches, graph replays)
    cudaStream_t cap_stream = nullptr;  // private stream used only for capture
    cudaStream_t cap_side = nullptr;    // second capture branch (predictor)
    cudaStream_t cap_side2 = nullptr;   // third capture branch (planner)
    cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
    nb_params p{};
    int64_t n = 0;
    int32_t nc = 1;
    std::vector<int64_t> h_offsets, h_jofs;
    std::vector<int32_t> h_chunk0;       // first chunk of each cluster [nc + 1]
    int64_t max_cluster = 0;
    Dev d{};
    Dev d_pot{};  // FP64 view for energy
    std::vector<void *> allocs;
    int sm_count = 0;
    int grid_eval = 0, grid_pot = 0;
    int64_t cap_items = 0;
    std::vector<PlanEntry> table;
    PlanEntry *d_table = nullptr;
    cudaGraphExec_t g_step = nullptr;    // one block step
    cudaGraphExec_t g_multi = nullptr;   // kMultiSteps block steps + busy readback
    int32_t *h_busy = nullptr;           // pinned
    double *h_tend = nullptr;            // pinned
    std::string err;
    // launch accounting and evaluation timing (NB_TIME_EVAL)
    int64_t launches = 0;
    int64_t eval_launches = 0;
    double eval_ms = 0.0;
    std::vector<cudaEvent_t> ev;         // [2 * (kMultiSteps + 1)]: start/end pairs
};

namespace {
constexpr int kMultiSteps = 16;
thread_local std::string g_init_err;

nb_status fail(nb_ctx *ctx, nb_status s, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_init_err = msg;
    return s;
}
nb_status cuda_fail(nb_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, NB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define NB_CU(ctx, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

bool is_pow2(double x) {
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

template <typename T>
cudaError_t dalloc(nb_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

// Default plan: lanes per i from the active-set size; splits aim at a few
// waves of the persistent grid.  nb_autotune replaces it with measurements.
void default_table(nb_ctx *ctx) {
    ctx->table.assign(kBuckets, PlanEntry{1, 1});
    for (int b = 0; b < kBuckets; ++b) {
        const double A = std::ldexp(1.0, b);
        int gl = 1;
        if (A < 64) gl = 32;
        else if (A < 1024) gl = 8;
        else if (A < 4096) gl = 2;
        // per-cluster split target: a few waves of the grid for one cluster,
        // shared out when many clusters advance together
        // (a batch keeps the grid busy with many clusters; its per-cluster
        // target shrinks with the fourth root of the cluster count: for 512
        // clusters the measured FP64 rate rose from 7.2e9 at 9 items per
        // cluster to 1.10e10 at 215 and 1.12e10 at 1216)
        const int64_t tgt = std::max<int64_t>(
            1, (int64_t)(8.0 * ctx->grid_eval / std::pow((double)ctx->nc, 0.25)));
        ctx->table[b] = PlanEntry{gl, (int32_t)tgt};
    }
}

nb_status upload_table(nb_ctx *ctx) {
    NB_CU(ctx, cudaMemcpyAsync(ctx->d_table, ctx->table.data(), kBuckets * sizeof(PlanEntry),
                               cudaMemcpyHostToDevice, ctx->stream));
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return NB_OK;
}

nb_status check_device_error(nb_ctx *ctx) {
    uint32_t err = 0;
    NB_CU(ctx, cudaMemcpy(&err, ctx->d.err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err & kErrTimeout) return fail(ctx, NB_ETIMEOUT, "device: a bounded wait timed out");
    if (err & kErrIndex) return fail(ctx, NB_EINVAL, "device: an active index lies outside its cluster");
    if (err & kErrNonFinite) return fail(ctx, NB_ENONFINITE, "device: non-finite value in the state");
    return NB_OK;
}

constexpr int kKernelsPerStep = 5;

// Enqueue one block step (all clusters) on stream st; `slot` selects the
// event pair timing its evaluation launch (-1: none).
cudaError_t enqueue_step(nb_ctx *ctx, cudaStream_t st, int slot) {
    cudaError_t e;
    if ((e = launch_select_min(ctx->d, st)) != cudaSuccess) return e;
    // the compaction, the planner and the predictor all need only pass 1's
    // t_next and counts: three graph branches, joined before the evaluation
    if ((e = cudaEventRecord(ctx->fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->cap_side, ctx->fork, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(ctx->cap_side2, ctx->fork, 0)) != cudaSuccess) return e;
    if ((e = launch_predict(ctx->d, 0, 0, 0.0, ctx->cap_side)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ctx->join, ctx->cap_side)) != cudaSuccess) return e;
    if ((e = launch_plan_ex(ctx->d, 0, 1, ctx->cap_side2)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ctx->join2, ctx->cap_side2)) != cudaSuccess) return e;
    if ((e = launch_select_compact(ctx->d, 0.0, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, ctx->join, 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, ctx->join2, 0)) != cudaSuccess) return e;
    EvalLaunch L{};
    if (slot >= 0 && (e = cudaEventRecordWithFlags(ctx->ev[2 * slot], st, cudaEventRecordExternal)) != cudaSuccess)
        return e;
    const int mode = ctx->d.order == 4 ? kModeStep4 : kModeStep;
    if ((e = launch_eval(ctx->d, mode, L, ctx->grid_eval, st)) != cudaSuccess) return e;
    if (slot >= 0 && (e = cudaEventRecordWithFlags(ctx->ev[2 * slot + 1], st, cudaEventRecordExternal)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// After a synchronised replay: add the timed evaluation launches.
void harvest_events(nb_ctx *ctx, int first, int count) {
    if (ctx->ev.empty()) return;
    for (int k = first; k < first + count; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * k], ctx->ev[2 * k + 1]) == cudaSuccess) {
            ctx->eval_ms += ms;
            ctx->eval_launches += 1;
        }
    }
}

nb_status build_graphs(nb_ctx *ctx) {
    if (ctx->g_step) return NB_OK;
    for (int which = 0; which < 2; ++which) {
        cudaGraph_t g = nullptr;
        NB_CU(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        const int steps = which == 0 ? 1 : kMultiSteps;
        const bool timed = !ctx->ev.empty();
        for (int k = 0; k < steps && e == cudaSuccess; ++k)
            e = enqueue_step(ctx, ctx->cap_stream, !timed ? -1 : (which == 0 ? kMultiSteps : k));
        if (e == cudaSuccess && which == 1)
            e = cudaMemcpyAsync(ctx->h_busy, ctx->d.busy, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                ctx->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "capture");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        (which == 0 ? ctx->g_step : ctx->g_multi) = ex;
    }
    return NB_OK;
}

nb_status set_tend(nb_ctx *ctx, double t_end) {
    *ctx->h_tend = t_end;
    NB_CU(ctx, cudaMemcpyAsync(ctx->d.t_end, ctx->h_tend, sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream));
    return NB_OK;
}

// Plan a direct (host-driven) evaluation of n_active particles of one cluster.
void plan_direct(const nb_ctx *ctx, int cluster, int32_t n_active, int &gl, int &split, int &tiles,
                 int &streamk, int64_t jtiles = -1) {
    const int b = 31 - __builtin_clz((unsigned)std::max(n_active, 1));
    const PlanEntry e = ctx->table[b];
    gl = e.gl;
    tiles = (int)cdiv(n_active, kTPB / gl);
    const int64_t ncl = ctx->h_offsets[cluster + 1] - ctx->h_offsets[cluster];
    const int64_t ntj = jtiles >= 0 ? jtiles : cdiv(ncl, kTJ);  // j-tiles evaluated
    streamk = !(ctx->p.flags & NB_NO_STREAMK) &&
              sk_use(tiles, kTPB / gl, ntj, ctx->grid_eval, ctx->d.partial_cap) ? 1 : 0;
    if (streamk) {
        split = 1;
        return;
    }
    int64_t S = choose_split(tiles, ntj, e.target_items, ctx->grid_eval);
    const int64_t per_item = 10LL * (kTPB / gl);  // partial doubles per item
    if (S > 1 && (int64_t)tiles * S * per_item > ctx->d.partial_cap)
        S = std::max<int64_t>(1, ctx->d.partial_cap / (per_item * tiles));
    split = (int)S;
}
nb_status eval_direct(nb_ctx *ctx, int cluster, const int32_t *active, int32_t n_active, double *out,
                      int gl, int split, int tiles, int streamk, int32_t jt0 = 0, int32_t jt1 = 0) {
    EvalLaunch L{};
    L.direct = 1;
    L.cluster = cluster;
    L.n_active = n_active;
    L.gl = gl;
    L.split = split;
    L.tiles = tiles;
    L.active = active;
    L.out = out;
    L.streamk = streamk;
    L.jt0 = jt0;
    L.jt1 = jt1;
    const int64_t items = (int64_t)tiles * split;
    // stream-K ranges were cut for the whole persistent grid
    const int grid = streamk ? ctx->grid_eval : (int)std::min<int64_t>(items, ctx->grid_eval);
    NB_CU(ctx, launch_eval(ctx->d, ctx->d.order == 4 ? kModeOut4 : kModeOut, L, grid, ctx->stream));
    return NB_OK;
}

// Start-up: the two evaluation passes (a, jerk with a = 0; then snap), dt0;
// the 4th-order scheme takes the first pass only (a, jerk; dt0 from |a|/|j|).
nb_status startup(nb_ctx *ctx) {
    NB_CU(ctx, launch_init_clear(ctx->d, ctx->stream));
    const bool order4 = ctx->d.order == 4;
    for (int pass = 0; pass < (order4 ? 1 : 2); ++pass) {
        NB_CU(ctx, launch_predict(ctx->d, 0, 1, 0.0, ctx->stream));
        NB_CU(ctx, launch_plan_ex(ctx->d, 1, 0, ctx->stream));
        EvalLaunch L{};
        L.identity = 1;
        const int mode = order4 ? kModeInit4 : (pass == 0 ? kModeInit1 : kModeInit2);
        NB_CU(ctx, launch_eval(ctx->d, mode, L, ctx->grid_eval, ctx->stream));
    }
    return NB_OK;
}
}  // namespace

namespace nb {
// Message for nb_last_error(NULL) from calls that have no context.
void set_global_error(const char *msg) { g_init_err = msg; }
}  // namespace nb

// =================================================================== ABI
extern "C" {

const char *nb_status_string(nb_status s) {
    switch (s) {
    case NB_OK: return "NB_OK";
    case NB_EINVAL: return "NB_EINVAL";
    case NB_ENOMEM: return "NB_ENOMEM";
    case NB_ECUDA: return "NB_ECUDA";
    case NB_ENONFINITE: return "NB_ENONFINITE";
    case NB_EDTUNDERFLOW: return "NB_EDTUNDERFLOW";
    case NB_ETIMEOUT: return "NB_ETIMEOUT";
    case NB_ESTATE: return "NB_ESTATE";
    }
    return "NB_UNKNOWN";
}

const char *nb_last_error(const nb_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_init_err.c_str();
}

void nb_free(nb_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->g_step) cudaGraphExecDestroy(ctx->g_step);
    if (ctx->g_multi) cudaGraphExecDestroy(ctx->g_multi);
    for (void *q : ctx->allocs) cudaFree(q);
    if (ctx->h_busy) cudaFreeHost(ctx->h_busy);
    if (ctx->h_tend) cudaFreeHost(ctx->h_tend);
    for (cudaEvent_t ev : ctx->ev) cudaEventDestroy(ev);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cap_side) cudaStreamDestroy(ctx->cap_side);
    if (ctx->cap_side2) cudaStreamDestroy(ctx->cap_side2);
    if (ctx->join2) cudaEventDestroy(ctx->join2);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    delete ctx;
}

nb_status nb_init(nb_ctx **out, const nb_params *p, int64_t n, const nb_state *st, int32_t n_clusters,
                  const int64_t *cluster_offsets, void *stream) {
    if (!out) return fail(nullptr, NB_EINVAL, "nb_init: out is NULL");
    *out = nullptr;
    if (!p || !st) return fail(nullptr, NB_EINVAL, "nb_init: NULL params or state");
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(nullptr, NB_EINVAL, "nb_init: n out of range");
    if (n_clusters < 1 || n_clusters > n) return fail(nullptr, NB_EINVAL, "nb_init: bad n_clusters");
    if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return fail(nullptr, NB_EINVAL, "nb_init: eps < 0");
    if (!(p->eta > 0.0) || !(p->eta_init > 0.0)) return fail(nullptr, NB_EINVAL, "nb_init: eta <= 0");
    if (!is_pow2(p->dt_min) || !is_pow2(p->dt_max) || p->dt_min > p->dt_max)
        return fail(nullptr, NB_EINVAL, "nb_init: dt_min/dt_max must be powers of two, min <= max");
    if (p->precision < NB_FP64 || p->precision > NB_FP32X)
        return fail(nullptr, NB_EINVAL, "nb_init: unknown precision");
    if (p->order != 0 && p->order != 4 && p->order != 6)
        return fail(nullptr, NB_EINVAL, "nb_init: order must be 4 or 6 (0 = 6)");
    if (p->reserved != 0) return fail(nullptr, NB_EINVAL, "nb_init: reserved must be 0");
    if (!st->m || !st->x || !st->v || !st->a || !st->j || !st->s || !st->c || !st->t || !st->dt || !st->pot)
        return fail(nullptr, NB_EINVAL, "nb_init: NULL state buffer");
    std::vector<int64_t> offs(n_clusters + 1);
    if (cluster_offsets) {
        for (int c = 0; c <= n_clusters; ++c) offs[c] = cluster_offsets[c];
        if (offs[0] != 0 || offs[n_clusters] != n)
            return fail(nullptr, NB_EINVAL, "nb_init: offsets must start at 0 and end at n");
        for (int c = 0; c < n_clusters; ++c)
            if (offs[c + 1] <= offs[c]) return fail(nullptr, NB_EINVAL, "nb_init: empty or decreasing cluster");
    } else {
        if (n_clusters != 1) return fail(nullptr, NB_EINVAL, "nb_init: offsets required for n_clusters > 1");
        offs[0] = 0;
        offs[1] = n;
    }

    nb_ctx *ctx = new nb_ctx();
    ctx->p = *p;
    ctx->n = n;
    ctx->nc = n_clusters;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->h_offsets = offs;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_side2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_busy, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_tend, sizeof(double));
    if (e != cudaSuccess) {
        nb_status s = cuda_fail(nullptr, e, "nb_init: setup");
        nb_free(ctx);
        return s;
    }
    // chunks and padded j offsets
    std::vector<int32_t> chunk_cluster, cluster_chunk0(n_clusters + 1);
    std::vector<int64_t> chunk_begin, chunk_end;
    ctx->h_jofs.assign(n_clusters + 1, 0);
    for (int c = 0; c < n_clusters; ++c) {
        cluster_chunk0[c] = (int32_t)chunk_cluster.size();
        for (int64_t b = offs[c]; b < offs[c + 1]; b += kChunk) {
            chunk_cluster.push_back(c);
            chunk_begin.push_back(b);
            chunk_end.push_back(std::min<int64_t>(b + kChunk, offs[c + 1]));
        }
        const int64_t ncl = offs[c + 1] - offs[c];
        ctx->max_cluster = std::max(ctx->max_cluster, ncl);
        ctx->h_jofs[c + 1] = ctx->h_jofs[c] + cdiv(ncl, kTJ) * kTJ;
    }
    cluster_chunk0[n_clusters] = (int32_t)chunk_cluster.size();
    ctx->h_chunk0 = cluster_chunk0;
    const int n_chunks = (int)chunk_cluster.size();
    const int64_t nj = ctx->h_jofs[n_clusters];

    Dev &d = ctx->d;
    d.n = n;
    d.n_clusters = n_clusters;
    d.n_chunks = n_chunks;
    d.precision = p->precision;
    d.order = p->order == 4 ? 4 : 6;
    d.streamk_off = (p->flags & NB_NO_STREAMK) ? 1 : 0;
    d.m = st->m; d.x = st->x; d.v = st->v; d.a = st->a; d.j = st->j; d.s = st->s; d.c = st->c;
    d.t = st->t; d.dt = st->dt; d.pot = st->pot;
    set_eps2(d, p->eps);
    d.eta = p->eta;
    d.eta_init = p->eta_init;
    d.dt_min = p->dt_min;
    d.dt_max = p->dt_max;
    d.neg_one = -1.0;
    d.neg_zero = -0.0;

    const int occ = std::max(1, eval_occupancy(p->precision, d.order == 4 ? kModeStep4 : kModeStep));
    ctx->grid_eval = occ * ctx->sm_count;
    ctx->grid_pot = std::max(1, eval_occupancy(NB_FP64, kModePot)) * ctx->sm_count;
    d.grid_eval = ctx->grid_eval;
    // split partial sums, in full-width items (10 x 128 doubles): 32 waves of
    // the grid for one cluster; a batch gets room for every cluster at twice
    // its default target (at most 2 GB), so the planner's fall-back to
    // unsplit work stays an exception
    {
        const double batch = 2.0 * n_clusters * (8.0 * ctx->grid_eval / std::pow((double)n_clusters, 0.25));
        const double two_gb_items = 2.0e9 / (10.0 * kTPB * sizeof(double));
        ctx->cap_items = (int64_t)std::max(32.0 * ctx->grid_eval, std::min(batch, two_gb_items));
    }
    d.partial_cap = ctx->cap_items * 10 * kTPB;  // doubles

    int64_t *d_offs = nullptr, *d_jofs = nullptr, *d_cb = nullptr, *d_ce = nullptr;
    int32_t *d_ccl = nullptr, *d_cc0 = nullptr;
    size_t jbytes = p->precision == NB_FP64 ? sizeof(J64)
                    : (p->precision == NB_FP32 ? sizeof(J32) : sizeof(JEX));  // EX, FP32X
#define ALLOC(ptr, cnt)                                                                      \
    do {                                                                                     \
        cudaError_t ee = dalloc(ctx, &(ptr), (cnt));                                         \
        if (ee != cudaSuccess) {                                                             \
            nb_status s = fail(nullptr, NB_ENOMEM, std::string("nb_init: cudaMalloc ") + #ptr); \
            cudaGetLastError();                                                              \
            nb_free(ctx);                                                                    \
            return s;                                                                        \
        }                                                                                    \
    } while (0)
    ALLOC(d_offs, n_clusters + 1);
    ALLOC(d_jofs, n_clusters + 1);
    ALLOC(d_cb, n_chunks);
    ALLOC(d_ce, n_chunks);
    ALLOC(d_ccl, n_chunks);
    ALLOC(d_cc0, n_clusters + 1);
    unsigned char *jraw = nullptr;
    ALLOC(jraw, nj * jbytes);
    d.jarr = jraw;
    if (p->precision == NB_FP64) {
        d.jarr64 = reinterpret_cast<J64 *>(jraw);
    } else {
        ALLOC(d.jarr64, nj);
    }
    ALLOC(d.chunk_min, n_chunks);
    ALLOC(d.chunk_cnt, n_chunks);
    ALLOC(d.tnext, n_clusters);
    ALLOC(d.nact, n_clusters);
    ALLOC(d.active, n);
    ALLOC(d.plan, n_clusters);
    ALLOC(d.n_items, 1);
    ALLOC(d.item_ctr, 1);
    ALLOC(d.sel_ctr, 1);
    ALLOC(ctx->d_table, kBuckets);
    ALLOC(d.partial, ctx->cap_items * 10 * kTPB);
    const int64_t max_tiles = n + n_clusters + 1;
    ALLOC(d.tile_cnt, max_tiles);
    ALLOC(d.ctr_steps, 1);
    ALLOC(d.ctr_inter, 1);
    ALLOC(d.ctr_underflow, 1);
    ALLOC(d.err, 1);
    ALLOC(d.busy, 1);
    ALLOC(d.t_end, 1);
    ALLOC(d.pot_tmp, n);
    ALLOC(d.energy_part, (int64_t)n_chunks * 8);
#undef ALLOC
    d.offsets = d_offs;
    d.jofs = d_jofs;
    d.chunk_begin = d_cb;
    d.chunk_end = d_ce;
    d.chunk_cluster = d_ccl;
    d.cluster_chunk0 = d_cc0;
    d.table = ctx->d_table;
    ctx->d_pot = d;
    ctx->d_pot.jarr = d.jarr64;
    ctx->d_pot.precision = NB_FP64;
    ctx->d_pot.grid_eval = ctx->grid_pot;

    default_table(ctx);
    if (p->flags & NB_TIME_EVAL) {
        ctx->ev.resize(2 * (kMultiSteps + 1));
        for (auto &ev : ctx->ev) {
            if (cudaEventCreate(&ev) != cudaSuccess) {
                nb_status s = cuda_fail(nullptr, cudaGetLastError(), "nb_init: cudaEventCreate");
                nb_free(ctx);
                return s;
            }
        }
    }
    cudaStream_t s0 = ctx->stream;
    bool ok = true;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (ok && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s0) != cudaSuccess) ok = false;
    };
    up(d_offs, offs.data(), offs.size() * sizeof(int64_t));
    up(d_jofs, ctx->h_jofs.data(), ctx->h_jofs.size() * sizeof(int64_t));
    up(d_cb, chunk_begin.data(), chunk_begin.size() * sizeof(int64_t));
    up(d_ce, chunk_end.data(), chunk_end.size() * sizeof(int64_t));
    up(d_ccl, chunk_cluster.data(), chunk_cluster.size() * sizeof(int32_t));
    up(d_cc0, cluster_chunk0.data(), cluster_chunk0.size() * sizeof(int32_t));
    up(ctx->d_table, ctx->table.data(), kBuckets * sizeof(PlanEntry));
    if (ok && cudaMemsetAsync(d.tile_cnt, 0, max_tiles * sizeof(int32_t), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.ctr_steps, 0, sizeof(unsigned long long), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.ctr_inter, 0, sizeof(double), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.ctr_underflow, 0, sizeof(unsigned long long), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.err, 0, sizeof(uint32_t), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.busy, 0, sizeof(int32_t), s0) != cudaSuccess) ok = false;
    if (ok && cudaMemsetAsync(d.sel_ctr, 0, sizeof(unsigned int), s0) != cudaSuccess) ok = false;
    // the chunk tables live in pageable host vectors: finish the copies here
    if (ok && cudaStreamSynchronize(s0) != cudaSuccess) ok = false;
    if (!ok) {
        nb_status s = cuda_fail(nullptr, cudaGetLastError(), "nb_init: upload");
        nb_free(ctx);
        return s;
    }
    nb_status s = NB_OK;
    if (launch_pad(d, s0) != cudaSuccess) s = cuda_fail(ctx, cudaGetLastError(), "pad");
    if (s == NB_OK && !(p->flags & NB_INIT_KEEP_STATE)) s = startup(ctx);
    if (s == NB_OK && set_tend(ctx, INFINITY) != NB_OK) s = NB_ECUDA;
    if (s == NB_OK && cudaStreamSynchronize(s0) != cudaSuccess) s = cuda_fail(ctx, cudaGetLastError(), "nb_init");
    if (s == NB_OK) s = check_device_error(ctx);
    if (s != NB_OK) {
        g_init_err = ctx->err;
        nb_free(ctx);
        return s;
    }
    *out = ctx;
    return NB_OK;
}

nb_status nb_predict(nb_ctx *ctx, double t_next, double *out) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_predict: NULL context");
    if (!std::isfinite(t_next)) return fail(ctx, NB_EINVAL, "nb_predict: t_next not finite");
    NB_CU(ctx, launch_predict(ctx->d, out != nullptr, 1, t_next, ctx->stream));
    if (out) NB_CU(ctx, launch_unpack64(ctx->d, out, ctx->stream));
    return NB_OK;
}

nb_status nb_evaluate(nb_ctx *ctx, int32_t cluster, const int32_t *active, int32_t n_active,
                      double *out_ajs) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_evaluate: NULL context");
    if (cluster < 0 || cluster >= ctx->nc) return fail(ctx, NB_EINVAL, "nb_evaluate: cluster out of range");
    const int64_t ncl = ctx->h_offsets[cluster + 1] - ctx->h_offsets[cluster];
    if (n_active < 0 || n_active > ncl) return fail(ctx, NB_EINVAL, "nb_evaluate: n_active out of range");
    if (n_active == 0) return NB_OK;
    if (!active || !out_ajs) return fail(ctx, NB_EINVAL, "nb_evaluate: NULL pointer");
    int gl, split, tiles, streamk;
    plan_direct(ctx, cluster, n_active, gl, split, tiles, streamk);
    return eval_direct(ctx, cluster, active, n_active, out_ajs, gl, split, tiles, streamk);
}

nb_status nb_evaluate_range(nb_ctx *ctx, int32_t cluster, const int32_t *active, int32_t n_active,
                            int64_t j_begin, int64_t j_end, double *out_ajs) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_evaluate_range: NULL context");
    if (cluster < 0 || cluster >= ctx->nc)
        return fail(ctx, NB_EINVAL, "nb_evaluate_range: cluster out of range");
    const int64_t ncl = ctx->h_offsets[cluster + 1] - ctx->h_offsets[cluster];
    if (n_active < 0 || n_active > ncl)
        return fail(ctx, NB_EINVAL, "nb_evaluate_range: n_active out of range");
    if (j_begin < 0 || j_end < j_begin || j_end > ncl || j_begin % kTJ != 0 ||
        (j_end % kTJ != 0 && j_end != ncl))
        return fail(ctx, NB_EINVAL,
                    "nb_evaluate_range: need 0 <= j_begin <= j_end <= n_cluster, j_begin a multiple "
                    "of 64, j_end a multiple of 64 or n_cluster");
    if (n_active == 0) return NB_OK;
    if (!active || !out_ajs) return fail(ctx, NB_EINVAL, "nb_evaluate_range: NULL pointer");
    if (j_end == j_begin) {  // an empty range sums nothing
        NB_CU(ctx, cudaMemsetAsync(out_ajs, 0, sizeof(double) * 10 * (size_t)n_active, ctx->stream));
        return NB_OK;
    }
    const int32_t jt0 = (int32_t)(j_begin / kTJ), jt1 = (int32_t)cdiv(j_end, kTJ);
    int gl, split, tiles, streamk;
    plan_direct(ctx, cluster, n_active, gl, split, tiles, streamk, jt1 - jt0);
    return eval_direct(ctx, cluster, active, n_active, out_ajs, gl, split, tiles, streamk, jt0, jt1);
}

nb_status nb_correct_and_timestep(nb_ctx *ctx, int32_t cluster, const int32_t *active,
                                  int32_t n_active, double t_next, const double *ajs) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_correct_and_timestep: NULL context");
    if (cluster < 0 || cluster >= ctx->nc) return fail(ctx, NB_EINVAL, "nb_correct_and_timestep: bad cluster");
    const int64_t ncl = ctx->h_offsets[cluster + 1] - ctx->h_offsets[cluster];
    if (n_active < 0 || n_active > ncl) return fail(ctx, NB_EINVAL, "nb_correct_and_timestep: n_active");
    if (n_active == 0) return NB_OK;
    if (!active || !ajs || !std::isfinite(t_next))
        return fail(ctx, NB_EINVAL, "nb_correct_and_timestep: NULL pointer or bad t_next");
    NB_CU(ctx, launch_correct(ctx->d, ctx->h_offsets[cluster], ctx->h_offsets[cluster + 1], active,
                              n_active, t_next, ajs, ctx->stream));
    return NB_OK;
}

nb_status nb_step(nb_ctx *ctx, double *t_next_out, int32_t *n_active_out) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_step: NULL context");
    nb_status s = build_graphs(ctx);
    if (s != NB_OK) return s;
    if ((s = set_tend(ctx, INFINITY)) != NB_OK) return s;
    NB_CU(ctx, cudaGraphLaunch(ctx->g_step, ctx->stream));
    ctx->launches += kKernelsPerStep;
    if (!ctx->ev.empty()) {  // timing needs the replay to finish before the events are read
        NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
        harvest_events(ctx, kMultiSteps, 1);
    }
    if (t_next_out || n_active_out) {
        std::vector<double> tn(ctx->nc);
        std::vector<int32_t> na(ctx->nc);
        NB_CU(ctx, cudaMemcpyAsync(tn.data(), ctx->d.tnext, ctx->nc * sizeof(double),
                                   cudaMemcpyDeviceToHost, ctx->stream));
        NB_CU(ctx, cudaMemcpyAsync(na.data(), ctx->d.nact, ctx->nc * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, ctx->stream));
        NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
        if (t_next_out) *t_next_out = *std::min_element(tn.begin(), tn.end());
        if (n_active_out) {
            int64_t tot = 0;
            for (int32_t v : na) tot += v;
            *n_active_out = (int32_t)tot;
        }
        return check_device_error(ctx);
    }
    return NB_OK;
}

nb_status nb_run(nb_ctx *ctx, double t_end, int64_t max_block_steps, int64_t *block_steps_out,
                 double *interactions_out) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_run: NULL context");
    if (std::isnan(t_end)) return fail(ctx, NB_EINVAL, "nb_run: t_end is NaN");
    nb_status s = build_graphs(ctx);
    if (s != NB_OK) return s;
    unsigned long long steps0 = 0;
    double inter0 = 0.0;
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    NB_CU(ctx, cudaMemcpy(&steps0, ctx->d.ctr_steps, sizeof(steps0), cudaMemcpyDeviceToHost));
    NB_CU(ctx, cudaMemcpy(&inter0, ctx->d.ctr_inter, sizeof(inter0), cudaMemcpyDeviceToHost));
    if ((s = set_tend(ctx, t_end)) != NB_OK) return s;
    int64_t done_batches = 0;
    while (true) {
        const int64_t left = max_block_steps < 0 ? INT64_MAX : max_block_steps - done_batches;
        if (left <= 0) break;
        const bool multi = left >= kMultiSteps;
        if (multi) {
            NB_CU(ctx, cudaGraphLaunch(ctx->g_multi, ctx->stream));
            done_batches += kMultiSteps;
            ctx->launches += (int64_t)kKernelsPerStep * kMultiSteps;
        } else {
            NB_CU(ctx, cudaGraphLaunch(ctx->g_step, ctx->stream));
            NB_CU(ctx, cudaMemcpyAsync(ctx->h_busy, ctx->d.busy, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, ctx->stream));
            done_batches += 1;
            ctx->launches += kKernelsPerStep;
        }
        NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
        if (multi) harvest_events(ctx, 0, kMultiSteps);
        else harvest_events(ctx, kMultiSteps, 1);
        if (*ctx->h_busy == 0) break;
        // a device-side failure stops time from advancing: never spin on it
        if ((s = check_device_error(ctx)) != NB_OK) {
            set_tend(ctx, INFINITY);
            return s;
        }
    }
    if ((s = set_tend(ctx, INFINITY)) != NB_OK) return s;
    unsigned long long steps1 = 0;
    double inter1 = 0.0;
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    NB_CU(ctx, cudaMemcpy(&steps1, ctx->d.ctr_steps, sizeof(steps1), cudaMemcpyDeviceToHost));
    NB_CU(ctx, cudaMemcpy(&inter1, ctx->d.ctr_inter, sizeof(inter1), cudaMemcpyDeviceToHost));
    if (block_steps_out) *block_steps_out = (int64_t)(steps1 - steps0);
    if (interactions_out) *interactions_out = inter1 - inter0;
    return check_device_error(ctx);
}

nb_status nb_energy(nb_ctx *ctx, int32_t cluster, double t, double *ekin, double *epot, double P[3],
                    double L[3]) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_energy: NULL context");
    if (cluster < -1 || cluster >= ctx->nc) return fail(ctx, NB_EINVAL, "nb_energy: bad cluster");
    if (!std::isfinite(t)) return fail(ctx, NB_EINVAL, "nb_energy: t not finite");
    NB_CU(ctx, launch_predict(ctx->d, 1, 1, t, ctx->stream));
    NB_CU(ctx, launch_plan_ex(ctx->d_pot, 1, 0, ctx->stream));
    EvalLaunch Lz{};
    Lz.identity = 1;
    NB_CU(ctx, launch_eval(ctx->d_pot, kModePot, Lz, ctx->grid_pot, ctx->stream));
    const int64_t b = cluster < 0 ? 0 : ctx->h_offsets[cluster];
    const int64_t e = cluster < 0 ? ctx->n : ctx->h_offsets[cluster + 1];
    NB_CU(ctx, launch_energy(ctx->d, b, e, 0, ctx->stream));
    std::vector<double> part((size_t)ctx->d.n_chunks * 8);
    NB_CU(ctx, cudaMemcpyAsync(part.data(), ctx->d.energy_part, part.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < ctx->d.n_chunks; ++k)
        for (int q = 0; q < 8; ++q) acc[q] += part[(size_t)k * 8 + q];
    if (ekin) *ekin = acc[0];
    if (epot) *epot = acc[1];
    if (P) for (int q = 0; q < 3; ++q) P[q] = acc[2 + q];
    if (L) for (int q = 0; q < 3; ++q) L[q] = acc[5 + q];
    return check_device_error(ctx);
}

nb_status nb_energy_all(nb_ctx *ctx, double t, double *out) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_energy_all: NULL context");
    if (!out || !std::isfinite(t)) return fail(ctx, NB_EINVAL, "nb_energy_all: NULL out or bad t");
    NB_CU(ctx, launch_predict(ctx->d, 1, 1, t, ctx->stream));
    NB_CU(ctx, launch_plan_ex(ctx->d_pot, 1, 0, ctx->stream));
    EvalLaunch Lz{};
    Lz.identity = 1;
    NB_CU(ctx, launch_eval(ctx->d_pot, kModePot, Lz, ctx->grid_pot, ctx->stream));
    NB_CU(ctx, launch_energy(ctx->d, 0, ctx->n, 0, ctx->stream));
    std::vector<double> part((size_t)ctx->d.n_chunks * 8);
    NB_CU(ctx, cudaMemcpyAsync(part.data(), ctx->d.energy_part, part.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, ctx->stream));
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    // chunks never straddle clusters and are numbered cluster by cluster
    for (int c = 0; c < ctx->nc; ++c) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = ctx->h_chunk0[c]; k < ctx->h_chunk0[c + 1]; ++k)
            for (int q = 0; q < 8; ++q) acc[q] += part[(size_t)k * 8 + q];
        for (int q = 0; q < 8; ++q) out[(size_t)c * 8 + q] = acc[q];
    }
    return check_device_error(ctx);
}

static nb_status copy_state(nb_ctx *ctx, const nb_state *dst, const nb_state *src) {
    const size_t n = (size_t)ctx->n;
    const size_t sc = n * sizeof(double), vc = 3 * sc;
    struct F { double *dst; const double *src; size_t bytes; } f[] = {
        {dst->m, src->m, sc},   {dst->x, src->x, vc}, {dst->v, src->v, vc}, {dst->a, src->a, vc},
        {dst->j, src->j, vc},   {dst->s, src->s, vc}, {dst->c, src->c, vc}, {dst->t, src->t, sc},
        {dst->dt, src->dt, sc}, {dst->pot, src->pot, sc}};
    for (auto &q : f) {
        if (!q.dst || !q.src) return fail(ctx, NB_EINVAL, "nb_get/set_state: NULL buffer");
        if (q.dst == q.src) continue;
        NB_CU(ctx, cudaMemcpyAsync(q.dst, q.src, q.bytes, cudaMemcpyDefault, ctx->stream));
    }
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return NB_OK;
}

static nb_state ctx_state(const nb_ctx *ctx) {
    const Dev &d = ctx->d;
    return nb_state{d.m, d.x, d.v, d.a, d.j, d.s, d.c, d.t, d.dt, d.pot};
}

nb_status nb_get_state(nb_ctx *ctx, const nb_state *dst) {
    if (!ctx || !dst) return fail(ctx, NB_EINVAL, "nb_get_state: NULL argument");
    nb_state me = ctx_state(ctx);
    return copy_state(ctx, dst, &me);
}

nb_status nb_set_state(nb_ctx *ctx, const nb_state *src) {
    if (!ctx || !src) return fail(ctx, NB_EINVAL, "nb_set_state: NULL argument");
    nb_state me = ctx_state(ctx);
    return copy_state(ctx, &me, src);
}

nb_status nb_get_counters(nb_ctx *ctx, nb_counters *out) {
    if (!ctx || !out) return fail(ctx, NB_EINVAL, "nb_get_counters: NULL argument");
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned long long steps = 0, uf = 0;
    double inter = 0.0;
    uint32_t err = 0;
    NB_CU(ctx, cudaMemcpy(&steps, ctx->d.ctr_steps, sizeof(steps), cudaMemcpyDeviceToHost));
    NB_CU(ctx, cudaMemcpy(&inter, ctx->d.ctr_inter, sizeof(inter), cudaMemcpyDeviceToHost));
    NB_CU(ctx, cudaMemcpy(&uf, ctx->d.ctr_underflow, sizeof(uf), cudaMemcpyDeviceToHost));
    NB_CU(ctx, cudaMemcpy(&err, ctx->d.err, sizeof(err), cudaMemcpyDeviceToHost));
    out->block_steps = (int64_t)steps;
    out->interactions = inter;
    out->dt_underflows = (int64_t)uf;
    out->device_errors = err;
    out->kernel_launches = ctx->launches;
    out->eval_launches = ctx->eval_launches;
    out->eval_ms = ctx->eval_ms;
    return NB_OK;
}

nb_status nb_sync(nb_ctx *ctx) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_sync: NULL context");
    NB_CU(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

nb_status nb_autotune(nb_ctx *ctx, const char *cache_path) {
    if (!ctx) return fail(nullptr, NB_EINVAL, "nb_autotune: NULL context");
    // cached table?
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "r");
        if (f) {
            std::vector<PlanEntry> t(kBuckets);
            int prec = -1, grid = -1, okc = 1;
            if (std::fscanf(f, "nbtune %d %d", &prec, &grid) != 2) okc = 0;
            for (int b = 0; okc && b < kBuckets; ++b)
                if (std::fscanf(f, "%d %d", &t[b].gl, &t[b].target_items) != 2) okc = 0;
            std::fclose(f);
            if (okc && prec == ctx->p.precision) {
                ctx->table = t;
                return upload_table(ctx);
            }
        }
    }
    // largest cluster: time evaluations of its first A particles
    int cmax = 0;
    for (int c = 0; c < ctx->nc; ++c)
        if (ctx->h_offsets[c + 1] - ctx->h_offsets[c] == ctx->max_cluster) { cmax = c; break; }
    const int64_t ncl = ctx->max_cluster;
    int32_t *d_act = nullptr;
    double *d_out = nullptr;
    NB_CU(ctx, cudaMalloc(&d_act, ncl * sizeof(int32_t)));
    cudaError_t e = cudaMalloc(&d_out, ncl * 10 * sizeof(double));
    if (e != cudaSuccess) { cudaFree(d_act); return cuda_fail(ctx, e, "nb_autotune: cudaMalloc"); }
    std::vector<int32_t> h_act(ncl);
    for (int64_t k = 0; k < ncl; ++k) h_act[k] = (int32_t)(ctx->h_offsets[cmax] + k);
    e = cudaMemcpy(d_act, h_act.data(), ncl * sizeof(int32_t), cudaMemcpyHostToDevice);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int G = ctx->grid_eval;
    const int64_t targets[] = {G / 2, G, 2LL * G, 4LL * G, 8LL * G, 16LL * G};
    const int gls[] = {1, 2, 4, 8, 16, 32};
    nb_status st = NB_OK;
    for (int b = 0; b < kBuckets && e == cudaSuccess; ++b) {
        const double A0 = std::ldexp(1.0, b);
        if (A0 > (double)ncl) break;
        const int32_t A = (int32_t)std::min<double>(std::floor(A0 * 1.5), (double)ncl);
        float best = 1e30f;
        PlanEntry bestE = ctx->table[b];
        int reps = 2;
        for (int gl : gls) {
            if (A >= 4096 && gl > 2) continue;   // wide i-sets: j broadcast wins
            for (int64_t tg : targets) {
                if (tg > ctx->cap_items / 2) continue;
                ctx->table[b] = PlanEntry{gl, (int32_t)tg};
                int g2, sp, tl, skm;
                plan_direct(ctx, cmax, A, g2, sp, tl, skm);
                float ms_best = 1e30f;
                for (int rep = 0; rep < reps; ++rep) {
                    if ((e = cudaEventRecord(e0, ctx->stream)) != cudaSuccess) break;
                    st = eval_direct(ctx, cmax, d_act, A, d_out, g2, sp, tl, skm);
                    if (st != NB_OK) break;
                    if ((e = cudaEventRecord(e1, ctx->stream)) != cudaSuccess) break;
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    float ms = 0.f;
                    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
                    ms_best = std::min(ms_best, ms);
                }
                if (st != NB_OK || e != cudaSuccess) break;
                if (ms_best > 50.f) reps = 1;    // long launches: one timing is enough
                if (ms_best < best) {
                    best = ms_best;
                    bestE = ctx->table[b];
                }
            }
            if (st != NB_OK || e != cudaSuccess) break;
        }
        ctx->table[b] = bestE;
        // buckets above the largest timed one reuse its choice
        for (int b2 = b + 1; b2 < kBuckets; ++b2) ctx->table[b2] = bestE;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_act);
    cudaFree(d_out);
    if (st != NB_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nb_autotune");
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "w");
        if (f) {
            std::fprintf(f, "nbtune %d %d\n", ctx->p.precision, ctx->grid_eval);
            for (int b = 0; b < kBuckets; ++b) std::fprintf(f, "%d %d\n", ctx->table[b].gl, ctx->table[b].target_items);
            std::fclose(f);
        }
    }
    return upload_table(ctx);
}

}  // extern "C"
