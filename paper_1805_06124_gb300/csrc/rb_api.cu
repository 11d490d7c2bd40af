// rb_api.cu -- host runtime behind the C ABI of include/rb.h: context,
// device workspace, argument checks and the device-driven greedy loop.
//
// The loop never waits on the device per iteration: it queues
// iters_per_sync iterations (IMGS launches + one sweep each), then reads the
// 100-byte device state once.  Kernels queued after the stop flag was set
// return immediately.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "rb_internal.cuh"

struct rb_ctx {
    int device = 0;
    int sms = 152;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    rb_options opt{};
    char err[512] = {0};
    void *ws = nullptr;          // main workspace (split copy + vectors)
    size_t ws_cap = 0;
    void *stage = nullptr;       // device staging for rb_greedy_host
    size_t stage_cap = 0;
    void *gen = nullptr;         // rb_generate tables
    size_t gen_cap = 0;
    void *aux = nullptr;         // rb_validate coefficients
    size_t aux_cap = 0;
    rbk::DevState *st_host = nullptr;  // pinned copy of the device state
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> sweep_ev;
    std::vector<cudaEvent_t> imgs_ev;   // IMGS events per iteration of the FP64 form (RB_FLAG_TIMING)
    std::vector<int> trace_passes;      // last FP64-form call: IMGS passes per iteration
    std::vector<double> trace_sweep_ms, trace_imgs_ms;  // and phase times (RB_FLAG_TIMING)
    std::vector<cudaEvent_t> recon_ev;  // phase events of rb_reconstruct (RB_FLAG_TIMING)
    double recon_ms[7] = {0};           // phase times of the last rb_reconstruct
    int recon_counts[4] = {0};          // Jacobi sweeps / rotations, pass 1 and pass 2
    int grid_cache[2] = {0, 0};
    // last rb_greedy_streamed: resident columns, chunks, columns per chunk,
    // chunk updates, bytes read from host memory
    long long str_stats[4] = {0, 0, 0, 0};
    double str_host_bytes = 0.0;
    double str_ms_init = 0.0;
    std::map<std::tuple<int, long long, long long>, std::pair<int, int>> tune;  // batch shape -> (variant, CW)
};

namespace {

rb_status fail(rb_ctx *c, rb_status s, const char *fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

rb_status cuda_fail(rb_ctx *c, cudaError_t e, const char *what) {
    return fail(c, RB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RB_CK(call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t off = 0;
    size_t add(size_t bytes) {
        size_t o = align_up(off, 512);
        off = o + bytes;
        return o;
    }
};

rb_status ensure(rb_ctx *ctx, void **buf, size_t *cap, size_t need) {
    if (getenv("RB_TEST_FAIL_ALLOC"))  // fault injection for the tests (host side only)
        return fail(ctx, RB_ENOMEM, "device allocation refused (RB_TEST_FAIL_ALLOC is set)");
    if (*cap >= need && *buf) return RB_OK;
    if (*buf) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, RB_ENOMEM, "cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
    }
    *cap = need;
    return RB_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int grid_for_variant(rb_ctx *ctx, int variant) {
    if (!ctx->grid_cache[variant]) ctx->grid_cache[variant] = rbk::sweep_grid(variant, ctx->device);
    return ctx->grid_cache[variant];
}

}  // namespace

namespace rbk {
cudaStream_t ctx_stream(rb_ctx *ctx) { return ctx->stream; }
int ctx_device(rb_ctx *ctx) { return ctx->device; }
unsigned long long ctx_wait_cycles(const rb_ctx *ctx) {
    return ctx->opt.timeout_cycles ? ctx->opt.timeout_cycles : kWaitCyclesDefault;
}
const rb_options &ctx_options(const rb_ctx *ctx) { return ctx->opt; }
int ctx_sweep_grid(rb_ctx *ctx, int variant) { return grid_for_variant(ctx, variant); }
rb_status ctx_fail(rb_ctx *ctx, rb_status s, const char *msg) { return fail(ctx, s, "%s", msg); }
}  // namespace rbk

extern "C" {

void rb_default_options(rb_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->device = 0;
    opt->sweep = RB_SWEEP_DF32;
    opt->imgs_kappa = 2.0;
    opt->imgs_max_passes = 4;
    opt->switch_err = 0.0;
    opt->iters_per_sync = 8;
    opt->recompute_period = 16;
    opt->stream = nullptr;
    opt->flags = 0;
    opt->batched_variant = -1;
    opt->timeout_cycles = 0;
}

rb_status rb_create(const rb_options *opt, rb_ctx **out) {
    if (!out) return RB_EINVAL;
    *out = nullptr;
    rb_options o;
    if (opt)
        o = *opt;
    else
        rb_default_options(&o);
    if (!(o.imgs_kappa > 1.0) || o.imgs_max_passes < 1 || o.iters_per_sync < 1 || o.recompute_period < 0 ||
        (o.sweep != RB_SWEEP_DF32 && o.sweep != RB_SWEEP_FP64) || !(o.switch_err >= 0.0) || !std::isfinite(o.switch_err) ||
        o.batched_variant < -1 || o.batched_variant > 23 || (o.timeout_cycles && o.timeout_cycles < (1ull << 20)))
        return RB_EINVAL;
    rb_ctx *ctx = new (std::nothrow) rb_ctx();
    if (!ctx) return RB_ENOMEM;
    ctx->opt = o;
    ctx->device = o.device;
    cudaError_t e = cudaSetDevice(o.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e == cudaSuccess) {
        if (o.stream) {
            ctx->stream = (cudaStream_t)o.stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->st_host, sizeof(rbk::DevState));
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        rb_destroy(ctx);
        return RB_ECUDA;
    }
    *out = ctx;
    return RB_OK;
}

void rb_destroy(rb_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t ev : ctx->sweep_ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : ctx->recon_ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : ctx->imgs_ev) cudaEventDestroy(ev);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->gen) cudaFree(ctx->gen);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->st_host) cudaFreeHost(ctx->st_host);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *rb_last_error(const rb_ctx *ctx) { return ctx ? ctx->err : "null context"; }

rb_status rb_generate(rb_ctx *ctx, const double *q, const double *m, long long N, long long M, void *S,
                      long long ldS) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || M < 1 || ldS < N || !q || !m || !S || !aligned(S, 16))
        return fail(ctx, RB_EINVAL, "rb_generate: bad arguments (N=%lld M=%lld ldS=%lld)", N, M, ldS);
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    rb_status s = ensure(ctx, &ctx->gen, &ctx->gen_cap, (size_t)N * 2 * sizeof(double));
    if (s != RB_OK) return s;
    double *amp = (double *)ctx->gen, *ph = amp + N;
    RB_CK(rbk::launch_generate_tables(amp, ph, N, ctx->stream), "generate tables");
    RB_CK(rbk::launch_generate(q, m, amp, ph, N, M, (double2 *)S, ldS, ctx->stream), "generate");
    return RB_OK;
}

rb_status rb_split(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, void *hi, void *lo,
                   long long ldH) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || M < 1 || ldS < N || ldH < N || !S || !hi || !lo || !aligned(S, 16) || !aligned(hi, 8) ||
        !aligned(lo, 8))
        return fail(ctx, RB_EINVAL, "rb_split: bad arguments (N=%lld M=%lld ldS=%lld ldH=%lld)", N, M, ldS, ldH);
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    RB_CK(rbk::launch_split((const double2 *)S, N, M, ldS, (float2 *)hi, (float2 *)lo, ldH, nullptr, ctx->stream),
          "split");
    return RB_OK;
}

rb_status rb_project(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ, const void *X, long long Mx,
                     long long ldX, void *C, long long ldC) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || k < 0 || Mx < 0 || ldQ < N || ldX < N || ldC < Mx || (k > 0 && (!Q || !X || !C)) ||
        !aligned(Q, 16) || !aligned(X, 16) || !aligned(C, 16))
        return fail(ctx, RB_EINVAL, "rb_project: bad arguments (N=%lld k=%d Mx=%lld)", N, k, Mx);
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (k == 0 || Mx == 0) return RB_OK;
    if (ctx->opt.flags & RB_FLAG_PROJECT_FP64) {
        RB_CK(rbk::launch_project((const double2 *)Q, N, k, ldQ, (const double2 *)X, Mx, ldX, (double2 *)C, ldC,
                                  ctx->stream),
              "project");
        return RB_OK;
    }
    // tensor-core path, in column batches whose workspace (the basis slice planes and the
    // column scales) stays under ~4 GB
    long long Mb = Mx;
    while (Mb > 64 && rbk::oz_workspace(N, k, Mb) > (4ull << 30)) Mb = (Mb + 1) / 2;
    const size_t need = rbk::oz_workspace(N, k, Mb) + 256;
    rb_status s = ensure(ctx, &ctx->gen, &ctx->gen_cap, need);
    if (s != RB_OK) return s;
    int *err = (int *)((char *)ctx->gen + need - 256);
    cudaStream_t sm = ctx->stream;
    RB_CK(cudaMemsetAsync(err, 0, sizeof(int), sm), "memset flag");
    for (long long c0 = 0; c0 < Mx; c0 += Mb) {
        long long nb = Mx - c0 < Mb ? Mx - c0 : Mb;
        RB_CK(rbk::launch_project_tc((const double2 *)Q, N, k, ldQ, (const double2 *)X + c0 * ldX, nb, ldX,
                                     (double2 *)C, ldC, c0, ctx->gen, err, rbk::ctx_wait_cycles(ctx), sm),
              "project (tensor cores)");
    }
    int herr = 0;
    RB_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, sm), "flag copy");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    if (herr) return fail(ctx, RB_ETIMEOUT, "rb_project: a tensor-core wait ran out");
    return RB_OK;
}

rb_status rb_reconstruct(rb_ctx *ctx, const void *Q, long long N, int j, long long ldQ, const void *C, long long M,
                         long long ldC, double tau2, void *X, long long ldX, double *sigma, void *V, int *k_out) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || M < 1 || j < 0 || j > RB_RECON_MAX_J || ldQ < N || ldC < M || ldX < N || !k_out ||
        !(tau2 >= 0.0) || (j > 0 && (!Q || !C || !X || !sigma)) || !aligned(Q, 16) || !aligned(C, 16) ||
        !aligned(X, 16) || !aligned(V, 16))
        return fail(ctx, RB_EINVAL, "rb_reconstruct: bad arguments (N=%lld M=%lld j=%d, j <= %d)", N, M, j,
                    RB_RECON_MAX_J);
    *k_out = 0;
    for (double &t : ctx->recon_ms) t = 0.0;
    for (int &c : ctx->recon_counts) c = 0;
    if (j == 0) return RB_OK;
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t wsb = (rbk::recon_workspace(j, M) + 255) & ~(size_t)255;
    const size_t vbytes = ((size_t)j * j * 16 + 255) & ~(size_t)255;
    rb_status s = ensure(ctx, &ctx->gen, &ctx->gen_cap, wsb + vbytes + 256);
    if (s != RB_OK) return s;
    double2 *Vw = V ? (double2 *)V : (double2 *)((char *)ctx->gen + wsb);
    int *stats = (int *)((char *)ctx->gen + wsb + vbytes);
    const bool timing = (ctx->opt.flags & RB_FLAG_TIMING) != 0;
    if (timing && ctx->recon_ev.empty()) {
        ctx->recon_ev.resize(8);
        for (cudaEvent_t &ev : ctx->recon_ev) RB_CK(cudaEventCreate(&ev), "cudaEventCreate");
    }
    cudaEvent_t *ev = timing ? ctx->recon_ev.data() : nullptr;
    cudaStream_t sm = ctx->stream;
    RB_CK(rbk::launch_recon_svd((const double2 *)C, ldC, j, M, ctx->gen, sigma, Vw, stats, ev, sm), "reconstruct svd");
    std::vector<double> hs(j);
    RB_CK(cudaMemcpyAsync(hs.data(), sigma, (size_t)j * 8, cudaMemcpyDeviceToHost, sm), "sigma copy");
    RB_CK(cudaMemcpyAsync(ctx->recon_counts, stats, 4 * sizeof(int), cudaMemcpyDeviceToHost, sm), "stats copy");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    int k = 0;
    while (k < j && hs[k] > tau2) k++;
    RB_CK(rbk::launch_recon_basis((const double2 *)Q, ldQ, N, j, Vw, k, (double2 *)X, ldX, sm), "reconstruct basis");
    if (ev) RB_CK(cudaEventRecord(ev[7], sm), "cudaEventRecord");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    if (ev)
        for (int i = 0; i < 7; i++) {
            float t = 0.f;
            RB_CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]), "cudaEventElapsedTime");
            ctx->recon_ms[i] = t;
        }
    *k_out = k;
    return RB_OK;
}

rb_status rb_eim(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ, long long *nodes, void *V, void *B,
                 long long ldB, void *Vinv) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || k < 0 || k > N || ldQ < N || (k > 0 && (!Q || !nodes)) || (B && ldB < N) || !aligned(Q, 16) ||
        !aligned(V, 16) || !aligned(B, 16) || !aligned(Vinv, 16) || !aligned(nodes, 8))
        return fail(ctx, RB_EINVAL, "rb_eim: bad arguments (N=%lld k=%d ldQ=%lld ldB=%lld)", N, k, ldQ, ldB);
    if (k == 0) return RB_OK;
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t wsb = (rbk::eim_workspace(N, k) + 255) & ~(size_t)255;
    const size_t bws = (!B && Vinv) ? (((size_t)N * k * 16 + 255) & ~(size_t)255) : 0;
    rb_status s = ensure(ctx, &ctx->gen, &ctx->gen_cap, wsb + bws + 256);
    if (s != RB_OK) return s;
    double2 *Bw = B ? (double2 *)B : (Vinv ? (double2 *)((char *)ctx->gen + wsb) : nullptr);
    const long long ldBw = B ? ldB : N;
    int *flag = (int *)((char *)ctx->gen + wsb + bws);
    cudaStream_t sm = ctx->stream;
    RB_CK(cudaMemsetAsync(flag, 0, sizeof(int), sm), "memset flag");
    RB_CK(rbk::launch_eim((const double2 *)Q, N, k, ldQ, ctx->gen, nodes, (double2 *)V, Bw, ldBw, flag, sm), "eim");
    if (Vinv)  // V^{-1} = Q^H B for an orthonormal basis
        RB_CK(rbk::launch_project((const double2 *)Q, N, k, ldQ, Bw, k, ldBw, (double2 *)Vinv, k, sm), "eim V^-1");
    int hf = 0;
    RB_CK(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, sm), "flag copy");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    if (hf) return fail(ctx, RB_ESTATE, "rb_eim: a residual vanished on every free grid point (dependent basis)");
    return RB_OK;
}

rb_status rb_validate(rb_ctx *ctx, const void *Q, long long N, int k, long long ldQ, const long long *nodes,
                      const void *Vinv, const void *T, long long Mt, long long ldT, double *err_proj, double *err_eim) {
    if (!ctx) return RB_EINVAL;
    if (N < 1 || k < 0 || Mt < 0 || ldQ < N || ldT < N || (Mt > 0 && (!T || !err_proj)) || (k > 0 && !Q) ||
        (err_eim && k > 0 && (!nodes || !Vinv)) || (err_eim && k > RB_VALIDATE_MAX_K) || !aligned(Q, 16) ||
        !aligned(T, 16) || !aligned(Vinv, 16))
        return fail(ctx, RB_EINVAL, "rb_validate: bad arguments (N=%lld k=%d Mt=%lld)", N, k, Mt);
    if (Mt == 0) return RB_OK;
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    double2 *Cv = nullptr;
    if (k > 0) {
        rb_status s = ensure(ctx, &ctx->aux, &ctx->aux_cap, (size_t)k * Mt * 16);
        if (s != RB_OK) return s;
        Cv = (double2 *)ctx->aux;
        s = rb_project(ctx, Q, N, k, ldQ, T, Mt, ldT, Cv, Mt);
        if (s != RB_OK) return s;
    }
    cudaStream_t sm = ctx->stream;
    RB_CK(rbk::launch_validate((const double2 *)T, N, Mt, ldT, Cv, Mt, k, nodes, (const double2 *)Vinv, err_proj,
                               err_eim, sm),
          "validate");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    return RB_OK;
}

rb_status rb_trace(const rb_ctx *ctx, int *imgs_passes, double *sweep_ms, double *imgs_ms, int cap, int *n) {
    if (!ctx || cap < 0 || !n) return RB_EINVAL;
    const int np = (int)ctx->trace_passes.size();
    *n = np;
    for (int i = 0; i < np && i < cap; i++) {
        if (imgs_passes) imgs_passes[i] = ctx->trace_passes[i];
        if (sweep_ms) sweep_ms[i] = i < (int)ctx->trace_sweep_ms.size() ? ctx->trace_sweep_ms[i] : 0.0;
        if (imgs_ms) imgs_ms[i] = i < (int)ctx->trace_imgs_ms.size() ? ctx->trace_imgs_ms[i] : 0.0;
    }
    return RB_OK;
}

rb_status rb_reconstruct_stats(const rb_ctx *ctx, double *ms, int *counts) {
    if (!ctx) return RB_EINVAL;
    if (ms)
        for (int i = 0; i < 7; i++) ms[i] = ctx->recon_ms[i];
    if (counts)
        for (int i = 0; i < 4; i++) counts[i] = ctx->recon_counts[i];
    return RB_OK;
}

// k0 > 0: resume from a checkpoint of k0 vectors held in out (Q, pivots, C,
// err_curve, rdiag rows 0..k0-1; C complete for all M columns).
static rb_status greedy_device(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol,
                               int kmax, rb_result *out, int k0 = 0) {
    const rb_options &o = ctx->opt;
    const int variant = o.sweep;
    const bool df = (variant == RB_SWEEP_DF32);
    const int G = grid_for_variant(ctx, variant);
    const long long ldH = (long long)align_up((size_t)N, 64);
    const int chunk = 2048;
    const int nchunk = (int)((N + chunk - 1) / chunk);
    const int gN = (int)((N + rbk::kThreads - 1) / rbk::kThreads);
    const int kcap = kmax > 0 ? kmax : 1;

    Layout L;
    size_t o_hi = 0, o_lo = 0;
    if (df) {
        o_hi = L.add((size_t)M * ldH * sizeof(float2));
        o_lo = L.add((size_t)M * ldH * sizeof(float2));
    }
    size_t o_norm = L.add((size_t)M * 8), o_acc = L.add((size_t)M * 8), o_pick = L.add((size_t)M);
    size_t o_qh = L.add((size_t)(N + 2) * sizeof(float2)), o_ql = L.add((size_t)(N + 2) * sizeof(float2));
    size_t o_v = L.add((size_t)N * sizeof(double2));
    size_t o_hp = L.add((size_t)kcap * nchunk * sizeof(double2));
    size_t np = (size_t)(G > gN ? G : gN);
    size_t o_np = L.add(np * 8), o_be = L.add((size_t)G * 8), o_bi = L.add((size_t)G * 8);
    size_t o_st = L.add(sizeof(rbk::DevState));
    size_t o_pass = L.add((size_t)kcap * sizeof(int));
    // the periodic recompute reads the stored coefficients: keep them in the
    // workspace when the caller does not ask for C
    const bool ws_C = !out->C && o.recompute_period > 0;
    size_t o_C = ws_C ? L.add((size_t)kcap * M * sizeof(double2)) : 0;
    rb_status s = ensure(ctx, &ctx->ws, &ctx->ws_cap, L.off);
    if (s != RB_OK) return s;
    char *w = (char *)ctx->ws;

    rbk::Prob p{};
    p.N = N;
    p.M = M;
    p.ldS = ldS;
    p.ldH = ldH;
    p.ldQ = out->ldQ;
    p.ldC = ws_C ? M : out->ldC;
    p.minNM = N < M ? N : M;
    p.kmax = kmax;
    p.max_passes = o.imgs_max_passes;
    p.nchunk = nchunk;
    p.chunk = chunk;
    p.tol = tol;
    p.kappa2 = o.imgs_kappa * o.imgs_kappa;
    p.S = (const double2 *)S;
    p.hi = df ? (const float2 *)(w + o_hi) : nullptr;
    p.lo = df ? (const float2 *)(w + o_lo) : nullptr;
    p.Q = (double2 *)out->Q;
    p.pivots = out->pivots;
    p.err_curve = out->err_curve;
    p.C = ws_C ? (double2 *)(w + o_C) : (double2 *)out->C;
    p.rdiag = out->rdiag;
    p.norm2 = (double *)(w + o_norm);
    p.acc = (double *)(w + o_acc);
    p.picked = (unsigned char *)(w + o_pick);
    p.qh = df ? (float2 *)(w + o_qh) : nullptr;
    p.ql = df ? (float2 *)(w + o_ql) : nullptr;
    p.v = (double2 *)(w + o_v);
    p.hpart = (double2 *)(w + o_hp);
    p.npart = (double *)(w + o_np);
    p.bpart_err = (double *)(w + o_be);
    p.bpart_idx = (long long *)(w + o_bi);
    p.st = (rbk::DevState *)(w + o_st);
    p.passes_out = (int *)(w + o_pass);

    cudaStream_t sm = ctx->stream;
    const bool timing = (o.flags & RB_FLAG_TIMING) != 0;
    if (timing && (int)ctx->sweep_ev.size() < 2 * kcap) {
        while ((int)ctx->sweep_ev.size() < 2 * kcap) {
            cudaEvent_t ev;
            RB_CK(cudaEventCreate(&ev), "cudaEventCreate");
            ctx->sweep_ev.push_back(ev);
        }
    }
    if (timing && (int)ctx->imgs_ev.size() < 2 * kcap) {
        while ((int)ctx->imgs_ev.size() < 2 * kcap) {
            cudaEvent_t ev;
            RB_CK(cudaEventCreate(&ev), "cudaEventCreate");
            ctx->imgs_ev.push_back(ev);
        }
    }
    ctx->trace_passes.clear();
    ctx->trace_sweep_ms.clear();
    ctx->trace_imgs_ms.clear();
    int nlaunch = 0;
    RB_CK(cudaEventRecord(ctx->ev0, sm), "cudaEventRecord");
    RB_CK(cudaMemsetAsync(p.st, 0, sizeof(rbk::DevState), sm), "memset state");
    if (df)
        RB_CK(rbk::launch_split(p.S, N, M, ldS, (float2 *)p.hi, (float2 *)p.lo, ldH, p.norm2, sm), "split");
    else
        RB_CK(rbk::launch_norms(p.S, N, M, ldS, p.norm2, sm), "norms");
    if (k0 > 0) {
        RB_CK(rbk::launch_resume(p, k0, G, sm), "resume");
        nlaunch += 4;
    } else {
        RB_CK(rbk::launch_init(p, G, sm), "init");
        nlaunch += 2;
    }

    int it = k0;
    bool stopped = false;
    while (!stopped) {
        for (int t = 0; t < o.iters_per_sync && it < kcap; t++, it++) {
            if (timing) RB_CK(cudaEventRecord(ctx->imgs_ev[2 * it], sm), "cudaEventRecord");
            RB_CK(rbk::launch_imgs(p, G, false, sm, &nlaunch), "imgs");
            if (timing) RB_CK(cudaEventRecord(ctx->imgs_ev[2 * it + 1], sm), "cudaEventRecord");
            if (o.recompute_period > 0) {
                RB_CK(rbk::launch_recompute(p, o.recompute_period, G, sm), "recompute");
                nlaunch += 1;
            }
            if (timing) RB_CK(cudaEventRecord(ctx->sweep_ev[2 * it], sm), "cudaEventRecord");
            RB_CK(rbk::launch_sweep(p, variant, G, sm), "sweep");
            if (timing) RB_CK(cudaEventRecord(ctx->sweep_ev[2 * it + 1], sm), "cudaEventRecord");
            nlaunch += 1;
        }
        RB_CK(cudaMemcpyAsync(ctx->st_host, p.st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm), "state copy");
        RB_CK(cudaStreamSynchronize(sm), "stream sync");
        stopped = ctx->st_host->stop != 0;
        if (!stopped && it >= kcap) return fail(ctx, RB_ESTATE, "greedy loop did not stop after kmax iterations");
    }
    if (out->final_err) {
        RB_CK(rbk::launch_final_err(p, out->final_err, sm), "final_err");
        nlaunch += 1;
    }
    RB_CK(cudaEventRecord(ctx->ev1, sm), "cudaEventRecord");
    RB_CK(cudaEventSynchronize(ctx->ev1), "cudaEventSynchronize");
    const rbk::DevState &hs = *ctx->st_host;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    out->k = hs.k;
    out->status = hs.status;
    out->imgs_passes = hs.total_passes;
    out->switch_iter = -1;
    out->n_launches = nlaunch;
    out->n_sweeps = hs.n_sweeps;
    out->ms_total = ms;
    out->ms_sweep = 0.0;
    if (timing) {
        for (int i = k0; i < k0 + hs.n_sweeps && i < it; i++) {
            float t = 0.f, ti = 0.f;
            cudaEventElapsedTime(&t, ctx->sweep_ev[2 * i], ctx->sweep_ev[2 * i + 1]);
            cudaEventElapsedTime(&ti, ctx->imgs_ev[2 * i], ctx->imgs_ev[2 * i + 1]);
            out->ms_sweep += t;
            ctx->trace_sweep_ms.push_back(t);
            ctx->trace_imgs_ms.push_back(ti);
        }
    }
    if (hs.k > k0) {
        ctx->trace_passes.resize((size_t)(hs.k - k0));
        RB_CK(cudaMemcpy(ctx->trace_passes.data(), p.passes_out + k0, (size_t)(hs.k - k0) * sizeof(int),
                         cudaMemcpyDeviceToHost),
              "passes copy");
    }
    // algorithmic bytes of one sweep: S (16 N M: complex128, or hi+lo complex64),
    // q (16 N), norm2 + acc reads (16 M), picked (M), C row + acc writes (24 M)
    out->sweep_bytes = (double)hs.n_sweeps * (16.0 * N * M + 16.0 * N + 41.0 * M);
    if (hs.status < 0) {
        const char *why = hs.status == RB_ENONFINITE ? "NaN or Inf in S"
                          : hs.status == RB_EORTHO   ? "IMGS did not pass the kappa test within imgs_max_passes"
                                                     : "device error";
        return fail(ctx, (rb_status)hs.status, "rb_greedy: %s", why);
    }
    return (rb_status)hs.status;
}

static rb_status greedy_split_device(rb_ctx *ctx, const void *hi, const void *lo, long long N, long long M,
                                     long long ld, double tol, int kmax, rb_result *out) {
    const rb_options &o = ctx->opt;
    const int G = grid_for_variant(ctx, RB_SWEEP_DF32);
    const int chunk = 2048;
    const int nchunk = (int)((N + chunk - 1) / chunk);
    const int gN = (int)((N + rbk::kThreads - 1) / rbk::kThreads);
    const int kcap = kmax > 0 ? kmax : 1;
    const int lgcap = (kcap + 7) / 8;
    const long long qs = (long long)align_up((size_t)N, 64);

    Layout L;
    size_t o_norm = L.add((size_t)M * 8), o_acc = L.add((size_t)M * 8), o_pick = L.add((size_t)M);
    size_t o_nh = L.add((size_t)M * 8), o_ln = L.add((size_t)M * 4), o_sn = L.add((size_t)M * 64 * 4);
    size_t o_sa = L.add((size_t)M * 8);
    size_t o_da = L.add((size_t)M * 8), o_dc = L.add((size_t)M * 4);
    size_t o_qh = L.add((size_t)kcap * qs * sizeof(float2)), o_ql = L.add((size_t)kcap * qs * sizeof(float2));
    size_t o_v = L.add((size_t)N * sizeof(double2));
    size_t o_hp = L.add((size_t)kcap * nchunk * sizeof(double2));
    size_t np = (size_t)(G > gN ? G : gN);
    size_t o_np = L.add(np * 8), o_be = L.add((size_t)G * 8), o_bi = L.add((size_t)G * 8);
    size_t o_cd = L.add((size_t)M * 8), o_ce = L.add((size_t)M * 8);
    size_t o_pv = L.add((size_t)M * lgcap * 8);
    // FP16 pieces of the basis for the projection onto lo, and their scales
    size_t o_ap = L.add(rbk::lo_pieces_bytes(N, kcap));
    size_t o_qs = L.add((size_t)kcap * sizeof(int));
    // re-check chunk partials and counters (2048 pairs x 8 chunks x 32 doubles)
    size_t o_rp = L.add((size_t)2048 * 8 * 32 * 8), o_rt = L.add((size_t)2048 * 4);
    size_t o_C = out->C ? 0 : L.add((size_t)kcap * M * sizeof(double2));
    size_t o_st = L.add(sizeof(rbk::DevState));
    size_t o_te = L.add(sizeof(int));
    rb_status s = ensure(ctx, &ctx->ws, &ctx->ws_cap, L.off);
    if (s != RB_OK) return s;
    char *w = (char *)ctx->ws;

    rbk::Prob p{};
    p.N = N;
    p.M = M;
    p.ldS = 0;
    p.ldH = ld;
    p.ldQ = out->ldQ;
    p.ldC = out->C ? out->ldC : M;
    p.minNM = N < M ? N : M;
    p.kmax = kmax;
    p.max_passes = o.imgs_max_passes;
    p.nchunk = nchunk;
    p.chunk = chunk;
    p.tol = tol;
    p.kappa2 = o.imgs_kappa * o.imgs_kappa;
    p.S = nullptr;
    p.hi = (const float2 *)hi;
    p.lo = (const float2 *)lo;
    p.Q = (double2 *)out->Q;
    p.pivots = out->pivots;
    p.err_curve = out->err_curve;
    p.C = out->C ? (double2 *)out->C : (double2 *)(w + o_C);
    p.rdiag = out->rdiag;
    p.norm2 = (double *)(w + o_norm);
    p.acc = (double *)(w + o_acc);
    p.picked = (unsigned char *)(w + o_pick);
    p.qh = (float2 *)(w + o_qh);
    p.ql = (float2 *)(w + o_ql);
    p.qs_stride = qs;
    p.v = (double2 *)(w + o_v);
    p.hpart = (double2 *)(w + o_hp);
    p.npart = (double *)(w + o_np);
    p.bpart_err = (double *)(w + o_be);
    p.bpart_idx = (long long *)(w + o_bi);
    p.st = (rbk::DevState *)(w + o_st);
    p.norm2_hi = (double *)(w + o_nh);
    p.lonrm = (float *)(w + o_ln);
    p.snorm = (float *)(w + o_sn);
    p.sabs = (double *)(w + o_sa);
    // bound on the hi-only sweep's rounding relative to ||hi_j||: 2^-46 sqrt(N)
    // (measured maxima near 2^-42.4 at N = 16384, i.e. 2^-49.4 sqrt(N))
    p.eta = std::ldexp(1.0, -46) * std::sqrt((double)N);
    p.dacc = (double *)(w + o_da);
    p.dcnt = (int *)(w + o_dc);
    p.nblk_cand = G;
    p.cand = (long long *)(w + o_cd);
    p.cand_err = (double *)(w + o_ce);
    p.pv = (double *)(w + o_pv);
    p.apieces = (uint8_t *)(w + o_ap);
    p.qscale = (int *)(w + o_qs);
    p.rpart = (double *)(w + o_rp);
    p.rtick = (int *)(w + o_rt);
    p.lgcap = lgcap;
    p.tc_err = (int *)(w + o_te);
    p.wait_cycles = rbk::ctx_wait_cycles(ctx);
    p.switch_err = o.switch_err;
    // re-checking more than this many candidates costs more than sweeping hi + lo
    p.switch_cand = (o.flags & RB_FLAG_SPLIT_NO_SWITCH) ? INT_MAX : (int)std::max<long long>(M / 8, 256);

    cudaStream_t sm = ctx->stream;
    int nlaunch = 0;
    RB_CK(cudaEventRecord(ctx->ev0, sm), "cudaEventRecord");
    RB_CK(cudaMemsetAsync(p.st, 0, sizeof(rbk::DevState), sm), "memset state");
    RB_CK(cudaMemsetAsync(p.tc_err, 0, sizeof(int), sm), "memset tc flag");
    RB_CK(cudaMemsetAsync(p.rtick, 0, 2048 * sizeof(int), sm), "memset re-check counters");
    RB_CK(rbk::launch_split_init(p, sm), "split init");
    RB_CK(rbk::launch_init(p, G, sm), "init");
    nlaunch += 2;
    int it = 0;
    bool stopped = false;
    // one more round than kmax: a loop that ends at kmax still queues its
    // projection onto lo after the last sweep
    while (!stopped) {
        for (int t = 0; t < o.iters_per_sync && it <= kcap; t++, it++) {
            RB_CK(rbk::launch_imgs(p, G, true, sm, &nlaunch), "imgs");
            // hi-only phase (these return at once after the switch) ...
            RB_CK(rbk::launch_split_iteration(p, G, sm, &nlaunch), "split iteration");
            // ... or the hi + lo sweep after it (returns at once before it)
            RB_CK(rbk::launch_sweep(p, RB_SWEEP_DF32, G, sm), "hi+lo sweep");
            nlaunch += 1;
            // the projection onto lo, queued at the switch or when the loop ends
            RB_CK(rbk::launch_split_finish(p, G, sm, &nlaunch), "split finish");
        }
        RB_CK(cudaMemcpyAsync(ctx->st_host, p.st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm), "state copy");
        RB_CK(cudaStreamSynchronize(sm), "stream sync");
        stopped = ctx->st_host->stop != 0;
        if (!stopped && it > kcap) return fail(ctx, RB_ESTATE, "split greedy did not stop after kmax iterations");
    }
    if (out->final_err) {
        RB_CK(rbk::launch_final_err(p, out->final_err, sm), "final_err");
        nlaunch += 1;
    }
    RB_CK(cudaEventRecord(ctx->ev1, sm), "cudaEventRecord");
    RB_CK(cudaEventSynchronize(ctx->ev1), "cudaEventSynchronize");
    const rbk::DevState &hs = *ctx->st_host;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    out->k = hs.k;
    out->status = hs.status;
    out->imgs_passes = hs.total_passes;
    out->switch_iter = hs.phase ? hs.switch_iter : -1;
    out->n_launches = nlaunch;
    out->n_sweeps = hs.n_sweeps;
    out->ms_total = ms;
    out->ms_sweep = 0.0;
    int tc_err = 0;
    RB_CK(cudaMemcpy(&tc_err, p.tc_err, sizeof(int), cudaMemcpyDeviceToHost), "tc flag");
    if (tc_err) return fail(ctx, RB_ETIMEOUT, "rb_greedy_split: a tensor-core wait ran out");
    // per hi-only sweep: hi (8 N M), chain norms (256 M), q (16 N), the column
    // scalars read and written (acc, sabs, C row, norm2, norm2_hi, lonrm, picked);
    // per hi + lo sweep after the switch, the FP64 form's sweep bytes
    out->sweep_bytes = (double)(hs.n_sweeps - hs.n_sweeps_hl) * (8.0 * N * M + 256.0 * M + 16.0 * N + 69.0 * M) +
                       (double)hs.n_sweeps_hl * (16.0 * N * M + 16.0 * N + 41.0 * M);
    if (hs.status < 0) {
        const char *why = hs.status == RB_ENONFINITE ? "NaN or Inf in hi/lo"
                          : hs.status == RB_EORTHO   ? "IMGS did not pass the kappa test within imgs_max_passes"
                                                     : "device error";
        return fail(ctx, (rb_status)hs.status, "rb_greedy_split: %s", why);
    }
    return (rb_status)hs.status;
}

static int rb_log_level() {
    const char *e = getenv("RB_LOG");
    return e ? atoi(e) : 0;
}

rb_status rb_greedy_batched(rb_ctx *ctx, int nprob, const rb_problem *probs, double tol, int kmax,
                            rb_result *outs) {
    if (!ctx) return RB_EINVAL;
    if (nprob < 1 || !probs || !outs) return fail(ctx, RB_EINVAL, "rb_greedy_batched: bad problem list");
    if (!(tol >= 0.0) || !std::isfinite(tol) || kmax < 0) return fail(ctx, RB_EINVAL, "rb_greedy_batched: bad tol/kmax");
    long long maxN = 0, sumNM = 0;
    for (int b = 0; b < nprob; b++) {
        const rb_problem &pr = probs[b];
        const rb_result &o = outs[b];
        if (!pr.S || pr.N < 1 || pr.M < 1 || pr.ldS < pr.N || !aligned(pr.S, 16) || !o.Q || !o.pivots ||
            !o.err_curve || o.ldQ < pr.N || !aligned(o.Q, 16) || (o.C && (o.ldC < pr.M || !aligned(o.C, 16))))
            return fail(ctx, RB_EINVAL, "rb_greedy_batched: bad arguments for problem %d", b);
        maxN = pr.N > maxN ? pr.N : maxN;
        sumNM += pr.N * pr.M;
    }
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const rb_options &o = ctx->opt;
    const int G = grid_for_variant(ctx, RB_SWEEP_DF32);
    const int chunk = 2048;
    const int kcap = kmax > 0 ? kmax : 1;
    const int CWs[2] = {32, 128};
    // workspace layout
    Layout L;
    std::vector<size_t> o_norm(nprob), o_acc(nprob), o_pick(nprob), o_qh(nprob), o_ql(nprob), o_v(nprob),
        o_hp(nprob), o_np(nprob), o_be(nprob), o_bi(nprob), o_st(nprob);
    long long chunks_min_cw = 0, total_cols = 0;
    for (int b = 0; b < nprob; b++) {
        const long long N = probs[b].N, M = probs[b].M;
        const int nchunk = (int)((N + chunk - 1) / chunk), gN = (int)((N + rbk::kThreads - 1) / rbk::kThreads);
        o_norm[b] = L.add((size_t)M * 8);
        o_acc[b] = L.add((size_t)M * 8);
        o_pick[b] = L.add((size_t)M);
        o_qh[b] = L.add((size_t)(N + 2) * 8);
        o_ql[b] = L.add((size_t)(N + 2) * 8);
        o_v[b] = L.add((size_t)N * 16);
        o_hp[b] = L.add((size_t)kcap * nchunk * 16);
        const int gNmax = (int)((maxN + rbk::kThreads - 1) / rbk::kThreads);
        const int np_b = G > gN ? G : gN;
        o_np[b] = L.add((size_t)(np_b > gNmax ? np_b : gNmax) * 8);
        o_be[b] = L.add((size_t)G * 8);
        o_bi[b] = L.add((size_t)G * 8);
        o_st[b] = L.add(sizeof(rbk::DevState));
        chunks_min_cw += (M + CWs[0] - 1) / CWs[0];
        total_cols += M;
    }
    // pre-split hi/lo copy when it fits in free device memory (sweeps then stream
    // 16 bytes per element without the in-register split)
    std::vector<size_t> o_hi(nprob), o_lo(nprob);
    std::vector<long long> ldHs(nprob);
    size_t split_bytes = 0;
    for (int b = 0; b < nprob; b++) {
        ldHs[b] = (long long)align_up((size_t)probs[b].N, 64);
        split_bytes += 2 * (size_t)probs[b].M * ldHs[b] * sizeof(float2) + 1024;
    }
    size_t freeb = 0, totalb = 0;
    RB_CK(cudaMemGetInfo(&freeb, &totalb), "cudaMemGetInfo");
    const size_t have = ctx->ws_cap;
    const bool fits = (split_bytes + L.off + (4ull << 30)) < (size_t)(0.95 * (double)(freeb + have));
    // a forced sweep variant (rb_options.batched_variant) fixes the layout too
    const int force = o.batched_variant;
    if (force >= 12 && !fits)
        return fail(ctx, RB_EINVAL, "rb_greedy_batched: forced pre-split variant %d, but the copy does not fit",
                    force / 2);
    const bool presplit = force >= 0 ? force >= 12 : fits;
    if (presplit)
        for (int b = 0; b < nprob; b++) {
            o_hi[b] = L.add((size_t)probs[b].M * ldHs[b] * sizeof(float2));
            o_lo[b] = L.add((size_t)probs[b].M * ldHs[b] * sizeof(float2));
        }
    size_t o_P = L.add((size_t)nprob * sizeof(rbk::BProb));
    size_t o_PP = L.add((size_t)nprob * sizeof(rbk::Prob));
    size_t o_ch = L.add((size_t)(nprob + 1) * 8), o_col = L.add((size_t)(nprob + 1) * 8);
    size_t o_pe = L.add((size_t)chunks_min_cw * 8), o_pi = L.add((size_t)chunks_min_cw * 8);
    rb_status s = ensure(ctx, &ctx->ws, &ctx->ws_cap, L.off);
    if (s != RB_OK) return s;
    char *w = (char *)ctx->ws;
    cudaStream_t sm = ctx->stream;
    RB_CK(cudaMemsetAsync(w, 0, L.off, sm), "memset workspace");

    std::vector<rbk::Prob> pp(nprob);
    std::vector<rbk::BProb> bp(nprob);
    std::vector<long long> col0(nprob + 1, 0);
    for (int b = 0; b < nprob; b++) {
        const long long N = probs[b].N, M = probs[b].M;
        rbk::Prob &p = pp[b];
        p = rbk::Prob{};
        p.N = N;
        p.M = M;
        p.ldS = probs[b].ldS;
        p.ldQ = outs[b].ldQ;
        p.ldC = outs[b].ldC;
        p.minNM = N < M ? N : M;
        p.kmax = kmax;
        p.max_passes = o.imgs_max_passes;
        p.chunk = chunk;
        p.nchunk = (int)((N + chunk - 1) / chunk);
        p.tol = tol;
        p.kappa2 = o.imgs_kappa * o.imgs_kappa;
        p.S = (const double2 *)probs[b].S;
        p.Q = (double2 *)outs[b].Q;
        p.pivots = outs[b].pivots;
        p.err_curve = outs[b].err_curve;
        p.C = (double2 *)outs[b].C;
        p.rdiag = outs[b].rdiag;
        p.norm2 = (double *)(w + o_norm[b]);
        p.acc = (double *)(w + o_acc[b]);
        p.picked = (unsigned char *)(w + o_pick[b]);
        p.qh = (float2 *)(w + o_qh[b]);
        p.ql = (float2 *)(w + o_ql[b]);
        p.v = (double2 *)(w + o_v[b]);
        p.hpart = (double2 *)(w + o_hp[b]);
        p.npart = (double *)(w + o_np[b]);
        p.bpart_err = (double *)(w + o_be[b]);
        p.bpart_idx = (long long *)(w + o_bi[b]);
        p.st = (rbk::DevState *)(w + o_st[b]);
        rbk::BProb &q = bp[b];
        q = rbk::BProb{};
        q.N = N;
        q.M = M;
        q.ldS = p.ldS;
        q.ldC = p.ldC;
        q.S = p.S;
        q.C = p.C;
        q.err_curve = p.err_curve;
        q.norm2 = p.norm2;
        q.acc = p.acc;
        q.picked = p.picked;
        q.qh = p.qh;
        q.ql = p.ql;
        q.st = p.st;
        q.kmax = kmax;
        q.minNM = p.minNM;
        q.tol = tol;
        if (presplit) {
            q.hi = (const float2 *)(w + o_hi[b]);
            q.lo = (const float2 *)(w + o_lo[b]);
            q.ldH = ldHs[b];
        }
        col0[b + 1] = col0[b] + M;
    }
    rbk::BProb *dP = (rbk::BProb *)(w + o_P);
    long long *dch = (long long *)(w + o_ch), *dcol = (long long *)(w + o_col);
    double *dpe = (double *)(w + o_pe);
    long long *dpi = (long long *)(w + o_pi);
    rbk::Prob *dPP = (rbk::Prob *)(w + o_PP);
    RB_CK(cudaMemcpyAsync(dP, bp.data(), nprob * sizeof(rbk::BProb), cudaMemcpyHostToDevice, sm), "copy problems");
    RB_CK(cudaMemcpyAsync(dPP, pp.data(), nprob * sizeof(rbk::Prob), cudaMemcpyHostToDevice, sm), "copy problems");
    RB_CK(cudaMemcpyAsync(dcol, col0.data(), (nprob + 1) * 8, cudaMemcpyHostToDevice, sm), "copy prefix");
    auto chunk_prefix = [&](int CW) {
        std::vector<long long> c(nprob + 1, 0);
        for (int b = 0; b < nprob; b++) c[b + 1] = c[b] + (probs[b].M + CW - 1) / CW;
        return c;
    };
    // chunk prefix sums on the device
    auto upload_chunks = [&](int CW) -> cudaError_t {
        std::vector<long long> c = chunk_prefix(CW);
        cudaError_t e1 = cudaMemcpyAsync(dch, c.data(), (nprob + 1) * 8, cudaMemcpyHostToDevice, sm);
        if (e1 != cudaSuccess) return e1;
        return cudaStreamSynchronize(sm);
    };
    // ---- autotune (dry sweeps of this batch), cached per batch shape
    const int v0 = presplit ? 6 : 0;
    auto key = std::make_tuple(nprob * (presplit ? -1 : 1), sumNM, maxN);
    if (presplit && force < 0 && ctx->tune.find(key) == ctx->tune.end())  // the tuning sweeps read the copy
        for (int b = 0; b < nprob; b++)
            RB_CK(rbk::launch_split(pp[b].S, probs[b].N, probs[b].M, probs[b].ldS, (float2 *)bp[b].hi,
                                    (float2 *)bp[b].lo, ldHs[b], pp[b].norm2, sm),
                  "split");
    int best_v = v0 + 3, best_cw = 32;
    auto it_t = ctx->tune.find(key);
    if (force >= 0) {
        best_v = force / 2;
        best_cw = CWs[force % 2];
    } else if (it_t != ctx->tune.end()) {
        best_v = it_t->second.first;
        best_cw = it_t->second.second;
    } else {
        float best_ms = 1e30f;
        for (int ci = 0; ci < 2; ci++) {
            RB_CK(upload_chunks(CWs[ci]), "copy chunks");
            for (int v = v0; v < v0 + 6; v++) {
                int g = rbk::bsweep_grid(v, ctx->device);
                float ms = 0.f;
                for (int rep = 0; rep < 2; rep++) {
                    RB_CK(cudaEventRecord(ctx->ev0, sm), "cudaEventRecord");
                    RB_CK(rbk::launch_bsweep(v, g, dP, nprob, dch, CWs[ci], dpe, dpi, 1, sm), "dry sweep");
                    RB_CK(cudaEventRecord(ctx->ev1, sm), "cudaEventRecord");
                    RB_CK(cudaEventSynchronize(ctx->ev1), "cudaEventSynchronize");
                    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
                }
                if (rb_log_level() > 0)
                    fprintf(stderr, "rb autotune: %s U=%d threads=%d CW=%d  %.3f ms\n",
                            presplit ? "hi/lo" : "complex128", 2 << (v % 3), rbk::bsweep_threads(v), CWs[ci], ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    best_v = v;
                    best_cw = CWs[ci];
                }
            }
        }
        ctx->tune[key] = std::make_pair(best_v, best_cw);
    }
    RB_CK(upload_chunks(best_cw), "copy chunks");
    const int gv = rbk::bsweep_grid(best_v, ctx->device);
    for (int b = 0; b < nprob; b++) RB_CK(cudaMemsetAsync(pp[b].st, 0, sizeof(rbk::DevState), sm), "memset state");
    RB_CK(cudaEventRecord(ctx->ev0, sm), "cudaEventRecord");
    int nlaunch = 0;
    if (presplit) {
        // timed region starts after the copy made for tuning: redo it here
        for (int b = 0; b < nprob; b++) {
            RB_CK(rbk::launch_split(pp[b].S, probs[b].N, probs[b].M, probs[b].ldS, (float2 *)bp[b].hi,
                                    (float2 *)bp[b].lo, ldHs[b], pp[b].norm2, sm),
                  "split");
            nlaunch++;
        }
    } else {
        RB_CK(rbk::launch_bnorms(dP, nprob, dcol, total_cols, sm), "norms");
        nlaunch++;
    }
    for (int b = 0; b < nprob; b++) {
        RB_CK(rbk::launch_init(pp[b], G, sm), "init");
        nlaunch++;
    }
    // ---- capture one iteration: the IMGS steps of all problems (one launch per
    // step, grid.y = problem), then the sweep and the per-problem reduction
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    int per_iter = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rbk::launch_imgs_batched(dPP, nprob, maxN, o.imgs_max_passes, G, cap, &per_iter);
        rbk::launch_bsweep(best_v, gv, dP, nprob, dch, best_cw, dpe, dpi, 0, cap);
        rbk::launch_breduce(dP, nprob, dch, dpe, dpi, cap);
        per_iter += 2;
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    // ---- replay until every problem has stopped
    std::vector<rbk::DevState> hs(nprob);
    int it = 0;
    bool all = false;
    while (e == cudaSuccess && !all) {
        for (int t = 0; t < o.iters_per_sync && it <= kcap && e == cudaSuccess; t++, it++) {
            e = cudaGraphLaunch(exec, sm);
            nlaunch += per_iter;
        }
        for (int b = 0; b < nprob && e == cudaSuccess; b++)
            e = cudaMemcpyAsync(&hs[b], pp[b].st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
        all = true;
        for (int b = 0; b < nprob; b++) all = all && hs[b].stop;
        if (!all && it > kcap) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_greedy_batched loop");
    if (!all) return fail(ctx, RB_ESTATE, "rb_greedy_batched: a problem did not stop after kmax iterations");
    for (int b = 0; b < nprob; b++)
        if (outs[b].final_err) {
            RB_CK(rbk::launch_final_err(pp[b], outs[b].final_err, sm), "final_err");
            nlaunch++;
        }
    RB_CK(cudaEventRecord(ctx->ev1, sm), "cudaEventRecord");
    RB_CK(cudaEventSynchronize(ctx->ev1), "cudaEventSynchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    rb_status worst = RB_OK;
    for (int b = 0; b < nprob; b++) {
        rb_result &out = outs[b];
        const long long N = probs[b].N, M = probs[b].M;
        out.k = hs[b].k;
        out.status = hs[b].status;
        out.imgs_passes = hs[b].total_passes;
        out.switch_iter = -1;
        out.n_launches = nlaunch;
        out.n_sweeps = hs[b].n_sweeps;
        out.ms_total = ms;
        out.ms_sweep = 0.0;
        out.sweep_bytes = (double)hs[b].n_sweeps * (16.0 * N * M + 16.0 * N + 41.0 * M);
        rb_status sb = (rb_status)hs[b].status;
        if (sb < 0 && (worst >= 0 || sb < worst)) worst = sb;
        else if (worst == RB_OK && sb == RB_KMAX_REACHED) worst = sb;
    }
    if (worst < 0) return fail(ctx, worst, "rb_greedy_batched: a problem failed (status %d)", (int)worst);
    return worst;
}

static rb_status check_greedy_args(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol,
                                   int kmax, const rb_result *out) {
    if (!ctx) return RB_EINVAL;
    if (!out || !S) return fail(ctx, RB_EINVAL, "null S or result");
    if (N < 1 || M < 1 || ldS < N) return fail(ctx, RB_EINVAL, "bad sizes N=%lld M=%lld ldS=%lld", N, M, ldS);
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(ctx, RB_EINVAL, "tol must be finite and >= 0");
    if (kmax < 0) return fail(ctx, RB_EINVAL, "kmax must be >= 0");
    if (!out->Q || !out->pivots || !out->err_curve) return fail(ctx, RB_EINVAL, "Q, pivots, err_curve are required");
    if (out->ldQ < N) return fail(ctx, RB_EINVAL, "ldQ < N");
    if (out->C && out->ldC < M) return fail(ctx, RB_EINVAL, "ldC < M");
    return RB_OK;
}

rb_status rb_greedy(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                    rb_result *out) {
    rb_status s = check_greedy_args(ctx, S, N, M, ldS, tol, kmax, out);
    if (s != RB_OK) return s;
    if (!aligned(S, 16) || !aligned(out->Q, 16) || (out->C && !aligned(out->C, 16)))
        return fail(ctx, RB_EINVAL, "complex128 arrays must be 16-byte aligned");
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    return greedy_device(ctx, S, N, M, ldS, tol, kmax, out);
}

rb_status rb_greedy_resume(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                           int k0, long long Mc, rb_result *out) {
    rb_status s = check_greedy_args(ctx, S, N, M, ldS, tol, kmax, out);
    if (s != RB_OK) return s;
    const long long minNM = N < M ? N : M;
    if (k0 < 0 || k0 > kmax || k0 > minNM || Mc < 0 || Mc > M || (k0 > 0 && !out->C))
        return fail(ctx, RB_EINVAL, "rb_greedy_resume: need 0 <= k0 <= min(kmax, N, M), 0 <= Mc <= M and C (k0=%d)", k0);
    if (!aligned(S, 16) || !aligned(out->Q, 16) || (out->C && !aligned(out->C, 16)))
        return fail(ctx, RB_EINVAL, "complex128 arrays must be 16-byte aligned");
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (k0 == 0) return greedy_device(ctx, S, N, M, ldS, tol, kmax, out);
    // the checkpoint's pivots: distinct columns of S
    std::vector<long long> piv(k0);
    RB_CK(cudaMemcpyAsync(piv.data(), out->pivots, (size_t)k0 * 8, cudaMemcpyDeviceToHost, ctx->stream), "pivot copy");
    RB_CK(cudaStreamSynchronize(ctx->stream), "stream sync");
    std::vector<long long> sorted(piv);
    std::sort(sorted.begin(), sorted.end());
    for (int l = 0; l < k0; l++)
        if (sorted[l] < 0 || sorted[l] >= M || (l > 0 && sorted[l] == sorted[l - 1]))
            return fail(ctx, RB_EINVAL, "rb_greedy_resume: checkpoint pivots must be distinct columns of S");
    // coefficients of the columns the checkpoint has not seen
    if (Mc < M) {
        s = rb_project(ctx, out->Q, N, k0, out->ldQ, (const double2 *)S + Mc * ldS, M - Mc, ldS,
                       (double2 *)out->C + Mc, out->ldC);
        if (s != RB_OK) return s;
    }
    return greedy_device(ctx, S, N, M, ldS, tol, kmax, out, k0);
}

// Host pointer of S as the device sees it; registers pageable memory for the
// call (*registered = true) and rejects device memory.
static rb_status host_view(rb_ctx *ctx, const void *S, size_t bytes, const double2 **dptr, bool *registered) {
    *registered = false;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, S);
    if (e != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return fail(ctx, RB_EINVAL, "rb_greedy_streamed: S must be host memory (device arrays go to rb_greedy)");
    if (at.type == cudaMemoryTypeUnregistered) {
        RB_CK(cudaHostRegister(const_cast<void *>(S), bytes, cudaHostRegisterMapped), "cudaHostRegister of S");
        *registered = true;
    }
    // pinned memory under unified addressing: the attributes carry the device
    // view; otherwise ask for the mapping
    void *d = nullptr;
    if (cudaPointerGetAttributes(&at, S) == cudaSuccess && at.type == cudaMemoryTypeHost) d = at.devicePointer;
    cudaGetLastError();
    if (!d) {
        e = cudaHostGetDevicePointer(&d, const_cast<void *>(S), 0);
        if (e != cudaSuccess) cudaGetLastError();
    }
    if (!d) {
        if (*registered) cudaHostUnregister(const_cast<void *>(S));
        *registered = false;
        return fail(ctx, RB_ECUDA, "rb_greedy_streamed: S has no device mapping (host memory not mapped)");
    }
    *dptr = (const double2 *)d;
    return RB_OK;
}

// Sd: S in host memory (device-visible pointer); columns Mr.. are read lazily
// over the host link.
static rb_status greedy_streamed_device(rb_ctx *ctx, const double2 *Sd, long long N, long long M, long long ldS,
                                       double tol, int kmax, long long Mr, long long cols, rb_result *out) {
    const rb_options &o = ctx->opt;
    const int G = grid_for_variant(ctx, RB_SWEEP_DF32);
    const long long ldH = (long long)align_up((size_t)N, 64);
    const int chunk = 2048;
    const int nchunk = (int)((N + chunk - 1) / chunk);
    const int gN = (int)((N + rbk::kThreads - 1) / rbk::kThreads);
    const int kcap = kmax > 0 ? kmax : 1;
    const int nch = (int)((M - Mr + cols - 1) / cols);
    const int Gs = rbk::stream_sweep_grid(ctx->device);
    const int nwarps = Gs * (rbk::kThreads / 32);

    Layout L;
    size_t o_hi = L.add((size_t)Mr * ldH * sizeof(float2)), o_lo = L.add((size_t)Mr * ldH * sizeof(float2));
    size_t o_norm = L.add((size_t)M * 8), o_acc = L.add((size_t)M * 8), o_pick = L.add((size_t)M);
    size_t o_qh = L.add((size_t)kcap * ldH * sizeof(float2)), o_ql = L.add((size_t)kcap * ldH * sizeof(float2));
    size_t o_v = L.add((size_t)N * sizeof(double2));
    size_t o_hp = L.add((size_t)kcap * nchunk * sizeof(double2));
    size_t np = (size_t)std::max(std::max(G, gN), Gs);
    size_t o_np = L.add(np * 8), o_be = L.add(np * 8), o_bi = L.add(np * 8);
    size_t o_st = L.add(sizeof(rbk::DevState));
    size_t o_pass = L.add((size_t)kcap * sizeof(int));
    const bool ws_C = !out->C && o.recompute_period > 0;
    size_t o_C = ws_C ? L.add((size_t)kcap * M * sizeof(double2)) : 0;
    size_t o_last = L.add((size_t)nch * 4), o_bound = L.add((size_t)nch * 8), o_nmax = L.add((size_t)nch * 8);
    size_t o_list = L.add((size_t)nch * 4), o_cnt = L.add(16), o_upd = L.add(8), o_part = L.add(1024 * 8);
    size_t o_stage = nch ? L.add((size_t)nwarps * 2 * ldH * sizeof(float2)) : 0;
    rb_status s = ensure(ctx, &ctx->ws, &ctx->ws_cap, L.off);
    if (s != RB_OK) return s;
    char *w = (char *)ctx->ws;

    rbk::Prob p{};
    p.N = N;
    p.M = M;
    p.ldS = ldS;
    p.ldH = ldH;
    p.ldQ = out->ldQ;
    p.ldC = ws_C ? M : out->ldC;
    p.minNM = N < M ? N : M;
    p.kmax = kmax;
    p.max_passes = o.imgs_max_passes;
    p.nchunk = nchunk;
    p.chunk = chunk;
    p.tol = tol;
    p.kappa2 = o.imgs_kappa * o.imgs_kappa;
    p.S = Sd;  // the IMGS steps read the pivot column from host memory
    p.hi = (const float2 *)(w + o_hi);
    p.lo = (const float2 *)(w + o_lo);
    p.Q = (double2 *)out->Q;
    p.pivots = out->pivots;
    p.err_curve = out->err_curve;
    p.C = ws_C ? (double2 *)(w + o_C) : (double2 *)out->C;
    p.rdiag = out->rdiag;
    p.norm2 = (double *)(w + o_norm);
    p.acc = (double *)(w + o_acc);
    p.picked = (unsigned char *)(w + o_pick);
    p.qh = (float2 *)(w + o_qh);
    p.ql = (float2 *)(w + o_ql);
    p.qs_stride = ldH;  // one FP32 slot per basis vector: lazy chunks apply old vectors
    p.v = (double2 *)(w + o_v);
    p.hpart = (double2 *)(w + o_hp);
    p.npart = (double *)(w + o_np);
    p.bpart_err = (double *)(w + o_be);
    p.bpart_idx = (long long *)(w + o_bi);
    p.st = (rbk::DevState *)(w + o_st);
    p.passes_out = (int *)(w + o_pass);

    rbk::StreamPart sp{};
    sp.Sd = Sd;
    sp.part = (double *)(w + o_part);
    sp.Mr = Mr;
    sp.cols = cols;
    sp.nch = nch;
    sp.period = o.recompute_period;
    sp.gamma = 0.99;
    sp.last = (int *)(w + o_last);
    sp.bound = (double *)(w + o_bound);
    sp.nmax = (double *)(w + o_nmax);
    sp.list = (int *)(w + o_list);
    sp.cnt = (int *)(w + o_cnt);
    sp.updates = (unsigned long long *)(w + o_upd);
    sp.stage = nch ? (float2 *)(w + o_stage) : nullptr;
    sp.stage_ld = ldH;

    cudaStream_t sm = ctx->stream;
    const bool timing = (o.flags & RB_FLAG_TIMING) != 0;
    if (timing) {
        while ((int)ctx->sweep_ev.size() < 2 * kcap) {
            cudaEvent_t ev;
            RB_CK(cudaEventCreate(&ev), "cudaEventCreate");
            ctx->sweep_ev.push_back(ev);
        }
        while ((int)ctx->imgs_ev.size() < 2 * kcap) {
            cudaEvent_t ev;
            RB_CK(cudaEventCreate(&ev), "cudaEventCreate");
            ctx->imgs_ev.push_back(ev);
        }
    }
    ctx->trace_passes.clear();
    ctx->trace_sweep_ms.clear();
    ctx->trace_imgs_ms.clear();
    int nlaunch = 0;
    cudaEvent_t ev_init = timing ? ctx->sweep_ev[0] : nullptr;
    RB_CK(cudaEventRecord(ctx->ev0, sm), "cudaEventRecord");
    RB_CK(cudaMemsetAsync(p.st, 0, sizeof(rbk::DevState), sm), "memset state");
    RB_CK(cudaMemsetAsync(sp.updates, 0, 8, sm), "memset counters");
    // one read of S from host memory: the resident split and every norm
    if (Mr > 0) RB_CK(rbk::launch_split(Sd, N, Mr, ldS, (float2 *)p.hi, (float2 *)p.lo, ldH, p.norm2, sm), "split");
    if (M > Mr)
        RB_CK(rbk::launch_split(Sd + Mr * ldS, N, M - Mr, ldS, nullptr, nullptr, ldH, p.norm2 + Mr, sm), "norms");
    RB_CK(rbk::launch_init(p, G, sm), "init");
    RB_CK(rbk::launch_stream_init(p, sp, sm), "stream init");
    nlaunch += 2 + (Mr > 0) + (M > Mr);
    float ms_init = 0.f;
    if (timing) {
        RB_CK(cudaEventRecord(ev_init, sm), "cudaEventRecord");
        RB_CK(cudaEventSynchronize(ev_init), "cudaEventSynchronize");
        cudaEventElapsedTime(&ms_init, ctx->ev0, ev_init);
    }
    rbk::Prob pres = p;  // the recompute of the resident columns
    pres.M = Mr;
    const int per_iter = 1 + 5 * (nch > 0) + 1;

    int it = 0;
    bool stopped = false;
    while (!stopped) {
        for (int t = 0; t < o.iters_per_sync && it < kcap; t++, it++) {
            if (timing) RB_CK(cudaEventRecord(ctx->imgs_ev[2 * it], sm), "cudaEventRecord");
            RB_CK(rbk::launch_imgs(p, G, false, sm, &nlaunch), "imgs");
            if (timing) RB_CK(cudaEventRecord(ctx->imgs_ev[2 * it + 1], sm), "cudaEventRecord");
            if (o.recompute_period > 0 && Mr > 0) {
                RB_CK(rbk::launch_recompute(pres, o.recompute_period, G, sm), "recompute");
                nlaunch += 1;
            }
            if (timing) RB_CK(cudaEventRecord(ctx->sweep_ev[2 * it], sm), "cudaEventRecord");
            RB_CK(rbk::launch_stream_iteration(p, sp, G, Gs, sm), "streamed sweep");
            if (timing) RB_CK(cudaEventRecord(ctx->sweep_ev[2 * it + 1], sm), "cudaEventRecord");
            nlaunch += per_iter;
        }
        RB_CK(cudaMemcpyAsync(ctx->st_host, p.st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm), "state copy");
        RB_CK(cudaStreamSynchronize(sm), "stream sync");
        stopped = ctx->st_host->stop != 0;
        if (!stopped && it >= kcap) return fail(ctx, RB_ESTATE, "greedy loop did not stop after kmax iterations");
    }
    RB_CK(rbk::launch_stream_flush(p, sp, Gs, sm), "flush");
    nlaunch += nch > 0 ? 2 : 0;
    if (out->final_err) {
        RB_CK(rbk::launch_final_err(p, out->final_err, sm), "final_err");
        nlaunch += 1;
    }
    RB_CK(cudaEventRecord(ctx->ev1, sm), "cudaEventRecord");
    RB_CK(cudaEventSynchronize(ctx->ev1), "cudaEventSynchronize");
    unsigned long long updates = 0;
    RB_CK(cudaMemcpy(&updates, sp.updates, 8, cudaMemcpyDeviceToHost), "counter copy");
    const rbk::DevState &hs = *ctx->st_host;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    out->k = hs.k;
    out->status = hs.status;
    out->imgs_passes = hs.total_passes;
    out->switch_iter = -1;
    out->n_launches = nlaunch;
    out->n_sweeps = hs.n_sweeps;
    out->ms_total = ms;
    out->ms_sweep = 0.0;
    if (timing) {
        for (int i = 0; i < hs.n_sweeps && i < it; i++) {
            float t = 0.f, ti = 0.f;
            cudaEventElapsedTime(&t, ctx->sweep_ev[2 * i], ctx->sweep_ev[2 * i + 1]);
            cudaEventElapsedTime(&ti, ctx->imgs_ev[2 * i], ctx->imgs_ev[2 * i + 1]);
            out->ms_sweep += t;
            ctx->trace_sweep_ms.push_back(t);
            ctx->trace_imgs_ms.push_back(ti);
        }
    }
    if (hs.k > 0) {
        ctx->trace_passes.resize((size_t)hs.k);
        RB_CK(cudaMemcpy(ctx->trace_passes.data(), p.passes_out, (size_t)hs.k * sizeof(int), cudaMemcpyDeviceToHost),
              "passes copy");
    }
    // device bytes of the resident sweeps (hi + lo, q, bookkeeping)
    out->sweep_bytes = (double)hs.n_sweeps * (16.0 * N * Mr + 16.0 * N + 41.0 * Mr);
    ctx->str_stats[0] = Mr;
    ctx->str_stats[1] = nch;
    ctx->str_stats[2] = cols;
    ctx->str_stats[3] = (long long)updates;
    // host bytes: the initial pass over all of S, one column per IMGS step, and
    // the non-resident columns of every chunk update
    double host = 16.0 * (double)N * (double)M + 16.0 * (double)N * hs.k;
    if (nch > 0) host += 16.0 * (double)N * (double)(M - Mr) / nch * (double)updates;
    ctx->str_host_bytes = host;
    ctx->str_ms_init = ms_init;
    if (hs.status < 0) {
        const char *why = hs.status == RB_ENONFINITE ? "NaN or Inf in S"
                          : hs.status == RB_EORTHO   ? "IMGS did not pass the kappa test within imgs_max_passes"
                                                     : "device error";
        return fail(ctx, (rb_status)hs.status, "rb_greedy_streamed: %s", why);
    }
    return (rb_status)hs.status;
}

rb_status rb_greedy_streamed(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol,
                             int kmax, long long resident, long long chunk_cols, rb_result *out) {
    rb_status s = check_greedy_args(ctx, S, N, M, ldS, tol, kmax, out);
    if (s != RB_OK) return s;
    if (!aligned(S, 16) || !aligned(out->Q, 16) || (out->C && !aligned(out->C, 16)))
        return fail(ctx, RB_EINVAL, "complex128 arrays must be 16-byte aligned");
    if (ctx->opt.sweep != RB_SWEEP_DF32)
        return fail(ctx, RB_EINVAL, "rb_greedy_streamed: needs the double-float sweep (RB_SWEEP_DF32)");
    if (chunk_cols < 0 || chunk_cols > (1LL << 20))
        return fail(ctx, RB_EINVAL, "rb_greedy_streamed: chunk_cols must be in [0, 2^20]");
    if (chunk_cols == 0) chunk_cols = 1;
    if ((M + chunk_cols - 1) / chunk_cols > (1LL << 30))
        return fail(ctx, RB_EINVAL, "rb_greedy_streamed: too many chunks");
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const long long ldH = (long long)align_up((size_t)N, 64);
    long long Mr = resident;
    if (Mr < 0) {
        // as many resident columns as the free device memory holds after the
        // per-column state, C, the basis slots and 4 GB of headroom
        size_t fr = 0, tot = 0;
        RB_CK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        const int kcap = kmax > 0 ? kmax : 1;
        double other = 17.0 * M + (out->C ? 0.0 : 16.0 * kcap * M) + 16.0 * kcap * ldH + 4e9 + (double)ctx->ws_cap;
        double room = (double)fr + (double)ctx->ws_cap - other;
        Mr = room > 0 ? (long long)(room / (16.0 * ldH)) : 0;
    }
    if (Mr > M) Mr = M;
    const size_t bytes = ((size_t)(M - 1) * (size_t)ldS + (size_t)N) * 16;
    const double2 *Sd = nullptr;
    bool reg = false;
    s = host_view(ctx, S, bytes, &Sd, &reg);
    if (s != RB_OK) return s;
    s = greedy_streamed_device(ctx, Sd, N, M, ldS, tol, kmax, Mr, chunk_cols, out);
    if (reg) {
        cudaStreamSynchronize(ctx->stream);
        cudaHostUnregister(const_cast<void *>(S));
    }
    return s;
}

rb_status rb_streamed_stats(const rb_ctx *ctx, long long *counts, double *host_bytes, double *ms_init) {
    if (!ctx) return RB_EINVAL;
    if (counts)
        for (int i = 0; i < 4; i++) counts[i] = ctx->str_stats[i];
    if (host_bytes) *host_bytes = ctx->str_host_bytes;
    if (ms_init) *ms_init = ctx->str_ms_init;
    return RB_OK;
}

rb_status rb_greedy_split(rb_ctx *ctx, const void *hi, const void *lo, long long N, long long M, long long ld,
                          double tol, int kmax, rb_result *out) {
    rb_status s = check_greedy_args(ctx, hi, N, M, ld, tol, kmax, out);
    if (s != RB_OK) return s;
    if (!lo || (ld & 1) || !aligned(hi, 16) || !aligned(lo, 16) || !aligned(out->Q, 16) ||
        (out->C && !aligned(out->C, 16)))
        return fail(ctx, RB_EINVAL, "rb_greedy_split: lo required, ld must be even and hi/lo 16-byte aligned");
    if (N > (1LL << 22)) return fail(ctx, RB_EINVAL, "rb_greedy_split: N must not exceed 2^22");
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    return greedy_split_device(ctx, hi, lo, N, M, ld, tol, kmax, out);
}

rb_status rb_debug_wait_selftest(rb_ctx *ctx, long long cycles, int arrive) {
    if (!ctx || cycles < 1) return RB_EINVAL;
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    rb_status s = ensure(ctx, &ctx->gen, &ctx->gen_cap, 256);
    if (s != RB_OK) return s;
    int *flag = (int *)ctx->gen;
    cudaStream_t sm = ctx->stream;
    RB_CK(cudaMemsetAsync(flag, 0, sizeof(int), sm), "memset flag");
    RB_CK(rbk::launch_wait_selftest(cycles, arrive, flag, sm), "wait selftest");
    int h = 0;
    RB_CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, sm), "flag copy");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    if (h) return fail(ctx, RB_ETIMEOUT, "bounded wait ran out after %lld cycles (self-test)", cycles);
    return RB_OK;
}

rb_status rb_greedy_host(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, double tol, int kmax,
                         rb_result *out) {
    rb_status s = check_greedy_args(ctx, S, N, M, ldS, tol, kmax, out);
    if (s != RB_OK) return s;
    RB_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    // pinned S under the double-float sweep: the kernels read it in place over
    // the host link (rb_greedy_streamed; no device copy of S, identical
    // results); otherwise one copy of S to the device
    bool in_place = false;
    if (ctx->opt.sweep == RB_SWEEP_DF32 && aligned(S, 16)) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, S) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
            in_place = true;
        cudaGetLastError();
    }
    const int kcap = kmax > 0 ? kmax : 1;
    Layout L;
    size_t o_S = in_place ? 0 : L.add((size_t)M * N * 16);
    size_t o_Q = L.add((size_t)kcap * N * 16), o_p = L.add((size_t)kcap * 8);
    size_t o_e = L.add((size_t)(kcap + 1) * 8);
    size_t o_C = out->C ? L.add((size_t)kcap * M * 16) : 0;
    size_t o_f = out->final_err ? L.add((size_t)M * 8) : 0;
    size_t o_r = out->rdiag ? L.add((size_t)kcap * 8) : 0;
    s = ensure(ctx, &ctx->stage, &ctx->stage_cap, L.off);
    if (s != RB_OK) return s;
    char *w = (char *)ctx->stage;
    cudaStream_t sm = ctx->stream;
    if (!in_place) {
        // a contiguous S goes in one linear copy (the 2D copy engine path is
        // about 2.5x slower for a 34 GB transfer from pinned memory)
        if (ldS == N)
            RB_CK(cudaMemcpyAsync(w + o_S, S, (size_t)M * N * 16, cudaMemcpyHostToDevice, sm), "copy S to device");
        else
            RB_CK(cudaMemcpy2DAsync(w + o_S, (size_t)N * 16, S, (size_t)ldS * 16, (size_t)N * 16, (size_t)M,
                                    cudaMemcpyHostToDevice, sm),
                  "copy S to device");
    }
    rb_result d = *out;
    d.Q = w + o_Q;
    d.ldQ = N;
    d.pivots = (long long *)(w + o_p);
    d.err_curve = (double *)(w + o_e);
    d.C = out->C ? (void *)(w + o_C) : nullptr;
    d.ldC = M;
    d.final_err = out->final_err ? (double *)(w + o_f) : nullptr;
    d.rdiag = out->rdiag ? (double *)(w + o_r) : nullptr;
    rb_status st = in_place ? rb_greedy_streamed(ctx, S, N, M, ldS, tol, kmax, -1, 0, &d)
                            : greedy_device(ctx, w + o_S, N, M, N, tol, kmax, &d);
    if (st < 0) return st;
    const int k = d.k;
    if (k > 0) {
        RB_CK(cudaMemcpy2DAsync(out->Q, (size_t)out->ldQ * 16, d.Q, (size_t)N * 16, (size_t)N * 16, (size_t)k,
                                cudaMemcpyDeviceToHost, sm),
              "copy Q");
        RB_CK(cudaMemcpyAsync(out->pivots, d.pivots, (size_t)k * 8, cudaMemcpyDeviceToHost, sm), "copy pivots");
        if (out->C && out->ldC == M)
            RB_CK(cudaMemcpyAsync(out->C, d.C, (size_t)k * M * 16, cudaMemcpyDeviceToHost, sm), "copy C");
        else if (out->C)
            RB_CK(cudaMemcpy2DAsync(out->C, (size_t)out->ldC * 16, d.C, (size_t)M * 16, (size_t)M * 16, (size_t)k,
                                    cudaMemcpyDeviceToHost, sm),
                  "copy C");
        if (out->rdiag)
            RB_CK(cudaMemcpyAsync(out->rdiag, d.rdiag, (size_t)k * 8, cudaMemcpyDeviceToHost, sm), "copy rdiag");
    }
    RB_CK(cudaMemcpyAsync(out->err_curve, d.err_curve, (size_t)(k + 1) * 8, cudaMemcpyDeviceToHost, sm),
          "copy err_curve");
    if (out->final_err)
        RB_CK(cudaMemcpyAsync(out->final_err, d.final_err, (size_t)M * 8, cudaMemcpyDeviceToHost, sm),
              "copy final_err");
    RB_CK(cudaStreamSynchronize(sm), "stream sync");
    void *keepQ = out->Q, *keepC = out->C;
    long long *keepP = out->pivots;
    double *keepE = out->err_curve, *keepF = out->final_err, *keepR = out->rdiag;
    long long kldQ = out->ldQ, kldC = out->ldC;
    *out = d;
    out->Q = keepQ;
    out->C = keepC;
    out->pivots = keepP;
    out->err_curve = keepE;
    out->final_err = keepF;
    out->rdiag = keepR;
    out->ldQ = kldQ;
    out->ldC = kldC;
    return st;
}

}  // extern "C"
