// rb_shard.cu -- one rank's part of the column-sharded greedy (the paper's
// parallel scheme, Sec. 6.1.4 and Sec. 6.2: every process owns a block of
// snapshot columns, finds its local pivot candidate, the candidates meet in a
// max-loc reduction, the owner of the winner sends that column, and every
// process orthogonalises it against its own full copy of the basis).
//
// A shard holds columns col0 .. col0 + M_local - 1 of the global snapshot
// matrix: their hi/lo split copy, norms, the Eq. (Residual) bookkeeping, the
// picked flags and their rows of C.  The exchange itself (max-loc, broadcast)
// is the caller's, between calls:
//   rb_shard_init    norms and the first local candidate;
//   rb_shard_column  the pivot column (owner only) and its norm;
//   rb_shard_append  IMGS of the received column against the shard's basis
//                    (every rank, the same deterministic kernels on the same
//                    bytes, so all ranks build bit-identical vectors), then
//                    the sweep of the local columns: the next local candidate;
//   rb_shard_finish  final errors of the local columns.
// The kernels are the FP64 form's (double-float sweep, FP64 IMGS and
// bookkeeping, periodic recompute); only the pivot's source and the stopping
// rule move to the caller.
#include <cmath>
#include <cstdio>
#include <new>

#include "rb_internal.cuh"

struct rb_shard {
    rb_ctx *ctx = nullptr;
    rbk::Prob p{};
    void *ws = nullptr;
    rbk::DevState *st_host = nullptr;  // pinned copy of the state
    long long col0 = 0;
    int kcap = 1;
    int G = 0;
    int period = 0;
    int k = 0;          // vectors appended so far
    int status = 0;     // RB_OK, or an error / RB_EORTHO from the device
    bool rank_end = false;  // the last received column lay in the span of the basis
};

namespace rbk {

// v = the received pivot column; IMGS state for basis size k.
__global__ void __launch_bounds__(kThreads) k_shard_begin(Prob p, const double2 *vin, double vnorm2) {
    DevState *st = p.st;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
         i += (long long)gridDim.x * blockDim.x)
        p.v[i] = vin[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // a negative norm from the host: the owner's norm travels in vin[N].x
        const double n2 = vnorm2 >= 0.0 ? vnorm2 : vin[p.N].x;
        st->stop = 0;
        st->force_stop = 0;
        st->status = RB_OK;
        st->passes = 0;
        st->accepted = (st->k == 0);
        st->before2 = n2;
        st->after2 = n2;
    }
}

// q_k = v / ||v||, its FP32 hi/lo split for the sweep, the global pivot index,
// R(k,k); the pivot is marked picked on its owner.  A zero v (the column lies
// in the span: exact rank) stops the shard without appending.
__global__ void __launch_bounds__(kThreads) k_shard_finalize(Prob p, long long jglobal, long long jlocal) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    const int k = st->k;
    const double nv2 = st->after2;
    if (!(nv2 > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->status = RB_OK;
            st->stop = 1;
            st->force_stop = 1;
        }
        return;
    }
    const double nv = sqrt(nv2);
    double2 *qk = p.Q + (long long)k * p.ldQ;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
         i += (long long)gridDim.x * blockDim.x) {
        double2 x = p.v[i];
        double2 q = make_double2(x.x / nv, x.y / nv);
        qk[i] = q;
        float hr = __double2float_rn(q.x), hm = __double2float_rn(q.y);
        p.qh[i] = make_float2(hr, hm);
        p.ql[i] = make_float2(__double2float_rn(q.x - (double)hr), __double2float_rn(q.y - (double)hm));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.pivots[k] = jglobal;
        if (p.rdiag) p.rdiag[k] = nv;
        if (p.passes_out) p.passes_out[k] = st->passes;
        if (jlocal >= 0) p.picked[jlocal] = 1;
    }
}

}  // namespace rbk

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

rb_status shard_fail(rb_shard *sh, rb_status s, const char *msg) {
    if (sh && sh->ctx) return rbk::ctx_fail(sh->ctx, s, msg);
    return s;
}

rb_status cuda_fail(rb_shard *sh, cudaError_t e, const char *what) {
    char m[256];
    snprintf(m, sizeof(m), "rb_shard: %s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return shard_fail(sh, RB_ECUDA, m);
}

#define SH_CK(call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(sh, e_, what); \
    } while (0)

// Reads the device state; the local candidate as a global index (-1: none).
rb_status read_best(rb_shard *sh, double *best_err, long long *best_idx) {
    cudaStream_t sm = rbk::ctx_stream(sh->ctx);
    SH_CK(cudaMemcpyAsync(sh->st_host, sh->p.st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm), "state copy");
    SH_CK(cudaStreamSynchronize(sm), "stream sync");
    const rbk::DevState &h = *sh->st_host;
    if (h.nonfinite) sh->status = RB_ENONFINITE;
    else if (h.status < 0) sh->status = h.status;
    const bool none = h.J == rbk::kNoIdx;
    if (best_err) *best_err = none ? -INFINITY : h.errJ;
    if (best_idx) *best_idx = none ? -1 : sh->col0 + h.J;
    return (rb_status)sh->status;
}

}  // namespace

extern "C" {

rb_status rb_shard_create(rb_ctx *ctx, const void *S, long long N, long long M, long long ldS, long long col0,
                          int kmax, rb_result *out, rb_shard **sh_out) {
    if (!ctx || !sh_out) return RB_EINVAL;
    *sh_out = nullptr;
    if (!S || !out || !out->Q || !out->pivots || N < 1 || M < 1 || ldS < N || col0 < 0 || kmax < 0 ||
        out->ldQ < N || (out->C && out->ldC < M))
        return rbk::ctx_fail(ctx, RB_EINVAL, "rb_shard_create: bad arguments");
    if ((reinterpret_cast<uintptr_t>(S) % 16) || (reinterpret_cast<uintptr_t>(out->Q) % 16) ||
        (out->C && (reinterpret_cast<uintptr_t>(out->C) % 16)))
        return rbk::ctx_fail(ctx, RB_EINVAL, "rb_shard_create: complex128 arrays must be 16-byte aligned");
    rb_shard *sh = new (std::nothrow) rb_shard();
    if (!sh) return RB_ENOMEM;
    sh->ctx = ctx;
    sh->col0 = col0;
    const rb_options &o = rbk::ctx_options(ctx);
    cudaError_t e = cudaSetDevice(rbk::ctx_device(ctx));
    if (e != cudaSuccess) {
        delete sh;
        return rbk::ctx_fail(ctx, RB_ECUDA, "rb_shard_create: cudaSetDevice failed");
    }
    const int G = rbk::ctx_sweep_grid(ctx, RB_SWEEP_DF32);
    const long long ldH = (long long)align_up((size_t)N, 64);
    const int chunk = 2048;
    const int nchunk = (int)((N + chunk - 1) / chunk);
    const int gN = (int)((N + rbk::kThreads - 1) / rbk::kThreads);
    const int kcap = kmax > 0 ? kmax : 1;
    sh->kcap = kcap;
    sh->G = G;
    sh->period = out->C ? o.recompute_period : 0;  // the recompute reads the shard's rows of C
    // workspace layout
    size_t off = 0;
    auto add = [&](size_t bytes) {
        size_t a = align_up(off, 512);
        off = a + bytes;
        return a;
    };
    const size_t o_hi = add((size_t)M * ldH * sizeof(float2)), o_lo = add((size_t)M * ldH * sizeof(float2));
    const size_t o_norm = add((size_t)M * 8), o_acc = add((size_t)M * 8), o_pick = add((size_t)M);
    const size_t o_qh = add((size_t)(N + 2) * sizeof(float2)), o_ql = add((size_t)(N + 2) * sizeof(float2));
    const size_t o_v = add((size_t)N * sizeof(double2));
    const size_t o_hp = add((size_t)kcap * nchunk * sizeof(double2));
    const size_t np = (size_t)(G > gN ? G : gN);
    const size_t o_np = add(np * 8), o_be = add((size_t)G * 8), o_bi = add((size_t)G * 8);
    const size_t o_st = add(sizeof(rbk::DevState));
    const size_t o_ec = add((size_t)(kcap + 1) * 8);
    e = cudaMalloc(&sh->ws, off);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sh->st_host, sizeof(rbk::DevState));
    if (e != cudaSuccess) {
        cudaGetLastError();
        rb_shard_destroy(sh);
        return rbk::ctx_fail(ctx, RB_ENOMEM, "rb_shard_create: device workspace could not be allocated");
    }
    char *w = (char *)sh->ws;
    rbk::Prob &p = sh->p;
    p.N = N;
    p.M = M;
    p.ldS = ldS;
    p.ldH = ldH;
    p.ldQ = out->ldQ;
    p.ldC = out->ldC;
    // the caller applies the stopping rule; the shard's kernels never stop on
    // their own (tolerance below every error, no size limits)
    p.minNM = 1LL << 62;
    p.kmax = 1 << 30;
    p.tol = -1.0;
    p.max_passes = o.imgs_max_passes;
    p.nchunk = nchunk;
    p.chunk = chunk;
    p.kappa2 = o.imgs_kappa * o.imgs_kappa;
    p.S = (const double2 *)S;
    p.hi = (const float2 *)(w + o_hi);
    p.lo = (const float2 *)(w + o_lo);
    p.Q = (double2 *)out->Q;
    p.pivots = out->pivots;
    p.err_curve = (double *)(w + o_ec);  // local candidates' errors (the caller keeps the global curve)
    p.C = (double2 *)out->C;
    p.rdiag = out->rdiag;
    p.norm2 = (double *)(w + o_norm);
    p.acc = (double *)(w + o_acc);
    p.picked = (unsigned char *)(w + o_pick);
    p.qh = (float2 *)(w + o_qh);
    p.ql = (float2 *)(w + o_ql);
    p.qs_stride = 0;
    p.v = (double2 *)(w + o_v);
    p.hpart = (double2 *)(w + o_hp);
    p.npart = (double *)(w + o_np);
    p.bpart_err = (double *)(w + o_be);
    p.bpart_idx = (long long *)(w + o_bi);
    p.st = (rbk::DevState *)(w + o_st);
    *sh_out = sh;
    return RB_OK;
}

void rb_shard_destroy(rb_shard *sh) {
    if (!sh) return;
    if (sh->ws) {
        cudaStreamSynchronize(rbk::ctx_stream(sh->ctx));
        cudaFree(sh->ws);
    }
    if (sh->st_host) cudaFreeHost(sh->st_host);
    delete sh;
}

rb_status rb_shard_init(rb_shard *sh, double *best_err, long long *best_idx) {
    if (!sh) return RB_EINVAL;
    rbk::Prob &p = sh->p;
    cudaStream_t sm = rbk::ctx_stream(sh->ctx);
    SH_CK(cudaSetDevice(rbk::ctx_device(sh->ctx)), "cudaSetDevice");
    SH_CK(cudaMemsetAsync(p.st, 0, sizeof(rbk::DevState), sm), "memset state");
    SH_CK(rbk::launch_split(p.S, p.N, p.M, p.ldS, (float2 *)p.hi, (float2 *)p.lo, p.ldH, p.norm2, sm), "split");
    SH_CK(rbk::launch_init(p, sh->G, sm), "init");
    sh->k = 0;
    sh->status = RB_OK;
    sh->rank_end = false;
    return read_best(sh, best_err, best_idx);
}

rb_status rb_shard_column(rb_shard *sh, long long j, void *dst, double *norm2) {
    if (!sh || !dst) return RB_EINVAL;
    const long long jl = j - sh->col0;
    if (jl < 0 || jl >= sh->p.M) return shard_fail(sh, RB_EINVAL, "rb_shard_column: column not owned by this shard");
    cudaStream_t sm = rbk::ctx_stream(sh->ctx);
    SH_CK(cudaSetDevice(rbk::ctx_device(sh->ctx)), "cudaSetDevice");
    SH_CK(cudaMemcpyAsync(dst, sh->p.S + jl * sh->p.ldS, (size_t)sh->p.N * sizeof(double2), cudaMemcpyDeviceToDevice,
                          sm),
          "column copy");
    if (norm2) {
        SH_CK(cudaMemcpyAsync(norm2, sh->p.norm2 + jl, sizeof(double), cudaMemcpyDeviceToHost, sm), "norm copy");
        SH_CK(cudaStreamSynchronize(sm), "stream sync");
    } else {
        // the norm into dst[N] (real part, imaginary part zero), on the device
        double2 *d = (double2 *)dst + sh->p.N;
        SH_CK(cudaMemcpyAsync(d, sh->p.norm2 + jl, sizeof(double), cudaMemcpyDeviceToDevice, sm), "norm copy");
        SH_CK(cudaMemsetAsync((double *)d + 1, 0, sizeof(double), sm), "norm copy");
    }
    return RB_OK;
}

rb_status rb_shard_append(rb_shard *sh, const void *v, double vnorm2, long long j, double *best_err,
                          long long *best_idx, int *appended) {
    if (!sh || !v || std::isnan(vnorm2) || j < 0)
        return sh ? shard_fail(sh, RB_EINVAL, "rb_shard_append: bad arguments") : RB_EINVAL;
    if (appended) *appended = 0;
    if (sh->status < 0) return shard_fail(sh, (rb_status)sh->status, "rb_shard_append: the shard has failed");
    if (sh->rank_end) return shard_fail(sh, RB_ESTATE, "rb_shard_append: the basis is already complete");
    if (sh->k >= sh->kcap) return shard_fail(sh, RB_EINVAL, "rb_shard_append: kmax vectors already built");
    if (reinterpret_cast<uintptr_t>(v) % 16) return shard_fail(sh, RB_EINVAL, "rb_shard_append: v must be 16-byte aligned");
    rbk::Prob &p = sh->p;
    cudaStream_t sm = rbk::ctx_stream(sh->ctx);
    SH_CK(cudaSetDevice(rbk::ctx_device(sh->ctx)), "cudaSetDevice");
    const long long jl = j - sh->col0;
    const long long jlocal = (jl >= 0 && jl < p.M) ? jl : -1;
    const int gN = (int)((p.N + rbk::kThreads - 1) / rbk::kThreads);
    const int gcopy = gN < sh->G ? gN : sh->G;
    rbk::k_shard_begin<<<gcopy, rbk::kThreads, 0, sm>>>(p, (const double2 *)v, vnorm2);
    SH_CK(cudaGetLastError(), "shard begin");
    SH_CK(rbk::launch_imgs_passes(p, sh->G, sm, nullptr), "imgs");
    rbk::k_shard_finalize<<<gcopy, rbk::kThreads, 0, sm>>>(p, j, jlocal);
    SH_CK(cudaGetLastError(), "shard finalize");
    if (sh->period > 0) SH_CK(rbk::launch_recompute(p, sh->period, sh->G, sm), "recompute");
    SH_CK(rbk::launch_sweep(p, RB_SWEEP_DF32, sh->G, sm), "sweep");
    SH_CK(cudaMemcpyAsync(sh->st_host, p.st, sizeof(rbk::DevState), cudaMemcpyDeviceToHost, sm), "state copy");
    SH_CK(cudaStreamSynchronize(sm), "stream sync");
    const rbk::DevState &h = *sh->st_host;
    if (h.status == RB_EORTHO) {
        sh->status = RB_EORTHO;
        return shard_fail(sh, RB_EORTHO, "rb_shard_append: IMGS did not pass the kappa test within imgs_max_passes");
    }
    if (h.force_stop) {  // exact rank: nothing appended
        sh->rank_end = true;
        if (best_err) *best_err = -INFINITY;
        if (best_idx) *best_idx = -1;
        return RB_OK;
    }
    sh->k += 1;
    if (appended) *appended = 1;
    return read_best(sh, best_err, best_idx);
}

rb_status rb_shard_finish(rb_shard *sh, double *final_err, int *k) {
    if (!sh) return RB_EINVAL;
    cudaStream_t sm = rbk::ctx_stream(sh->ctx);
    SH_CK(cudaSetDevice(rbk::ctx_device(sh->ctx)), "cudaSetDevice");
    if (final_err) {
        SH_CK(rbk::launch_final_err(sh->p, final_err, sm), "final_err");
        SH_CK(cudaStreamSynchronize(sm), "stream sync");
    }
    if (k) *k = sh->k;
    return (rb_status)(sh->status < 0 ? sh->status : RB_OK);
}

}  // extern "C"
