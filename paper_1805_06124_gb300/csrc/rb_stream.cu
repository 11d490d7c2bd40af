// rb_stream.cu -- the FP64-form greedy (Alg. 3 with the Eq. (Residual)
// bookkeeping) on a snapshot matrix that stays in host memory.
//
// The paper's largest runs hold S of about half a terabyte (Sec. 1, Sec. 6),
// more than one GPU's HBM.  Here the hi/lo split copy of the leading
// `resident` columns lives on the device and every other column is read from
// host memory (mapped, over the host link) in chunks of `cols` columns (one
// column by default: the finest bounds, the fewest reads).
//
// Lazy chunk updates.  A chunk keeps `last` (the first basis vector it has
// not seen) and `bound` (the largest error of its unpicked columns when it
// was last brought up to date).  The errors err_j = ||s_j||^2 - acc_j never
// grow in exact arithmetic, and in floating point by at most
// (k + 16) 2^-51 max_j ||s_j||^2 across a periodic recompute (the running sum
// only adds non-negative terms, so between recomputes they do not grow at
// all).  A chunk whose bound plus that margin is below the best error known
// in this iteration cannot hold the pivot and is skipped; when it is next
// read, it applies every pending basis vector in order, with the same
// arithmetic as the in-core sweep (the same hi/lo split, double-float dot
// product, running sum and recompute).  The pivots, C, the errors and the
// basis are therefore bit-identical to those of the in-core form.
//
// One iteration: the resident sweep gives the best resident error R; round A
// brings up to date every stale chunk whose bound reaches
// max(R, gamma * largest bound); round B every remaining chunk whose bound
// reaches the best error after round A (gamma only steers the work, never
// the result).  After the loop a flush applies the vectors each chunk has
// not seen, so C and the errors are complete.
#include "rb_internal.cuh"

namespace rbk {

enum { ST_ROUND_A = 0, ST_ROUND_B = 1, ST_FLUSH = 2 };

__device__ __forceinline__ double stream_margin(int k, double nmax) { return (double)(k + 16) * 0x1p-51 * nmax; }

// Resident sweep: the in-core DF32 sweep over columns 0..Mr-1, ending with
// the best (err, idx) in the state instead of a published pivot.
__global__ void __launch_bounds__(kThreads) k_str_resident(Prob p, StreamPart sp) {
    const long long Mr = sp.Mr;
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    const int k = st->k;
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float2 *qh = p.qh + (long long)k * p.qs_stride, *ql = p.ql + (long long)k * p.qs_stride;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long j = gw; j < Mr; j += nw) {
        const double2 c = col_dot_df32<4>(p.hi + j * p.ldH, p.lo + j * p.ldH, qh, ql, p.N, lane);
        if (lane == 0) {
            if (p.C) p.C[(long long)k * p.ldC + j] = c;
            const double a = acc_add(p.acc[j], c);
            p.acc[j] = a;
            const double e = p.norm2[j] - a;
            if (!p.picked[j] && better(e, j, be, bi)) { be = e; bi = j; }
        }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = be;
        p.bpart_idx[blockIdx.x] = bi;
    }
    if (!last_block(&st->ticket_host)) return;
    be = -INFINITY;
    bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const double e = __ldcg(p.bpart_err + b);
        const long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_host = 0;
        st->hbest_err = be;
        st->hbest_idx = bi;
        if (sp.cnt) {
            sp.cnt[0] = 0;
            sp.cnt[1] = 0;
        }
    }
}

// Largest stale bound (plus margin) over the chunks not yet brought up to
// this iteration (grid; the last block stores it in the state).
__global__ void __launch_bounds__(kThreads) k_str_maxub(Prob p, StreamPart sp) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    const int k = st->k;
    double mx = -INFINITY;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < sp.nch; c += gridDim.x * blockDim.x)
        if (sp.last[c] <= k && sp.bound[c] > -INFINITY) mx = fmax(mx, sp.bound[c] + stream_margin(k, sp.nmax[c]));
    long long dummy = 0;
    block_best(mx, dummy);
    if (threadIdx.x == 0) sp.part[blockIdx.x] = mx;
    if (!last_block(&st->ticket_sel)) return;
    mx = -INFINITY;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) mx = fmax(mx, __ldcg(sp.part + b));
    block_best(mx, dummy);
    if (threadIdx.x == 0) {
        st->ticket_sel = 0;
        st->sel_max = mx;
    }
}

// Chunk selection (grid).  Round A: stale chunks with bound + margin >=
// max(R, gamma * largest such value); round B: stale chunks with bound +
// margin >= the best error so far; flush: every chunk that has not seen all
// basis vectors.  List order does not matter: every chunk's result and the
// (err, idx) order are independent of it.
__global__ void __launch_bounds__(kThreads) k_str_select(Prob p, StreamPart sp, int mode) {
    DevState *st = p.st;
    const int k = st->k;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    if (mode == ST_FLUSH) {
        for (int c = g0; c < sp.nch; c += gs)
            if (sp.last[c] < k) sp.list[atomicAdd(sp.cnt + 2, 1)] = c;
        return;
    }
    if (ld_volatile(&st->stop)) return;
    double th = st->hbest_idx == kNoIdx ? -INFINITY : st->hbest_err;
    if (mode == ST_ROUND_A) {
        const double mx = st->sel_max;
        if (mx > 0.0) th = fmax(th, sp.gamma * mx);
    }
    for (int c = g0; c < sp.nch; c += gs)
        if (sp.last[c] <= k && sp.bound[c] > -INFINITY && sp.bound[c] + stream_margin(k, sp.nmax[c]) >= th)
            sp.list[atomicAdd(sp.cnt + mode, 1)] = c;
}

// c = q^H s_j from the complex128 column in host memory, split on the fly
// exactly as the split kernel stores it, in the per-lane order of
// col_dot_df32 (pair t = lane, lane + 32, ..., two elements per pair, then
// the odd last element on lane 0).  With hs != null the split is also kept.
__device__ __forceinline__ double2 dot_from_host(const double2 *__restrict__ s, const float2 *__restrict__ qh,
                                                 const float2 *__restrict__ ql, long long N, int lane, float2 *hs,
                                                 float2 *ls) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const long long n2 = N >> 1;
    const float4 *qh4 = reinterpret_cast<const float4 *>(qh);
    const float4 *ql4 = reinterpret_cast<const float4 *>(ql);
    float4 *hs4 = reinterpret_cast<float4 *>(hs);
    float4 *ls4 = reinterpret_cast<float4 *>(ls);
    constexpr int U = 4;
    for (long long t0 = lane; t0 < n2; t0 += 32 * U) {
        double2 x[2 * U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long t = t0 + 32 * u;
            if (t < n2) {
                x[2 * u] = __ldcs(s + 2 * t);
                x[2 * u + 1] = __ldcs(s + 2 * t + 1);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const long long t = t0 + 32 * u;
            if (t >= n2) break;
            float2 h0, l0, h1, l1;
            split_c(x[2 * u], h0, l0);
            split_c(x[2 * u + 1], h1, l1);
            if (hs) {
                hs4[t] = make_float4(h0.x, h0.y, h1.x, h1.y);
                ls4[t] = make_float4(l0.x, l0.y, l1.x, l1.y);
            }
            const float4 qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
            df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, h0.x, h0.y, l0.x, l0.y);
            df_cmac(rh, rl, ih, il, qa.z, qa.w, qb.z, qb.w, h1.x, h1.y, l1.x, l1.y);
        }
    }
    if ((N & 1) && lane == 0) {
        const long long i = N - 1;
        float2 h, l;
        split_c(__ldcs(s + i), h, l);
        if (hs) {
            hs[i] = h;
            ls[i] = l;
        }
        const float2 qa = qh[i], qb = ql[i];
        df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, h.x, h.y, l.x, l.y);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

// The same product from the staged split (written earlier by this thread:
// plain coherent loads, not the read-only path).
__device__ __forceinline__ double2 dot_from_stage(const float2 *hs, const float2 *ls, const float2 *__restrict__ qh,
                                                  const float2 *__restrict__ ql, long long N, int lane) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const long long n2 = N >> 1;
    const float4 *h4 = reinterpret_cast<const float4 *>(hs);
    const float4 *l4 = reinterpret_cast<const float4 *>(ls);
    const float4 *qh4 = reinterpret_cast<const float4 *>(qh);
    const float4 *ql4 = reinterpret_cast<const float4 *>(ql);
    for (long long t = lane; t < n2; t += 32) {
        const float4 a = __ldcg(h4 + t), b = __ldcg(l4 + t);
        const float4 qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, a.x, a.y, b.x, b.y);
        df_cmac(rh, rl, ih, il, qa.z, qa.w, qb.z, qb.w, a.z, a.w, b.z, b.w);
    }
    if ((N & 1) && lane == 0) {
        const long long i = N - 1;
        const float2 a = __ldcg(hs + i), b = __ldcg(ls + i), qa = qh[i], qb = ql[i];
        df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, a.x, a.y, b.x, b.y);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

// Brings the listed chunks up to date, one warp per chunk: for each column,
// every pending basis vector l = last..kend in order (recompute first where l
// is a positive multiple of the period, as the in-core loop does before its
// sweep l).  In rounds A and B the best (err, idx) is merged into the state;
// a flush only completes C and acc.
__global__ void __launch_bounds__(kThreads, 2) k_str_sweep(Prob p, StreamPart sp, int mode) {
    DevState *st = p.st;
    if (mode != ST_FLUSH && ld_volatile(&st->stop)) return;
    const int kend = mode == ST_FLUSH ? st->k - 1 : st->k;
    const int n = sp.cnt[mode];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int gwarp = blockIdx.x * nwarp + warp, twarps = gridDim.x * nwarp;
    float2 *hs = sp.stage + (long long)gwarp * 2 * sp.stage_ld;
    float2 *ls = hs + sp.stage_ld;
    double tbe = -INFINITY;  // lane 0: best over this warp's chunks
    long long tbi = kNoIdx;
    for (int e = gwarp; e < n; e += twarps) {
        const int c = sp.list[e];
        const int l0 = sp.last[c];
        const long long j0 = sp.Mr + (long long)c * sp.cols;
        long long j1 = j0 + sp.cols;
        if (j1 > p.M) j1 = p.M;
        double be = -INFINITY;
        long long bi = kNoIdx;
        for (long long j = j0; j < j1; j++) {
            double a = lane == 0 ? p.acc[j] : 0.0;
            for (int l = l0; l <= kend; l++) {
                if (lane == 0 && l > 0 && sp.period > 0 && l % sp.period == 0)
                    a = acc_recompute(p.C, p.ldC, j, l);
                const float2 *qh = p.qh + (long long)l * p.qs_stride, *ql = p.ql + (long long)l * p.qs_stride;
                const double2 c2 = l == l0 ? dot_from_host(sp.Sd + j * p.ldS, qh, ql, p.N, lane,
                                                           l < kend ? hs : nullptr, ls)
                                           : dot_from_stage(hs, ls, qh, ql, p.N, lane);
                if (lane == 0) {
                    if (p.C) p.C[(long long)l * p.ldC + j] = c2;
                    a = acc_add(a, c2);
                }
            }
            if (lane == 0) {
                p.acc[j] = a;
                const double err = p.norm2[j] - a;
                if (!p.picked[j] && better(err, j, be, bi)) { be = err; bi = j; }
            }
        }
        if (lane == 0) {
            sp.bound[c] = bi == kNoIdx ? -INFINITY : be;
            sp.last[c] = kend + 1;
            atomicAdd(sp.updates, 1ull);
            if (better(be, bi, tbe, tbi)) { tbe = be; tbi = bi; }
        }
    }
    if (mode == ST_FLUSH) return;
    if (lane != 0) {
        tbe = -INFINITY;
        tbi = kNoIdx;
    }
    block_best(tbe, tbi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = tbe;
        p.bpart_idx[blockIdx.x] = tbi;
    }
    if (!last_block(&st->ticket_host)) return;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const double e = __ldcg(p.bpart_err + b);
        const long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_host = 0;
        const double he = st->hbest_err;
        const long long hi = st->hbest_idx;
        if (better(be, bi, he, hi)) {
            st->hbest_err = be;
            st->hbest_idx = bi;
        }
    }
}

// The iteration's pivot from the merged best, as the in-core sweep's last block.
__global__ void k_str_publish(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    if (threadIdx.x == 0) sweep_publish(p, st, st->k, st->hbest_err, st->hbest_idx);
}

// Chunk state after the norms: nothing applied, bound = largest norm (the
// error with acc = 0), and the state flag that makes the IMGS kernels keep
// one FP32 basis slot per vector (as the split form's second phase does).
__global__ void __launch_bounds__(kThreads) k_str_init(Prob p, StreamPart sp) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((long long)gridDim.x * blockDim.x) >> 5);
    if (gw == 0 && lane == 0) {
        p.st->phase = 1;
        sp.cnt[0] = sp.cnt[1] = sp.cnt[2] = 0;
    }
    for (int c = gw; c < sp.nch; c += nw) {
        const long long j0 = sp.Mr + (long long)c * sp.cols;
        long long j1 = j0 + sp.cols;
        if (j1 > p.M) j1 = p.M;
        double mx = -INFINITY;
        for (long long j = j0 + lane; j < j1; j += 32) mx = fmax(mx, p.norm2[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            sp.last[c] = 0;
            sp.bound[c] = mx;
            sp.nmax[c] = mx;
        }
    }
}

int stream_sweep_grid(int device) {
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_str_sweep, kThreads, 0);
    if (per < 1) per = 1;
    if (per > 2) per = 2;
    return sms * per;
}

cudaError_t launch_stream_init(const Prob &p, const StreamPart &sp, cudaStream_t s) {
    int g = (int)((sp.nch + 7) / 8);
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    k_str_init<<<g, kThreads, 0, s>>>(p, sp);
    return cudaGetLastError();
}

int stream_select_grid(const StreamPart &sp) {
    long long g = ((long long)sp.nch + kThreads - 1) / kThreads;
    if (g > 1024) g = 1024;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_stream_iteration(const Prob &p, const StreamPart &sp, int res_grid, int str_grid,
                                    cudaStream_t s) {
    long long g = (sp.Mr * 32 + kThreads - 1) / kThreads;
    if (g > res_grid) g = res_grid;
    if (g < 1) g = 1;
    k_str_resident<<<(int)g, kThreads, 0, s>>>(p, sp);
    if (sp.nch > 0) {
        const int gs = stream_select_grid(sp);
        k_str_maxub<<<gs, kThreads, 0, s>>>(p, sp);
        k_str_select<<<gs, kThreads, 0, s>>>(p, sp, ST_ROUND_A);
        k_str_sweep<<<str_grid, kThreads, 0, s>>>(p, sp, ST_ROUND_A);
        k_str_select<<<gs, kThreads, 0, s>>>(p, sp, ST_ROUND_B);
        k_str_sweep<<<str_grid, kThreads, 0, s>>>(p, sp, ST_ROUND_B);
    }
    k_str_publish<<<1, 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_stream_flush(const Prob &p, const StreamPart &sp, int str_grid, cudaStream_t s) {
    if (sp.nch == 0) return cudaSuccess;
    k_str_select<<<stream_select_grid(sp), kThreads, 0, s>>>(p, sp, ST_FLUSH);
    k_str_sweep<<<str_grid, kThreads, 0, s>>>(p, sp, ST_FLUSH);
    return cudaGetLastError();
}

}  // namespace rbk
