// rb_sweep.cu -- the fused pivot-search sweep of RB-greedy (Alg. 3 with the
// bookkeeping of Eq. (Residual), Sec. 6.1.2).
//
// One launch streams all of S once: for every column j it forms
// c_kj = q_k^H s_j, stores C[k, j], updates acc_j += |c_kj|^2 in FP64,
// err_j = ||s_j||^2 - acc_j, and folds (err_j, j) into a warp -> block ->
// grid argmax over unpicked columns (ties to the lowest index).  The last
// block to finish reduces the per-block partials, appends err_curve[k+1],
// publishes the next pivot and applies the stopping rule.
//
// Work split: one warp owns a whole column at a time (lanes stride over
// rows with 128-bit loads, warp-shuffle reduction at the end), so no
// shared-memory traffic or __syncthreads sits inside the streaming loop.
#include "rb_internal.cuh"

namespace rbk {

enum { SWEEP_DF32 = 0, SWEEP_FP64 = 1 };

// Column dot product c = q^H s_j in plain FP64 straight from complex128.
__device__ __forceinline__ double2 col_dot_fp64(const double2 *__restrict__ s, const double2 *__restrict__ q,
                                                long long N, int lane) {
    double re = 0.0, im = 0.0;
    long long i = lane;
    constexpr int U = 4;
    for (; i + 32 * (U - 1) < N; i += 32 * U) {
        double2 a[U];
#pragma unroll
        for (int u = 0; u < U; u++) a[u] = ld_stream_d2(s + i + 32 * u);
#pragma unroll
        for (int u = 0; u < U; u++) {
            double2 b = __ldg(q + i + 32 * u);
            re = fma(b.x, a[u].x, fma(b.y, a[u].y, re));
            im = fma(b.x, a[u].y, fma(-b.y, a[u].x, im));
        }
    }
    for (; i < N; i += 32) {
        double2 a = ld_stream_d2(s + i), b = __ldg(q + i);
        re = fma(b.x, a.x, fma(b.y, a.y, re));
        im = fma(b.x, a.y, fma(-b.y, a.x, im));
    }
    return make_double2(warp_sum(re), warp_sum(im));
}

template <int VARIANT>
__global__ void __launch_bounds__(kThreads) k_sweep(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    if (p.qs_stride && (ld_volatile(&st->phase) == 0 || ld_volatile(&st->switch_pending))) return;  // split form before the switch
    const int k = st->k;  // row of C written by this sweep; q_k is the newest vector
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    double be = -INFINITY;
    long long bi = kNoIdx;
    const double2 *qk = p.Q + (long long)k * p.ldQ;
    for (long long j = gw; j < p.M; j += nw) {
        double2 c;
        if (VARIANT == SWEEP_DF32)
            c = col_dot_df32<4>(p.hi + j * p.ldH, p.lo + j * p.ldH, p.qh + (long long)k * p.qs_stride,
                             p.ql + (long long)k * p.qs_stride, p.N, lane);
        else
            c = col_dot_fp64(p.S + j * p.ldS, qk, p.N, lane);
        if (lane == 0) {
            if (p.C) p.C[(long long)k * p.ldC + j] = c;
            double a = acc_add(p.acc[j], c);
            p.acc[j] = a;
            double e = p.norm2[j] - a;
            if (!p.picked[j] && better(e, j, be, bi)) { be = e; bi = j; }
        }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = be;
        p.bpart_idx[blockIdx.x] = bi;
    }
    if (!last_block(&st->ticket_sweep)) return;
    be = -INFINITY;
    bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double e = __ldcg(p.bpart_err + b);
        long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_sweep = 0;
        if (p.qs_stride) st->n_sweeps_hl += 1;
        sweep_publish(p, st, k, be, bi);
    }
}

int sweep_grid(int variant, int device) {
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (variant == SWEEP_DF32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<SWEEP_DF32>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<SWEEP_FP64>, kThreads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

// Periodic exact recompute of the bookkeeping: before the sweep of iteration
// k (k a positive multiple of `period`), acc_j = sum_{l<k} |C[l, j]|^2 is
// rebuilt from the stored coefficients with error-free products (FMA) and a
// compensated (TwoSum) running sum, replacing the k rounded updates of Eq.
// (Residual)'s running sum by one sum accurate to about one unit in the last
// place.  In exact arithmetic nothing changes.
__global__ void __launch_bounds__(kThreads) k_recompute(Prob p, int period) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    const int k = st->k;
    if (k == 0 || k % period != 0) return;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x)
        p.acc[j] = acc_recompute(p.C, p.ldC, j, k);
}

cudaError_t launch_recompute(const Prob &p, int period, int grid, cudaStream_t s) {
    long long g = (p.M + kThreads - 1) / kThreads;
    if (g > grid) g = grid;
    k_recompute<<<(int)g, kThreads, 0, s>>>(p, period);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const Prob &p, int variant, int grid, cudaStream_t s) {
    if (variant == SWEEP_DF32)
        k_sweep<SWEEP_DF32><<<grid, kThreads, 0, s>>>(p);
    else
        k_sweep<SWEEP_FP64><<<grid, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace rbk
