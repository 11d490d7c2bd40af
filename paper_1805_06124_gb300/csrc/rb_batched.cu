// rb_batched.cu -- many independent greedy problems of uneven N and M.
//
// The sweep of every active problem runs in ONE persistent launch: the
// column ranges of all problems are cut into chunks of CW columns, the chunks
// are numbered across problems (prefix sums), and each block takes chunks in
// a grid-stride loop, finds their problem by binary search, and streams the
// columns warp by warp.  When a hi/lo copy of the batch fits in free device
// memory the sweep streams it (16 bytes per element, as the FP64 form);
// otherwise it reads complex128 and splits each element into hi/lo FP32 pairs
// in registers (integer round-to-nearest split), needing no copy.  Either way
// the dot products are the FP64 form's double-float arithmetic.  Per-chunk argmax partials are reduced per
// problem by a second small kernel, which also applies each problem's own
// stopping rule; stopped problems' chunks return at once.
//
// The tunables -- loads in flight per lane (U), threads per block and
// columns per chunk (CW) -- are picked by timing every variant on a dry sweep
// of the batch itself (see rb_api.cu).
#include "rb_internal.cuh"

namespace rbk {

__device__ __forceinline__ int find_problem(const long long *prefix, int nprob, long long x) {
    int lo = 0, hi = nprob;  // prefix[lo] <= x < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// c = q^H s with s read as complex128 and split on the fly; pairs of elements
// per lane step (two 16-byte loads of s, one 16-byte load each of q's hi/lo).
template <int U>
__device__ __forceinline__ double2 col_dot_c128(const double2 *__restrict__ s, const float2 *__restrict__ qh,
                                                const float2 *__restrict__ ql, long long N, int lane) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4 *qh4 = reinterpret_cast<const float4 *>(qh);
    const float4 *ql4 = reinterpret_cast<const float4 *>(ql);
    const long long n2 = N >> 1;
    long long t = lane;
    for (; t + 32 * (U - 1) < n2; t += 32 * U) {
        double2 a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            a[u] = ld_stream_d2(s + 2 * (t + 32 * u));
            b[u] = ld_stream_d2(s + 2 * (t + 32 * u) + 1);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            float4 qa = __ldg(qh4 + t + 32 * u), qb = __ldg(ql4 + t + 32 * u);
            float h0, l0, h1, l1, h2, l2, h3, l3;
            split_rn(a[u].x, h0, l0);
            split_rn(a[u].y, h1, l1);
            split_rn(b[u].x, h2, l2);
            split_rn(b[u].y, h3, l3);
            df_mac(rh, rl, qa.x, qb.x, h0, l0);
            df_mac(rh, rl, qa.y, qb.y, h1, l1);
            df_mac(ih, il, qa.x, qb.x, h1, l1);
            df_mac(ih, il, -qa.y, -qb.y, h0, l0);
            df_mac(rh, rl, qa.z, qb.z, h2, l2);
            df_mac(rh, rl, qa.w, qb.w, h3, l3);
            df_mac(ih, il, qa.z, qb.z, h3, l3);
            df_mac(ih, il, -qa.w, -qb.w, h2, l2);
        }
    }
    for (; t < n2; t += 32) {
        double2 a = ld_stream_d2(s + 2 * t), b = ld_stream_d2(s + 2 * t + 1);
        float4 qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        float h0, l0, h1, l1, h2, l2, h3, l3;
        split_rn(a.x, h0, l0);
        split_rn(a.y, h1, l1);
        split_rn(b.x, h2, l2);
        split_rn(b.y, h3, l3);
        df_mac(rh, rl, qa.x, qb.x, h0, l0);
        df_mac(rh, rl, qa.y, qb.y, h1, l1);
        df_mac(ih, il, qa.x, qb.x, h1, l1);
        df_mac(ih, il, -qa.y, -qb.y, h0, l0);
        df_mac(rh, rl, qa.z, qb.z, h2, l2);
        df_mac(rh, rl, qa.w, qb.w, h3, l3);
        df_mac(ih, il, qa.z, qb.z, h3, l3);
        df_mac(ih, il, -qa.w, -qb.w, h2, l2);
    }
    if ((N & 1) && lane == 0) {
        long long i = N - 1;
        double2 a = s[i];
        float2 qa = qh[i], qb = ql[i];
        float h0, l0, h1, l1;
        split_rn(a.x, h0, l0);
        split_rn(a.y, h1, l1);
        df_mac(rh, rl, qa.x, qb.x, h0, l0);
        df_mac(rh, rl, qa.y, qb.y, h1, l1);
        df_mac(ih, il, qa.x, qb.x, h1, l1);
        df_mac(ih, il, -qa.y, -qb.y, h0, l0);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

// ||hi + lo||^2 of every column of every problem, hi/lo the same split the
// sweep forms in registers (so the bookkeeping is self-consistent).
__global__ void __launch_bounds__(kThreads) k_bnorms(const BProb *__restrict__ P, int nprob,
                                                     const long long *__restrict__ col0) {
    const int lane = threadIdx.x & 31;
    const long long total = col0[nprob];
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < total;
         g += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int b = find_problem(col0, nprob, g);
        const BProb &pr = P[b];
        const long long j = g - col0[b];
        const double2 *s = pr.S + j * pr.ldS;
        float nh = 0.f, nl = 0.f;
        for (long long i = lane; i < pr.N; i += 32) {
            double2 x = ld_stream_d2(s + i);
            float h0, l0, h1, l1;
            split_rn(x.x, h0, l0);
            split_rn(x.y, h1, l1);
            df_sq(nh, nl, h0, l0);
            df_sq(nh, nl, h1, l1);
        }
        double n2 = warp_sum((double)nh + (double)nl);
        if (lane == 0) pr.norm2[j] = n2;
    }
}

// The pre-split variants are held to 64 registers (32 warps per SM, as the
// single-problem sweep) so that enough loads are in flight per SM.
template <int U, int THREADS, bool SPLIT>
__global__ void __launch_bounds__(THREADS, SPLIT ? 1024 / THREADS : 1) k_bsweep(const BProb *__restrict__ P, int nprob,
                                                    const long long *__restrict__ chunk0, int CW,
                                                    double *__restrict__ part_err, long long *__restrict__ part_idx,
                                                    int dry) {
    __shared__ int s_b, s_skip, s_k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = THREADS / 32;
    const long long total = chunk0[nprob];
    for (long long ch = blockIdx.x; ch < total; ch += gridDim.x) {
        if (threadIdx.x == 0) {
            int b = find_problem(chunk0, nprob, ch);
            s_b = b;
            s_skip = dry ? 0 : ld_volatile(&P[b].st->stop);
            s_k = P[b].st->k;
        }
        __syncthreads();
        const int b = s_b;
        if (!s_skip) {
            const BProb &pr = P[b];
            const int k = s_k;
            const long long j0 = (ch - chunk0[b]) * CW;
            const long long j1 = j0 + CW < pr.M ? j0 + CW : pr.M;
            double be = -INFINITY;
            long long bi = kNoIdx;
            for (long long j = j0 + warp; j < j1; j += NW) {
                double2 c = SPLIT ? col_dot_df32<U>(pr.hi + j * pr.ldH, pr.lo + j * pr.ldH, pr.qh, pr.ql, pr.N, lane)
                                  : col_dot_c128<U>(pr.S + j * pr.ldS, pr.qh, pr.ql, pr.N, lane);
                if (lane == 0) {
                    if (dry) {
                        if (better(c.x, j, be, bi)) { be = c.x; bi = j; }
                    } else {
                        if (pr.C) pr.C[(long long)k * pr.ldC + j] = c;
                        double a = pr.acc[j] + (c.x * c.x + c.y * c.y);
                        pr.acc[j] = a;
                        double e = pr.norm2[j] - a;
                        if (!pr.picked[j] && better(e, j, be, bi)) { be = e; bi = j; }
                    }
                }
            }
            block_best(be, bi);
            if (threadIdx.x == 0) {
                part_err[ch] = be;
                part_idx[ch] = bi;
            }
        }
        __syncthreads();
    }
}

// Per problem: reduce its chunk partials, append err_curve[k+1], next pivot,
// stopping rule.  One block per problem.
__global__ void __launch_bounds__(kThreads) k_breduce(const BProb *__restrict__ P, int nprob,
                                                      const long long *__restrict__ chunk0,
                                                      const double *__restrict__ part_err,
                                                      const long long *__restrict__ part_idx) {
    const BProb &pr = P[blockIdx.x];
    DevState *st = pr.st;
    if (ld_volatile(&st->stop)) return;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long c = chunk0[blockIdx.x] + threadIdx.x; c < chunk0[blockIdx.x + 1]; c += blockDim.x) {
        double e = part_err[c];
        long long i = part_idx[c];
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        const int k1 = st->k + 1;
        st->k = k1;
        st->n_sweeps += 1;
        double emax = bi == kNoIdx ? 0.0 : be;
        pr.err_curve[k1] = emax;
        st->J = bi;
        st->errJ = emax;
        if (bi == kNoIdx || emax < pr.tol) {
            st->status = RB_OK;
            st->stop = 1;
        } else if (k1 >= pr.kmax) {
            st->status = RB_KMAX_REACHED;
            st->stop = 1;
        } else if (k1 >= pr.minNM) {
            st->status = RB_OK;
            st->stop = 1;
        }
    }
}

cudaError_t launch_bnorms(const BProb *P, int nprob, const long long *col0, long long total_cols, cudaStream_t s) {
    long long g = (total_cols * 32 + kThreads - 1) / kThreads;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    k_bnorms<<<(int)g, kThreads, 0, s>>>(P, nprob, col0);
    return cudaGetLastError();
}

// variant index v: U = {2, 4, 8}[v % 3], THREADS = {128, 256}[(v / 3) % 2],
// v >= 6: the sweep reads a pre-split hi/lo copy instead of complex128.
#define RB_BSWEEP_CASES(X)                                                                             \
    X(0, 2, 128, false) X(1, 4, 128, false) X(2, 8, 128, false) X(3, 2, 256, false) X(4, 4, 256, false) \
    X(5, 8, 256, false) X(6, 2, 128, true) X(7, 4, 128, true) X(8, 8, 128, true) X(9, 2, 256, true)     \
    X(10, 4, 256, true) X(11, 8, 256, true)

static void *bsweep_fn(int v) {
#define RB_FN(i, u, t, sp) \
    if (v == i) return (void *)k_bsweep<u, t, sp>;
    RB_BSWEEP_CASES(RB_FN)
#undef RB_FN
    return (void *)k_bsweep<4, 256, false>;
}

int bsweep_threads(int v) { return (v / 3) % 2 ? 256 : 128; }

int bsweep_grid(int v, int device) {
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bsweep_fn(v), bsweep_threads(v), 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_bsweep(int v, int grid, const BProb *P, int nprob, const long long *chunk0, int CW,
                          double *part_err, long long *part_idx, int dry, cudaStream_t s) {
#define RB_LAUNCH(i, u, t, sp) \
    if (v == i) k_bsweep<u, t, sp><<<grid, t, 0, s>>>(P, nprob, chunk0, CW, part_err, part_idx, dry);
    RB_BSWEEP_CASES(RB_LAUNCH)
#undef RB_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_breduce(const BProb *P, int nprob, const long long *chunk0, const double *part_err,
                           const long long *part_idx, cudaStream_t s) {
    k_breduce<<<nprob, kThreads, 0, s>>>(P, nprob, chunk0, part_err, part_idx);
    return cudaGetLastError();
}

}  // namespace rbk
