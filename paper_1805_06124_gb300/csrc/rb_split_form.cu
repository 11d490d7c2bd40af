// rb_split_form.cu -- the split-precision form of the greedy sweep.
//
// S is stored as complex64 hi + lo (hi = fl32(s), lo = fl32(s - hi)).  Two
// phases, decided on the device:
//
// Phase 0 (hi only, 8 bytes per element).  The sweep forms c_hi = q^H hi with
// exact FP32 products (the FMA form of TwoProduct) summed in double-float, so
// the FP64 bookkeeping err_hi_j = ||hi_j||^2 - sum_l |c_hi,lj|^2 tracks the
// projection error of hi_j itself, not an estimate of it.  Because the
// orthogonal projector P applied to s_j = hi_j + lo_j moves it by at most
// ||lo_j||, the true error obeys
//     |sqrt(err_j) - sqrt(err_hi_j)| <= ||P lo_j|| <= ||lo_j||,
// so U_j = err_hi_j + 2 sqrt(err_hi_j) ||lo_j|| + ||lo_j||^2 bounds it from
// above and L_j = err_hi_j - 2 sqrt(err_hi_j) ||lo_j|| from below.  Every
// column whose U_j reaches max_i L_i is a candidate for the pivot; the
// candidates are re-checked exactly (FP64 bookkeeping of
// |c_hi,lj + q_l^H lo_j|^2 for all l) and the exact argmax is the pivot.
//
// Switch.  Once the exact max error falls below switch_err (where the lo
// margin starts to matter) -- or the loop ends in phase 0 -- one projection of
// the basis onto lo, d_lj = q_l^H lo_j for all l and j, turns every stored
// c_hi,lj into c_lj, rebuilds acc_j = sum_l |c_lj|^2 exactly and re-takes the
// argmax.  d only needs FP32 relative accuracy (|lo| <= 2^-24 |s|).
//
// Phase 1 (hi + lo, 16 bytes per element): the FP64 form's double-float sweep.
#include "rb_internal.cuh"

namespace rbk {

// certified upper / lower bounds of the true error from the hi-only error
__device__ __forceinline__ void split_bounds(double ehi, float lonrm, double n2, int k, double &U, double &L) {
    double e = ehi > 0.0 ? ehi : 0.0;
    double ln = (double)lonrm;
    double r = sqrt(e);
    double E = 2.0 * r * ln * (1.0 + 1e-6) + ln * ln;
    // FP64 noise of the bookkeeping itself
    E += 8.0 * (k + 16) * 1.1102230246251565e-16 * n2;
    U = ehi + E;
    L = ehi - E;
}

// ---------------------------------------------------------------- init
// Warp per column: ||hi + lo||^2 and ||hi||^2 in double-float, ||lo|| in
// FP32 (inflated to stay an upper bound).
__global__ void __launch_bounds__(kThreads) k_split_init(Prob p) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long j = gw; j < p.M; j += nw) {
        const float2 *h = p.hi + j * p.ldH;
        const float2 *l = p.lo + j * p.ldH;
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, lsq = 0.f;
        for (long long i = lane; i < p.N; i += 32) {
            float2 x = h[i], y = l[i];
            df_mac(ah, al, x.x, y.x, x.x, y.x);
            df_mac(ah, al, x.y, y.y, x.y, y.y);
            df_mac(bh, bl, x.x, 0.f, x.x, 0.f);
            df_mac(bh, bl, x.y, 0.f, x.y, 0.f);
            lsq = fmaf(y.x, y.x, fmaf(y.y, y.y, lsq));
        }
        // the lo^2 term dropped by df_mac (2^-48 relative) is added back here
        double n2 = warp_sum((double)ah + (double)al + (double)lsq);
        double nh = warp_sum((double)bh + (double)bl);
        double ls = warp_sum((double)lsq);
        if (lane == 0) {
            p.norm2[j] = n2;
            p.norm2_hi[j] = nh;
            p.lonrm[j] = (float)(sqrt(ls) * (1.0 + 1e-4));
        }
    }
}

// ------------------------------------------------------- phase 0 sweep
// c_hi = q^H hi with q = qh + ql (double-float), hi exact.
__device__ __forceinline__ double2 col_dot_hi(const float2 *__restrict__ hcol, const float2 *__restrict__ qh,
                                              const float2 *__restrict__ ql, long long N, int lane) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4 *h4 = reinterpret_cast<const float4 *>(hcol);
    const float4 *qh4 = reinterpret_cast<const float4 *>(qh);
    const float4 *ql4 = reinterpret_cast<const float4 *>(ql);
    const long long n2 = N >> 1;
    long long t = lane;
    constexpr int U = 4;
    for (; t + 32 * (U - 1) < n2; t += 32 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; u++) a[u] = ld_stream(h4 + t + 32 * u);
#pragma unroll
        for (int u = 0; u < U; u++) {
            float4 qa = __ldg(qh4 + t + 32 * u), qb = __ldg(ql4 + t + 32 * u);
            df_mac(rh, rl, qa.x, qb.x, a[u].x, 0.f);
            df_mac(rh, rl, qa.y, qb.y, a[u].y, 0.f);
            df_mac(ih, il, qa.x, qb.x, a[u].y, 0.f);
            df_mac(ih, il, -qa.y, -qb.y, a[u].x, 0.f);
            df_mac(rh, rl, qa.z, qb.z, a[u].z, 0.f);
            df_mac(rh, rl, qa.w, qb.w, a[u].w, 0.f);
            df_mac(ih, il, qa.z, qb.z, a[u].w, 0.f);
            df_mac(ih, il, -qa.w, -qb.w, a[u].z, 0.f);
        }
    }
    for (; t < n2; t += 32) {
        float4 a = ld_stream(h4 + t), qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        df_mac(rh, rl, qa.x, qb.x, a.x, 0.f);
        df_mac(rh, rl, qa.y, qb.y, a.y, 0.f);
        df_mac(ih, il, qa.x, qb.x, a.y, 0.f);
        df_mac(ih, il, -qa.y, -qb.y, a.x, 0.f);
        df_mac(rh, rl, qa.z, qb.z, a.z, 0.f);
        df_mac(rh, rl, qa.w, qb.w, a.w, 0.f);
        df_mac(ih, il, qa.z, qb.z, a.w, 0.f);
        df_mac(ih, il, -qa.w, -qb.w, a.z, 0.f);
    }
    if ((N & 1) && lane == 0) {
        long long i = N - 1;
        float2 a = hcol[i], qa = qh[i], qb = ql[i];
        df_mac(rh, rl, qa.x, qb.x, a.x, 0.f);
        df_mac(rh, rl, qa.y, qb.y, a.y, 0.f);
        df_mac(ih, il, qa.x, qb.x, a.y, 0.f);
        df_mac(ih, il, -qa.y, -qb.y, a.x, 0.f);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

__device__ __forceinline__ bool phase0_active(const DevState *st) {
    return !ld_volatile(&st->stop) && ld_volatile(&st->phase) == 0 && !ld_volatile(&st->switch_pending);
}

__global__ void __launch_bounds__(kThreads) k_sweep_hi(Prob p) {
    DevState *st = p.st;
    if (!phase0_active(st)) return;
    const int k = st->k;
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float2 *qh = p.qh + (long long)k * p.qs_stride;
    const float2 *ql = p.ql + (long long)k * p.qs_stride;
    double bu = -INFINITY, bl = -INFINITY;
    long long bi = kNoIdx, li = kNoIdx;
    for (long long j = gw; j < p.M; j += nw) {
        double2 c = col_dot_hi(p.hi + j * p.ldH, qh, ql, p.N, lane);
        if (lane == 0) {
            p.C[(long long)k * p.ldC + j] = c;
            double a = p.acc[j] + (c.x * c.x + c.y * c.y);
            p.acc[j] = a;
            if (!p.picked[j]) {
                double U, L;
                split_bounds(p.norm2_hi[j] - a, p.lonrm[j], p.norm2[j], k + 1, U, L);
                if (better(U, j, bu, bi)) { bu = U; bi = j; }
                if (better(L, j, bl, li)) { bl = L; li = j; }
            }
        }
    }
    block_best(bu, bi);
    __shared__ double s_u;
    __shared__ long long s_i;
    if (threadIdx.x == 0) { s_u = bu; s_i = bi; }
    block_best(bl, li);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = bl;        // lower bounds
        p.bpart_idx[blockIdx.x] = s_i;       // argmax of the upper bound
        p.npart[blockIdx.x] = s_u;
    }
    if (!last_block(&st->ticket_sweep)) return;
    double gl = -INFINITY, gu = -INFINITY;
    long long gi = kNoIdx, dummy = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double l = __ldcg(p.bpart_err + b);
        if (l > gl) gl = l;
        double u = __ldcg(p.npart + b);
        long long i = __ldcg(p.bpart_idx + b);
        if (better(u, i, gu, gi)) { gu = u; gi = i; }
    }
    block_best(gl, dummy);
    __shared__ double s_gl;
    if (threadIdx.x == 0) s_gl = gl;
    block_best(gu, gi);
    if (threadIdx.x == 0) {
        st->ticket_sweep = 0;
        const int k1 = k + 1;
        st->k = k1;
        st->n_sweeps += 1;
        st->Lmax = s_gl;
        st->J = gi;
        st->errJ = gu;  // provisional (an upper bound); replaced by the recheck or the projection
        p.err_curve[k1] = gu;
        if (gi == kNoIdx || k1 >= p.kmax || k1 >= p.minNM) {
            // the loop ends in phase 0: make C and the errors exact first
            st->switch_pending = 1;
            st->ncand = 0;
        } else {
            st->ncand = -1;  // recheck needed
        }
    }
}

// ------------------------------------------------------- candidates
__device__ __forceinline__ bool is_candidate(const Prob &p, long long j, int k1, double Lmax) {
    if (p.picked[j]) return false;
    double U, L;
    split_bounds(p.norm2_hi[j] - p.acc[j], p.lonrm[j], p.norm2[j], k1, U, L);
    return U >= Lmax;
}

__device__ __forceinline__ bool recheck_active(const DevState *st) {
    return phase0_active(st) && ld_volatile(&st->ncand) == -1;
}

// Deterministic gathering: block b owns the contiguous column range
// [b*chunk, (b+1)*chunk); counts first, then writes at its exclusive prefix.
__global__ void __launch_bounds__(kThreads) k_cand_count(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    const int k1 = st->k;
    const double Lmax = st->Lmax;
    const long long per = (p.M + gridDim.x - 1) / gridDim.x;
    const long long j0 = blockIdx.x * per, j1 = j0 + per < p.M ? j0 + per : p.M;
    int c = 0;
    for (long long j = j0 + threadIdx.x; j < j1; j += blockDim.x) c += is_candidate(p, j, k1, Lmax);
    c = (int)block_sum((double)c);
    if (threadIdx.x == 0) p.bcount[blockIdx.x] = c;
}

__global__ void __launch_bounds__(kThreads) k_cand_write(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    const int k1 = st->k;
    const double Lmax = st->Lmax;
    __shared__ int base;
    __shared__ int wcount[kThreads / 32];
    if (threadIdx.x == 0) {
        int b0 = 0;
        for (int b = 0; b < (int)blockIdx.x; b++) b0 += p.bcount[b];
        base = b0;
    }
    __syncthreads();
    const long long per = (p.M + gridDim.x - 1) / gridDim.x;
    const long long j0 = blockIdx.x * per, j1 = j0 + per < p.M ? j0 + per : p.M;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int off = base;
    // process the range in rounds of blockDim.x columns, in index order
    for (long long r = j0; r < j1; r += blockDim.x) {
        long long j = r + threadIdx.x;
        bool c = j < j1 && is_candidate(p, j, k1, Lmax);
        unsigned m = __ballot_sync(0xffffffffu, c);
        if (lane == 0) wcount[w] = __popc(m);
        __syncthreads();
        int before = 0, round = 0;
        for (int x = 0; x < (int)(blockDim.x >> 5); x++) {
            if (x < w) before += wcount[x];
            round += wcount[x];
        }
        if (c) {
            int pos = off + before + __popc(m & ((1u << lane) - 1u));
            if (pos < p.cand_cap) p.cand[pos] = j;
        }
        off += round;
        __syncthreads();
    }
}

// Exact error of each candidate: err_j = ||hi_j + lo_j||^2 - sum_l |c_hi,lj + q_l^H lo_j|^2.
__global__ void __launch_bounds__(kThreads) k_recheck(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    __shared__ int s_total;
    if (threadIdx.x == 0) {
        int t = 0;
        for (int b = 0; b < p.nblk_cand; b++) t += __ldcg(p.bcount + b);
        s_total = t;
    }
    __syncthreads();
    const int total = s_total;
    const int n = total < p.cand_cap ? total : p.cand_cap;
    const int k1 = st->k;
    if ((int)blockIdx.x < n) {
        const long long j = p.cand[blockIdx.x];
        const float2 *lcol = p.lo + j * p.ldH;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        double accp = 0.0;
        for (int l = w; l < k1; l += nwarp) {
            const float2 *q = p.qh + (long long)l * p.qs_stride;
            float re = 0.f, im = 0.f;
            for (long long i = lane; i < p.N; i += 32) {
                float2 a = q[i], b = lcol[i];
                re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
                im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
            }
            double dre = warp_sum((double)re), dim = warp_sum((double)im);
            double2 c = p.C[(long long)l * p.ldC + j];
            double cr = c.x + dre, ci = c.y + dim;
            accp += cr * cr + ci * ci;
        }
        double acc = block_sum(lane == 0 ? accp : 0.0);
        if (threadIdx.x == 0) p.cand_err[blockIdx.x] = p.norm2[j] - acc;
    }
    if (!last_block(&st->ticket_aux)) return;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double e = __ldcg(p.cand_err + b);
        long long i = __ldcg(p.cand + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_aux = 0;
        st->ncand = n;
        if (total > p.cand_cap) st->cand_overflow = 1;
        if (n > st->max_cand) st->max_cand = n;
        st->J = bi;
        st->errJ = be;
        p.err_curve[k1] = be;
        if (bi == kNoIdx || be < p.switch_err || be < p.tol) st->switch_pending = 1;
    }
}

// ------------------------------------------------------- projection onto lo
// d = Qh^H lo for the k1 basis vectors, C[l, j] += d, acc_j = sum_l |C[l, j]|^2,
// then the exact argmax and the stopping rule.  Tiled FP32 complex GEMM:
// a block owns 64 columns and up to 64 basis vectors at a time, staging 32
// rows of both operands in shared memory.
constexpr int RJ = 64, RL = 64, RK = 32;

__global__ void __launch_bounds__(kThreads) k_rebase(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    __shared__ float2 qs[RL][RK + 1];
    __shared__ float2 ls[RJ][RK + 1];
    __shared__ double accs[RJ];
    __shared__ double parts[16][RJ];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 4 columns x 4 vectors per thread
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long j0 = (long long)blockIdx.x * RJ; j0 < p.M; j0 += (long long)gridDim.x * RJ) {
        if (threadIdx.x < RJ) accs[threadIdx.x] = 0.0;
        for (int l0 = 0; l0 < k1; l0 += RL) {
            float dr[4][4], di[4][4];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) dr[a][b] = di[a][b] = 0.f;
            for (long long i0 = 0; i0 < p.N; i0 += RK) {
                __syncthreads();
                for (int t = threadIdx.x; t < RL * RK; t += blockDim.x) {
                    int r = t / RK, c = t % RK;
                    long long i = i0 + c;
                    qs[r][c] = (l0 + r < k1 && i < p.N) ? p.qh[(long long)(l0 + r) * p.qs_stride + i]
                                                        : make_float2(0.f, 0.f);
                    ls[r][c] = (j0 + r < p.M && i < p.N) ? p.lo[(j0 + r) * p.ldH + i] : make_float2(0.f, 0.f);
                }
                __syncthreads();
#pragma unroll 4
                for (int c = 0; c < RK; c++) {
                    float2 q[4], x[4];
#pragma unroll
                    for (int a = 0; a < 4; a++) q[a] = qs[ty * 4 + a][c];
#pragma unroll
                    for (int b = 0; b < 4; b++) x[b] = ls[tx * 4 + b][c];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int b = 0; b < 4; b++) {
                            dr[a][b] = fmaf(q[a].x, x[b].x, fmaf(q[a].y, x[b].y, dr[a][b]));
                            di[a][b] = fmaf(q[a].x, x[b].y, fmaf(-q[a].y, x[b].x, di[a][b]));
                        }
                }
            }
            // fold d into C and the per-column sums
#pragma unroll
            for (int b = 0; b < 4; b++) {
                long long j = j0 + tx * 4 + b;
                double part = 0.0;
                if (j < p.M) {
#pragma unroll
                    for (int a = 0; a < 4; a++) {
                        int l = l0 + ty * 4 + a;
                        if (l < k1) {
                            double2 *cp = p.C + (long long)l * p.ldC + j;
                            double2 c = *cp;
                            c.x += (double)dr[a][b];
                            c.y += (double)di[a][b];
                            *cp = c;
                            part += c.x * c.x + c.y * c.y;
                        }
                    }
                }
                parts[ty][tx * 4 + b] = part;
            }
            __syncthreads();
            if (threadIdx.x < RJ) {
                double a = accs[threadIdx.x];
                for (int g = 0; g < 16; g++) a += parts[g][threadIdx.x];  // fixed order
                accs[threadIdx.x] = a;
            }
        }
        __syncthreads();
        if (threadIdx.x < RJ) {
            long long j = j0 + threadIdx.x;
            if (j < p.M) {
                double a = accs[threadIdx.x];
                p.acc[j] = a;
                double e = p.norm2[j] - a;
                if (!p.picked[j] && better(e, j, be, bi)) { be = e; bi = j; }
            }
        }
        __syncthreads();
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = be;
        p.bpart_idx[blockIdx.x] = bi;
    }
    if (!last_block(&st->ticket_aux)) return;
    be = -INFINITY;
    bi = kNoIdx;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        double e = __ldcg(p.bpart_err + b);
        long long i = __ldcg(p.bpart_idx + b);
        if (better(e, i, be, bi)) { be = e; bi = i; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_aux = 0;
        st->switch_pending = 0;
        st->phase = 1;
        st->switch_iter = k1;
        double emax = bi == kNoIdx ? 0.0 : be;
        p.err_curve[k1] = emax;
        st->J = bi;
        st->errJ = emax;
        if (bi == kNoIdx || emax < p.tol || st->force_stop) {
            st->status = RB_OK;
            st->stop = 1;
        } else if (k1 >= p.kmax) {
            st->status = RB_KMAX_REACHED;
            st->stop = 1;
        } else if (k1 >= p.minNM) {
            st->status = RB_OK;
            st->stop = 1;
        }
    }
}

cudaError_t launch_split_init(const Prob &p, cudaStream_t s) {
    long long g = (p.M * 32 + kThreads - 1) / kThreads;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    k_split_init<<<(int)g, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_split_iteration(const Prob &p, int grid, cudaStream_t s, int *nlaunch) {
    k_sweep_hi<<<grid, kThreads, 0, s>>>(p);
    cudaError_t e = launch_sweep(p, 0, grid, s);
    if (e != cudaSuccess) return e;
    k_cand_count<<<grid, kThreads, 0, s>>>(p);
    k_cand_write<<<grid, kThreads, 0, s>>>(p);
    k_recheck<<<p.cand_cap, kThreads, 0, s>>>(p);
    long long rb = (p.M + RJ - 1) / RJ;
    if (rb > grid) rb = grid;
    k_rebase<<<(int)rb, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 6;
    return cudaGetLastError();
}

}  // namespace rbk
