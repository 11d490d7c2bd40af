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
#include "rb_tc.cuh"

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
            p.dacc[j] = 0.0;
            p.dcnt[j] = 0;
        }
    }
}

// ------------------------------------------------------- phase 0 sweep
// (sh, sl) += (ah + al) * b for an exact FP32 b: TwoProduct of ah*b by FMA,
// the al*b term into the low part, TwoSum into the high part.
__device__ __forceinline__ void df_mac1(float &sh, float &sl, float ah, float al, float b) {
    float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// c_hi = q^H hi with q = qh + ql (double-float), hi exact.
__device__ __forceinline__ double2 col_dot_hi(const float2 *__restrict__ hcol, const float2 *__restrict__ qh,
                                              const float2 *__restrict__ ql, long long N, int lane) {
    // two independent (re, im) double-float chains (even / odd element of each
    // 16-byte pair) so consecutive TwoSums do not wait on each other
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f, rh2 = 0.f, rl2 = 0.f, ih2 = 0.f, il2 = 0.f;
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
            df_mac1(rh, rl, qa.x, qb.x, a[u].x);
            df_mac1(ih, il, qa.x, qb.x, a[u].y);
            df_mac1(rh2, rl2, qa.z, qb.z, a[u].z);
            df_mac1(ih2, il2, qa.z, qb.z, a[u].w);
            df_mac1(rh, rl, qa.y, qb.y, a[u].y);
            df_mac1(ih, il, -qa.y, -qb.y, a[u].x);
            df_mac1(rh2, rl2, qa.w, qb.w, a[u].w);
            df_mac1(ih2, il2, -qa.w, -qb.w, a[u].z);
        }
    }
    for (; t < n2; t += 32) {
        float4 a = ld_stream(h4 + t), qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        df_mac1(rh, rl, qa.x, qb.x, a.x);
        df_mac1(ih, il, qa.x, qb.x, a.y);
        df_mac1(rh2, rl2, qa.z, qb.z, a.z);
        df_mac1(ih2, il2, qa.z, qb.z, a.w);
        df_mac1(rh, rl, qa.y, qb.y, a.y);
        df_mac1(ih, il, -qa.y, -qb.y, a.x);
        df_mac1(rh2, rl2, qa.w, qb.w, a.w);
        df_mac1(ih2, il2, -qa.w, -qb.w, a.z);
    }
    if ((N & 1) && lane == 0) {
        long long i = N - 1;
        float2 a = hcol[i], qa = qh[i], qb = ql[i];
        df_mac1(rh, rl, qa.x, qb.x, a.x);
        df_mac1(rh, rl, qa.y, qb.y, a.y);
        df_mac1(ih, il, qa.x, qb.x, a.y);
        df_mac1(ih, il, -qa.y, -qb.y, a.x);
    }
    df_add(rh, rl, rh2, rl2);
    df_add(ih, il, ih2, il2);
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
    // the last block turns the counts into exclusive prefixes (bases of the
    // write pass) and publishes the total, once, through shared memory
    if (!last_block(&st->ticket_aux)) return;
    __shared__ int sc[4096];
    const int G = gridDim.x;
    for (int b = threadIdx.x; b < G; b += blockDim.x) sc[b] = __ldcg(p.bcount + b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < G; b++) {
            int x = sc[b];
            sc[b] = run;
            run += x;
        }
        st->cand_total = run;
        st->ticket_aux = 0;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < G; b += blockDim.x) p.bcount[b] = sc[b];
}

__global__ void __launch_bounds__(kThreads) k_cand_write(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    const int k1 = st->k;
    const double Lmax = st->Lmax;
    __shared__ int wcount[kThreads / 32];
    const int base = p.bcount[blockIdx.x];  // exclusive prefix from k_cand_count
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

// Exact error of each candidate: err_j = ||hi_j + lo_j||^2 - sum_l |c_hi,lj + q_l^H lo_j|^2
// = norm2_j - acc_hi_j - D_j with D_j = sum_l (2 Re(conj(c_hi,lj) d_lj) + |d_lj|^2),
// d_lj = q_l^H lo_j.  D_j is kept per column with the number of basis vectors it
// covers, so a column that stays a candidate over many iterations only adds the
// new vectors' terms.  One block per candidate; the block sweeps the rows once
// per group of 8 basis vectors (8 complex FP32 dots per thread).
constexpr int RG = 8;

__global__ void __launch_bounds__(kThreads) k_recheck(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    __shared__ float red[2 * RG][kThreads / 32];
    __shared__ double s_acc;
    __shared__ double vals[RG];
    const int total = st->cand_total;
    const int n = total < p.cand_cap ? total : p.cand_cap;
    const int k1 = st->k;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if ((int)blockIdx.x < n) {
        const long long j = p.cand[blockIdx.x];
        const float2 *lcol = p.lo + j * p.ldH;
        // basis vectors already folded into D_j by earlier rechecks of this column
        const int lstart = p.dcnt[j];
        if (threadIdx.x == 0) s_acc = p.dacc[j];
        __syncthreads();
        for (int l0 = lstart; l0 < k1; l0 += RG) {
            float re[RG], im[RG];
#pragma unroll
            for (int g = 0; g < RG; g++) re[g] = im[g] = 0.f;
            for (long long i = threadIdx.x; i < p.N; i += blockDim.x) {
                float2 b = lcol[i];
#pragma unroll
                for (int g = 0; g < RG; g++) {
                    if (l0 + g < k1) {
                        float2 a = p.qh[(long long)(l0 + g) * p.qs_stride + i];
                        re[g] = fmaf(a.x, b.x, fmaf(a.y, b.y, re[g]));
                        im[g] = fmaf(a.x, b.y, fmaf(-a.y, b.x, im[g]));
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < RG; g++) {
                float r = re[g], m = im[g];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r += __shfl_xor_sync(0xffffffffu, r, o);
                    m += __shfl_xor_sync(0xffffffffu, m, o);
                }
                if (lane == 0) {
                    red[2 * g][w] = r;
                    red[2 * g + 1][w] = m;
                }
            }
            __syncthreads();
            if (threadIdx.x < RG) {
                int g = threadIdx.x;
                double v = 0.0;
                if (l0 + g < k1) {
                    double dre = 0.0, dim = 0.0;
                    for (int x = 0; x < (int)(blockDim.x >> 5); x++) {
                        dre += (double)red[2 * g][x];
                        dim += (double)red[2 * g + 1][x];
                    }
                    // |c_hi + d|^2 - |c_hi|^2 = 2 Re(conj(c_hi) d) + |d|^2
                    double2 c = p.C[(long long)(l0 + g) * p.ldC + j];
                    v = 2.0 * (c.x * dre + c.y * dim) + (dre * dre + dim * dim);
                }
                vals[g] = v;
            }
            __syncthreads();
            if (threadIdx.x == 0)
                for (int g = 0; g < RG; g++) s_acc += vals[g];  // fixed order
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            p.dacc[j] = s_acc;
            p.dcnt[j] = k1;
            // err_j = ||hi + lo||^2 - sum_l |c_hi,lj + d_lj|^2 = norm2 - acc_hi - D_j
            p.cand_err[blockIdx.x] = p.norm2[j] - p.acc[j] - s_acc;
        }
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
// d = Qh^H lo for the k1 basis vectors on the tensor cores, then C[l, j] += d.
// As a real GEMM with K = 2N interleaved (re, im): A rows 2l = (a_i, b_i) and
// 2l+1 = (-b_i, a_i) for q_l = a + ib; B row j = (u_i, v_i) for lo_j = u + iv.
// Every FP32 value is split exactly into three BF16 pieces (x = x1 + x2 + x3);
// the six piece products with s + t <= 4 accumulate into one FP32 TMEM
// accumulator, which leaves a relative error of a few 2^-24 -- what d needs,
// since |lo| <= 2^-24 |s|.
constexpr int PT = 128;  // tile rows (A) and columns (B)
constexpr int PKC = 64;  // K per stage
constexpr int PSL = 3;   // BF16 pieces per FP32 value

__device__ __forceinline__ void split3(float x, __nv_bfloat16 *o) {
    __nv_bfloat16 x1 = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(x1);
    __nv_bfloat16 x2 = __float2bfloat16_rn(r);
    r -= __bfloat162float(x2);
    o[0] = x1;
    o[1] = x2;
    o[2] = __float2bfloat16_rn(r);
}

// Stage 8 consecutive K entries (4 complex elements) of one tile row into the
// three piece tiles: one 16-byte core-matrix row per piece.
__device__ __forceinline__ void stage_row8(uint8_t *base, int r, int kk, const float v[8]) {
    __nv_bfloat16 pc[PSL][8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        __nv_bfloat16 o[PSL];
        split3(v[e], o);
#pragma unroll
        for (int s = 0; s < PSL; s++) pc[s][e] = o[s];
    }
#pragma unroll
    for (int s = 0; s < PSL; s++)
        *(uint4 *)(base + s * (PT * PKC * 2) + kmajor_off(r, kk, PKC)) = *(const uint4 *)pc[s];
}

__global__ void __launch_bounds__(128) k_lo_project_tc(Prob p, int *err) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    const int r0 = blockIdx.y * PT;  // first A row of this tile
    if (r0 >= 2 * k1) return;
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t *sA = dsm, *sB = dsm + PSL * PT * PKC * 2;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    const long long j0 = (long long)blockIdx.x * PT;
    if (warp == 0) tmem_alloc(&tslot, PT);
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(PT, PT);
    const long long K = 2 * p.N;
    uint32_t phase = 0;
    bool ok = true;
    int nst = 0;
    for (long long k0 = 0; k0 < K; k0 += PKC, nst++) {
        // A: 128 rows x 64 K; each thread fills (row, 8 K) pieces, 8 per thread
        for (int t = threadIdx.x; t < PT * (PKC / 8); t += blockDim.x) {
            int r = t / (PKC / 8), kk = (t % (PKC / 8)) * 8;
            int gr = r0 + r;
            float v[8];
            long long i0 = (k0 + kk) >> 1;  // first complex element
#pragma unroll
            for (int e = 0; e < 4; e++) {
                long long i = i0 + e;
                float2 q = (gr < 2 * k1 && i < p.N) ? p.qh[(long long)(gr >> 1) * p.qs_stride + i] : make_float2(0.f, 0.f);
                if ((gr & 1) == 0) { v[2 * e] = q.x; v[2 * e + 1] = q.y; }
                else { v[2 * e] = -q.y; v[2 * e + 1] = q.x; }
            }
            stage_row8(sA, r, kk, v);
        }
        // B: 128 columns x 64 K from lo
        for (int t = threadIdx.x; t < PT * (PKC / 8); t += blockDim.x) {
            int r = t / (PKC / 8), kk = (t % (PKC / 8)) * 8;
            long long j = j0 + r;
            float v[8];
            long long i0 = (k0 + kk) >> 1;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                long long i = i0 + e;
                float2 x = (j < p.M && i < p.N) ? p.lo[j * p.ldH + i] : make_float2(0.f, 0.f);
                v[2 * e] = x.x;
                v[2 * e + 1] = x.y;
            }
            stage_row8(sB, r, kk, v);
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            int first = 1;
#pragma unroll
            for (int sa = 0; sa < PSL; sa++)
#pragma unroll
                for (int sb = 0; sb < PSL; sb++) {
                    if (sa + sb > 2) continue;  // pieces s + t <= 4 (0-based sa + sb <= 2)
#pragma unroll
                    for (int kk = 0; kk < PKC / 16; kk++) {
                        uint64_t ad = smem_desc(smem_u32(sA) + sa * (PT * PKC * 2) + kk * 256, 128, (PKC / 8) * 128);
                        uint64_t bd = smem_desc(smem_u32(sB) + sb * (PT * PKC * 2) + kk * 256, 128, (PKC / 8) * 128);
                        tc_mma_bf16(tmem, ad, bd, idesc, (nst > 0 || !first) ? 1u : 0u);
                        first = 0;
                    }
                }
            tc_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase) && ok;
        phase ^= 1;
        tc_fence_after();
        __syncthreads();
    }
    if (!ok) atomicExch(err, 1);
    // epilogue: thread = A row (TMEM lane); row 2l adds to Re C[l, j], row 2l+1 to Im
    const int r = r0 + threadIdx.x;
    for (int c0 = 0; c0 < PT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (r < 2 * k1) {
            double *crow = (double *)(p.C + (long long)(r >> 1) * p.ldC) + (r & 1);
#pragma unroll
            for (int e = 0; e < 16; e++) {
                long long j = j0 + c0 + e;
                if (j < p.M) crow[2 * j] += (double)v[e];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, PT);
}

// acc_j = sum_l |C[l, j]|^2 after the projection onto lo, the exact argmax,
// the switch to the hi + lo phase and the stopping rule.
__global__ void __launch_bounds__(kThreads) k_rebase_finish(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M; j += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int l = 0; l < k1; l++) {
            double2 c = p.C[(long long)l * p.ldC + j];
            a += c.x * c.x + c.y * c.y;
        }
        p.acc[j] = a;
        double e = p.norm2[j] - a;
        if (!p.picked[j] && better(e, j, be, bi)) { be = e; bi = j; }
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
    const size_t dsmem = 2 * PSL * PT * PKC * 2;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_lo_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
        attr_set = true;
    }
    dim3 pg((unsigned)((p.M + PT - 1) / PT), (unsigned)((2LL * (p.kmax > 0 ? p.kmax : 1) + PT - 1) / PT));
    k_lo_project_tc<<<pg, 128, dsmem, s>>>(p, p.tc_err);
    long long rf = (p.M + kThreads - 1) / kThreads;
    if (rf > grid) rf = grid;
    k_rebase_finish<<<(int)rf, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 7;
    return cudaGetLastError();
}

}  // namespace rbk
