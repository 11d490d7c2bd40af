// rb_split_form.cu -- the split-precision form of the greedy sweep.
//
// S is stored as complex64 hi + lo (hi = fl32(s), lo = fl32(s - hi)).  Every
// sweep reads hi only (8 bytes per element); lo is read for the candidate
// columns of the exact re-check and once, at the end, by the projection of
// the basis onto lo.
//
// Hi-only sweep.  c~ = q^H hi_j is accumulated against a fixed offset: each of
// the 64 lane chains of a column (lane, element parity) keeps S = 1.5 sigma +
// (sum so far) with sigma a power of two >= 4 ||q_I|| ||hi_I|| (Cauchy-Schwarz
// over the chain I), so S never leaves its binade.  One FMA adds a product
// qh*hi to S on that grid, the difference is exact, a second FMA recovers the
// product's part below ulp(sigma) into an FP32 remainder that is folded back
// into S after every two products; the ql*hi terms (2^-24 relative) go to a
// plain FP32 sum.  Five FP32 operations per real product keep the sweep at
// HBM speed.  Relative to ||hi_j|| the result is accurate to about 2^-42 at
// N = 16384 (growing like sqrt(N)); eta = 2^-46 sqrt(N) bounds it with a wide
// margin (measured, see the tests).
//
// Bounds.  With acc~_j = sum_l |c~_lj|^2 and sigma_j = sum_l |c~_lj|,
//     |err(hi_j) - (||hi_j||^2 - acc~_j)| <= Ec_j = 2 eta ||hi_j|| sigma_j + 3 k eta^2 ||hi_j||^2,
// and, the orthogonal projector P moving s_j = hi_j + lo_j by at most ||lo_j||,
//     |sqrt(err_j) - sqrt(err(hi_j))| <= ||lo_j||.
// Together they give U_j >= err_j >= L_j.  Every column whose U_j reaches
// max_i L_i is a candidate for the pivot.
//
// Re-check.  For each candidate the rows not yet re-checked are recomputed
// exactly, c_lj = q_l^H hi_j (double-float, TwoSum accumulation) + q_l^H lo_j
// (FP32, |lo| <= 2^-24 |s|), and D_j = sum_l (|c_lj|^2 - |c~_lj|^2) is kept
// per column, so err_j = ||s_j||^2 - acc~_j - D_j exactly and the exact argmax
// over the candidates is the pivot.  A column that stays a candidate only
// adds the newest row.
//
// End.  When every upper bound is below tol (or the exact pivot error is, or
// kmax is reached), the basis is projected onto lo on the tensor cores, C +=
// Q^H lo, and the final errors and argmax are taken from C.
#include "rb_internal.cuh"
#include "rb_tc.cuh"

namespace rbk {

// Rounding allowance of the FP32 chain norms (sums of at most 2^16 squares).
constexpr float kNormUp = 1.001f;

// Certified bounds of the true error from the hi-only bookkeeping.
//   e   = ||hi_j||^2 - acc~_j          ln  = ||lo_j|| (rounded up)
//   Ec  = bound on |err(hi_j) - e|     n2  = ||s_j||^2 (FP64 bookkeeping slack)
__device__ __forceinline__ void split_bounds(double e, double Ec, float lonrm, double n2, int k, double &U,
                                             double &L) {
    const double ln = (double)lonrm;
    const double ehi_up = e + Ec > 0.0 ? e + Ec : 0.0;
    const double r = sqrt(ehi_up) * (1.0 + 1e-15);
    const double slack = 8.0 * (k + 16) * 1.1102230246251565e-16 * n2;
    U = ehi_up + 2.0 * r * ln + ln * ln + slack;
    L = e - Ec - 2.0 * r * ln - slack;
}

__device__ __forceinline__ double col_ec(const Prob &p, long long j, int k1) {
    const double nh2 = p.norm2_hi[j];
    return 2.0 * p.eta * sqrt(nh2) * p.sabs[j] + 3.0 * k1 * p.eta * p.eta * nh2;
}

// ---------------------------------------------------------------- init
// Warp per column: ||hi + lo||^2 and ||hi||^2 in double-float, ||lo|| and the
// 64 chain norms of hi in FP32 (rounded up).  Chain (lane, c) holds the
// elements 2t + c with t = lane (mod 32): the float4 slots the sweep's lane
// reads.  An odd last element belongs to no chain (the sweep adds it exactly).
__global__ void __launch_bounds__(kThreads) k_split_init(Prob p) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n2 = p.N >> 1;
    for (long long j = gw; j < p.M; j += nw) {
        const float2 *h = p.hi + j * p.ldH;
        const float2 *l = p.lo + j * p.ldH;
        const float4 *h4 = reinterpret_cast<const float4 *>(h);
        const float4 *l4 = reinterpret_cast<const float4 *>(l);
        Norm2Acc a{0.f, 0.f, 0.f};
        float bh = 0.f, bl = 0.f, c0 = 0.f, c1 = 0.f;
        for (long long t = lane; t < n2; t += 32) {
            float4 x = h4[t], y = l4[t];
            norm2_acc4(a, x, y);
            df_mac(bh, bl, x.x, 0.f, x.x, 0.f);
            df_mac(bh, bl, x.y, 0.f, x.y, 0.f);
            df_mac(bh, bl, x.z, 0.f, x.z, 0.f);
            df_mac(bh, bl, x.w, 0.f, x.w, 0.f);
            c0 = fmaf(x.x, x.x, fmaf(x.y, x.y, c0));
            c1 = fmaf(x.z, x.z, fmaf(x.w, x.w, c1));
        }
        if ((p.N & 1) && lane == 0) {
            float2 x = h[p.N - 1], y = l[p.N - 1];
            norm2_acc2(a, x, y);
            df_mac(bh, bl, x.x, 0.f, x.x, 0.f);
            df_mac(bh, bl, x.y, 0.f, x.y, 0.f);
        }
        p.snorm[j * 64 + lane] = sqrtf(c0) * kNormUp;
        p.snorm[j * 64 + 32 + lane] = sqrtf(c1) * kNormUp;
        // ||hi + lo||^2 with the steps of the FP64 form's split kernel
        double n2s = norm2_finish(a);
        double nh = warp_sum((double)bh + (double)bl);
        double ls = warp_sum((double)a.lsq);
        if (lane == 0) {
            p.norm2[j] = n2s;
            p.norm2_hi[j] = nh;
            p.lonrm[j] = (float)(sqrt(ls) * (1.0 + 1e-4));
            p.sabs[j] = 0.0;
            p.dacc[j] = 0.0;
            p.dcnt[j] = 0;
        }
    }
}

// ------------------------------------------------------- hi-only sweep
// Smallest power of two >= 4 B (B >= 0 finite), at least 2^-96.
__device__ __forceinline__ float sigma_of(float B) {
    const uint32_t b = __float_as_uint(__fmul_rn(4.f, B));
    uint32_t e = b & 0x7f800000u;
    if (b & 0x007fffffu) e += 0x00800000u;
    if (e < 0x0f800000u) e = 0x0f800000u;
    return __uint_as_float(e);
}

// S + lo += a * b.  t = fl(S + a*b) by one FMA lands on the grid of S, which
// stays in [sigma, 2 sigma) because every partial sum is below sigma / 4 in
// magnitude; z = t - S is then exact (Sterbenz) and r = a*b - z, formed by a
// second FMA, is at most ulp(sigma) and rounded once on its way into lo.
__device__ __forceinline__ void sg_mac(float &S, float &lo, float a, float b) {
    const float t = __fmaf_rn(a, b, S);
    const float z = __fsub_rn(t, S);
    const float r = __fmaf_rn(a, b, -z);
    S = t;
    lo = __fadd_rn(lo, r);
}

// Moves the part of lo on the grid of S into S (error-free).
__device__ __forceinline__ void sg_fold(float &S, float &lo) {
    const float t = __fadd_rn(S, lo);
    const float z = __fsub_rn(t, S);
    lo = __fsub_rn(lo, z);
    S = t;
}

// (sh, sl) += (ah + al) * b with TwoSum accumulation (no offset needed).
__device__ __forceinline__ void df_mac1(float &sh, float &sl, float ah, float al, float b) {
    const float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// The 8 products of one float4 (two complex elements) with qh into the two
// chains, the ql terms (2^-24 relative, FP32 accuracy suffices) into xr, xi,
// and the fold of every chain.
#define RB_SG_ELEM2(a, qa, qb)                                                                                  \
    do {                                                                                                        \
        sg_mac(R0, r0, qa.x, a.x);                                                                              \
        sg_mac(I0, i0, qa.x, a.y);                                                                              \
        sg_mac(R1, r1, qa.z, a.z);                                                                              \
        sg_mac(I1, i1, qa.z, a.w);                                                                              \
        sg_mac(R0, r0, qa.y, a.y);                                                                              \
        sg_mac(I0, i0, -qa.y, a.x);                                                                             \
        sg_mac(R1, r1, qa.w, a.w);                                                                              \
        sg_mac(I1, i1, -qa.w, a.z);                                                                             \
        xr = __fmaf_rn(qb.x, a.x, __fmaf_rn(qb.y, a.y, __fmaf_rn(qb.z, a.z, __fmaf_rn(qb.w, a.w, xr))));      \
        xi = __fmaf_rn(qb.x, a.y, __fmaf_rn(-qb.y, a.x, __fmaf_rn(qb.z, a.w, __fmaf_rn(-qb.w, a.z, xi))));    \
        sg_fold(R0, r0);                                                                                        \
        sg_fold(I0, i0);                                                                                        \
        sg_fold(R1, r1);                                                                                        \
        sg_fold(I1, i1);                                                                                        \
    } while (0)

// c~ = q^H hi for one column; o0, o1 = 1.5 sigma of this lane's two chains.
__device__ __forceinline__ double2 col_dot_sig(const float2 *__restrict__ hcol, const float2 *__restrict__ qh,
                                               const float2 *__restrict__ ql, long long N, int lane, float o0,
                                               float o1) {
    float R0 = o0, I0 = o0, R1 = o1, I1 = o1, r0 = 0.f, i0 = 0.f, r1 = 0.f, i1 = 0.f, xr = 0.f, xi = 0.f;
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
            const float4 qa = __ldg(qh4 + t + 32 * u), qb = __ldg(ql4 + t + 32 * u);
            RB_SG_ELEM2(a[u], qa, qb);
        }
    }
    for (; t < n2; t += 32) {
        const float4 a = ld_stream(h4 + t), qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        RB_SG_ELEM2(a, qa, qb);
    }
    // S - 1.5 sigma is exact (same binade)
    float rh = __fsub_rn(R0, o0), rl = __fadd_rn(r0, xr), ih = __fsub_rn(I0, o0), il = __fadd_rn(i0, xi);
    df_add(rh, rl, __fsub_rn(R1, o1), r1);
    df_add(ih, il, __fsub_rn(I1, o1), i1);
    if ((N & 1) && lane == 0) {
        const float2 a = hcol[N - 1], qa = qh[N - 1], qb = ql[N - 1];
        df_mac1(rh, rl, qa.x, qb.x, a.x);
        df_mac1(rh, rl, qa.y, qb.y, a.y);
        df_mac1(ih, il, qa.x, qb.x, a.y);
        df_mac1(ih, il, -qa.y, -qb.y, a.x);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

__device__ __forceinline__ bool loop_active(const DevState *st) {
    return !ld_volatile(&st->stop) && !ld_volatile(&st->switch_pending);
}

__global__ void __launch_bounds__(kThreads, 4) k_sweep_hi(Prob p) {
    DevState *st = p.st;
    if (!loop_active(st)) return;
    const int k = st->k;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float2 *qh = p.qh + (long long)k * p.qs_stride;
    const float2 *ql = p.ql + (long long)k * p.qs_stride;
    const long long n2 = p.N >> 1;
    // chain norms of qh: thread x sums the slots t = x (mod kThreads), all of
    // lane x & 31; the kThreads/32 partials of a lane are added in order
    __shared__ float s_part[kThreads / 32][64];
    __shared__ float s_qn[64];
    {
        const float4 *q4 = reinterpret_cast<const float4 *>(qh);
        float a0 = 0.f, a1 = 0.f;
        for (long long t = threadIdx.x; t < n2; t += blockDim.x) {
            const float4 v = __ldg(q4 + t);
            a0 = fmaf(v.x, v.x, fmaf(v.y, v.y, a0));
            a1 = fmaf(v.z, v.z, fmaf(v.w, v.w, a1));
        }
        s_part[w][lane] = a0;
        s_part[w][32 + lane] = a1;
        __syncthreads();
        if (threadIdx.x < 64) {
            float s = 0.f;
#pragma unroll
            for (int x = 0; x < kThreads / 32; x++) s += s_part[x][threadIdx.x];
            s_qn[threadIdx.x] = sqrtf(s) * kNormUp;
        }
        __syncthreads();
    }
    const float qn0 = s_qn[lane], qn1 = s_qn[32 + lane];
    double2 *Crow = p.C + (long long)k * p.ldC;
    for (long long j = gw; j < p.M; j += nw) {
        const float *sn = p.snorm + j * 64;
        const float o0 = 1.5f * sigma_of(__fmul_rn(qn0, __ldg(sn + lane)));
        const float o1 = 1.5f * sigma_of(__fmul_rn(qn1, __ldg(sn + 32 + lane)));
        const double2 c = col_dot_sig(p.hi + j * p.ldH, qh, ql, p.N, lane, o0, o1);
        // every lane holds c: lane 0 keeps C and acc, lane 1 sum |c|
        const double cc = c.x * c.x + c.y * c.y;
        if (lane == 0) {
            Crow[j] = c;
            p.acc[j] += cc;
        } else if (lane == 1) {
            p.sabs[j] += sqrt(cc);
        }
    }
}

// Bounds of every unpicked column, the largest lower bound and the argmax of
// the upper bound; the last block decides whether the loop ends here.
__global__ void __launch_bounds__(kThreads) k_bounds(Prob p) {
    DevState *st = p.st;
    if (!loop_active(st)) return;
    const int k1 = st->k + 1;
    double bu = -INFINITY, bl = -INFINITY;
    long long bi = kNoIdx, li = kNoIdx;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M;
         j += (long long)gridDim.x * blockDim.x) {
        if (p.picked[j]) continue;
        double U, L;
        split_bounds(p.norm2_hi[j] - p.acc[j], col_ec(p, j, k1), p.lonrm[j], p.norm2[j], k1, U, L);
        if (better(U, j, bu, bi)) { bu = U; bi = j; }
        if (better(L, j, bl, li)) { bl = L; li = j; }
    }
    block_best(bu, bi);
    __shared__ double s_u;
    __shared__ long long s_i;
    if (threadIdx.x == 0) { s_u = bu; s_i = bi; }
    block_best(bl, li);
    if (threadIdx.x == 0) {
        p.bpart_err[blockIdx.x] = bl;   // lower bounds
        p.bpart_idx[blockIdx.x] = s_i;  // argmax of the upper bound
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
        st->k = k1;
        st->n_sweeps += 1;
        st->Lmax = s_gl;
        st->J = gi;
        st->errJ = gu;  // provisional (an upper bound); replaced by the re-check or the projection
        p.err_curve[k1] = gu;
        if (gi == kNoIdx || k1 >= p.kmax || k1 >= p.minNM || gu < p.tol) {
            // the loop ends: complete C on lo first (gu < tol certifies every error below tol)
            st->switch_pending = 1;
            st->ncand = 0;
        } else {
            st->ncand = -1;  // re-check needed
        }
    }
}

// ------------------------------------------------------- candidates
__device__ __forceinline__ bool is_candidate(const Prob &p, long long j, int k1, double Lmax) {
    if (p.picked[j]) return false;
    double U, L;
    split_bounds(p.norm2_hi[j] - p.acc[j], col_ec(p, j, k1), p.lonrm[j], p.norm2[j], k1, U, L);
    return U >= Lmax;
}

__device__ __forceinline__ bool recheck_active(const DevState *st) {
    return loop_active(st) && ld_volatile(&st->ncand) == -1;
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
        if (c) p.cand[off + before + __popc(m & ((1u << lane) - 1u))] = j;
        off += round;
        __syncthreads();
    }
}

// Exact re-check.  Work item = (candidate c, group g of RG basis vectors, row
// chunk h).  When the candidates are few, each (c, g) is split into RCH row
// chunks so that many blocks share the work; the last chunk block of a (c, g)
// adds the chunks in order.  Either way pv[c][g] = sum over the group's rows
// l >= dcnt_j of (|c_lj|^2 - |c~_lj|^2), in a fixed order, and the last block
// folds the groups into D_j and takes the exact argmax.
constexpr int RG = 8;
constexpr int RCH = 8;             // row chunks per (candidate, group) when few
constexpr int RPCAP = 2048;        // (candidate, group) pairs that may be chunked

__global__ void __launch_bounds__(kThreads) k_recheck(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    constexpr int NW = kThreads / 32;
    __shared__ double s_red[RG][4][NW];
    __shared__ double s_v[RG];
    __shared__ int s_last;
    const int n = st->cand_total;
    const int k1 = st->k;
    const int LG = (k1 + RG - 1) / RG;
    const long long pairs = (long long)n * LG;
    const int nch = pairs <= RPCAP ? RCH : 1;
    const long long items = pairs * nch;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long n2 = p.N >> 1;
    const long long per = (n2 + nch - 1) / nch;  // float4 slots per chunk
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const long long pr = it / nch;
        const int h = (int)(it % nch);
        const int c = (int)(pr / LG), g = (int)(pr % LG);
        const long long j = p.cand[c];
        const int l0 = g * RG;
        const int lstart = p.dcnt[j];
        const int la = l0 > lstart ? l0 : lstart;
        const int lb = l0 + RG < k1 ? l0 + RG : k1;
        if (la >= lb) {
            if (threadIdx.x == 0 && h == 0) p.pv[(long long)c * p.lgcap + g] = 0.0;
            continue;
        }
        const float4 *h4 = reinterpret_cast<const float4 *>(p.hi + j * p.ldH);
        const float4 *o4 = reinterpret_cast<const float4 *>(p.lo + j * p.ldH);
        const long long t_lo = (long long)h * per, t_hi = t_lo + per < n2 ? t_lo + per : n2;
        float rh[RG], rl[RG], ih[RG], il[RG], dr[RG], di[RG];
#pragma unroll
        for (int e = 0; e < RG; e++) rh[e] = rl[e] = ih[e] = il[e] = dr[e] = di[e] = 0.f;
        // the column's hi and lo are loaded RU slots at a time so that their
        // HBM latency overlaps; the basis rows come from L2
        constexpr int RU = 4;
        for (long long t0 = t_lo + threadIdx.x; t0 < t_hi; t0 += (long long)RU * blockDim.x) {
            float4 a[RU], b[RU];
#pragma unroll
            for (int u = 0; u < RU; u++) {
                const long long t = t0 + (long long)u * blockDim.x;
                a[u] = t < t_hi ? __ldg(h4 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
                b[u] = t < t_hi ? __ldg(o4 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int e = 0; e < RG; e++) {
                const int l = l0 + e;
                if (l >= la && l < lb) {
                    const float4 *qh4 = reinterpret_cast<const float4 *>(p.qh + (long long)l * p.qs_stride);
                    const float4 *ql4 = reinterpret_cast<const float4 *>(p.ql + (long long)l * p.qs_stride);
#pragma unroll
                    for (int u = 0; u < RU; u++) {
                        const long long t = t0 + (long long)u * blockDim.x;
                        if (t < t_hi) {
                            const float4 qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
                            df_mac1(rh[e], rl[e], qa.x, qb.x, a[u].x);
                            df_mac1(rh[e], rl[e], qa.y, qb.y, a[u].y);
                            df_mac1(rh[e], rl[e], qa.z, qb.z, a[u].z);
                            df_mac1(rh[e], rl[e], qa.w, qb.w, a[u].w);
                            df_mac1(ih[e], il[e], qa.x, qb.x, a[u].y);
                            df_mac1(ih[e], il[e], -qa.y, -qb.y, a[u].x);
                            df_mac1(ih[e], il[e], qa.z, qb.z, a[u].w);
                            df_mac1(ih[e], il[e], -qa.w, -qb.w, a[u].z);
                            dr[e] = fmaf(qa.x, b[u].x, fmaf(qa.y, b[u].y, fmaf(qa.z, b[u].z, fmaf(qa.w, b[u].w, dr[e]))));
                            di[e] = fmaf(qa.x, b[u].y, fmaf(-qa.y, b[u].x, fmaf(qa.z, b[u].w, fmaf(-qa.w, b[u].z, di[e]))));
                        }
                    }
                }
            }
        }
        if ((p.N & 1) && h == nch - 1 && threadIdx.x == 0) {
            const long long i = p.N - 1;
            const float2 a = p.hi[j * p.ldH + i], b = p.lo[j * p.ldH + i];
#pragma unroll
            for (int e = 0; e < RG; e++) {
                const int l = l0 + e;
                if (l >= la && l < lb) {
                    const float2 qa = p.qh[(long long)l * p.qs_stride + i], qb = p.ql[(long long)l * p.qs_stride + i];
                    df_mac1(rh[e], rl[e], qa.x, qb.x, a.x);
                    df_mac1(rh[e], rl[e], qa.y, qb.y, a.y);
                    df_mac1(ih[e], il[e], qa.x, qb.x, a.y);
                    df_mac1(ih[e], il[e], -qa.y, -qb.y, a.x);
                    dr[e] = fmaf(qa.x, b.x, fmaf(qa.y, b.y, dr[e]));
                    di[e] = fmaf(qa.x, b.y, fmaf(-qa.y, b.x, di[e]));
                }
            }
        }
#pragma unroll
        for (int e = 0; e < RG; e++) {
            warp_df_sum(rh[e], rl[e]);
            warp_df_sum(ih[e], il[e]);
            float x = dr[e], y = di[e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                y += __shfl_xor_sync(0xffffffffu, y, o);
            }
            if (lane == 0) {
                s_red[e][0][w] = (double)rh[e] + (double)rl[e];
                s_red[e][1][w] = (double)ih[e] + (double)il[e];
                s_red[e][2][w] = (double)x;
                s_red[e][3][w] = (double)y;
            }
        }
        __syncthreads();
        // this block's sums of the four parts per row (fixed warp order)
        if (threadIdx.x < 4 * RG) {
            const int e = threadIdx.x >> 2, q = threadIdx.x & 3;
            double a = 0.0;
            for (int x = 0; x < NW; x++) a += s_red[e][q][x];
            if (nch > 1) p.rpart[(pr * RCH + h) * (4 * RG) + threadIdx.x] = a;
            else s_red[e][q][0] = a;
        }
        if (nch > 1) {
            // the last chunk of this (candidate, group) adds the chunks in order
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                s_last = atomicAdd(p.rtick + pr, 1) == nch - 1;
            }
            __syncthreads();
            if (!s_last) continue;
            __threadfence();
            if (threadIdx.x < 4 * RG) {
                double a = 0.0;
                for (int x = 0; x < nch; x++) a += __ldcg(p.rpart + (pr * RCH + x) * (4 * RG) + threadIdx.x);
                s_red[threadIdx.x >> 2][threadIdx.x & 3][0] = a;
            }
            if (threadIdx.x == 0) p.rtick[pr] = 0;
        }
        __syncthreads();
        if (threadIdx.x < RG) {
            const int e = threadIdx.x, l = l0 + e;
            double v = 0.0;
            if (l >= la && l < lb) {
                // exact c = q^H hi + q^H lo; v = |c|^2 - |c~|^2 without cancellation
                const double xr = s_red[e][0][0] + s_red[e][2][0], xi = s_red[e][1][0] + s_red[e][3][0];
                const double2 ct = p.C[(long long)l * p.ldC + j];
                v = (xr - ct.x) * (xr + ct.x) + (xi - ct.y) * (xi + ct.y);
            }
            s_v[e] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sv = 0.0;
            for (int e = 0; e < RG; e++) sv += s_v[e];  // fixed order
            p.pv[(long long)c * p.lgcap + g] = sv;
        }
        __syncthreads();
    }
    if (!last_block(&st->ticket_aux)) return;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const long long j = __ldcg(p.cand + c);
        const int lstart = __ldcg(p.dcnt + j);
        double D = __ldcg(p.dacc + j);
        for (int g = lstart / RG; g < LG; g++) D += __ldcg(p.pv + (long long)c * p.lgcap + g);
        p.dacc[j] = D;
        p.dcnt[j] = k1;
        // err_j = ||s_j||^2 - sum_l |c_lj|^2 = norm2 - acc~ - D
        const double e = p.norm2[j] - p.acc[j] - D;
        p.cand_err[c] = e;
        if (better(e, j, be, bi)) { be = e; bi = j; }
    }
    block_best(be, bi);
    if (threadIdx.x == 0) {
        st->ticket_aux = 0;
        st->ncand = n;
        if (n > st->max_cand) st->max_cand = n;
        st->J = bi;
        st->errJ = be;
        p.err_curve[k1] = be;
        if (bi == kNoIdx || be < p.tol) st->switch_pending = 1;
    }
}

// ------------------------------------------------------- projection onto lo
// d = Qh^H lo for the k1 basis vectors on the tensor cores, then C[l, j] += d.
// As a real GEMM with K = 2N interleaved (re, im): A rows 2l = (a_i, b_i) and
// 2l+1 = (-b_i, a_i) for q_l = a + ib; B row j = (u_i, v_i) for lo_j = u + iv.
// Every FP32 value is split exactly into three BF16 pieces (x = x1 + x2 + x3);
// the six piece products with s + t <= 4 accumulate into one FP32 TMEM
// accumulator, which leaves a relative error of a few 2^-24 -- what d needs,
// since |lo| <= 2^-24 |s|.  Blocks loop over (row tile, column tile) pairs.
constexpr int PT = 128;  // tile rows (A) and columns (B)
constexpr int PKC = 32;  // K per stage
constexpr int PSL = 3;   // BF16 pieces per FP32 value

// x rounded to BF16 (nearest, ties to even), as the FP32 bit pattern with the
// low 16 bits cleared: BF16 is the top half of an FP32, so the rounding is an
// integer add and mask (finite x; conversion instructions run at a low rate on
// this GPU).
__device__ __forceinline__ uint32_t bf16_round_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
}

// Exact split x = x1 + x2 + x3 into BF16 pieces (each difference is exact in
// FP32); o[s] = the FP32 bit pattern of piece s (its BF16 value in the top half).
__device__ __forceinline__ void split3_bits(float x, uint32_t o[PSL]) {
    o[0] = bf16_round_bits(x);
    const float r = x - __uint_as_float(o[0]);
    o[1] = bf16_round_bits(r);
    o[2] = bf16_round_bits(r - __uint_as_float(o[1]));
}

// Stage 8 consecutive K entries (4 complex elements) of one tile row into the
// three piece tiles: one 16-byte core-matrix row per piece.
__device__ __forceinline__ void stage_row8(uint8_t *base, int r, int kk, const float v[8]) {
    uint32_t pc[PSL][8];
#pragma unroll
    for (int e = 0; e < 8; e++) {
        uint32_t o[PSL];
        split3_bits(v[e], o);
#pragma unroll
        for (int s = 0; s < PSL; s++) pc[s][e] = o[s];
    }
#pragma unroll
    for (int s = 0; s < PSL; s++) {
        // pairs of BF16 values: element 2i in the low half of word i
        const uint4 w = make_uint4(__byte_perm(pc[s][0], pc[s][1], 0x7632), __byte_perm(pc[s][2], pc[s][3], 0x7632),
                                   __byte_perm(pc[s][4], pc[s][5], 0x7632), __byte_perm(pc[s][6], pc[s][7], 0x7632));
        *(uint4 *)(base + s * (PT * PKC * 2) + kmajor_off(r, kk, PKC)) = w;
    }
}

// A operand pieces, built once when the loop ends: for row tile rt and K
// stage st the three BF16 piece tiles lie contiguously (48 KB) in the layout
// the MMA reads, so a block stages them with plain 16-byte copies.
constexpr int PTILE = PSL * PT * PKC * 2;  // bytes of one stage's three piece tiles

__global__ void __launch_bounds__(kThreads) k_qpieces(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    const int nrt = (2 * k1 + PT - 1) / PT;
    const long long nstg = (2 * p.N + PKC - 1) / PKC;
    const long long units = (long long)nrt * nstg * PT * (PKC / 8);
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        const long long ts = u / (PT * (PKC / 8));  // (rt, stage) index = rt * nstg + stage
        const int w = (int)(u % (PT * (PKC / 8)));
        const int r = w / (PKC / 8), kk = (w % (PKC / 8)) * 8;
        const int rt = (int)(ts / nstg);
        const long long stg = ts % nstg;
        const int gr = rt * PT + r;
        float v[8];
        const long long i0 = (stg * PKC + kk) >> 1;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const long long i = i0 + e;
            const float2 q = (gr < 2 * k1 && i < p.N) ? p.qh[(long long)(gr >> 1) * p.qs_stride + i] : make_float2(0.f, 0.f);
            if ((gr & 1) == 0) { v[2 * e] = q.x; v[2 * e + 1] = q.y; }
            else { v[2 * e] = -q.y; v[2 * e + 1] = q.x; }
        }
        stage_row8(p.apieces + ts * PTILE, r, kk, v);
    }
}

// One stage of B (lo columns j0..j0+127, K entries [64 stg, +64)) into
// registers: thread t holds units t + u * kThreads, each 8 K entries.
constexpr int PBU = PT * (PKC / 8) / kThreads;

// Unit t -> (row r, first K entry kk) such that the 8 threads of each quarter
// warp store the 8 rows of one core matrix (128 contiguous bytes: no bank
// conflicts), while each warp still reads whole 128-byte runs of lo.
__device__ __forceinline__ void proj_unit(int t, int &r, int &kk) {
    r = (t & 7) + 8 * (t / (8 * (PKC / 8)));
    kk = ((t >> 3) % (PKC / 8)) * 8;
}

__device__ __forceinline__ void proj_load_b(const Prob &p, long long j0, long long stg, float4 bx[PBU], float4 by[PBU]) {
#pragma unroll
    for (int u = 0; u < PBU; u++) {
        const int t = threadIdx.x + u * kThreads;
        int r, kk;
        proj_unit(t, r, kk);
        const long long j = j0 + r;
        const long long i0 = (stg * PKC + kk) >> 1;  // a multiple of 4
        if (j < p.M && i0 + 3 < p.N) {
            const float4 *l4 = reinterpret_cast<const float4 *>(p.lo + j * p.ldH + i0);
            bx[u] = ld_stream(l4);
            by[u] = ld_stream(l4 + 1);
        } else {
            float v[8];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const long long i = i0 + e;
                const float2 x = (j < p.M && i < p.N) ? p.lo[j * p.ldH + i] : make_float2(0.f, 0.f);
                v[2 * e] = x.x;
                v[2 * e + 1] = x.y;
            }
            bx[u] = make_float4(v[0], v[1], v[2], v[3]);
            by[u] = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
}

__device__ __forceinline__ void proj_store_b(uint8_t *sB, const float4 bx[PBU], const float4 by[PBU]) {
#pragma unroll
    for (int u = 0; u < PBU; u++) {
        const int t = threadIdx.x + u * kThreads;
        int r, kk;
        proj_unit(t, r, kk);
        const float v[8] = {bx[u].x, bx[u].y, bx[u].z, bx[u].w, by[u].x, by[u].y, by[u].z, by[u].w};
        stage_row8(sB, r, kk, v);
    }
}

// d = Qh^H lo on the tensor cores, C += d.  One block per SM (persistent over
// tiles), warp-specialised around a ring of LP_NBUF stage buffers (A pieces,
// then B pieces):
//   warps 0-7 (producers) convert the lo values of stage s (loaded into
//     registers LP_AHEAD stages earlier) into the B pieces of buffer s % LP_NBUF
//     once the MMAs of stage s - LP_NBUF are done, then arrive on bfull;
//   warp 8, lane 0 waits for the A bytes (afull) and the B pieces (bfull) of
//     stage s, issues its MMAs, commits them to done, and bulk-copies the A
//     pieces of stage s + LP_NBUF - 1 into the buffer of stage s - 1 once the
//     MMAs of stage s - 1 are done;
//   warps 0-3 (TMEM lanes 0-127) run the epilogue of each tile.
// Barrier phases follow a running stage count g over all tiles of the block:
// buffer g % LP_NBUF, phase (g / LP_NBUF) & 1.  No role can run a full ring
// ahead of another (each refill waits for the MMAs that emptied the buffer),
// so no wait can be two phases behind.
constexpr int LP_NBUF = 4;
constexpr int LP_AHEAD = 4;                    // stages of lo loaded ahead into registers
constexpr int LP_PRODUCERS = kThreads;         // 256 converting threads
constexpr int LP_THREADS = kThreads + 32;      // + the MMA warp

__global__ void __launch_bounds__(LP_THREADS) k_lo_project_tc(Prob p, int *err) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    const int nrt = (2 * k1 + PT - 1) / PT;
    const long long nct = (p.M + PT - 1) / PT;
    const long long ntiles = (long long)nrt * nct;
    if (k1 <= 0 || (long long)blockIdx.x >= ntiles) return;
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t afull[LP_NBUF], bfull[LP_NBUF], done[LP_NBUF];
    __shared__ uint32_t tslot;
    __shared__ int s_bad;
    const int warp = threadIdx.x >> 5;
    const bool producer = threadIdx.x < LP_PRODUCERS;
    const bool issuer = threadIdx.x == LP_PRODUCERS;  // lane 0 of warp 8
    if (warp == 0) tmem_alloc(&tslot, PT);
    if (threadIdx.x == 0) {
        s_bad = 0;
        for (int b = 0; b < LP_NBUF; b++) {
            mbar_init(&afull[b], 1);
            mbar_init(&bfull[b], LP_PRODUCERS);  // one arrive per producer thread
            mbar_init(&done[b], 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(PT, PT);
    const long long nstg = (2 * p.N + PKC - 1) / PKC;
    bool ok = true;
    long long gs = 0;  // stages run by this block so far (all tiles)
    auto bufA = [&](long long g) { return dsm + (int)(g % LP_NBUF) * 2 * PTILE; };
    auto par = [&](long long g) { return (uint32_t)((g / LP_NBUF) & 1); };
    float4 bx0[PBU], by0[PBU], bx1[PBU], by1[PBU], bx2[PBU], by2[PBU], bx3[PBU], by3[PBU];
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int rt = (int)(tile % nrt);
        const long long j0 = (tile / nrt) * PT;
        const uint8_t *ga = p.apieces + (long long)rt * nstg * PTILE;
        const long long g0 = gs;
        if (producer) {
            // register sets: stage s uses set s % 4
            proj_load_b(p, j0, 0, bx0, by0);
            if (nstg > 1) proj_load_b(p, j0, 1, bx1, by1);
            if (nstg > 2) proj_load_b(p, j0, 2, bx2, by2);
            if (nstg > 3) proj_load_b(p, j0, 3, bx3, by3);
            auto produce = [&](long long s, float4 (&BX)[PBU], float4 (&BY)[PBU]) {
                const long long g = g0 + s;
                if (g >= LP_NBUF) ok = mbar_wait(&done[g % LP_NBUF], par(g - LP_NBUF), p.wait_cycles) && ok;
                proj_store_b(bufA(g) + PTILE, BX, BY);
                if (s + LP_AHEAD < nstg) proj_load_b(p, j0, s + LP_AHEAD, BX, BY);
                // each thread makes its own stores visible to the tensor core
                // (async proxy), then arrives
                fence_async_smem();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull[g % LP_NBUF])) : "memory");
            };
            for (long long s = 0; s < nstg; s += 4) {
                produce(s, bx0, by0);
                if (s + 1 < nstg) produce(s + 1, bx1, by1);
                if (s + 2 < nstg) produce(s + 2, bx2, by2);
                if (s + 3 < nstg) produce(s + 3, bx3, by3);
            }
        } else if (issuer) {
            auto load_a = [&](long long s) {
                uint64_t *fb = &afull[(g0 + s) % LP_NBUF];
                mbar_expect_tx(fb, PTILE);
                bulk_g2s(bufA(g0 + s), ga + s * PTILE, PTILE, fb);
            };
            // the first LP_NBUF - 1 stages: their buffers' MMAs (previous tile)
            // are complete
            for (long long s = 0; s < LP_NBUF - 1 && s < nstg; s++) load_a(s);
            for (long long s = 0; s < nstg; s++) {
                const long long g = g0 + s;
                const int b = (int)(g % LP_NBUF);
                ok = mbar_wait(&afull[b], par(g), p.wait_cycles) && ok;
                ok = mbar_wait(&bfull[b], par(g), p.wait_cycles) && ok;
                tc_fence_after();
                const uint64_t ad0 = smem_desc(smem_u32(bufA(g)), 128, (PKC / 8) * 128);
                const uint64_t bd0 = smem_desc(smem_u32(bufA(g) + PTILE), 128, (PKC / 8) * 128);
                bool first = true;
#pragma unroll
                for (int sa = 0; sa < PSL; sa++)
#pragma unroll
                    for (int sb = 0; sb < PSL; sb++) {
                        if (sa + sb > 2) continue;  // pieces s + t <= 4 (0-based sa + sb <= 2)
#pragma unroll
                        for (int kk = 0; kk < PKC / 16; kk++) {
                            const uint64_t ad = ad0 + (uint64_t)((sa * (PT * PKC * 2) + kk * 256) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((sb * (PT * PKC * 2) + kk * 256) >> 4);
                            tc_mma_bf16(tmem, ad, bd, idesc, (s > 0 || !first) ? 1u : 0u);
                            first = false;
                        }
                    }
                tc_commit(&done[b]);
                // A of stage s + LP_NBUF - 1 into the buffer of stage s - 1
                if (s + LP_NBUF - 1 < nstg) {
                    if (s >= 1) ok = mbar_wait(&done[(g - 1) % LP_NBUF], par(g - 1), p.wait_cycles) && ok;
                    load_a(s + LP_NBUF - 1);
                }
            }
        }
        gs = g0 + nstg;
        // every thread: the tile's last MMAs (the latest phase of that barrier)
        ok = mbar_wait(&done[(gs - 1) % LP_NBUF], par(gs - 1), p.wait_cycles) && ok;
        tc_fence_after();
        // epilogue: thread = A row (TMEM lane); row 2l adds to Re C[l, j], row 2l+1 to Im
        if (warp < 4) {
            const int r = rt * PT + threadIdx.x;
            for (int c0 = 0; c0 < PT; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                if (r < 2 * k1 && ok) {
                    double *crow = (double *)(p.C + (long long)(r >> 1) * p.ldC) + (r & 1);
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const long long j = j0 + c0 + e;
                        if (j < p.M) crow[2 * j] += (double)v[e];
                    }
                }
            }
        }
        if (!ok) s_bad = 1;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s_bad) break;
    }
    if (s_bad && threadIdx.x == 0) atomicExch(err, 1);
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, PT);
}

// acc_j = sum_l |C[l, j]|^2 after the projection onto lo, the final argmax and
// the stopping status.
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
        st->status = (bi != kNoIdx && !(emax < p.tol) && !st->force_stop && k1 >= p.kmax && k1 < p.minNM)
                         ? RB_KMAX_REACHED
                         : RB_OK;
        st->stop = 1;
    }
}

cudaError_t launch_split_init(const Prob &p, cudaStream_t s) {
    long long g = (p.M * 32 + kThreads - 1) / kThreads;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    k_split_init<<<(int)g, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

// Blocks of a persistent launch: SMs times the resident blocks per SM, so no
// block waits for a second wave (grid-stride loops assign work statically).
template <typename K>
static int resident_grid(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    return sms * (per > 0 ? per : 1);
}

cudaError_t launch_split_iteration(const Prob &p, int grid, cudaStream_t s, int *nlaunch) {
    static int g_sweep = 0, g_re = 0;
    if (!g_sweep) g_sweep = resident_grid(k_sweep_hi, kThreads, 0);
    if (!g_re) g_re = resident_grid(k_recheck, kThreads, 0);
    (void)grid;
    k_sweep_hi<<<g_sweep, kThreads, 0, s>>>(p);
    k_bounds<<<p.nblk_cand, kThreads, 0, s>>>(p);
    k_cand_count<<<p.nblk_cand, kThreads, 0, s>>>(p);
    k_cand_write<<<p.nblk_cand, kThreads, 0, s>>>(p);
    k_recheck<<<g_re, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 5;
    return cudaGetLastError();
}

// Queued after every iteration; both kernels return at once unless the loop
// has just ended.
size_t lo_pieces_bytes(long long N, int kcap) {
    const long long nrt = (2LL * kcap + PT - 1) / PT, nstg = (2 * N + PKC - 1) / PKC;
    return (size_t)nrt * (size_t)nstg * PTILE;
}

cudaError_t launch_split_finish(const Prob &p, int grid, cudaStream_t s, int *nlaunch) {
    const size_t dsmem = (size_t)LP_NBUF * 2 * PTILE;  // 192 KB
    static int g_proj = 0;
    if (!g_proj) {
        cudaFuncSetAttribute(k_lo_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
        cudaFuncSetAttribute(k_lo_project_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        // one block per SM (144 KB ring)
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_proj = sms;
    }
    k_qpieces<<<grid, kThreads, 0, s>>>(p);
    k_lo_project_tc<<<g_proj, LP_THREADS, dsmem, s>>>(p, p.tc_err);
    long long rf = (p.M + kThreads - 1) / kThreads;
    if (rf > grid) rf = grid;
    k_rebase_finish<<<(int)rf, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 3;
    return cudaGetLastError();
}

}  // namespace rbk
