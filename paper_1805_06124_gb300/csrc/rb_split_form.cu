// rb_split_form.cu -- the split-precision form of the greedy sweep.
//
// S is stored as complex64 hi + lo (hi = fl32(s), lo = fl32(s - hi)).  Every
// sweep of the hi-only phase reads hi only (8 bytes per element); lo is read
// for the candidate columns of the exact re-check and once by the projection
// of the basis onto lo (at the switch or at the end).
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
// Switch.  When more columns are candidates than the switch count (the
// bounds no longer separate them), or every error is certified below
// switch_err * max ||s_j||^2, the basis so far is projected onto lo on the
// tensor cores (C += Q^H lo), acc is rebuilt from the now exact C, and every
// later sweep is the FP64 form's double-float sweep over hi + lo (k_sweep in
// rb_sweep.cu, gated on the phase).
//
// End.  When every upper bound is below tol (or the exact pivot error is, or
// kmax is reached) in the hi-only phase, the basis is projected onto lo the
// same way and the final errors and argmax are taken from C.
#include "rb_internal.cuh"
#include "rb_tc.cuh"

namespace rbk {

// Rounding allowance of the FP32 chain norms (sums of at most 2^16 squares).
constexpr float kNormUp = 1.001f;

// An upper bound of sqrt(x) for x >= 0 from the FP32 square root: x rounded
// up to FP32, the correctly rounded sqrtf (within half an ulp), and a factor
// 1 + 2^-22 that covers that half ulp and the rounding of the product.  It
// only scales the small terms of the bounds, so FP32 accuracy is ample, and
// it keeps the FP64 square roots (long sequences on this GPU's FP64 pipe) out
// of the per-column work.  x beyond the FP32 range gives +inf (a looser,
// still valid bound).
__device__ __forceinline__ double sqrt_up(double x) {
    return (double)(sqrtf(__double2float_ru(x)) * 1.0000002384185791f);
}

// Certified bounds of the true error from the hi-only bookkeeping.
//   e   = ||hi_j||^2 - acc~_j          ln  = ||lo_j|| (rounded up)
//   Ec  = bound on |err(hi_j) - e|     n2  = ||s_j||^2 (FP64 bookkeeping slack)
__device__ __forceinline__ void split_bounds(double e, double Ec, float lonrm, double n2, int k, double &U,
                                             double &L) {
    const double ln = (double)lonrm;
    const double ehi_up = e + Ec > 0.0 ? e + Ec : 0.0;
    const double r = sqrt_up(ehi_up);
    const double slack = 8.0 * (k + 16) * 1.1102230246251565e-16 * n2;
    U = ehi_up + 2.0 * r * ln + ln * ln + slack;
    L = e - Ec - 2.0 * r * ln - slack;
}

__device__ __forceinline__ double ec_of(double eta, double nh2, double sabs, int k1) {
    return 2.0 * eta * sqrt_up(nh2) * sabs + 3.0 * k1 * eta * eta * nh2;
}

__device__ __forceinline__ double col_ec(const Prob &p, long long j, int k1) {
    return ec_of(p.eta, p.norm2_hi[j], p.sabs[j], k1);
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
        auto slot = [&](const float4 &x, const float4 &y) {
            norm2_acc4(a, x, y);
            df_mac(bh, bl, x.x, 0.f, x.x, 0.f);
            df_mac(bh, bl, x.y, 0.f, x.y, 0.f);
            df_mac(bh, bl, x.z, 0.f, x.z, 0.f);
            df_mac(bh, bl, x.w, 0.f, x.w, 0.f);
            c0 = fmaf(x.x, x.x, fmaf(x.y, x.y, c0));
            c1 = fmaf(x.z, x.z, fmaf(x.w, x.w, c1));
        };
        // U slots of hi and lo in flight per lane; each lane still takes its
        // slots in increasing order
        constexpr int U = 4;
        long long t = lane;
        for (; t + 32 * (U - 1) < n2; t += 32 * U) {
            float4 x[U], y[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                x[u] = ld_stream(h4 + t + 32 * u);
                y[u] = ld_stream(l4 + t + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < U; u++) slot(x[u], y[u]);
        }
        for (; t < n2; t += 32) slot(ld_stream(h4 + t), ld_stream(l4 + t));
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

// The hi-only phase is running (no projection onto lo queued, no switch yet).
__device__ __forceinline__ bool loop_active(const DevState *st) {
    return !ld_volatile(&st->stop) && !ld_volatile(&st->switch_pending) && !ld_volatile(&st->phase);
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
        } else if (gu < p.switch_err * p.err_curve[0]) {
            // every error is certified below switch_err * max ||s_j||^2: switch to hi + lo sweeps
            st->switch_pending = 2;
            st->ncand = 0;
        } else {
            st->ncand = -1;  // re-check needed
            st->cand_total = 0;
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

// The candidate list: every unpicked column whose upper bound reaches the
// largest lower bound, gathered with one atomic per warp.  The order of the
// list does not matter: each candidate's re-check is its own and the exact
// argmax breaks ties by column index.  The last block applies the switch rule
// on the count.
__global__ void __launch_bounds__(kThreads) k_cand(Prob p) {
    DevState *st = p.st;
    if (!recheck_active(st)) return;
    const int k1 = st->k;
    const double Lmax = st->Lmax;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j0 = blockIdx.x * (long long)blockDim.x + threadIdx.x - lane; j0 < p.M; j0 += stride) {
        const long long j = j0 + lane;
        const bool c = j < p.M && is_candidate(p, j, k1, Lmax);
        const unsigned m = __ballot_sync(0xffffffffu, c);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&st->cand_total, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (c) p.cand[base + __popc(m & ((1u << lane) - 1u))] = j;
        }
    }
    if (!last_block(&st->ticket_aux)) return;
    if (threadIdx.x == 0) {
        st->ticket_aux = 0;
        if (ld_volatile(&st->cand_total) > p.switch_cand) {
            // the bounds no longer separate the columns: re-checking this many
            // would cost more than sweeping hi + lo, so switch instead
            st->switch_pending = 2;
            st->ncand = 0;
        }
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
// Every FP32 value is scaled by a power of two (per basis vector for A, per
// column for B, so that the largest scaled magnitude is at most 2^14) and
// split into two FP16 pieces: hi = the value with its low 13 mantissa bits
// cleared, lo = the exact remainder (|lo| < 2^-10 |x|) rounded to FP16
// (lp_enc2).  The three products hiA hiB + hiA loB + loA hiB accumulate in
// one FP32 TMEM accumulator; the dropped loA loB and the rounding of the lo
// pieces leave a relative error below 2^-19 per product, i.e. below
// 2^-43 ||s_j|| on d since |lo_j| <= 2^-24 |s_j|.  The epilogue undoes the
// two scales exactly.  Tiles are LT_M = 128 rows of A by nt <= 128 columns of
// lo, stages of LKC = 64 K entries; blocks loop over (row tile, column tile)
// pairs.
constexpr int LT_M = 128;      // A rows per tile
constexpr int LT_NMAX = 128;   // lo columns per tile (at most)
constexpr int LKC = 64;        // K entries per stage (32 complex elements, 256 bytes of lo per column)
constexpr int LA_PIECE = LT_M * LKC * 2;       // bytes of one FP16 piece of an A stage (16 KB)
constexpr int LA_STAGE = 2 * LA_PIECE;         // both pieces (32 KB)
// B pieces in shared memory: the K-major no-swizzle canonical layout with the
// core matrices (8 rows x 16 bytes) of one 8-row group LB_LBO = 144 bytes
// apart along K (128 + 16: consecutive K core matrices of a row fall in
// different banks) and 8-row groups LB_SBO = 4 x 144 bytes apart; the lo
// piece starts 64 bytes (mod 128) after the hi piece.  A row's 4 hi and 4 lo
// 16-byte pieces then cover all 8 bank groups (see lp_store).
constexpr int LB_LBO = 144;
constexpr int LB_SBO = (LKC / 8) * LB_LBO;       // 1152
constexpr int LB_PIECE = (LT_NMAX / 8) * LB_SBO;  // one FP16 piece of a B stage (18 KB)
constexpr int LB_LO = LB_PIECE + 64;              // offset of the lo piece
constexpr int LSTAGE = LA_STAGE + LB_LO + LB_PIECE;  // one ring buffer (68 KB + 64 B)
static_assert(LSTAGE % 16 == 0 && LB_LO % 128 == 64, "B layout");

__device__ __forceinline__ uint32_t lb_off(int r, int k) {
    return (uint32_t)((r >> 3) * LB_SBO + (k >> 3) * LB_LBO + (r & 7) * 16 + (k & 7) * 2);
}

// Power-of-two exponent e with 2^e * x_max <= 2^14 for x_max > 0 (0 for
// x_max == 0), clamped so that 2^e is a normal FP32 number.
__device__ __forceinline__ int lp_scale_exp(float xmax) {
    const uint32_t b = __float_as_uint(xmax) & 0x7FFFFFFFu;
    if (b == 0u) return 0;
    int e = (int)(b >> 23) - 127;  // xmax in [2^e, 2^(e+1)) (normal); subnormal -> -127
    if (b & 0x007FFFFFu) e += 1;   // ceil(log2(xmax))
    int s = 14 - e;
    return s > 126 ? 126 : (s < -126 ? -126 : s);
}

__device__ __forceinline__ float lp_pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Two FP16 pieces of a pair of values y = x * f (|y| < 2^15): hi = y with
// its low 13 mantissa bits cleared (on the FP16 grid on the FP16 normal
// range, so its conversion is exact there), lo = the exact remainder y - hi
// rounded to FP16; each pair is converted by one packed conversion (element
// a in the low half).  |y - hi - lo| <= 2^-21 |y| on the FP16 normal range and
// below 2^-24 absolutely under it.
__device__ __forceinline__ void lp_enc2(float a, float b, float f, uint32_t &hw, uint32_t &lw) {
    const float ya = __fmul_rn(a, f), yb = __fmul_rn(b, f);
    const float ta = __uint_as_float(__float_as_uint(ya) & 0xFFFFE000u);
    const float tb = __uint_as_float(__float_as_uint(yb) & 0xFFFFE000u);
    const __half2 h = __floats2half2_rn(ta, tb);
    const __half2 l = __floats2half2_rn(__fsub_rn(ya, ta), __fsub_rn(yb, tb));
    hw = *reinterpret_cast<const uint32_t *>(&h);
    lw = *reinterpret_cast<const uint32_t *>(&l);
}

// Per basis vector l < k1: sa[l] = lp_scale_exp(max_i max(|Re qh_i|, |Im qh_i|)).
__global__ void __launch_bounds__(kThreads) k_qscale(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    __shared__ float s_m[kThreads / 32];
    for (int l = blockIdx.x; l < k1; l += gridDim.x) {
        const float2 *q = p.qh + (long long)l * p.qs_stride;
        float m = 0.f;
        for (long long i = threadIdx.x; i < p.N; i += blockDim.x) {
            const float2 v = q[i];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float x = 0.f;
            for (int w = 0; w < kThreads / 32; w++) x = fmaxf(x, s_m[w]);
            p.qscale[l] = lp_scale_exp(x);
        }
        __syncthreads();
    }
}

// A operand pieces, built once when the loop ends: for row tile rt and stage
// stg the two FP16 piece tiles (K-major canonical layout) lie contiguously
// (16 KB) at apieces + (rt * nstg + stg) * LA_STAGE, so a block stages them
// with one bulk copy.  Rows 2 k1 .. and K entries beyond 2N are zero.
__global__ void __launch_bounds__(kThreads) k_qpieces(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    const int nrt = (2 * k1 + LT_M - 1) / LT_M;
    const long long nstg = (2 * p.N + LKC - 1) / LKC;
    const long long units = (long long)nrt * nstg * LT_M * (LKC / 8);
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)gridDim.x * blockDim.x) {
        const long long ts = u / (LT_M * (LKC / 8));  // rt * nstg + stg
        const int w = (int)(u % (LT_M * (LKC / 8)));
        const int r = w / (LKC / 8), kk = (w % (LKC / 8)) * 8;
        const int rt = (int)(ts / nstg);
        const long long stg = ts % nstg;
        const int gr = rt * LT_M + r;
        const int l = gr >> 1;
        const float f = gr < 2 * k1 ? lp_pow2f(p.qscale[l]) : 0.f;
        const long long i0 = (stg * LKC + kk) >> 1;
        uint32_t hp[4], lp[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const long long i = i0 + e;
            const float2 q = (gr < 2 * k1 && i < p.N) ? p.qh[(long long)l * p.qs_stride + i] : make_float2(0.f, 0.f);
            const float x0 = (gr & 1) == 0 ? q.x : -q.y;
            const float x1 = (gr & 1) == 0 ? q.y : q.x;
            lp_enc2(x0, x1, f, hp[e], lp[e]);
        }
        uint8_t *base = p.apieces + ts * LA_STAGE + kmajor_off(r, kk, LKC);
        *(uint4 *)base = make_uint4(hp[0], hp[1], hp[2], hp[3]);
        *(uint4 *)(base + LA_PIECE) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
    }
}

// Producer side of one stage: warp w (of LP_PWARPS) handles the column
// groups g = w + LP_PWARPS x (x < LP_GROUPS, g < nt / 4) of 4 columns.  Lane
// L takes column 4 g + (L >> 3) and, per instruction i < LP_CH, the 16-byte
// chunk q = (L & 7) + 8 i of the column's LKC / 16 chunks (2 complex elements
// = K entries 4q .. 4q+3): each warp load reads whole 128-byte lines of 4
// columns.
constexpr int LP_PWARPS = 16;                       // producer warps
constexpr int LP_GROUPS = LT_NMAX / 4 / LP_PWARPS;  // column groups per producer warp
constexpr int LP_CH = LKC / 32;                     // 16-byte chunks per lane, column and stage
struct LpRegs {
    float4 v[LP_GROUPS][LP_CH];
};

// What a producer lane needs per tile, computed once.  A lane's columns are
// j0 + 4 w + (L >> 3) + 64 x: consecutive groups are 64 columns apart, so
// the tile state is one base pointer, a validity mask, the scales and one
// store offset (group x adds 8 row groups, chunk set i adds 4 core columns).
struct LpTile {
    const float4 *base;  // chunk (L & 7) of the lane's first column (x = 0)
    unsigned valid;      // bit x: group x in range
    float f[LP_GROUPS];
    uint32_t doff;       // store offset of group 0, chunk set 0
};

__device__ __forceinline__ void lp_tile(const Prob &p, long long j0, int nt, LpTile &T) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool even = (lane & 1) == 0;
    const int r0 = 4 * w + (lane >> 3);
    T.base = reinterpret_cast<const float4 *>(p.lo + (j0 + r0) * p.ldH) + (lane & 7);
    T.valid = 0u;
#pragma unroll
    for (int x = 0; x < LP_GROUPS; x++) {
        const int g = w + LP_PWARPS * x;
        const long long j = j0 + 4 * g + (lane >> 3);
        const bool ok = 4 * g < nt && j < p.M;
        if (ok) T.valid |= 1u << x;
        T.f[x] = ok ? lp_pow2f(lp_scale_exp(p.lonrm[j])) : 0.f;
    }
    T.doff = (even ? 0u : (uint32_t)LB_LO) + lb_off(r0, 8 * ((lane & 7) >> 1));
}

// Stage stg of this lane's columns: chunks (lane & 7) + 8 i of each, i.e.
// complex elements (LKC / 2) stg + 2 ((lane & 7) + 8 i) + {0, 1}; stages below
// nfull (= N / (LKC / 2)) lie wholly inside the columns.
__device__ __forceinline__ void lp_load(const Prob &p, const LpTile &T, long long stg, long long nfull, LpRegs &R) {
    const int lane = threadIdx.x & 31;
    const long long gstride = 64 * (p.ldH >> 1);  // float4 between a lane's groups
    if (stg < nfull && T.valid == (1u << LP_GROUPS) - 1u) {
        // the common case: a whole stage of full column groups, no tests
#pragma unroll
        for (int x = 0; x < LP_GROUPS; x++)
#pragma unroll
            for (int i = 0; i < LP_CH; i++) R.v[x][i] = ld_stream(T.base + x * gstride + stg * (LKC / 4) + 8 * i);
        return;
    }
#pragma unroll
    for (int x = 0; x < LP_GROUPS; x++) {
#pragma unroll
        for (int i = 0; i < LP_CH; i++) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (T.valid & (1u << x)) {
                const float4 *src = T.base + x * gstride + stg * (LKC / 4) + 8 * i;
                if (stg < nfull) {
                    v = ld_stream(src);
                } else {
                    const long long e0 = stg * (LKC / 2) + 2 * ((lane & 7) + 8 * i);
                    if (e0 + 1 < p.N) {
                        v = ld_stream(src);
                    } else if (e0 < p.N) {
                        const float2 a = *reinterpret_cast<const float2 *>(src);
                        v = make_float4(a.x, a.y, 0.f, 0.f);
                    }
                }
            }
            R.v[x][i] = v;
        }
    }
}

// L2 prefetch of this lane's lines of stage stg, by the lanes that start a
// 128-byte line ((lane & 7) == 0), for stages wholly inside the columns: the
// loads into registers (one stage ahead) then find their lines in L2, so the
// DRAM reads in flight do not depend on registers.
constexpr int LP_PF = 4;  // stages of lo prefetched into L2 ahead
__device__ __forceinline__ void lp_prefetch(const Prob &p, const LpTile &T, long long stg, long long nfull) {
    const int lane = threadIdx.x & 31;
    if (stg >= nfull) return;  // warp-uniform
    const long long gstride = 64 * (p.ldH >> 1);
    // one lane in eight issues it, by predicate rather than a branch (no divergence)
    const uint32_t lead = (lane & 7) == 0 ? 1u : 0u;
#pragma unroll
    for (int x = 0; x < LP_GROUPS; x++) {
        const uint32_t on = lead & (T.valid >> x);
#pragma unroll
        for (int i = 0; i < LP_CH; i++)
            asm volatile("{\n.reg .pred q;\nsetp.ne.u32 q, %1, 0;\n@q prefetch.global.L2 [%0];\n}\n" ::"l"(
                             T.base + x * gstride + stg * (LKC / 4) + 8 * i),
                         "r"(on & 1u));
    }
}

// Converts the stage held in R into the two B piece tiles of the buffer at
// sB: lanes L and L^1 hold the two halves (4 K entries each) of one 16-byte
// core-matrix row of column 4 g + (L >> 3); the lane with the lower half
// stores the hi row, its partner the lo row.  The 8 lanes of a quarter warp
// (one column, four core columns, both pieces) hit 8 different bank groups
// in the padded layout (lb_off, LB_LO).
__device__ __forceinline__ void lp_store(int nt, const LpTile &T, const LpRegs &R, uint8_t *sB) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool even = (lane & 1) == 0;
#pragma unroll
    for (int x = 0; x < LP_GROUPS; x++) {
        const int g = w + LP_PWARPS * x;
        if (4 * g >= nt) continue;  // warp-uniform
        const float f = T.f[x];
#pragma unroll
        for (int i = 0; i < LP_CH; i++) {
            const float4 v = R.v[x][i];
            const uint32_t doff = T.doff + (uint32_t)(x * 8 * LB_SBO + i * 4 * LB_LBO);
            uint32_t ha, la, hb, lb;
            lp_enc2(v.x, v.y, f, ha, la);
            lp_enc2(v.z, v.w, f, hb, lb);
            // the even lane keeps its hi half and receives the odd lane's hi
            // half; the odd lane keeps its lo half and receives the even lane's
            const uint32_t sa = even ? la : ha, sb = even ? lb : hb;
            const uint32_t ra = __shfl_xor_sync(0xffffffffu, sa, 1);
            const uint32_t rb = __shfl_xor_sync(0xffffffffu, sb, 1);
            *(uint4 *)(sB + doff) = even ? make_uint4(ha, hb, ra, rb) : make_uint4(ra, rb, la, lb);
        }
    }
}

// d = Qh^H lo on the tensor cores, C += d.  One block per SM (persistent over
// tiles of LT_M rows by nt columns), warp-specialised around a ring of
// LP_NBUF stage buffers (A pieces, then B pieces), one mbarrier pair per
// buffer:
//   warps 0-15 (producers), for stage s: issue the lo loads of stage
//     s + LP_AHEAD into the register set freed by stage s - 1; wait (one lane
//     per warp) until the MMAs of stage s - LP_NBUF are done (done); convert
//     the lo values into the B pieces, fence them for the tensor core and
//     arrive on bfull (one arrive per warp);
//   warp 17, lane 0, for stage s: waits for the same done, arrives on bfull
//     announcing the A bytes (so the phase needs them) and bulk-copies the
//     A pieces of stage s into the buffer;
//   warp 16, lane 0 waits for bfull of stage s (17 arrivals and the A bytes),
//     issues the stage's MMAs and commits them to done;
//   warps 0-15 run the epilogue of each tile (TMEM lanes 32 (w % 4) .., the
//     column quarter w / 4).
// Barrier phases follow a running stage count g over all tiles of the block:
// buffer g % LP_NBUF, phase (g / LP_NBUF) & 1.  The producers refill a buffer
// only after its MMAs are done and the MMAs of a stage need its bfull, so no
// role runs a full ring ahead of the other and no wait is two phases behind.
// Every wait is bounded (p.wait_cycles); a wait that runs out marks the block
// bad, which skips the epilogue and the later tiles and sets *err.
constexpr int LP_NBUF = 3;
constexpr int LP_SETS = 2;                     // register sets of lo stages per producer lane
constexpr int LP_AHEAD = LP_SETS - 1;          // stages of lo loaded ahead into registers
constexpr int LP_PRODUCERS = 32 * LP_PWARPS;   // 512 converting threads
constexpr int LP_THREADS = LP_PRODUCERS + 64;  // + the MMA warp + the A-copy warp

__global__ void __launch_bounds__(LP_THREADS, 1) k_lo_project_tc(Prob p, int nt, int *err) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    const int nrt = (2 * k1 + LT_M - 1) / LT_M;
    const long long nct = (p.M + nt - 1) / nt;
    const long long ntiles = (long long)nrt * nct;
    if (k1 <= 0 || (long long)blockIdx.x >= ntiles) return;
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t bfull[LP_NBUF], done[LP_NBUF];
    __shared__ uint32_t tslot;
    __shared__ int s_bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = threadIdx.x < LP_PRODUCERS;
    const bool issuer = threadIdx.x == LP_PRODUCERS;  // lane 0 of warp 16
    if (warp == 0) tmem_alloc(&tslot, LT_NMAX);
    if (threadIdx.x == 0) {
        s_bad = 0;
        for (int b = 0; b < LP_NBUF; b++) {
            mbar_init(&bfull[b], LP_PWARPS + 1);  // one arrive per producer warp, one with the A bytes
            mbar_init(&done[b], 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    // kind::f16 with FP16 A and B (format 0), FP32 accumulator, K-major
    const uint32_t idesc = (1u << 4) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(LT_M >> 4) << 24);
    const long long nstg = (2 * p.N + LKC - 1) / LKC;
    bool ok = true;
    long long gs = 0;  // stages run by this block so far (all tiles)
    // buffer and phase parity of the block's next stage, carried along by
    // every role (each runs every stage once), so no stage count is divided
    int cb = 0;
    uint32_t cph = 0;
    auto advance = [&]() {
        if (++cb == LP_NBUF) {
            cb = 0;
            cph ^= 1u;
        }
    };
    LpRegs R[LP_SETS];  // (warp 16 does not use them)
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int rt = (int)(tile % nrt);
        const long long j0 = (tile / nrt) * nt;
        const uint8_t *ga = p.apieces + (long long)rt * nstg * LA_STAGE;
        const long long g0 = gs;
        if (producer) {
            LpTile T;
            lp_tile(p, j0, nt, T);
            const long long nfull = p.N / (LKC / 2);
#pragma unroll
            for (int a = 0; a < LP_AHEAD; a++)
                if (a < nstg) lp_load(p, T, a, nfull, R[a]);
            for (int a = LP_AHEAD; a < LP_PF; a++) lp_prefetch(p, T, a, nfull);
            auto produce = [&](long long s, const LpRegs &Rc, LpRegs &Rn) {
                if (s + LP_AHEAD < nstg) lp_load(p, T, s + LP_AHEAD, nfull, Rn);
                lp_prefetch(p, T, s + LP_PF, nfull);
                uint64_t *fb = &bfull[cb];
                if (g0 + s >= LP_NBUF) {
                    // one lane polls (the MMAs of the buffer's previous stage);
                    // __syncwarp orders the warp's stores after it
                    bool wok = true;
                    if (lane == 0) wok = mbar_wait(&done[cb], cph ^ 1u, p.wait_cycles);
                    wok = __shfl_sync(0xffffffffu, wok ? 1 : 0, 0) != 0;
                    __syncwarp();
                    ok = ok && wok;
                }
                lp_store(nt, T, Rc, dsm + cb * LSTAGE + LA_STAGE);
                // each thread makes its own stores visible to the tensor core
                // (async proxy); after the warp's, lane 0 arrives for it
                fence_async_smem();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(fb)) : "memory");
                advance();
            };
            for (long long s = 0; s < nstg; s += LP_SETS) {
#pragma unroll
                for (int a = 0; a < LP_SETS; a++)
                    if (s + a < nstg) produce(s + a, R[a], R[(a + LP_AHEAD) % LP_SETS]);
            }
        } else if (threadIdx.x == LP_PRODUCERS + 32) {
            // lane 0 of warp 17: the A pieces of every stage, into a buffer
            // whose MMAs are done, announced on its bfull
            for (long long s = 0; s < nstg; s++) {
                uint64_t *fb = &bfull[cb];
                if (g0 + s >= LP_NBUF) ok = mbar_wait(&done[cb], cph ^ 1u, p.wait_cycles) && ok;
                // arrive and announce the bytes in one step, before the copy:
                // the phase cannot complete without them
                mbar_expect_tx(fb, LA_STAGE);
                bulk_g2s(dsm + cb * LSTAGE, ga + s * LA_STAGE, LA_STAGE, fb);
                advance();
            }
        } else if (issuer) {
            for (long long s = 0; s < nstg; s++) {
                const int b = cb;
                ok = mbar_wait(&bfull[b], cph, p.wait_cycles) && ok;
                tc_fence_after();
                const uint32_t sa = smem_u32(dsm + b * LSTAGE), sb = sa + LA_STAGE;
#pragma unroll
                for (int kk = 0; kk < LKC / 16; kk++) {
                    // K step kk: two core matrices along K
                    const uint64_t ah = smem_desc(sa + kk * 256, 128, (LKC / 8) * 128);
                    const uint64_t al = smem_desc(sa + LA_PIECE + kk * 256, 128, (LKC / 8) * 128);
                    const uint64_t bh = smem_desc(sb + kk * 2 * LB_LBO, LB_LBO, LB_SBO);
                    const uint64_t bl = smem_desc(sb + LB_LO + kk * 2 * LB_LBO, LB_LBO, LB_SBO);
                    tc_mma_bf16(tmem, ah, bh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    tc_mma_bf16(tmem, ah, bl, idesc, 1u);
                    tc_mma_bf16(tmem, al, bh, idesc, 1u);
                }
                tc_commit(&done[b]);
                advance();
            }
        } else {
            // the other lanes of warps 16 and 17 keep the stage count with their lane 0
            for (long long s = 0; s < nstg; s++) advance();
        }
        // the other lanes of the MMA and A-copy warps wait here, converged,
        // while their lane 0 works
        if (warp >= LP_PWARPS) __syncwarp();
        gs = g0 + nstg;
        // every thread: the tile's last MMAs (the latest phase of that barrier:
        // the stage before the next one)
        ok = mbar_wait(&done[cb == 0 ? LP_NBUF - 1 : cb - 1], cb == 0 ? cph ^ 1u : cph, p.wait_cycles) && ok;
        if (!ok) s_bad = 1;
        __syncthreads();
        tc_fence_after();
        // epilogue: thread = A row (TMEM lane); row 2l adds to Re C[l, j], row
        // 2l+1 to Im; warp w reads TMEM lanes 32 (w % 4) .. for the column
        // quarter w / 4
        if (warp < LP_PWARPS && !s_bad) {
            const int r = rt * LT_M + 32 * (warp & 3) + lane;
            const int qw = ((nt >> 2) + 15) & ~15;
            const int c_lo = qw * (warp >> 2);
            const int c_hi = c_lo + qw < nt ? c_lo + qw : nt;
            const int sa_l = r < 2 * k1 ? p.qscale[r >> 1] : 0;
            for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0, v);
                if (r < 2 * k1) {
                    double *crow = (double *)(p.C + (long long)(r >> 1) * p.ldC) + (r & 1);
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const long long j = j0 + c0 + e;
                        if (c0 + e < c_hi && j < p.M) {
                            const int sc = sa_l + lp_scale_exp(p.lonrm[j]);
                            const double f = __longlong_as_double((long long)(1023 - sc) << 52);
                            crow[2 * j] += (double)v[e] * f;
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s_bad) break;
    }
    if (s_bad && threadIdx.x == 0) atomicExch(err, 1);
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, LT_NMAX);
}

// After the projection onto lo: acc_j = sum_l |C[l, j]|^2 from the now exact
// coefficients (error-free squares, compensated sum) and the exact argmax.
// switch_pending 1 (the loop has ended): the stopping status.  switch_pending
// 2 (the switch): the sweeps read hi + lo from here on (phase 1, the FP64
// form's double-float sweep on the same hi/lo storage), err_curve[k] and the
// next pivot become exact, and the stopping rule is applied to them.
__global__ void __launch_bounds__(kThreads) k_rebase_finish(Prob p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || !ld_volatile(&st->switch_pending)) return;
    const int k1 = st->k;
    double be = -INFINITY;
    long long bi = kNoIdx;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p.M; j += (long long)gridDim.x * blockDim.x) {
        const double a = acc_recompute(p.C, p.ldC, j, k1);
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
        const bool ending = st->switch_pending == 1;
        st->switch_pending = 0;
        double emax = bi == kNoIdx ? 0.0 : be;
        p.err_curve[k1] = emax;
        st->J = bi;
        st->errJ = emax;
        if (ending) {
            st->status = (bi != kNoIdx && !(emax < p.tol) && !st->force_stop && k1 >= p.kmax && k1 < p.minNM)
                             ? RB_KMAX_REACHED
                             : RB_OK;
            st->stop = 1;
        } else {
            st->phase = 1;
            st->switch_iter = k1;
            if (bi == kNoIdx || emax < p.tol) {
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
    k_cand<<<p.nblk_cand, kThreads, 0, s>>>(p);
    k_recheck<<<g_re, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 4;
    return cudaGetLastError();
}

// Queued after every iteration; both kernels return at once unless the loop
// has just ended.
size_t lo_pieces_bytes(long long N, int kcap) {
    const long long nrt = (2LL * kcap + LT_M - 1) / LT_M, nstg = (2 * N + LKC - 1) / LKC;
    return (size_t)nrt * (size_t)nstg * LA_STAGE;
}

// Column tile width of the projection onto lo: a multiple of 16 in [32, 256]
// that minimises (waves of tiles over the SMs) x (tile width + a per-tile
// overhead), so the last wave is not mostly empty.
static int lp_tile_width(long long M, int sms) {
    int best = LT_NMAX;
    double best_cost = 1e300;
    for (int nt = LT_NMAX; nt >= 32; nt -= 16) {
        const long long tiles = (M + nt - 1) / nt;
        const long long waves = (tiles + sms - 1) / sms;
        const double cost = (double)waves * (nt + 24);
        if (cost < best_cost) {
            best_cost = cost;
            best = nt;
        }
    }
    return best;
}

cudaError_t launch_split_finish(const Prob &p, int grid, cudaStream_t s, int *nlaunch) {
    const size_t dsmem = (size_t)LP_NBUF * LSTAGE;  // 204 KB (3 x 68 KB)
    static int sms = 0;
    if (!sms) {
        cudaFuncSetAttribute(k_lo_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
        cudaFuncSetAttribute(k_lo_project_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        // one block per SM
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int nt = lp_tile_width(p.M, sms);
    k_qscale<<<256, kThreads, 0, s>>>(p);
    k_qpieces<<<grid, kThreads, 0, s>>>(p);
    k_lo_project_tc<<<sms, LP_THREADS, dsmem, s>>>(p, nt, p.tc_err);
    long long rf = (p.M + kThreads - 1) / kThreads;
    if (rf > grid) rf = grid;
    k_rebase_finish<<<(int)rf, kThreads, 0, s>>>(p);
    if (nlaunch) *nlaunch += 4;
    return cudaGetLastError();
}

}  // namespace rbk
