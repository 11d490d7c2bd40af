// rb_internal.cuh -- shared device-side definitions of the CUDA path.
//
// Every kernel of the greedy loop reads and writes one small DevState in
// device memory, so an iteration can be queued (or replayed) without the host
// knowing k, the pivot or whether the loop has already stopped: each kernel
// returns at once when `stop` is set.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rb.h"

namespace rbk {

// Default budget of a device-side wait (tensor-core mbarrier waits): 2^31 SM
// clock cycles, about one second at 2 GHz.
constexpr unsigned long long kWaitCyclesDefault = 1ull << 31;


constexpr int kThreads = 256;
constexpr long long kNoIdx = 0x7fffffffffffffffLL;

struct DevState {
    int k;             // basis vectors appended so far
    int stop;          // 1 once the greedy loop has ended
    int status;        // rb_status at stop
    int accepted;      // IMGS: the current v passed the kappa test
    int passes;        // IMGS passes in the current iteration
    int total_passes;  // IMGS passes over the whole call
    int nonfinite;     // a column norm was NaN/Inf
    int phase;         // split form: 1 once the sweeps read hi + lo (after the switch)
    int switch_iter;   // split form: basis size at the switch
    int n_sweeps;      // sweep launches that did work
    int ncand;         // split form: candidates in the last recheck
    int switch_pending;  // split form: the projection onto lo is queued; 1: the loop has ended,
                         // 2: the switch to hi + lo sweeps (the loop goes on)
    int n_sweeps_hl;     // split form: hi + lo sweeps after the switch
    int max_cand;        // split form: largest candidate list seen
    int force_stop;      // split form: exact rank reached (IMGS found a zero vector)
    int cand_total;      // split form: candidates counted in this iteration
    double Lmax;       // split form: largest certified lower bound of the error
    long long J;       // next pivot column (kNoIdx = none left)
    double errJ;       // its error
    double before2;    // IMGS: ||v||^2 before the current pass
    double after2;     // IMGS: ||v||^2 after the current pass
    unsigned int ticket_sweep;  // last-block-done counters (reset by the last block)
    unsigned int ticket_imgs;
    unsigned int ticket_init;
    unsigned int ticket_aux;
    unsigned int ticket_host;   // streamed form: last-block counter of the chunk sweeps
    int pad1;
    double hbest_err;           // streamed form: best (err, idx) of the current sweep so far
    long long hbest_idx;
    double sel_max;             // streamed form: largest stale bound of the iteration
    unsigned int ticket_sel;
    int pad2;
    unsigned int bar_count;     // grid barrier of the fused IMGS kernel: arrivals
    unsigned int bar_gen;       // and generation
};

// Problem description passed by value to every kernel of a greedy call.
struct Prob {
    long long N, M;
    long long ldS, ldH, ldQ, ldC;
    long long minNM;
    int kmax;
    int max_passes;
    int nchunk;        // IMGS dot-product row chunks
    int chunk;         // rows per chunk
    double tol;
    double kappa2;     // kappa^2 (the kappa test compares squared norms)
    const double2 *S;  // complex128 snapshots (FP64 form)
    const float2 *hi;  // split storage
    const float2 *lo;
    double2 *Q;
    long long *pivots;
    double *err_curve;
    double2 *C;        // may be null
    double *rdiag;     // may be null
    double *norm2;
    double *acc;
    unsigned char *picked;
    float2 *qh;        // basis vectors rounded to FP32 (slot k at qh + k * qs_stride)
    float2 *ql;        // their FP32 remainders
    long long qs_stride;  // 0: one slot reused every iteration; else N rounded up
    double2 *v;        // IMGS work vector
    double2 *hpart;    // IMGS partial dot products [kmax][nchunk]
    double *npart;     // per-block partial norms
    double *bpart_err; // per-block argmax partials
    long long *bpart_idx;
    DevState *st;
    // split form
    double *norm2_hi;  // ||hi_j||^2
    float *lonrm;      // ||lo_j|| (rounded up)
    float *snorm;      // [M][64] 2-norms of the 64 lane chains of hi_j (rounded up)
    double *sabs;      // sum_l |c~_lj| of the hi-only sweep results
    double eta;        // bound on |c~ - q^H hi| relative to ||hi_j|| for one sweep
    long long *cand;   // candidate columns (capacity M)
    double *cand_err;  // their exact errors
    double *pv;        // recheck partials [candidate][group of 8 basis vectors]
    uint8_t *apieces;  // FP16 pieces of the basis for the projection onto lo
    int *qscale;       // their power-of-two scale exponents, one per basis vector
    double *rpart;     // re-check row-chunk partials [pair][chunk][32]
    int *rtick;        // re-check chunk counters per (candidate, group) pair
    int lgcap;         // groups per candidate in pv
    int nblk_cand;     // blocks of the candidate kernel
    int *tc_err;       // set when a tensor-core wait ran out
    unsigned long long wait_cycles;  // budget of each tensor-core wait, SM clock cycles
    double switch_err; // split form: switch once every error is certified below switch_err * max ||s_j||^2 (0: off)
    int switch_cand;   // split form: switch once more than switch_cand columns are candidates
    double *dacc;      // D_j = sum_l (|c_lj|^2 - |c~_lj|^2) over the rows re-checked so far
    int *dcnt;         // rows covered by D_j
    int *passes_out;   // IMGS passes of iteration k at [k] (may be null)
};

// Streamed part of a problem: chunk bookkeeping and the per-warp staging of
// one column's hi/lo split (reused by the second and later pending vectors).
struct StreamPart {
    const double2 *Sd;    // device-visible pointer to S (host memory)
    long long Mr;         // resident columns 0..Mr-1
    long long cols;       // columns per chunk
    int nch;              // chunks over columns Mr..M-1
    int period;           // recompute period (0: none)
    double gamma;         // round-A threshold factor
    int *last;            // [nch] first basis vector not yet applied
    double *bound;        // [nch] largest unpicked error when last updated (-inf: none)
    double *nmax;         // [nch] largest ||s_j||^2 of the chunk
    double *part;         // [grid] per-block maxima of the selection
    int *list;            // [nch] chunks selected for the current launch
    int *cnt;             // list lengths: [0] round A, [1] round B, [2] flush
    unsigned long long *updates;  // chunk updates so far
    float2 *stage;        // per warp: hi then lo, stage_ld each
    long long stage_ld;
};

// One problem of a batch (rb_greedy_batched): what the persistent sweep and
// the per-problem reduction need.
struct BProb {
    long long N, M, ldS, ldC;
    const double2 *S;
    double2 *C;
    double *err_curve;
    double *norm2;
    double *acc;
    unsigned char *picked;
    const float2 *qh;
    const float2 *ql;
    DevState *st;
    int kmax;
    int pad;
    long long minNM;
    double tol;
    const float2 *hi;  // pre-split copy (null: split in registers)
    const float2 *lo;
    long long ldH;
};

// ---------------------------------------------------------------- argmax key
// (err, idx) is better than (err2, idx2) when err is larger, ties to the
// lower index.
__device__ __forceinline__ bool better(double e1, long long i1, double e2, long long i2) {
    return e1 > e2 || (e1 == e2 && i1 < i2);
}

__device__ __forceinline__ void warp_best(double &e, long long &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double e2 = __shfl_xor_sync(0xffffffffu, e, o);
        long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(e2, i2, e, i)) { e = e2; i = i2; }
    }
}

// Block-wide best; the result is valid in thread 0.
__device__ __forceinline__ void block_best(double &e, long long &i) {
    __shared__ double se[32];
    __shared__ long long si[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    warp_best(e, i);
    __syncthreads();
    if (lane == 0) { se[w] = e; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        e = lane < nw ? se[lane] : -INFINITY;
        i = lane < nw ? si[lane] : kNoIdx;
        warp_best(e, i);
    }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide sum in a fixed order; valid in thread 0.
__device__ __forceinline__ double block_sum(double x) {
    __shared__ double sx[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    x = warp_sum(x);
    __syncthreads();
    if (lane == 0) sx[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        x = lane < nw ? sx[lane] : 0.0;
        x = warp_sum(x);
    }
    return x;
}

__device__ __forceinline__ double2 block_sum2(double2 x) {
    double a = block_sum(x.x);
    double b = block_sum(x.y);
    return make_double2(a, b);
}

// Last-block-done ticket: returns true in every thread of the block that
// arrives last.  Each block must have published its partial (and fenced)
// before calling.
__device__ __forceinline__ bool last_block(unsigned int *ticket) {
    __shared__ int amlast;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        amlast = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (amlast) __threadfence();
    return amlast != 0;
}

// --------------------------------------------------------- double-float ops
// Error-free transformations (Knuth's TwoSum; the FMA form of Dekker's
// TwoProduct).  The __f*_rn intrinsics keep the compiler from contracting or
// reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (sh, sl) += (ah + al) * (bh + bl), dropping al*bl (below 2^-48 relative).
__device__ __forceinline__ void df_mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// (ah, al) += (bh, bl)
__device__ __forceinline__ void df_add(float &ah, float &al, float bh, float bl) {
    float s, t;
    two_sum(ah, bh, s, t);
    t = __fadd_rn(t, __fadd_rn(al, bl));
    ah = __fadd_rn(s, t);
    al = __fsub_rn(t, __fsub_rn(ah, s));
}

__device__ __forceinline__ void warp_df_sum(float &h, float &l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float h2 = __shfl_xor_sync(0xffffffffu, h, o);
        float l2 = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, h2, l2);
    }
}

// Streaming 128-bit load that does not allocate in L1 (S is read once per sweep).
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ double2 ld_stream_d2(const double2 *p) {
    double2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// Round-to-nearest split of one double into hi = fl32(x), lo = fl32(x - hi)
// with integer operations (the FP64 conversion units of this GPU run at the
// FP64 rate).  Valid when the biased exponent e of x is in [949, 1149]: hi is
// then a normal float and lo = (x - hi) is an integer of at most 29 bits
// times 2^(e-1075), a normal float after one rounding.  Returns false
// outside that range (zero, tiny, huge, Inf, NaN).
__device__ __forceinline__ bool split_rn_fast(double x, float &h, float &l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned int e = (unsigned int)(mag >> 52);
    if (e < 949u || e > 1149u) return false;
    const unsigned int w0 = (unsigned int)b;
    const unsigned int lsb = (w0 >> 29) & 1u;
    // round the 52-bit mantissa to 23 bits, ties to even; a carry moves
    // into the exponent field by itself
    const unsigned long long r = mag + 0x0FFFFFFFull + lsb;
    const unsigned int fb = (unsigned int)(r >> 29) - (896u << 23);
    h = __uint_as_float(fb | sign);
    // x - hi: the dropped 29 bits, minus 2^29 when the mantissa rounded up
    const unsigned int rem = w0 & 0x1FFFFFFFu;
    int ri = (int)rem - ((rem + lsb > 0x10000000u) ? 0x20000000 : 0);
    if (sign) ri = -ri;
    l = __int2float_rn(ri) * __uint_as_float((e - 948u) << 23);
    return true;
}

// (sh, sl) += (h + l)^2 in double-float.
__device__ __forceinline__ void df_sq(float &sh, float &sl, float h, float l) {
    float p = __fmul_rn(h, h);
    float e = __fmaf_rn(h, h, -p);
    e = __fmaf_rn(2.0f * h, l, e);
    e = __fmaf_rn(l, l, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// ||hi + lo||^2 of one column, the part of one lane: lane L owns the complex
// element pairs (2t, 2t+1) with t = L (mod 32), i.e. the float4 slots of
// hi/lo that the split form's sweep reads.  (ah, al) gathers (h + l)^2 - l^2
// per real component in double-float, in the order re(2t), im(2t), re(2t+1),
// im(2t+1); lsq gathers l^2 in FP32 (below 2^-48 relative).  An odd last
// element is added by lane 0 after the loop.  The FP64 form (k_split) and the
// split form (its init) both use exactly these steps, so the two forms start
// from bit-identical norms and resolve the first, tied, pivot alike.
struct Norm2Acc {
    float ah, al, lsq;
};

__device__ __forceinline__ void norm2_acc4(Norm2Acc &a, float4 h, float4 l) {
    df_mac(a.ah, a.al, h.x, l.x, h.x, l.x);
    df_mac(a.ah, a.al, h.y, l.y, h.y, l.y);
    df_mac(a.ah, a.al, h.z, l.z, h.z, l.z);
    df_mac(a.ah, a.al, h.w, l.w, h.w, l.w);
    a.lsq = __fmaf_rn(l.x, l.x, __fmaf_rn(l.y, l.y, __fmaf_rn(l.z, l.z, __fmaf_rn(l.w, l.w, a.lsq))));
}

__device__ __forceinline__ void norm2_acc2(Norm2Acc &a, float2 h, float2 l) {
    df_mac(a.ah, a.al, h.x, l.x, h.x, l.x);
    df_mac(a.ah, a.al, h.y, l.y, h.y, l.y);
    a.lsq = __fmaf_rn(l.x, l.x, __fmaf_rn(l.y, l.y, a.lsq));
}

// Whole-warp call: the column's norm, valid in every lane.
__device__ __forceinline__ double norm2_finish(const Norm2Acc &a) {
    return warp_sum((double)a.ah + (double)a.al + (double)a.lsq);
}

// Double-float product of a conjugated basis element (hi + lo parts) with a
// snapshot element (hi + lo parts), accumulated into (re_h, re_l), (im_h, im_l):
//   Re += qr*sr + qi*si,  Im += qr*si - qi*sr.
__device__ __forceinline__ void df_cmac(float &rh, float &rl, float &ih, float &il, float qrh, float qih, float qrl,
                                        float qil, float srh, float sih, float srl, float sil) {
    df_mac(rh, rl, qrh, qrl, srh, srl);
    df_mac(rh, rl, qih, qil, sih, sil);
    df_mac(ih, il, qrh, qrl, sih, sil);
    df_mac(ih, il, -qih, -qil, srh, srl);
}

// Column dot product c = q^H s_j over the hi/lo split storage (double-float);
// U 128-bit loads of hi and of lo in flight per lane.
template <int U = 4>
__device__ __forceinline__ double2 col_dot_df32(const float2 *__restrict__ hcol, const float2 *__restrict__ lcol,
                                                const float2 *__restrict__ qh, const float2 *__restrict__ ql,
                                                long long N, int lane) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    const float4 *h4 = reinterpret_cast<const float4 *>(hcol);
    const float4 *l4 = reinterpret_cast<const float4 *>(lcol);
    const float4 *qh4 = reinterpret_cast<const float4 *>(qh);
    const float4 *ql4 = reinterpret_cast<const float4 *>(ql);
    long long n2 = N >> 1;  // complex pairs
    long long t = lane;
    for (; t + 32 * (U - 1) < n2; t += 32 * U) {
        float4 a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            a[u] = ld_stream(h4 + t + 32 * u);
            b[u] = ld_stream(l4 + t + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            float4 qa = __ldg(qh4 + t + 32 * u);
            float4 qb = __ldg(ql4 + t + 32 * u);
            df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, a[u].x, a[u].y, b[u].x, b[u].y);
            df_cmac(rh, rl, ih, il, qa.z, qa.w, qb.z, qb.w, a[u].z, a[u].w, b[u].z, b[u].w);
        }
    }
    for (; t < n2; t += 32) {
        float4 a = ld_stream(h4 + t), b = ld_stream(l4 + t);
        float4 qa = __ldg(qh4 + t), qb = __ldg(ql4 + t);
        df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, a.x, a.y, b.x, b.y);
        df_cmac(rh, rl, ih, il, qa.z, qa.w, qb.z, qb.w, a.z, a.w, b.z, b.w);
    }
    if ((N & 1) && lane == 0) {
        long long i = N - 1;
        float2 a = hcol[i], b = lcol[i], qa = qh[i], qb = ql[i];
        df_cmac(rh, rl, ih, il, qa.x, qa.y, qb.x, qb.y, a.x, a.y, b.x, b.y);
    }
    warp_df_sum(rh, rl);
    warp_df_sum(ih, il);
    return make_double2((double)rh + (double)rl, (double)ih + (double)il);
}

// Split with the intrinsic conversions when the fast path does not apply.
__device__ __forceinline__ void split_rn(double x, float &h, float &l) {
    if (!split_rn_fast(x, h, l)) {
        h = __double2float_rn(x);
        l = __double2float_rn(x - (double)h);
    }
}

// hi/lo split of one complex128 element, exactly as the split kernel stores
// it: the integer fast path for both parts, else the conversions for both.
__device__ __forceinline__ void split_c(double2 x, float2 &h, float2 &l) {
    float hr, lr, hm, lm;
    bool ok = split_rn_fast(x.x, hr, lr);
    ok = split_rn_fast(x.y, hm, lm) && ok;
    if (!ok) {
        hr = __double2float_rn(x.x);
        hm = __double2float_rn(x.y);
        lr = __double2float_rn(x.x - (double)hr);
        lm = __double2float_rn(x.y - (double)hm);
    }
    h = make_float2(hr, hm);
    l = make_float2(lr, lm);
}

// Eq. (Residual) running update acc_j += |c_kj|^2 (one expression, shared by
// every sweep of the FP64 form so that all of them round it alike).
__device__ __forceinline__ double acc_add(double a, double2 c) { return a + (c.x * c.x + c.y * c.y); }

// acc_j = sum_{l<k} |C[l, j]|^2 from the stored coefficients, with
// error-free squares (FMA) and a compensated (TwoSum) running sum: the
// periodic exact recompute of the Eq. (Residual) bookkeeping.
__device__ __forceinline__ double acc_recompute(const double2 *C, long long ldC, long long j, int k) {
    double s = 0.0, e = 0.0;
    for (int l = 0; l < k; l++) {
        const double2 c = C[(long long)l * ldC + j];
        const double x = c.x * c.x, ex = fma(c.x, c.x, -x);
        const double y = c.y * c.y, ey = fma(c.y, c.y, -y);
        double t = s + x, b = t - s;
        e += ((s - (t - b)) + (x - b)) + ex;
        s = t;
        t = s + y;
        b = t - s;
        e += ((s - (t - b)) + (y - b)) + ey;
        s = t;
    }
    return s + e;
}

// End of a sweep of the FP64 form: append err_curve[k+1], publish the next
// pivot (bi, be) and apply the stopping rule (Alg. 3 while-test on the
// squared error, Cor. 5.4).  One thread.
__device__ __forceinline__ void sweep_publish(const Prob &p, DevState *st, int k, double be, long long bi) {
    const int k1 = k + 1;
    st->k = k1;
    st->n_sweeps += 1;
    const double emax = bi == kNoIdx ? 0.0 : be;
    p.err_curve[k1] = emax;
    st->J = bi;
    st->errJ = emax;
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

}  // namespace rbk

// ------------------------------------------------------------- host launchers
namespace rbk {
cudaError_t launch_generate_tables(double *amp, double *ph, long long N, cudaStream_t s);
cudaError_t launch_generate(const double *q, const double *m, const double *amp, const double *ph,
                            long long N, long long M, double2 *S, long long ldS, cudaStream_t s);
cudaError_t launch_split(const double2 *S, long long N, long long M, long long ldS, float2 *hi, float2 *lo,
                         long long ldH, double *norm2, cudaStream_t s);
cudaError_t launch_norms(const double2 *S, long long N, long long M, long long ldS, double *norm2,
                         cudaStream_t s);
cudaError_t launch_init(const Prob &p, int grid, cudaStream_t s);
cudaError_t launch_resume(const Prob &p, int k0, int grid, cudaStream_t s);
cudaError_t launch_sweep(const Prob &p, int variant, int grid, cudaStream_t s);
cudaError_t launch_recompute(const Prob &p, int period, int grid, cudaStream_t s);
cudaError_t launch_imgs(const Prob &p, int grid, bool from_split, cudaStream_t s, int *nlaunch);
int stream_sweep_grid(int device);
cudaError_t launch_stream_init(const Prob &p, const StreamPart &sp, cudaStream_t s);
cudaError_t launch_stream_iteration(const Prob &p, const StreamPart &sp, int res_grid, int str_grid, cudaStream_t s);
cudaError_t launch_stream_flush(const Prob &p, const StreamPart &sp, int str_grid, cudaStream_t s);
cudaError_t launch_imgs_batched(const Prob *pp_dev, int nprob, long long maxN, int max_passes, int grid,
                                cudaStream_t s, int *nlaunch);
cudaError_t launch_final_err(const Prob &p, double *final_err, cudaStream_t s);
cudaError_t launch_split_init(const Prob &p, cudaStream_t s);
cudaError_t launch_split_iteration(const Prob &p, int grid, cudaStream_t s, int *nlaunch);
cudaError_t launch_split_finish(const Prob &p, int grid, cudaStream_t s, int *nlaunch);
size_t lo_pieces_bytes(long long N, int kcap);
size_t recon_workspace(int j, long long M);
long long eim_blocks(long long N);
size_t eim_workspace(long long N, int k);
cudaError_t launch_eim(const double2 *Q, long long N, int k, long long ldQ, void *ws, long long *nodes, double2 *V,
                       double2 *B, long long ldB, int *flag, cudaStream_t s);
cudaError_t launch_validate(const double2 *T, long long N, long long Mt, long long ldT, const double2 *C, long long ldC,
                            int k, const long long *nodes, const double2 *Vinv, double *err_proj, double *err_eim,
                            cudaStream_t s);
cudaError_t launch_recon_svd(const double2 *C, long long ldC, int j, long long M, void *ws, double *sigma, double2 *V,
                             int *stats, cudaEvent_t *ev, cudaStream_t s);
cudaError_t launch_recon_basis(const double2 *Q, long long ldQ, long long N, int j, const double2 *V, int k,
                               double2 *X, long long ldX, cudaStream_t s);
size_t oz_workspace(long long N, int k, long long Mb);
cudaError_t launch_wait_selftest(long long cycles, int arrive, int *flag, cudaStream_t s);
cudaError_t launch_project_tc(const double2 *Q, long long N, int k, long long ldQ, const double2 *X, long long Mb,
                              long long ldX, double2 *C, long long ldC, long long col_off, void *ws, int *err,
                              unsigned long long wait, cudaStream_t s);
cudaError_t launch_project(const double2 *Q, long long N, int k, long long ldQ, const double2 *X, long long Mx,
                           long long ldX, double2 *C, long long ldC, cudaStream_t s);
int sweep_grid(int variant, int device);
cudaError_t launch_bnorms(const BProb *P, int nprob, const long long *col0, long long total_cols, cudaStream_t s);
int bsweep_threads(int v);
int bsweep_grid(int v, int device);
cudaError_t launch_bsweep(int v, int grid, const BProb *P, int nprob, const long long *chunk0, int CW,
                          double *part_err, long long *part_idx, int dry, cudaStream_t s);
cudaError_t launch_breduce(const BProb *P, int nprob, const long long *chunk0, const double *part_err,
                           const long long *part_idx, cudaStream_t s);
cudaStream_t ctx_stream(rb_ctx *ctx);
int ctx_device(rb_ctx *ctx);
unsigned long long ctx_wait_cycles(const rb_ctx *ctx);  // rb_options.timeout_cycles, 0 -> the default
const rb_options &ctx_options(const rb_ctx *ctx);
int ctx_sweep_grid(rb_ctx *ctx, int variant);             // cached grid of the FP64-form sweep
rb_status ctx_fail(rb_ctx *ctx, rb_status s, const char *msg);  // records msg for rb_last_error
cudaError_t launch_imgs_passes(const Prob &p, int grid, cudaStream_t s, int *nlaunch);
}  // namespace rbk
