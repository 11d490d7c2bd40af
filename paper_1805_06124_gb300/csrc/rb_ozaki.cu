// rb_ozaki.cu -- FP64-accurate projection C = Q^H X on the BF16 tensor cores.
//
// Real form: with q_l = a + ib and x_j = u + iv, interleave K = 2N as
// (re, im) pairs; A row 2l = (a_i, b_i), row 2l+1 = (-b_i, a_i); B row j =
// (u_i, v_i).  Then D = A B^T holds Re c_lj in row 2l and Im c_lj in row 2l+1.
//
// Error-free slicing (the fixed-point splitting idea of Ozaki et al.): each A
// row and each B row gets a power-of-two scale 2^E with max |value| < 2^(E-1),
// and every value is written as 2^E * sum_{s=1..7} alpha_s 2^(-7s) with
// integers |alpha_s| <= 64 (balanced rounding, 49 bits in all).  Every slice
// is exact in BF16.  A product of slices is an integer below 2^12 and the 28
// slice pairs with s + t <= 8 group into seven "levels" L = s + t sharing the
// factor 2^(-7L).  A level collects at most 7 pairs, so its sum over 512 K
// terms stays below 7 * 2^12 * 512 < 2^24: the FP32 tensor-core accumulation
// of a level is EXACT over such a chunk.  Each level has its own TMEM
// accumulator; every 512 K the levels are drained, combined with their powers
// of two in double-float, and added to a double-float running sum per output.
// Pairs with s + t > 8 are dropped (below 2^-49 relative); the result is
// accurate to a few 2^-48 of max|A_r| max|B_j| K.
#include "rb_internal.cuh"
#include "rb_tc.cuh"

namespace rbk {

constexpr int OZ_S = 7;          // slices per value
constexpr int OZ_BITS = 7;       // bits per slice
constexpr int OZ_LV = OZ_S;      // levels 2..8 -> 7 accumulators
constexpr int OZ_M = 128;        // A rows per tile
constexpr int OZ_N = 64;         // B rows (columns of C) per tile
constexpr int OZ_KS = 16;        // K per shared-memory stage (double-buffered)
constexpr int OZ_DRAIN = 512;    // K per exact TMEM chunk
constexpr int OZ_TCOLS = 512;    // TMEM columns allocated (7 levels x 64 used)

__device__ __forceinline__ int scale_exp(double mx) {
    if (!(mx > 0.0)) return 0;
    int e;
    frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): mx < 2^e
    return e + 1;   // max < 2^(E-1)
}

__device__ __forceinline__ long long oz_fixed(double v, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    long long X = 0;
    if (e != 0) {
        const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
        const int sh = e - 1026 - E;
        if (sh >= 0) X = m << sh;
        else if (sh > -64) X = (m + (1LL << (-sh - 1))) >> (-sh);
        if (b >> 63) X = -X;
    }
    return X;
}

// Slices of a (re, im) pair stored as BF16x2 into each of the 7 planes.
__device__ __forceinline__ void slice7_pair(double re, double im, int E, __nv_bfloat162 *out, long long stride2) {
    long long X = oz_fixed(re, E), Y = oz_fixed(im, E);
#pragma unroll
    for (int s = 0; s < OZ_S; s++) {
        const int sh = 49 - OZ_BITS * (s + 1);
        long long a = (sh > 0) ? ((X + (1LL << (sh - 1))) >> sh) : X;
        long long c = (sh > 0) ? ((Y + (1LL << (sh - 1))) >> sh) : Y;
        X -= a << sh;
        Y -= c << sh;
        // |a|, |c| <= 64: exact through a 32-bit conversion
        out[s * stride2] = __floats2bfloat162_rn(__int2float_rn((int)a), __int2float_rn((int)c));
    }
}

// value -> 7 balanced slices of 7 bits.  Integer arithmetic on the IEEE
// bits (the FP64 pipe of this GPU is slow): X = round(v 2^(49-E)), an integer
// below 2^48 in magnitude since |v| < 2^(E-1); then balanced base-128 digits
// from the top, alpha_s = round(X / 2^(49-7s)), X -= alpha_s 2^(49-7s).
__device__ __forceinline__ void slice7(double v, int E, __nv_bfloat16 *out, long long stride) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    long long X = 0;
    if (e != 0) {  // zero and subnormal inputs give zero slices
        const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
        const int sh = e - 1026 - E;  // v = m 2^(e-1075) -> X = m 2^(e-1075+49-E)
        if (sh >= 0) X = m << sh;
        else if (sh > -64) X = (m + (1LL << (-sh - 1))) >> (-sh);  // round half up
        if (b >> 63) X = -X;
    }
#pragma unroll
    for (int s = 0; s < OZ_S; s++) {
        const int sh = 49 - OZ_BITS * (s + 1);
        long long a = (sh > 0) ? ((X + (1LL << (sh - 1))) >> sh) : X;
        X -= a << sh;
        out[s * stride] = __float2bfloat16_rn((float)a);
    }
}

// A: one block per basis vector l; E_l from max |a_i|, |b_i|; slices of both rows.
__global__ void k_oz_slice_A(const double2 *__restrict__ Q, long long N, int k, long long ldQ, long long Kp,
                             long long Rp, __nv_bfloat16 *__restrict__ As, int *__restrict__ Ea) {
    const int l = blockIdx.x;
    if (l >= k) return;
    const double2 *q = Q + (long long)l * ldQ;
    double mx = 0.0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, fmax(fabs(q[i].x), fabs(q[i].y)));
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmax(m, sm[w]);
        sm[0] = m;
    }
    __syncthreads();
    const int E = scale_exp(sm[0]);
    if (threadIdx.x == 0) Ea[l] = E;
    const long long sstride = Rp * Kp;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        double2 v = q[i];
        __nv_bfloat162 *re = (__nv_bfloat162 *)(As + (long long)(2 * l) * Kp + 2 * i);
        __nv_bfloat162 *im = (__nv_bfloat162 *)(As + (long long)(2 * l + 1) * Kp + 2 * i);
        slice7_pair(v.x, v.y, E, re, sstride / 2);
        slice7_pair(-v.y, v.x, E, im, sstride / 2);
    }
}

// B: one block per column j of this batch.  The scale comes from the largest
// biased exponent (integer max over the IEEE bits, no FP64 work): max|x| <
// 2^(e_max - 1022), so E = e_max - 1021, as frexp of the maximum would give.
// K positions past 2N (padding to Kp) are written as zero slices here.
__global__ void k_oz_slice_B(const double2 *__restrict__ X, long long N, long long Mb, long long ldX, long long Kp,
                             long long Cp, __nv_bfloat16 *__restrict__ Bs, int *__restrict__ Eb) {
    const long long j = blockIdx.x;
    if (j >= Mb) return;
    const double2 *x = X + j * ldX;
    unsigned int em = 0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 v = x[i];
        const unsigned int a = ((unsigned int)(__double_as_longlong(v.x) >> 52)) & 0x7FFu;
        const unsigned int b = ((unsigned int)(__double_as_longlong(v.y) >> 52)) & 0x7FFu;
        em = max(em, max(a, b));
    }
    __shared__ unsigned int se[32];
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    if ((threadIdx.x & 31) == 0) se[threadIdx.x >> 5] = em;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, se[w]);
        se[0] = m;
    }
    __syncthreads();
    const int E = se[0] ? (int)se[0] - 1021 : 0;
    if (threadIdx.x == 0) Eb[j] = E;
    const long long sstride = Cp * Kp;
    const __nv_bfloat162 z2 = __floats2bfloat162_rn(0.f, 0.f);
    for (long long i = threadIdx.x; i < Kp / 2; i += blockDim.x) {
        __nv_bfloat162 *o = (__nv_bfloat162 *)(Bs + j * Kp + 2 * i);
        if (i < N) {
            const double2 v = x[i];
            slice7_pair(v.x, v.y, E, o, sstride / 2);
        } else {
#pragma unroll
            for (int sl = 0; sl < OZ_S; sl++) o[sl * (sstride / 2)] = z2;
        }
    }
}

// Asynchronous copy of rows [r0, r0+R) x K [k0, k0+OZ_KS) of the 7 slice
// planes (row-major, K contiguous) into K-major shared tiles, 16 bytes (one
// core-matrix row) per cp.async.  The 8 threads of each quarter warp fill the
// 8 rows of one core matrix (128 contiguous bytes, no bank conflicts).
__device__ __forceinline__ void oz_stage_async(uint8_t *dst, const __nv_bfloat16 *src, long long plane, long long Kp,
                                               int R, long long r0, long long k0) {
    constexpr int per_row = OZ_KS / 8;
    for (int t = threadIdx.x; t < OZ_S * R * per_row; t += blockDim.x) {
        int s = t / (R * per_row), rem = t % (R * per_row);
        int r = (rem & 7) + 8 * (rem / (8 * per_row)), kk = ((rem >> 3) % per_row) * 8;
        const void *g = src + s * plane + (r0 + r) * Kp + k0 + kk;
        uint32_t d = smem_u32(dst + s * (R * OZ_KS * 2) + kmajor_off(r, kk, OZ_KS));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g));
    }
    asm volatile("cp.async.commit_group;");
}

// (hi, lo) += x, both double-float
__device__ __forceinline__ void dfs_add(float &ah, float &al, float bh, float bl) { df_add(ah, al, bh, bl); }

__global__ void __launch_bounds__(128) k_oz_gemm(const __nv_bfloat16 *__restrict__ As, const __nv_bfloat16 *__restrict__ Bs,
                                                 const int *__restrict__ Ea, const int *__restrict__ Eb, int k, long long Mb,
                                                 long long Kp, long long Rp, long long Cp, double2 *__restrict__ C,
                                                 long long ldC, long long col_off, int *err) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    constexpr int SA = OZ_S * OZ_M * OZ_KS * 2, SB = OZ_S * OZ_N * OZ_KS * 2;  // 28 KB, 14 KB per buffer
    uint8_t *sAb[2] = {dsm, dsm + SA};
    uint8_t *sBb[2] = {dsm + 2 * SA, dsm + 2 * SA + SB};
    float *acc_h = (float *)(dsm + 2 * (SA + SB));  // 128 x 64 double-float running sums
    float *acc_l = acc_h + OZ_M * OZ_N;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    const long long j0 = (long long)blockIdx.x * OZ_N;
    const long long r0 = (long long)blockIdx.y * OZ_M;
    for (int t = threadIdx.x; t < OZ_M * OZ_N; t += blockDim.x) acc_h[t] = acc_l[t] = 0.f;
    if (warp == 0) tmem_alloc(&tslot, OZ_TCOLS);
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(OZ_M, OZ_N);
    uint32_t phase = 0;
    bool ok = true;
    const long long nst = Kp / OZ_KS;
    constexpr int per_drain = OZ_DRAIN / OZ_KS;
    const long long planeA = Rp * Kp, planeB = Cp * Kp;
    oz_stage_async(sAb[0], As, planeA, Kp, OZ_M, r0, 0);
    oz_stage_async(sBb[0], Bs, planeB, Kp, OZ_N, j0, 0);
    for (long long st = 0; st < nst; st++) {
        const int cur = (int)(st & 1);
        uint8_t *sA = sAb[cur], *sB = sBb[cur];
        if (st + 1 < nst) {  // prefetch the next stage into the other buffer
            oz_stage_async(sAb[cur ^ 1], As, planeA, Kp, OZ_M, r0, (st + 1) * OZ_KS);
            oz_stage_async(sBb[cur ^ 1], Bs, planeB, Kp, OZ_N, j0, (st + 1) * OZ_KS);
            asm volatile("cp.async.wait_group 2;");
        } else {
            asm volatile("cp.async.wait_group 0;");
        }
        fence_async_smem();
        __syncthreads();
        const bool fresh = (st % per_drain) == 0;
        if (threadIdx.x == 0) {
            tc_fence_after();
            bool started[OZ_LV];
#pragma unroll
            for (int L = 0; L < OZ_LV; L++) started[L] = !fresh;
#pragma unroll
            for (int sa = 0; sa < OZ_S; sa++)
#pragma unroll
                for (int sb = 0; sb < OZ_S; sb++) {
                    const int L = sa + sb;  // level - 2
                    if (L >= OZ_LV) continue;
#pragma unroll
                    for (int kk = 0; kk < OZ_KS / 16; kk++) {
                        uint64_t ad = smem_desc(smem_u32(sA) + sa * (OZ_M * OZ_KS * 2) + kk * 256, 128, (OZ_KS / 8) * 128);
                        uint64_t bd = smem_desc(smem_u32(sB) + sb * (OZ_N * OZ_KS * 2) + kk * 256, 128, (OZ_KS / 8) * 128);
                        tc_mma_bf16(tmem + (uint32_t)(L * OZ_N), ad, bd, idesc, started[L] ? 1u : 0u);
                        started[L] = true;
                    }
                }
            tc_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase) && ok;
        phase ^= 1;
        tc_fence_after();
        __syncthreads();
        if ((st % per_drain) == per_drain - 1 || st == nst - 1) {
            // drain: row = TMEM lane; levels combined smallest first, in double-float
            const int r = threadIdx.x;
            const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
            for (int c0 = 0; c0 < OZ_N; c0 += 16) {
                float v[OZ_LV][16];
#pragma unroll
                for (int L = 0; L < OZ_LV; L++) tmem_ld16(tmem + lane_off + (uint32_t)(L * OZ_N + c0), v[L]);
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    float th = 0.f, tl = 0.f;
#pragma unroll
                    for (int L = OZ_LV - 1; L >= 0; L--) {
                        // level L+2 carries 2^(-7 (L+2)): an exact power-of-two factor
                        float x = v[L][e] * __int_as_float((127 - OZ_BITS * (L + 2)) << 23);
                        dfs_add(th, tl, x, 0.f);
                    }
                    float &h = acc_h[r * OZ_N + c0 + e];
                    float &lo = acc_l[r * OZ_N + c0 + e];
                    dfs_add(h, lo, th, tl);
                }
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    if (!ok && err) atomicExch(err, 1);
    // write: row r of the tile -> basis vector (r0 + r) / 2, Re or Im part
    const long long R = r0 + threadIdx.x;
    if (R < 2LL * k) {
        const int l = (int)(R >> 1);
        const int Ex = Ea[l];
        double *crow = (double *)(C + (long long)l * ldC) + (R & 1);
        for (int c = 0; c < OZ_N; c++) {
            long long j = j0 + c;
            if (j >= Mb) break;
            double t = (double)acc_h[threadIdx.x * OZ_N + c] + (double)acc_l[threadIdx.x * OZ_N + c];
            crow[2 * (col_off + j)] = ldexp(t, Ex + Eb[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, OZ_TCOLS);
}

// Self-test of the bounded mbarrier wait used by every tensor-core kernel: one
// thread waits on a barrier that nothing arrives on (unless `arrive`), with a
// budget of `polls`, and records a time-out in *flag.  No tensor-core work is
// in flight, so running out of budget leaves nothing behind.
__global__ void k_wait_selftest(long long polls, int arrive, int *flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        if (arrive) {
            unsigned long long st;
            asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(smem_u32(&bar)));
        }
        if (!mbar_wait(&bar, 0, polls)) *flag = 1;
    }
}

cudaError_t launch_wait_selftest(long long polls, int arrive, int *flag, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(polls, arrive, flag);
    return cudaGetLastError();
}

size_t oz_workspace(long long N, int k, long long Mb) {
    long long Kp = (2 * N + OZ_KS - 1) / OZ_KS * OZ_KS;
    long long Rp = (2LL * k + OZ_M - 1) / OZ_M * OZ_M;
    long long Cp = (Mb + OZ_N - 1) / OZ_N * OZ_N;
    return (size_t)OZ_S * (Rp + Cp) * Kp * 2 + (size_t)(k + Cp) * 4 + 4096;
}

// C[:, col_off : col_off + Mb] for one batch of Mb columns; ws from oz_workspace.
cudaError_t launch_project_tc(const double2 *Q, long long N, int k, long long ldQ, const double2 *X, long long Mb,
                              long long ldX, double2 *C, long long ldC, long long col_off, void *ws, int *err,
                              cudaStream_t s) {
    if (k <= 0 || Mb <= 0) return cudaSuccess;
    const long long Kp = (2 * N + OZ_KS - 1) / OZ_KS * OZ_KS;
    const long long Rp = (2LL * k + OZ_M - 1) / OZ_M * OZ_M;
    const long long Cp = (Mb + OZ_N - 1) / OZ_N * OZ_N;
    __nv_bfloat16 *As = (__nv_bfloat16 *)ws;
    __nv_bfloat16 *Bs = As + (size_t)OZ_S * Rp * Kp;
    int *Ea = (int *)(Bs + (size_t)OZ_S * Cp * Kp);
    int *Eb = Ea + k;
    // zero fill: the A planes (small) and the padded B rows Mb..Cp-1 of each
    // plane; k_oz_slice_B writes every other B entry, K padding included
    cudaError_t e = cudaMemsetAsync(As, 0, (size_t)OZ_S * Rp * Kp * 2, s);
    if (e != cudaSuccess) return e;
    if (Cp > Mb)
        for (int sl = 0; sl < OZ_S; sl++) {
            e = cudaMemsetAsync(Bs + (size_t)sl * Cp * Kp + (size_t)Mb * Kp, 0, (size_t)(Cp - Mb) * Kp * 2, s);
            if (e != cudaSuccess) return e;
        }
    k_oz_slice_A<<<k, 256, 0, s>>>(Q, N, k, ldQ, Kp, Rp, As, Ea);
    k_oz_slice_B<<<(unsigned)Mb, 256, 0, s>>>(X, N, Mb, ldX, Kp, Cp, Bs, Eb);
    const size_t dsm = (size_t)2 * OZ_S * (OZ_M + OZ_N) * OZ_KS * 2 + (size_t)2 * OZ_M * OZ_N * 4;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        attr = true;
    }
    dim3 grid((unsigned)(Cp / OZ_N), (unsigned)(Rp / OZ_M));
    k_oz_gemm<<<grid, 128, dsm, s>>>(As, Bs, Ea, Eb, k, Mb, Kp, Rp, Cp, C, ldC, col_off, err);
    return cudaGetLastError();
}

}  // namespace rbk
