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
constexpr int OZ_KS = 16;        // K per shared-memory stage
constexpr int OZ_DRAIN = 512;    // K per exact TMEM chunk
constexpr int OZ_TCOLS = 512;    // TMEM columns allocated (7 levels x 64, then the running sums' high words)
constexpr int OZ_ACOL = OZ_LV * 64;  // first column of the running sums

// The basis slice planes are stored tile by tile in the K-major shared-memory
// layout the MMAs read (8-row x 16-byte core matrices, see kmajor_off), so that
// the A tile of one K stage (7 planes x 128 rows x OZ_KS) is one contiguous
// block that a single bulk copy moves:  block (tile t, stage st, plane s)
// starts at ((t * nst + st) * OZ_S + s) * OZ_M * OZ_KS elements.  The snapshot
// (B) slices use the same layout for 64 rows, written by the GEMM's producer
// warps straight into the stage buffer.
__device__ __forceinline__ long long oz_tile_off(long long r, long long kpos, int R, long long nst) {
    const long long t = r / R, st = kpos / OZ_KS;
    const int rr = (int)(r % R), kk = (int)(kpos % OZ_KS);
    return ((t * nst + st) * OZ_S) * (long long)(R * OZ_KS) + (kmajor_off(rr, kk, OZ_KS) >> 1);
}

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

// Balanced base-128 digits of a fixed-point value X (|X| < 2^48):
// alpha_s = round(X_s / 2^(49-7s)) (halves up), X_{s+1} = X_s - alpha_s 2^(49-7s),
// s = 1..7, computed in 32-bit pieces.  The digits with 2^(49-7s) >= 2^28
// depend only on the bits of X from 2^27 up, so they come from hi = X / 2^21
// (rounded down); the 2^21 digit adds the rounding bit of lo = X mod 2^21,
// and the remainder below it fits in 22 bits.  |alpha_s| <= 64.
__device__ __forceinline__ void digits7(long long X, int (&a)[OZ_S]) {
    int hi = (int)(X >> 21);
    const int lo = (int)(X & 0x1FFFFF);
    int d;
    d = (hi + (1 << 20)) >> 21;
    hi -= d * (1 << 21);
    a[0] = d;
    d = (hi + (1 << 13)) >> 14;
    hi -= d * (1 << 14);
    a[1] = d;
    d = (hi + (1 << 6)) >> 7;
    hi -= d * (1 << 7);
    a[2] = d;
    d = hi + ((lo + (1 << 20)) >> 21);
    int r = lo - (d - hi) * (1 << 21);
    a[3] = d;
    d = (r + (1 << 13)) >> 14;
    r -= d * (1 << 14);
    a[4] = d;
    d = (r + (1 << 6)) >> 7;
    r -= d * (1 << 7);
    a[5] = d;
    a[6] = r;
}

// Slices of a (re, im) pair stored as BF16x2 into each of the 7 planes.
__device__ __forceinline__ void slice7_pair(double re, double im, int E, __nv_bfloat162 *out, long long stride2) {
    int a[OZ_S], c[OZ_S];
    digits7(oz_fixed(re, E), a);
    digits7(oz_fixed(im, E), c);
#pragma unroll
    for (int s = 0; s < OZ_S; s++)  // |a|, |c| <= 64: exact in BF16
        out[s * stride2] = __floats2bfloat162_rn(__int2float_rn(a[s]), __int2float_rn(c[s]));
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
    const long long nst = Kp / OZ_KS;
    constexpr long long pstride2 = OZ_M * OZ_KS / 2;  // plane stride in BF16 pairs
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        double2 v = q[i];
        __nv_bfloat162 *re = (__nv_bfloat162 *)(As + oz_tile_off(2 * l, 2 * i, OZ_M, nst));
        __nv_bfloat162 *im = (__nv_bfloat162 *)(As + oz_tile_off(2 * l + 1, 2 * i, OZ_M, nst));
        slice7_pair(v.x, v.y, E, re, pstride2);
        slice7_pair(-v.y, v.x, E, im, pstride2);
    }
}

// B: one warp per column j of this batch finds its scale; the slices
// themselves are made inside the GEMM (k_oz_gemm).  The scale comes from the
// largest biased exponent (integer max over the IEEE bits, no FP64 work):
// max|x| < 2^(e_max - 1022), so E = e_max - 1021, as frexp of the maximum
// would give.
__global__ void k_oz_exp_B(const double2 *__restrict__ X, long long N, long long Mb, long long ldX, int *__restrict__ Eb) {
    const int lane = threadIdx.x & 31;
    for (long long j = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; j < Mb;
         j += ((long long)gridDim.x * blockDim.x) >> 5) {
        const double2 *x = X + j * ldX;
        unsigned int em = 0;
        for (long long i = lane; i < N; i += 32) {
            const double2 v = x[i];
            const unsigned int a = ((unsigned int)(__double_as_longlong(v.x) >> 52)) & 0x7FFu;
            const unsigned int b = ((unsigned int)(__double_as_longlong(v.y) >> 52)) & 0x7FFu;
            em = max(em, max(a, b));
        }
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (lane == 0) Eb[j] = em ? (int)em - 1021 : 0;
    }
}

// (hi, lo) += x, both double-float
__device__ __forceinline__ void dfs_add(float &ah, float &al, float bh, float bl) { df_add(ah, al, bh, bl); }

// Four FP32 columns of this thread's TMEM lane from each of the seven level
// accumulators (level L at column offset L * OZ_N) and from the running
// sums' high words (at tacc), with one wait for all 32 values: the wait
// names every register, so no use can move above it.
__device__ __forceinline__ void tmem_ld4_levels(uint32_t taddr, uint32_t tacc, float (&v)[OZ_LV][4], float (&a)[4]) {
    uint32_t r[OZ_LV + 1][4];
#pragma unroll
    for (int L = 0; L <= OZ_LV; L++)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[L][0]), "=r"(r[L][1]), "=r"(r[L][2]), "=r"(r[L][3])
                     : "r"(L < OZ_LV ? taddr + (uint32_t)(L * OZ_N) : tacc));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                   "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                   "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]), "+r"(r[4][0]), "+r"(r[4][1]),
                   "+r"(r[4][2]), "+r"(r[4][3]), "+r"(r[5][0]), "+r"(r[5][1]), "+r"(r[5][2]), "+r"(r[5][3]),
                   "+r"(r[6][0]), "+r"(r[6][1]), "+r"(r[6][2]), "+r"(r[6][3]), "+r"(r[7][0]), "+r"(r[7][1]),
                   "+r"(r[7][2]), "+r"(r[7][3]));
#pragma unroll
    for (int L = 0; L < OZ_LV; L++)
#pragma unroll
        for (int e = 0; e < 4; e++) v[L][e] = __uint_as_float(r[L][e]);
#pragma unroll
    for (int e = 0; e < 4; e++) a[e] = __uint_as_float(r[OZ_LV][e]);
}

// Four FP32 values into four consecutive columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const float (&a)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(__float_as_uint(a[0])),
                 "r"(__float_as_uint(a[1])), "r"(__float_as_uint(a[2])), "r"(__float_as_uint(a[3]))
                 : "memory");
}

// Four consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&a)[4]) {
    uint32_t r0, r1, r2, r3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3));
    a[0] = __uint_as_float(r0);
    a[1] = __uint_as_float(r1);
    a[2] = __uint_as_float(r2);
    a[3] = __uint_as_float(r3);
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Snapshot (B) slices inside the GEMM.  X = round(v 2^(49-E)) is formed as
// the magnitude |X| (one right shift of the 53-bit significand, at least 5
// bits since |v| < 2^(E-1)) and a sign.  The balanced digits of |X| < 2^48
// come from the unsigned 7-bit fields gamma_s of
// Y = |X| + 64 sum_s 2^(49-7s) > 0: |X| = sum_s (gamma_s - 64) 2^(49-7s), the
// top field taking every bit from 2^42 up (gamma_1 <= 128), so |alpha_s| <= 64
// as for digits7.  A signed digit becomes an FP32 value as
// sign * (2^23 + gamma) - sign * (2^23 + 64) in one FMA (both terms exact, the
// result an integer), and two FP32 digits (at most 8 significant bits) become
// one BF16x2 word by keeping their upper halves: no conversion instructions.
constexpr unsigned long long OZ_OFF =
    64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

__device__ __forceinline__ void digits7f(double v, int E, float (&f)[OZ_S]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(bits >> 32);
    const int e = (int)((hw >> 20) & 0x7FFu);
    const int sh = 1026 + E - e;
    unsigned long long mag = 0;
    if (e != 0 && sh < 64) {  // round half up: (m / 2^(sh-1) + 1) / 2
        const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        mag = ((m >> (sh - 1)) + 1ull) >> 1;
    }
    const unsigned long long Y = mag + OZ_OFF;
    const unsigned lo = (unsigned)Y, hi = (unsigned)(Y >> 32);
    const unsigned g[OZ_S] = {hi >> 10, (hi >> 3) & 127u, (unsigned)(Y >> 28) & 127u, (lo >> 21) & 127u,
                              (lo >> 14) & 127u, (lo >> 7) & 127u, lo & 127u};
    const float sg = (hw >> 31) ? -1.0f : 1.0f;
#pragma unroll
    for (int t = 0; t < OZ_S; t++) f[t] = fmaf(sg, __uint_as_float(0x4B000000u | g[t]), sg * -8388672.0f);
}

// The seven BF16x2 (re, im) slice words of one complex value.
__device__ __forceinline__ void slice7_words(double re, double im, int E, uint32_t (&w)[OZ_S]) {
    float a[OZ_S], c[OZ_S];
    digits7f(re, E, a);
    digits7f(im, E, c);
#pragma unroll
    for (int t = 0; t < OZ_S; t++) w[t] = __byte_perm(__float_as_uint(a[t]), __float_as_uint(c[t]), 0x7632);
}

// The GEMM with the snapshot slicing inside it, persistent and stream-K.
// A work unit is one exact chunk (OZ_DRAIN K values = OZ_CHUNK stages) of one
// tile of 128 basis rows by 64 snapshot columns (K is padded to whole chunks
// with zero basis planes); tile t is row tile t % nrt, column tile t / nrt.
// Block i of G takes the contiguous units [i U / G, (i+1) U / G), so every
// block does the same work whatever the tile count.  A tile whose chunks all
// fall to one block is written to C by it; a tile shared by blocks leaves
// each block's part (unscaled double sums) in that block's slot -- 2i when
// the tile is the block's first, 2i + 1 when it is its last -- and
// k_oz_fixup adds the parts in chunk order.
//
// Roles.  Warps 0-15 (512 producer threads) read X and write the seven B
// slice planes of each stage straight into the stage's shared-memory buffer:
// lane l of warp w owns column 64 ct + 8 (w / 2) + l / 4 and complex
// element 4 (w % 2) + l % 4 of every stage, and reads X in groups of OZ_FG
// stages (the 512 contiguous bytes of a column per group come from two
// warps), two groups ahead of the slicing.  Lane 0 of warp 17
// fills the A half of each buffer with one bulk copy of the pre-sliced basis
// (28 KB, L2-resident) as soon as the buffer's previous MMAs are done.  Lane
// 0 of warp 16 issues the stage's MMAs: slice sa of A against the
// consecutive B planes sb .. sb+g-1 as one operand of 64 g rows (the planes
// are 64 rows apart in the K-major layout), whose product lands on the TMEM
// levels sa+sb .. sa+sb+g-1 (the levels are 64 columns apart) -- 10 MMAs of
// N = 64 .. 256 per stage.  The producers and warp 16 meet at a named barrier
// after each unit (the levels drained before the next unit overwrites them);
// warp 17 stays out of it and copies ahead across units.
//
// Two rings: OZ_NA buffers for A (a copy from L2 takes a few stages to
// land) and OZ_NB for B (the producers run ahead of the MMAs).  Barriers per
// buffer: "afull" counts the A bytes, "bfull" one arrival per producer warp,
// "adone" / "bdone" receive the MMA commit of the buffer's stage; the n-th
// phase of buffer b of a ring of depth D belongs to the block's stage b + D n
// (buffer and phase parity are carried along with the stage count).  Before
// draining a unit the producers already store the first read group of the
// next unit of the same tile (its buffers were freed by this unit's MMAs),
// so that the MMAs restart as soon as the drain ends.  At the end of each
// unit the producers drain the TMEM levels into double-float running sums
// whose high words stay in TMEM (the 64 columns after the levels) and whose
// low words sit in shared memory (column-major, so a warp's 32 rows are 32
// consecutive words): thread (warp w, lane l) owns row 32 (w % 4) + l (its
// TMEM lane) and columns 16 (w / 4) .. + 15.  Keeping the high words out of
// shared memory leaves room for a fourth A buffer.
constexpr int OZ_NA = 4;  // A ring depth
constexpr int OZ_NB = 5;  // B ring depth
constexpr int OZ_PWARPS = 16;
constexpr int OZ_PRODUCERS = 32 * OZ_PWARPS;
constexpr int OZ_THREADS = OZ_PRODUCERS + 64;      // 18 warps: + the MMA warp and the copy warp
constexpr int OZ_FG = 4;                           // stages per X read group
constexpr int OZ_CHUNK = OZ_DRAIN / OZ_KS;         // stages per work unit (32)
constexpr int OZ_DC = OZ_N / (OZ_PWARPS / 4);      // columns drained per thread (16)
constexpr int OZ_SA = OZ_S * OZ_M * OZ_KS * 2;     // A part of a stage (28 KB)
constexpr int OZ_SB = OZ_S * OZ_N * OZ_KS * 2;     // B part (14 KB)
constexpr int OZ_ACC = OZ_M * OZ_N * 4;            // running sums' low words (32 KB)
constexpr int OZ_MAX_BLOCKS = 256;                 // blocks of the persistent launch (at most)
static_assert(OZ_CHUNK % (2 * OZ_FG) == 0 && OZ_FG % 2 == 0, "units hold whole pairs of read groups");
// the early read group of the next unit waits only for MMAs of this unit
static_assert(OZ_FG < OZ_NB, "B ring deeper than a read group");
static_assert(OZ_PRODUCERS == OZ_N * (OZ_KS / 2), "one complex element per producer and stage");
// the grouped MMAs: plane sb + 1 of a B stage starts where row OZ_N of plane sb
// would (8-row groups (OZ_KS / 8) * 128 bytes apart), and the levels fit TMEM
static_assert((OZ_N / 8) * ((OZ_KS / 8) * 128) == OZ_N * OZ_KS * 2, "B planes contiguous as rows");
static_assert(OZ_LV * OZ_N <= OZ_ACOL && OZ_ACOL + OZ_N <= OZ_TCOLS && 4 * OZ_N <= 256, "level columns");

// A position in a ring of D buffers: the buffer and the phase parity of its
// current use.
struct RingPos {
    int i;
    uint32_t ph;
};
template <int D>
__device__ __forceinline__ void ring_next(RingPos &r) {
    if (++r.i == D) {
        r.i = 0;
        r.ph ^= 1u;
    }
}

// First unit of block i of G over U units.
__host__ __device__ __forceinline__ long long oz_u0(long long i, long long U, long long G) { return i * U / G; }

// The block whose range holds unit x.
__device__ __forceinline__ int oz_block_of(long long x, long long U, int G) {
    int i = (int)(x * G / U);
    while (i + 1 < G && oz_u0(i + 1, U, G) <= x) i++;
    while (i > 0 && oz_u0(i, U, G) > x) i--;
    return i;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const __nv_bfloat16 *__restrict__ As,
                                                        const double2 *__restrict__ X, long long N, long long ldX,
                                                        const int *__restrict__ Ea, const int *__restrict__ Eb, int k,
                                                        long long Mb, long long Kp, int nrt, long long U,
                                                        double *__restrict__ part, double2 *__restrict__ C,
                                                        long long ldC, long long col_off, int *err,
                                                        unsigned long long wait) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    __shared__ __align__(8) uint64_t afull[OZ_NA], adone[OZ_NA], bfull[OZ_NB], bdone[OZ_NB], cdone;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp < OZ_PWARPS;
    const bool issuer = threadIdx.x == OZ_PRODUCERS;       // lane 0 of warp 16
    const bool copier = threadIdx.x == OZ_PRODUCERS + 32;  // lane 0 of warp 17
    const int row = 32 * (warp & 3) + lane, cbase = OZ_DC * ((warp >> 2) & 3);
    uint8_t *bring = dsm + OZ_NA * OZ_SA;                        // the B ring after the A ring
    float *acc_ls = (float *)(bring + OZ_NB * OZ_SB);            // low words, [column][row]
    if (producer)
#pragma unroll
        for (int c = 0; c < OZ_DC; c++) acc_ls[(cbase + c) * OZ_M + row] = 0.f;
    if (warp == 0) tmem_alloc(&tslot, OZ_TCOLS);
    if (threadIdx.x == 0) {
        for (int b = 0; b < OZ_NA; b++) {
            mbar_init(&afull[b], 1);
            mbar_init(&adone[b], 1);
        }
        for (int b = 0; b < OZ_NB; b++) {
            mbar_init(&bfull[b], OZ_PWARPS);
            mbar_init(&bdone[b], 1);
        }
        mbar_init(&cdone, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    // this thread's TMEM lane (its row) and the running sums' high words
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t tacc = tmem + lane_off + (uint32_t)(OZ_ACOL + cbase);
    if (producer) {
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int h = 0; h < OZ_DC / 4; h++) tmem_st4(tacc + 4 * h, z);
        tmem_wait_st();
    }
    bool ok = true;
    const int nst = (int)(Kp / OZ_KS);  // whole units, Kp <= 2^23
    const int nch = nst / OZ_CHUNK;
    const int G = (int)gridDim.x;
    const long long u0 = oz_u0(blockIdx.x, U, G), u1 = oz_u0(blockIdx.x + 1, U, G);
    const int nu = (int)(u1 - u0);  // units of this block
    // tile indices fit 32 bits: X (16 N bytes per column) and Q fit in device memory
    const int t_first = (int)(u0 / nch);
    const uint32_t dsm0 = smem_u32(dsm);
    // producer: this thread's column of a tile and its complex element of a stage
    // warp w covers 8 columns x 4 complex elements: its slice words of one plane
    // are 32 consecutive words of the K-major buffer (one store, no bank conflict)
    const int jj = 8 * ((warp >> 1) & 7) + (lane >> 2), p0 = 4 * (warp & 1) + (lane & 3);
    constexpr int pstride = OZ_N * OZ_KS / 2;  // plane stride in 32-bit words
    const uint32_t woff = kmajor_off(jj, 2 * p0, OZ_KS) >> 2;
    int E = 0, nlim = 0;                       // of the current tile's column
    const double2 *x = X;
    // two register sets of OZ_FG stages: read group q (stages OZ_FG q ..) uses set q % 2
    double2 xa[OZ_FG], xb[OZ_FG];
    const int ngr = nst / OZ_FG;
    auto fetch = [&](int q, double2 (&v)[OZ_FG]) {
#pragma unroll
        for (int u = 0; u < OZ_FG; u++) {
            const int st = q * OZ_FG + u;
            v[u] = st < nlim ? x[(long long)st * (OZ_KS / 2)] : make_double2(0.0, 0.0);
        }
    };
    const long long gtot = (long long)nu * OZ_CHUNK;  // stages of this block
    // this thread's position in each ring (buffer, phase parity of its use)
    // and its role's count of the block's stages
    RingPos ra{0, 0u}, rb{0, 0u};
    long long g = 0;
    // the barrier of the producers and the MMA warp at the end of a unit: the
    // levels are drained before the next unit's first MMAs overwrite them
    auto unit_sync = [&]() {
        tc_fence_before();
        asm volatile("bar.sync 1, %0;" ::"r"(OZ_PRODUCERS + 32) : "memory");
        tc_fence_after();
    };
    // the slice words of tile stage st (zeros past the column's end) into the
    // stage's B buffer, once the MMAs of stage g - OZ_NB are done with it
    auto store = [&](int st, const uint32_t (&w)[OZ_S]) {
        if (g >= OZ_NB) ok = mbar_wait(&bdone[rb.i], rb.ph ^ 1u, wait) && ok;
        uint32_t *o = (uint32_t *)(bring + rb.i * OZ_SB) + woff;
        const bool in = st < nlim;
#pragma unroll
        for (int t = 0; t < OZ_S; t++) o[t * pstride] = in ? w[t] : 0u;
    };
    // two consecutive stages: one fence makes both buffers visible to the
    // tensor core, then one lane arrives on each
    auto put2 = [&](int st, const uint32_t (&w0)[OZ_S], const uint32_t (&w1)[OZ_S]) {
        store(st, w0);
        const int b0 = rb.i;
        ring_next<OZ_NB>(rb);
        g++;
        store(st + 1, w1);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull[b0])) : "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull[rb.i])) : "memory");
        }
        ring_next<OZ_NB>(rb);
        g++;
    };
    // a read group in pairs of stages: both stages' values are sliced first
    // (independent work), then stored
    auto group = [&](int q, double2 (&v)[OZ_FG]) {
#pragma unroll
        for (int u = 0; u < OZ_FG; u += 2) {
            uint32_t w0[OZ_S], w1[OZ_S];
            slice7_words(v[u].x, v[u].y, E, w0);
            slice7_words(v[u + 1].x, v[u + 1].y, E, w1);
            put2(q * OZ_FG + u, w0, w1);
        }
        if (q + 2 < ngr) fetch(q + 2, v);
    };
    int seg_c0 = 0;    // first chunk of the current tile segment
    bool early = false;  // this unit's first read group was stored before the last drain
    if (producer) {
    for (int du = 0; du < nu; du++) {
        const long long u = u0 + du;
        const int t = (int)(u / nch);
        const int c = (int)(u - (long long)t * nch);
        const int rt = t % nrt;
        const int ct = t / nrt;
        if (du == 0 || c == 0) {  // a new tile: this thread's column, its scale and first reads
            seg_c0 = c;
            const long long j = (long long)ct * OZ_N + jj;
            const bool live = j < Mb;
            E = live ? Eb[j] : 0;
            x = X + (live ? j : 0) * ldX + p0;
            nlim = live ? (int)((N - p0 + (OZ_KS / 2) - 1) / (OZ_KS / 2)) : 0;  // stages holding the element
            fetch(c * (OZ_CHUNK / OZ_FG), xa);
            fetch(c * (OZ_CHUNK / OZ_FG) + 1, xb);
        }
        {
            // read group q uses register set q % 2 (a unit starts on an even group)
            const int q0 = c * (OZ_CHUNK / OZ_FG), q1 = q0 + OZ_CHUNK / OZ_FG;
            for (int q = q0 + (early ? 1 : 0); q < q1; q++) {
                if (q & 1) group(q, xb);
                else group(q, xa);
            }
            // the next unit's first read group, when that unit continues this
            // tile: its OZ_FG < OZ_NB buffers wait only for MMAs of this unit
            early = du + 1 < nu && c + 1 < nch;
            if (early) group(q1, xa);
            // drain: wait for the unit's MMAs (cdone completes once per unit and
            // no thread runs more than one unit behind), then read this
            // thread's TMEM lane; levels combined smallest first, in double-float
            ok = mbar_wait(&cdone, (uint32_t)(du & 1), wait) && ok;
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < OZ_DC / 4; h++) {
                float v[OZ_LV][4], ah[4];
                tmem_ld4_levels(tmem + lane_off + (uint32_t)(cbase + 4 * h), tacc + 4 * h, v, ah);
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    // levels added smallest first by TwoSum, the errors gathered
                    // in tl (normalised once, by the add into the running sums)
                    float th = 0.f, tl = 0.f;
#pragma unroll
                    for (int L = OZ_LV - 1; L >= 0; L--) {
                        // level L+2 carries 2^(-7 (L+2)): an exact power-of-two factor
                        const float xl = v[L][e] * __int_as_float((127 - OZ_BITS * (L + 2)) << 23);
                        float sh, se;
                        two_sum(th, xl, sh, se);
                        th = sh;
                        tl = __fadd_rn(tl, se);
                    }
                    const int a = (cbase + 4 * h + e) * OZ_M + row;
                    float al = acc_ls[a];
                    dfs_add(ah[e], al, th, tl);
                    acc_ls[a] = al;
                }
                tmem_st4(tacc + 4 * h, ah);
            }
            tmem_wait_st();
            if (du == nu - 1 || c == nch - 1) {
                // the tile segment ends: the whole tile goes to C, a part to the
                // block's slot; the sums restart at zero for the next tile
                const long long R = (long long)rt * OZ_M + row;
                const bool whole = seg_c0 == 0 && c == nch - 1;
                const long long slot = 2LL * blockIdx.x + (t == t_first ? 0 : 1);
#pragma unroll
                for (int h = 0; h < OZ_DC / 4; h++) {
                    float ah[4];
                    tmem_ld4(tacc + 4 * h, ah);
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int cl = cbase + 4 * h + e;
                        const double val = (double)ah[e] + (double)acc_ls[cl * OZ_M + row];
                        acc_ls[cl * OZ_M + row] = 0.f;
                        ah[e] = 0.f;
                        const long long jc = (long long)ct * OZ_N + cl;
                        if (whole) {
                            if (R < 2LL * k && jc < Mb)
                                ((double *)(C + (R >> 1) * ldC) + (R & 1))[2 * (col_off + jc)] =
                                    ldexp(val, Ea[R >> 1] + Eb[jc]);
                        } else {
                            part[(slot * OZ_N + cl) * OZ_M + row] = val;
                        }
                    }
                    tmem_st4(tacc + 4 * h, ah);
                }
                tmem_wait_st();
            }
        }
        unit_sync();
    }
    } else if (warp == OZ_PWARPS) {
        // warp 16: lane 0 issues; the unit barrier with the producers
        auto issue = [&](bool first_of_unit) {
            ok = mbar_wait(&afull[ra.i], ra.ph, wait) && ok;
            ok = mbar_wait(&bfull[rb.i], rb.ph, wait) && ok;
            tc_fence_after();
            // one descriptor per operand and stage; slices and K steps are
            // constant offsets of its 16-byte address field
            const uint64_t ad0 = smem_desc(dsm0 + (uint32_t)(ra.i * OZ_SA), 128, (OZ_KS / 8) * 128);
            const uint64_t bd0 = smem_desc(dsm0 + (uint32_t)(OZ_NA * OZ_SA + rb.i * OZ_SB), 128, (OZ_KS / 8) * 128);
            const uint32_t acc0 = first_of_unit ? 0u : 1u;  // a unit's first stage overwrites the levels
#pragma unroll
            for (int sa = 0; sa < OZ_S; sa++)
#pragma unroll
                for (int sb = 0; sb < OZ_S - sa; sb += 4) {
                    const int gg = OZ_S - sa - sb < 4 ? OZ_S - sa - sb : 4;
                    const int L = sa + sb;  // first level - 2
#pragma unroll
                    for (int kk = 0; kk < OZ_KS / 16; kk++) {
                        const uint64_t ad = ad0 + (uint64_t)((sa * (OZ_M * OZ_KS * 2) + kk * 256) >> 4);
                        const uint64_t bd = bd0 + (uint64_t)((sb * (OZ_N * OZ_KS * 2) + kk * 256) >> 4);
                        // every level is first reached at sa = 0 (sb = L <= 6)
                        const uint32_t ac = (sa == 0 && kk == 0) ? acc0 : 1u;
                        tc_mma_bf16(tmem + (uint32_t)(L * OZ_N), ad, bd, idesc_bf16_f32(OZ_M, gg * OZ_N), ac);
                    }
                }
            tc_commit(&adone[ra.i]);
            tc_commit(&bdone[rb.i]);
            ring_next<OZ_NA>(ra);
            ring_next<OZ_NB>(rb);
        };
        for (int du = 0; du < nu; du++) {
            if (issuer) {
                for (int s2 = 0; s2 < OZ_CHUNK; s2++) issue(s2 == 0);
                tc_commit(&cdone);
            }
            __syncwarp();
            unit_sync();
        }
    } else {
        // warp 17: lane 0 copies the basis planes of every stage into its
        // buffer once the buffer's previous MMAs are done, across unit
        // boundaries (it keeps out of the unit barrier)
        // The basis copies go out in the block's stage order (units u0 .. in
        // order, OZ_CHUNK stages each), so their source advances one stage at
        // a time and is recomputed once per unit
        constexpr long long a_stage = (long long)OZ_S * OZ_M * OZ_KS;  // elements per stage
        auto unit_a = [&](long long u) {
            const long long t = u / nch;
            return As + ((t % nrt) * nst + (u % nch) * OZ_CHUNK) * a_stage;
        };
        long long a_u = u0;
        int a_s = 0;
        const __nv_bfloat16 *a_base = unit_a(u0);
        auto load_a = [&](int bb) {  // the next stage's A into buffer bb
            uint64_t *fb = &afull[bb];
            mbar_expect_tx(fb, OZ_SA);
            bulk_g2s(dsm + bb * OZ_SA, a_base + a_s * a_stage, OZ_SA, fb);
            if (++a_s == OZ_CHUNK) {
                a_s = 0;
                if (++a_u < u1) a_base = unit_a(a_u);
            }
        };
        if (copier) {
            for (long long gg = 0; gg < gtot; gg++) {
                if (gg >= OZ_NA) ok = mbar_wait(&adone[ra.i], ra.ph ^ 1u, wait) && ok;  // the MMAs of stage gg - OZ_NA
                load_a(ra.i);
                ring_next<OZ_NA>(ra);
            }
        }
        __syncwarp();
    }
    if (!ok && err) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, OZ_TCOLS);
}

// The tiles that several blocks shared: the parts in chunk order (block
// order), then the two scales, into C.  One block per tile; a tile that one
// block finished returns at once.
__global__ void k_oz_fixup(const double *__restrict__ part, const int *__restrict__ Ea, const int *__restrict__ Eb,
                           int k, long long Mb, int nrt, int nch, long long U, int G, double2 *__restrict__ C,
                           long long ldC, long long col_off) {
    const long long t = blockIdx.x;
    const int i0 = oz_block_of(t * nch, U, G), i1 = oz_block_of(t * nch + nch - 1, U, G);
    if (i0 == i1) return;
    const int rt = (int)(t % nrt);
    const long long ct = t / nrt;
    // the sharing blocks' slots, once per block (64-bit divisions), not per element
    constexpr int MAXS = 64;
    __shared__ long long s_slot[MAXS];
    const int ns = i1 - i0 + 1;
    auto slot_of = [&](int i) { return 2LL * i + (oz_u0(i, U, G) / nch == t ? 0 : 1); };
    for (int j = threadIdx.x; j < ns && j < MAXS; j += blockDim.x) s_slot[j] = slot_of(i0 + j);
    __syncthreads();
    for (int e = threadIdx.x; e < OZ_M * OZ_N; e += blockDim.x) {
        const int row = e % OZ_M, col = e / OZ_M;
        const long long R = (long long)rt * OZ_M + row, jc = ct * OZ_N + col;
        if (R >= 2LL * k || jc >= Mb) continue;
        double sum = 0.0;
        for (int j = 0; j < ns; j++) {
            const long long slot = j < MAXS ? s_slot[j] : slot_of(i0 + j);
            sum += part[(slot * OZ_N + col) * OZ_M + row];
        }
        ((double *)(C + (R >> 1) * ldC) + (R & 1))[2 * (col_off + jc)] = ldexp(sum, Ea[R >> 1] + Eb[jc]);
    }
}

// Self-test of the bounded mbarrier wait used by every tensor-core kernel: one
// thread waits on a barrier that nothing arrives on (unless `arrive`), with a
// budget of `cycles` SM clock cycles, and records a time-out in *flag.  No tensor-core work is
// in flight, so running out of budget leaves nothing behind.
__global__ void k_wait_selftest(long long cycles, int arrive, int *flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        if (!mbar_wait(&bar, 0, (unsigned long long)cycles)) *flag = 1;
    }
}

cudaError_t launch_wait_selftest(long long cycles, int arrive, int *flag, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(cycles, arrive, flag);
    return cudaGetLastError();
}

// K padded to whole exact chunks (zero basis planes past 2N).
static long long oz_kp(long long N) { return (2 * N + OZ_DRAIN - 1) / OZ_DRAIN * OZ_DRAIN; }

size_t oz_workspace(long long N, int k, long long Mb) {
    const long long Kp = oz_kp(N);
    const long long Rp = (2LL * k + OZ_M - 1) / OZ_M * OZ_M;
    const size_t parts = (size_t)2 * OZ_MAX_BLOCKS * OZ_M * OZ_N * sizeof(double);
    return (size_t)OZ_S * Rp * Kp * 2 + parts + (size_t)(k + Mb) * 4 + 4096;
}

// C[:, col_off : col_off + Mb] for one batch of Mb columns; ws from oz_workspace.
cudaError_t launch_project_tc(const double2 *Q, long long N, int k, long long ldQ, const double2 *X, long long Mb,
                              long long ldX, double2 *C, long long ldC, long long col_off, void *ws, int *err,
                              unsigned long long wait, cudaStream_t s) {
    if (k <= 0 || Mb <= 0) return cudaSuccess;
    const long long Kp = oz_kp(N);
    const long long Rp = (2LL * k + OZ_M - 1) / OZ_M * OZ_M;
    const long long Cp = (Mb + OZ_N - 1) / OZ_N * OZ_N;
    __nv_bfloat16 *As = (__nv_bfloat16 *)ws;
    double *part = (double *)(As + (size_t)OZ_S * Rp * Kp);
    int *Ea = (int *)(part + (size_t)2 * OZ_MAX_BLOCKS * OZ_M * OZ_N);
    int *Eb = Ea + k;
    // zero fill of the A planes (small: rows 2k..Rp-1 and the K padding)
    cudaError_t e = cudaMemsetAsync(As, 0, (size_t)OZ_S * Rp * Kp * 2, s);
    if (e != cudaSuccess) return e;
    k_oz_slice_A<<<k, 256, 0, s>>>(Q, N, k, ldQ, Kp, Rp, As, Ea);
    const long long ge = (Mb * 32 + 255) / 256;
    k_oz_exp_B<<<(unsigned)(ge < 4096 ? ge : 4096), 256, 0, s>>>(X, N, Mb, ldX, Eb);
    const size_t dsm = (size_t)OZ_NA * OZ_SA + (size_t)OZ_NB * OZ_SB + OZ_ACC;  // 182 KB of rings + 32 KB of sums
    static int sms = 0;
    if (!sms) {
        cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int nrt = (int)(Rp / OZ_M);
    const long long tiles = (long long)nrt * (Cp / OZ_N);
    const int nch = (int)(Kp / OZ_DRAIN);
    const long long U = tiles * nch;  // work units
    long long G = sms < OZ_MAX_BLOCKS ? sms : OZ_MAX_BLOCKS;
    if (G > U) G = U;
    k_oz_gemm<<<(unsigned)G, OZ_THREADS, dsm, s>>>(As, X, N, ldX, Ea, Eb, k, Mb, Kp, nrt, U, part, C, ldC, col_off,
                                                  err, wait);
    k_oz_fixup<<<(unsigned)tiles, 256, 0, s>>>(part, Ea, Eb, k, Mb, nrt, nch, U, (int)G, C, ldC, col_off);
    return cudaGetLastError();
}

}  // namespace rbk
