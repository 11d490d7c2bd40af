// rb_imgs.cu -- orthogonalisation of the pivot column (Sec. 6.1.2: Hoffmann's
// iterated Gram-Schmidt, "MGSCI" with kappa = 2; the remark after Prop. 5.3).
//
// GPU form: each pass is one classical Gram-Schmidt step written as two
// GEMVs, h = Q_k^H v then v -= Q_k h (the paper notes that its MGS passes
// cannot be cast as matrix-vector products when the basis arrives one vector
// at a time; a CGS-form pass can).  Hoffmann's test is unchanged: a pass is
// accepted when ||v_after|| >= ||v_before|| / kappa, otherwise another pass
// runs, up to max_passes (then RB_EORTHO).  All arithmetic is FP64.
//
// The pass count is decided on the device: the host queues max_passes
// (dot, update) pairs and every launch returns at once when the state says
// the vector was already accepted or the loop has stopped.
#include "rb_internal.cuh"

namespace rbk {

// Every step is a device body over blockIdx.x / gridDim.x, launched either for
// one problem (Prob by value) or for a batch (blockIdx.y selects the problem
// in a device array), so a batch of problems takes one launch per step.

// v = s_J (FP64 copy of the pivot column), reset the pass counters.
__device__ __forceinline__ void imgs_begin(const Prob &p, int from_split) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    long long J = st->J;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
         i += (long long)gridDim.x * blockDim.x) {
        double2 x;
        if (from_split) {
            float2 a = p.hi[J * p.ldH + i], b = p.lo[J * p.ldH + i];
            x = make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
        } else {
            x = p.S[J * p.ldS + i];
        }
        p.v[i] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->passes = 0;
        st->accepted = (st->k == 0);
        st->before2 = p.norm2[J];
        st->after2 = p.norm2[J];
    }
}

// Partial h_l over one row chunk: hpart[l][c] = sum_{i in chunk c} conj(q_l[i]) v[i].
__device__ __forceinline__ void imgs_dot(const Prob &p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || ld_volatile(&st->accepted)) return;
    const int k = st->k;
    const long long items = (long long)k * p.nchunk;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        int l = (int)(it / p.nchunk), c = (int)(it % p.nchunk);
        long long i0 = (long long)c * p.chunk, i1 = i0 + p.chunk;
        if (i1 > p.N) i1 = p.N;
        const double2 *q = p.Q + (long long)l * p.ldQ;
        double re = 0.0, im = 0.0;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            double2 a = q[i], b = p.v[i];
            re = fma(a.x, b.x, fma(a.y, b.y, re));
            im = fma(a.x, b.y, fma(-a.y, b.x, im));
        }
        double2 h = block_sum2(make_double2(re, im));
        if (threadIdx.x == 0) p.hpart[(long long)l * p.nchunk + c] = h;
        __syncthreads();
    }
}

// v -= Q_k h with h_l = sum_c hpart[l][c]; ||v||^2; kappa test in the last block.
// One element per thread: gridDim.x * blockDim.x >= N.
__device__ __forceinline__ void imgs_update(const Prob &p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop) || ld_volatile(&st->accepted)) return;
    const int k = st->k;
    constexpr int TL = 256;
    __shared__ double2 hs[TL];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double2 d = make_double2(0.0, 0.0);
    for (int l0 = 0; l0 < k; l0 += TL) {
        int nl = k - l0 < TL ? k - l0 : TL;
        __syncthreads();
        for (int t = threadIdx.x; t < nl; t += blockDim.x) {
            double2 h = make_double2(0.0, 0.0);
            const double2 *hp = p.hpart + (long long)(l0 + t) * p.nchunk;
            for (int c = 0; c < p.nchunk; c++) {
                double2 x = hp[c];
                h.x += x.x;
                h.y += x.y;
            }
            hs[t] = h;
        }
        __syncthreads();
        if (i < p.N) {
            for (int t = 0; t < nl; t++) {
                double2 q = p.Q[(long long)(l0 + t) * p.ldQ + i];
                double2 h = hs[t];
                d.x = fma(q.x, h.x, fma(-q.y, h.y, d.x));
                d.y = fma(q.x, h.y, fma(q.y, h.x, d.y));
            }
        }
    }
    double n2 = 0.0;
    if (i < p.N) {
        double2 x = p.v[i];
        x.x -= d.x;
        x.y -= d.y;
        p.v[i] = x;
        n2 = x.x * x.x + x.y * x.y;
    }
    n2 = block_sum(n2);
    if (threadIdx.x == 0) p.npart[blockIdx.x] = n2;
    if (!last_block(&st->ticket_imgs)) return;
    double tot = 0.0;
    if (threadIdx.x == 0) {
        for (int b = 0; b < gridDim.x; b++) tot += __ldcg(p.npart + b);
        st->ticket_imgs = 0;
        st->after2 = tot;
        st->passes += 1;
        st->total_passes += 1;
        if (tot >= st->before2 / p.kappa2) {
            st->accepted = 1;
        } else {
            st->before2 = tot;
            if (st->passes >= p.max_passes) {
                st->status = RB_EORTHO;
                st->stop = 1;
            }
        }
    }
}

// q_k = v / ||v||; Q[:, k], its FP32 hi/lo split for the sweep, pivot, R(k,k).
__device__ __forceinline__ void imgs_finalize(const Prob &p) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;
    const int k = st->k;
    const double nv2 = st->after2;
    if (!(nv2 > 0.0)) {
        // the pivot column lies in the span already: exact rank reached
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (p.qs_stride && st->phase == 0) {
                // split form, hi-only phase: make C and the errors exact, then stop
                st->switch_pending = 1;
                st->force_stop = 1;
            } else {
                st->status = RB_OK;
                st->stop = 1;
            }
        }
        return;
    }
    const double nv = sqrt(nv2);
    double2 *qk = p.Q + (long long)k * p.ldQ;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
         i += (long long)gridDim.x * blockDim.x) {
        double2 x = p.v[i];
        double2 q = make_double2(x.x / nv, x.y / nv);
        qk[i] = q;
        if (p.qh) {
            float hr = __double2float_rn(q.x), hm = __double2float_rn(q.y);
            long long o = (long long)k * p.qs_stride + i;
            p.qh[o] = make_float2(hr, hm);
            p.ql[o] = make_float2(__double2float_rn(q.x - (double)hr), __double2float_rn(q.y - (double)hm));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long J = st->J;
        p.pivots[k] = J;
        if (p.rdiag) p.rdiag[k] = nv;
        if (p.passes_out) p.passes_out[k] = st->passes;
        p.picked[J] = 1;
    }
}

__global__ void __launch_bounds__(kThreads) k_imgs_begin(Prob p, int from_split) { imgs_begin(p, from_split); }
__global__ void __launch_bounds__(kThreads) k_imgs_dot(Prob p) { imgs_dot(p); }
__global__ void __launch_bounds__(kThreads) k_imgs_update(Prob p) { imgs_update(p); }
__global__ void __launch_bounds__(kThreads) k_imgs_finalize(Prob p) { imgs_finalize(p); }

__global__ void __launch_bounds__(kThreads) k_imgs_begin_b(const Prob *pp) { imgs_begin(pp[blockIdx.y], 0); }
__global__ void __launch_bounds__(kThreads) k_imgs_dot_b(const Prob *pp) { imgs_dot(pp[blockIdx.y]); }
__global__ void __launch_bounds__(kThreads) k_imgs_update_b(const Prob *pp) { imgs_update(pp[blockIdx.y]); }
__global__ void __launch_bounds__(kThreads) k_imgs_finalize_b(const Prob *pp) { imgs_finalize(pp[blockIdx.y]); }

cudaError_t launch_imgs(const Prob &p, int grid, bool from_split, cudaStream_t s, int *nlaunch) {
    int gN = (int)((p.N + kThreads - 1) / kThreads);
    int gcopy = gN < grid ? gN : grid;
    k_imgs_begin<<<gcopy, kThreads, 0, s>>>(p, from_split ? 1 : 0);
    int n = 1;
    for (int pass = 0; pass < p.max_passes; pass++) {
        k_imgs_dot<<<grid, kThreads, 0, s>>>(p);
        k_imgs_update<<<gN, kThreads, 0, s>>>(p);
        n += 2;
    }
    k_imgs_finalize<<<gcopy, kThreads, 0, s>>>(p);
    n += 1;
    if (nlaunch) *nlaunch += n;
    return cudaGetLastError();
}

// The (dot, update) pass pairs alone, for a caller that prepares p.v and the
// state itself (the column-sharded greedy).
cudaError_t launch_imgs_passes(const Prob &p, int grid, cudaStream_t s, int *nlaunch) {
    const int gN = (int)((p.N + kThreads - 1) / kThreads);
    for (int pass = 0; pass < p.max_passes; pass++) {
        k_imgs_dot<<<grid, kThreads, 0, s>>>(p);
        k_imgs_update<<<gN, kThreads, 0, s>>>(p);
    }
    if (nlaunch) *nlaunch += 2 * p.max_passes;
    return cudaGetLastError();
}

// The same steps for nprob problems at once (complex128 input): grid.y is the
// problem, grid.x is sized for the largest N (smaller problems leave the extra
// blocks idle; every problem's npart must hold gridDim.x entries).
cudaError_t launch_imgs_batched(const Prob *pp_dev, int nprob, long long maxN, int max_passes, int grid,
                                cudaStream_t s, int *nlaunch) {
    const int gN = (int)((maxN + kThreads - 1) / kThreads);
    const int gcopy = gN < grid ? gN : grid;
    k_imgs_begin_b<<<dim3(gcopy, nprob), kThreads, 0, s>>>(pp_dev);
    int n = 1;
    // the dot step's items are (basis vector, row chunk) pairs: k * nchunk,
    // a few hundred at most per problem
    const int gdot = grid < 128 ? grid : 128;
    for (int pass = 0; pass < max_passes; pass++) {
        k_imgs_dot_b<<<dim3(gdot, nprob), kThreads, 0, s>>>(pp_dev);
        k_imgs_update_b<<<dim3(gN, nprob), kThreads, 0, s>>>(pp_dev);
        n += 2;
    }
    k_imgs_finalize_b<<<dim3(gcopy, nprob), kThreads, 0, s>>>(pp_dev);
    n += 1;
    if (nlaunch) *nlaunch += n;
    return cudaGetLastError();
}

}  // namespace rbk
