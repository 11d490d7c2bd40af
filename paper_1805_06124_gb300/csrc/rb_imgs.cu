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
// The pass count is decided on the device.  A single problem's iteration is
// one cooperative launch that loops over the passes between grid barriers
// (k_imgs_fused); the batched and column-sharded forms queue max_passes
// (dot, update) launch pairs instead, each returning at once when the state
// says the vector was already accepted or the loop has stopped.
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

__global__ void __launch_bounds__(kThreads) k_imgs_dot(Prob p) { imgs_dot(p); }
__global__ void __launch_bounds__(kThreads) k_imgs_update(Prob p) { imgs_update(p); }

__global__ void __launch_bounds__(kThreads) k_imgs_begin_b(const Prob *pp) { imgs_begin(pp[blockIdx.y], 0); }
__global__ void __launch_bounds__(kThreads) k_imgs_dot_b(const Prob *pp) { imgs_dot(pp[blockIdx.y]); }
__global__ void __launch_bounds__(kThreads) k_imgs_update_b(const Prob *pp) { imgs_update(pp[blockIdx.y]); }
__global__ void __launch_bounds__(kThreads) k_imgs_finalize_b(const Prob *pp) { imgs_finalize(pp[blockIdx.y]); }

// ------------------------------------------------ one launch per iteration
// The same steps in one cooperative launch (every block resident): begin,
// the passes and finalize separated by grid-wide barriers, so an iteration
// costs one launch instead of 2 + 2 max_passes.  The arithmetic and its
// order are those of the separate kernels above (the dot items, the norm
// partials of 256-element "virtual blocks" summed in block order), so both
// give identical results.  Data that other blocks wrote during the launch
// (v, the partials) is read through L2.

// Bounded grid barrier on the state's arrival counter and generation; false
// in every thread of the block when the wait ran out of its budget.
__device__ bool imgs_grid_sync(DevState *st, unsigned long long budget) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &st->bar_gen;
        const unsigned int g0 = *gen;
        int ok = 1;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            st->bar_count = 0u;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const unsigned long long t0 = (unsigned long long)clock64();
            while (*gen == g0) {
                if ((unsigned long long)clock64() - t0 > budget) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kThreads) k_imgs_fused(Prob p, int from_split) {
    DevState *st = p.st;
    if (ld_volatile(&st->stop)) return;  // nothing in this launch sets it before the first barrier
    const unsigned long long budget = p.wait_cycles ? p.wait_cycles : kWaitCyclesDefault;
    auto timed_out = [&]() {
        if (threadIdx.x == 0) {
            st->status = RB_ETIMEOUT;
            st->stop = 1;
        }
    };
    const int k = st->k;
    const long long J = st->J;
    const long long N = p.N;
    // begin: v = s_J
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double2 x;
        if (from_split) {
            const float2 a = p.hi[J * p.ldH + i], b = p.lo[J * p.ldH + i];
            x = make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
        } else {
            x = p.S[J * p.ldS + i];
        }
        p.v[i] = x;
    }
    if (!imgs_grid_sync(st, budget)) return timed_out();
    bool accepted = (k == 0);
    double before2 = p.norm2[J], after2 = before2;
    int passes = 0;
    const int gN = (int)((N + kThreads - 1) / kThreads);  // the separate update's blocks
    constexpr int TL = 256;
    __shared__ double2 hs[TL];
    while (!accepted) {
        // dot: hpart[l][c] over the (basis vector, row chunk) items
        const long long items = (long long)k * p.nchunk;
        for (long long it = blockIdx.x; it < items; it += gridDim.x) {
            const int l = (int)(it / p.nchunk), c = (int)(it % p.nchunk);
            const long long i0 = (long long)c * p.chunk;
            const long long i1 = i0 + p.chunk < N ? i0 + p.chunk : N;
            const double2 *q = p.Q + (long long)l * p.ldQ;
            double re = 0.0, im = 0.0;
            for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const double2 a = q[i], b = __ldcg(p.v + i);
                re = fma(a.x, b.x, fma(a.y, b.y, re));
                im = fma(a.x, b.y, fma(-a.y, b.x, im));
            }
            const double2 h = block_sum2(make_double2(re, im));
            if (threadIdx.x == 0) p.hpart[(long long)l * p.nchunk + c] = h;
            __syncthreads();
        }
        if (!imgs_grid_sync(st, budget)) return timed_out();
        // update: v -= Q h, one element per thread of each 256-element virtual block
        for (int vb = blockIdx.x; vb < gN; vb += gridDim.x) {
            const long long i = (long long)vb * kThreads + threadIdx.x;
            double2 d = make_double2(0.0, 0.0);
            for (int l0 = 0; l0 < k; l0 += TL) {
                const int nl = k - l0 < TL ? k - l0 : TL;
                __syncthreads();
                for (int t = threadIdx.x; t < nl; t += blockDim.x) {
                    double2 h = make_double2(0.0, 0.0);
                    const double2 *hp = p.hpart + (long long)(l0 + t) * p.nchunk;
                    for (int c = 0; c < p.nchunk; c++) {
                        const double2 x = __ldcg(hp + c);
                        h.x += x.x;
                        h.y += x.y;
                    }
                    hs[t] = h;
                }
                __syncthreads();
                if (i < N) {
                    for (int t = 0; t < nl; t++) {
                        const double2 q = p.Q[(long long)(l0 + t) * p.ldQ + i];
                        const double2 h = hs[t];
                        d.x = fma(q.x, h.x, fma(-q.y, h.y, d.x));
                        d.y = fma(q.x, h.y, fma(q.y, h.x, d.y));
                    }
                }
            }
            double n2 = 0.0;
            if (i < N) {
                double2 x = __ldcg(p.v + i);
                x.x -= d.x;
                x.y -= d.y;
                p.v[i] = x;
                n2 = x.x * x.x + x.y * x.y;
            }
            n2 = block_sum(n2);
            if (threadIdx.x == 0) p.npart[vb] = n2;
        }
        if (!imgs_grid_sync(st, budget)) return timed_out();
        // every block forms the same total in the same order and takes the same decision
        double tot = 0.0;
        for (int b = 0; b < gN; b++) tot += __ldcg(p.npart + b);
        after2 = tot;
        passes += 1;
        if (tot >= before2 / p.kappa2) {
            accepted = true;
        } else {
            before2 = tot;
            if (passes >= p.max_passes) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    st->passes = passes;
                    st->total_passes += passes;
                    st->after2 = after2;
                    st->status = RB_EORTHO;
                    st->stop = 1;
                }
                return;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->passes = passes;
        st->total_passes += passes;
        st->accepted = 1;
        st->before2 = before2;
        st->after2 = after2;
    }
    // finalize: q_k = v / ||v|| (every block knows ||v||^2)
    if (!(after2 > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (p.qs_stride && st->phase == 0) {
                st->switch_pending = 1;
                st->force_stop = 1;
            } else {
                st->status = RB_OK;
                st->stop = 1;
            }
        }
        return;
    }
    const double nv = sqrt(after2);
    double2 *qk = p.Q + (long long)k * p.ldQ;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double2 x = __ldcg(p.v + i);
        const double2 q = make_double2(x.x / nv, x.y / nv);
        qk[i] = q;
        if (p.qh) {
            const float hr = __double2float_rn(q.x), hm = __double2float_rn(q.y);
            const long long o = (long long)k * p.qs_stride + i;
            p.qh[o] = make_float2(hr, hm);
            p.ql[o] = make_float2(__double2float_rn(q.x - (double)hr), __double2float_rn(q.y - (double)hm));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.pivots[k] = J;
        if (p.rdiag) p.rdiag[k] = nv;
        if (p.passes_out) p.passes_out[k] = passes;
        p.picked[J] = 1;
    }
}

// One cooperative launch per iteration: one block per SM (at most the blocks
// that can be resident at once, which a cooperative launch requires).
cudaError_t launch_imgs(const Prob &p, int grid, bool from_split, cudaStream_t s, int *nlaunch) {
    static int gcoop = 0;
    if (!gcoop) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_imgs_fused, kThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1 || sms < 1) return cudaErrorCooperativeLaunchTooLarge;
        gcoop = sms;
    }
    (void)grid;
    Prob pc = p;
    int fs = from_split ? 1 : 0;
    void *args[] = {&pc, &fs};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_imgs_fused, dim3(gcoop), dim3(kThreads), args, 0, s);
    if (nlaunch) *nlaunch += 1;
    return e;
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
