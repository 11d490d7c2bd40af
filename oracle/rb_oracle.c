/*
 * rb_oracle.c -- plain, slow FP64 CPU oracle for the greedy reduced-basis /
 * column-pivoted QR of a complex snapshot matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline arm of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path and must never be used as
 * a fallback for it.
 *
 * Paper: Antil, Chen, Field, "A Note on QR-Based Model Reduction:
 * Algorithm, Software, and Gravitational Wave Applications" (arXiv 1805.06124).
 *
 * Layout conventions (identical in meaning to the CUDA path, written
 * independently):
 *   S   complex128, column j (snapshot j) at S + j*ldS, N entries, ldS >= N.
 *   Q   complex128, basis vector l at Q + l*N (N x kmax, column-major).
 *   C   complex128, row-major kmax x M: C[l*M + j] = q_l^H s_j.
 *   err_curve has kmax+1 entries: err_curve[l] = max over unpicked columns of
 *   the squared projection error after l basis vectors.
 *
 * Readings of the paper taken here (each one a plain statement):
 *   - complex inner product: c = q^H s (conjugate on the basis vector), as the
 *     paper's code works on complex data and writes |c|^2 as c c^*  (Sec. 6.1.2,
 *     Eq. (Residual)).
 *   - the tolerance is on the SQUARED error: stop when max_j err_j < tol.
 *   - a basis vector is appended only while the current max error is >= tol
 *     (the stopping guarantee stated in Sec. 6.1), so k counts appended vectors
 *     and err_curve has k+1 meaningful entries.
 *   - ties in the argmax go to the lowest column index; columns already picked
 *     are excluded from the argmax.
 *   - Hoffmann's MGSCI with kappa: after a full MGS pass, accept when
 *     ||v_after|| >= ||v_before|| / kappa, otherwise repeat (cap max_passes).
 *
 * Parity pins: every function below is pinned by tests against brute-force
 * least squares, LAPACK pivoted QR, closed forms and invariants (see tests/).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_KMAX_REACHED 1
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENONFINITE (-4)
#define ORC_EORTHO (-5)

typedef long long i64;

/* Planted-mistake switch used only by the oracle's own mutation tests: the
 * default build (ORC_PLANT undefined or 0) is the oracle. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

/* c = q^H s over n complex entries, summed sequentially in FP64. */
static void cdot_conj(const double *q, const double *s, i64 n, double *cre, double *cim)
{
    double re = 0.0, im = 0.0;
    for (i64 i = 0; i < n; i++) {
        double qr = q[2 * i], qi = q[2 * i + 1];
        double sr = s[2 * i], si = s[2 * i + 1];
#if ORC_PLANT == 1
        /* planted: missing conjugate */
        re += qr * sr - qi * si;
        im += qr * si + qi * sr;
#else
        re += qr * sr + qi * si;
        im += qr * si - qi * sr;
#endif
    }
    *cre = re;
    *cim = im;
}

/* ||v||^2, sequential FP64. */
static double cnorm2(const double *v, i64 n)
{
    double s = 0.0;
    for (i64 i = 0; i < n; i++)
        s += v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1];
    return s;
}

/* argmax of err over columns with picked==0; ties -> lowest index.
 * Returns -1 when no column is left. */
static i64 argmax_unpicked(const double *err, const unsigned char *picked, i64 M)
{
    i64 best = -1;
    for (i64 j = 0; j < M; j++) {
        if (picked[j])
            continue;
#if ORC_PLANT == 3
        /* planted: ties go to the highest index */
        if (best < 0 || err[j] >= err[best])
            best = j;
#else
        if (best < 0 || err[j] > err[best])
            best = j;
#endif
    }
    return best;
}

/*
 * One Hoffmann MGSCI orthogonalisation of v (n entries) against the k
 * orthonormal columns of Q (Sec. 6.1.2: "iterative modified Gram-Schmidt ...
 * MGSCI with kappa = 2"; Remark after Prop. 5.3 on iterated Gram-Schmidt).
 * Each pass is a full modified Gram-Schmidt sweep over q_1..q_k.
 * Returns the number of passes, or -1 when max_passes did not satisfy the
 * kappa test.  With k == 0 no pass is made.
 */
static int mgsci(const double *Q, i64 N, int k, double *v, double kappa, int max_passes)
{
    if (k == 0)
        return 0;
    int passes = 0;
    for (;;) {
        double before = sqrt(cnorm2(v, N));
        for (int l = 0; l < k; l++) {
            const double *q = Q + 2 * (i64)l * N;
            double hr, hi;
            cdot_conj(q, v, N, &hr, &hi);
            for (i64 i = 0; i < N; i++) {
                double qr = q[2 * i], qi = q[2 * i + 1];
                /* v -= h * q */
                v[2 * i] -= hr * qr - hi * qi;
                v[2 * i + 1] -= hr * qi + hi * qr;
            }
        }
        passes++;
        double after = sqrt(cnorm2(v, N));
#if ORC_PLANT == 4
        /* planted: never re-orthogonalise */
        return passes;
#endif
        if (after >= before / kappa)
            return passes;
        if (passes >= max_passes)
            return -1;
    }
}

/*
 * RB-greedy, Alg. 3, with the incremental residual bookkeeping of
 * Eq. (Residual): err_j = ||s_j||^2 - sum_l |c_lj|^2, norms and sums stored
 * separately, no square roots in the argmax (Sec. 6.1.2).
 *
 * forced (optional, nforced entries): replay mode.  At step l < nforced the
 * given column is taken as the pivot instead of the oracle's own argmax; the
 * oracle still reports its own argmax (own_argmax[l]), its max error
 * (own_max[l]), the error of the forced column (forced_err[l]) and the
 * second-largest error (second_max[l]).  Any of the diagnostics pointers may
 * be NULL.
 *
 * Outputs: Q (N x kmax), pivots[kmax], err_curve[kmax+1], C (kmax x M
 * row-major), final_err[M] (may be NULL), rdiag[kmax] = ||v|| before
 * normalisation (R(l,l) of Alg. 2), passes[kmax] (may be NULL).
 */
int orc_rb_greedy(const double *S, i64 N, i64 M, i64 ldS, double tol, int kmax,
                  double kappa, int max_passes,
                  const i64 *forced, int nforced,
                  double *Q, i64 *pivots, double *err_curve, double *C,
                  double *final_err, double *rdiag, int *passes,
                  i64 *own_argmax, double *own_max, double *forced_err, double *second_max,
                  int *k_out)
{
    *k_out = 0;
    if (N <= 0 || M <= 0 || ldS < N || kmax < 0 || !(tol >= 0.0) || kappa <= 1.0 || max_passes < 1)
        return ORC_EINVAL;
    double *norm2 = (double *)calloc((size_t)M, sizeof(double));
    double *acc = (double *)calloc((size_t)M, sizeof(double));
    double *err = (double *)calloc((size_t)M, sizeof(double));
    unsigned char *picked = (unsigned char *)calloc((size_t)M, 1);
    double *v = (double *)malloc((size_t)N * 2 * sizeof(double));
    if (!norm2 || !acc || !err || !picked || !v) {
        free(norm2); free(acc); free(err); free(picked); free(v);
        return ORC_ENOMEM;
    }
    int status = ORC_OK, bad = 0;
    /* Alg. 3 steps "Define sigma_0(s_i) = ||s_i||" and "j(0) = arg sup".
     * Columns are independent; built with -fopenmp (the paper's shared-memory
     * scheme, Sec. 6.1.3) they are split over threads, each column still summed
     * sequentially, so the results do not depend on the thread count. */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (i64 j = 0; j < M; j++) {
        norm2[j] = cnorm2(S + 2 * j * ldS, N);
        if (!isfinite(norm2[j]))
            bad |= 1;
        err[j] = norm2[j];
    }
    if (bad)
        status = ORC_ENONFINITE;
    if (status != ORC_OK)
        goto done;
    i64 minNM = N < M ? N : M;
    int k = 0;
    for (;;) {
        i64 J = argmax_unpicked(err, picked, M);
        double emax = J >= 0 ? err[J] : 0.0;
        if (J >= 0) {
            double second = -INFINITY;
            for (i64 j = 0; j < M; j++)
                if (!picked[j] && j != J && err[j] > second)
                    second = err[j];
            if (own_argmax && k < nforced) own_argmax[k] = J;
            if (own_max && k < nforced) own_max[k] = emax;
            if (second_max && k < nforced) second_max[k] = second;
        }
        err_curve[k] = emax;
        /* Stopping test (Alg. 3 while-condition, squared-error reading). */
#if ORC_PLANT == 5
        /* planted: off-by-one, one vector too many */
        if (J < 0 || (k > 0 && err_curve[k - 1] < tol) || k >= kmax || k >= minNM) {
#else
        if (J < 0 || emax < tol || k >= kmax || k >= minNM) {
#endif
            if (J >= 0 && emax >= tol && k >= kmax)
                status = ORC_KMAX_REACHED;
            break;
        }
        if (forced && k < nforced) {
            J = forced[k];
            if (J < 0 || J >= M || picked[J]) {
                status = ORC_EINVAL;
                break;
            }
            if (forced_err) forced_err[k] = err[J];
        }
        /* q_{k+1} = s_J - Q_k Q_k^H s_J, normalised (Alg. 3), with MGSCI. */
        memcpy(v, S + 2 * J * ldS, (size_t)N * 2 * sizeof(double));
        int np = mgsci(Q, N, k, v, kappa, max_passes);
        if (np < 0) {
            status = ORC_EORTHO;
            break;
        }
        double nv = sqrt(cnorm2(v, N));
        if (!(nv > 0.0))
            break; /* column already in the span: exact rank reached */
        double *q = Q + 2 * (i64)k * N;
        for (i64 i = 0; i < 2 * N; i++)
            q[i] = v[i] / nv;
        pivots[k] = J;
        rdiag[k] = nv;
        if (passes) passes[k] = np;
        picked[J] = 1;
        /* Pivot search of the next step: c_j = q^H s_j, Eq. (Residual). */
#pragma omp parallel for schedule(static)
        for (i64 j = 0; j < M; j++) {
            double cr, ci;
            cdot_conj(q, S + 2 * j * ldS, N, &cr, &ci);
            C[2 * ((i64)k * M + j)] = cr;
            C[2 * ((i64)k * M + j) + 1] = ci;
#if ORC_PLANT == 2
            acc[j] += cr * cr; /* planted: imaginary part dropped */
#else
            acc[j] += cr * cr + ci * ci;
#endif
            err[j] = norm2[j] - acc[j];
        }
        k++;
    }
    *k_out = k;
done:
    if (final_err)
        for (i64 j = 0; j < M; j++)
            final_err[j] = err[j];
    free(norm2); free(acc); free(err); free(picked); free(v);
    return status;
}

/*
 * Modified Gram-Schmidt with column pivoting, Alg. 2, on a private copy V of
 * S (Businger-Golub reading: pivot over all not-yet-picked columns by the
 * directly recomputed ||V(:,j)||^2; R(k,j) = q_k^H V(:,j); V(:,j) -= R(k,j) q_k).
 * Stops when the largest remaining ||V(:,j)||^2 < tol, at kmax, or at min(N,M).
 * Outputs Q (N x kmax), pivots, rdiag[kmax] = R(k,k), R (kmax x M row-major,
 * zero for columns picked before step k), err_curve[kmax+1].
 * No re-orthogonalisation (the algorithm as the paper states it).
 */
int orc_mgs_pivot(const double *S, i64 N, i64 M, i64 ldS, double tol, int kmax,
                  double *Q, i64 *pivots, double *rdiag, double *R, double *err_curve, int *k_out)
{
    *k_out = 0;
    if (N <= 0 || M <= 0 || ldS < N || kmax < 0 || !(tol >= 0.0))
        return ORC_EINVAL;
    double *V = (double *)malloc((size_t)N * (size_t)M * 2 * sizeof(double));
    unsigned char *picked = (unsigned char *)calloc((size_t)M, 1);
    double *nrm = (double *)malloc((size_t)M * sizeof(double));
    if (!V || !picked || !nrm) {
        free(V); free(picked); free(nrm);
        return ORC_ENOMEM;
    }
    for (i64 j = 0; j < M; j++)
        memcpy(V + 2 * j * N, S + 2 * j * ldS, (size_t)N * 2 * sizeof(double));
    memset(R, 0, (size_t)kmax * (size_t)M * 2 * sizeof(double));
    i64 minNM = N < M ? N : M;
    int status = ORC_OK;
    int k = 0;
    for (;;) {
        i64 best = -1;
        for (i64 j = 0; j < M; j++) {
            if (picked[j])
                continue;
            nrm[j] = cnorm2(V + 2 * j * N, N);
            if (!isfinite(nrm[j])) {
                status = ORC_ENONFINITE;
                goto done;
            }
            if (best < 0 || nrm[j] > nrm[best])
                best = j;
        }
        double rkk2 = best >= 0 ? nrm[best] : 0.0;
        err_curve[k] = rkk2;
        if (best < 0 || rkk2 < tol || k >= kmax || k >= minNM) {
            if (best >= 0 && rkk2 >= tol && k >= kmax)
                status = ORC_KMAX_REACHED;
            break;
        }
        double rkk = sqrt(rkk2);
        if (!(rkk > 0.0))
            break;
        double *q = Q + 2 * (i64)k * N;
        const double *vb = V + 2 * best * N;
        for (i64 i = 0; i < 2 * N; i++)
            q[i] = vb[i] / rkk;
        pivots[k] = best;
        rdiag[k] = rkk;
        picked[best] = 1;
        R[2 * ((i64)k * M + best)] = rkk;
        for (i64 j = 0; j < M; j++) {
            if (picked[j])
                continue;
            double *vj = V + 2 * j * N;
            double hr, hi;
            cdot_conj(q, vj, N, &hr, &hi);
            R[2 * ((i64)k * M + j)] = hr;
            R[2 * ((i64)k * M + j) + 1] = hi;
            for (i64 i = 0; i < N; i++) {
                double qr = q[2 * i], qi = q[2 * i + 1];
                vj[2 * i] -= hr * qr - hi * qi;
                vj[2 * i + 1] -= hr * qi + hi * qr;
            }
        }
        k++;
    }
    *k_out = k;
done:
    free(V); free(picked); free(nrm);
    return status;
}

/*
 * Projection onto the basis: C[l*ldC + j] = q_l^H x_j for l < k, j < Mx
 * (Sec. 2: a column is represented by orthogonal projection onto the span
 * of the basis).  Sequential FP64 sums.
 */
int orc_project(const double *Q, i64 N, int k, i64 ldQ, const double *X, i64 Mx, i64 ldX,
                double *C, i64 ldC)
{
    if (N <= 0 || k < 0 || Mx < 0 || ldQ < N || ldX < N || ldC < Mx)
        return ORC_EINVAL;
    for (int l = 0; l < k; l++)
        for (i64 j = 0; j < Mx; j++) {
            double cr, ci;
            cdot_conj(Q + 2 * (i64)l * ldQ, X + 2 * j * ldX, N, &cr, &ci);
            C[2 * ((i64)l * ldC + j)] = cr;
            C[2 * ((i64)l * ldC + j) + 1] = ci;
        }
    return ORC_OK;
}

/*
 * hi/lo split of complex128 into two complex64 arrays: hi = fl32(x) rounded
 * to nearest, lo = fl32(x - hi) rounded to nearest, per real component.
 * Definition of the split storage used by the split-precision form.
 */
int orc_split(const double *S, i64 N, i64 M, i64 ldS, float *hi, float *lo, i64 ldH)
{
    if (N <= 0 || M < 0 || ldS < N || ldH < N)
        return ORC_EINVAL;
    for (i64 j = 0; j < M; j++)
        for (i64 i = 0; i < 2 * N; i++) {
            double x = S[2 * j * ldS + i];
            float h = (float)x;
            float l = (float)(x - (double)h);
            hi[2 * j * ldH + i] = h;
            lo[2 * j * ldH + i] = l;
        }
    return ORC_OK;
}
