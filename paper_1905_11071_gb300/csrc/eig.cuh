// Largest eigenvalue of a small symmetric matrix held in shared memory, by a
// group of threads (one warp, or a whole CTA):
//   1. Householder reduction to tridiagonal form (Golub & Van Loan, Sec. 8.3.1):
//      for each column j, the reflector I - beta v v^T annihilates A[j+2:, j],
//      and the trailing block is updated as A22 <- A22 - v q^T - q v^T with
//      p = beta A22 v, q = p - (beta/2)(p^T v) v;
//   2. Sturm-sequence multisection on the tridiagonal matrix: each thread of the
//      group counts the eigenvalues below its own trial point (LDL^T pivots),
//      so every round shrinks the bracket of the largest eigenvalue by a factor
//      (group size + 1).  The upper end of the final bracket is returned, so the
//      result does not underestimate the largest eigenvalue of the stored
//      matrix (a step 1/L_S computed from it never exceeds the exact one by
//      more than the FP32 error of the reduction).
// Used for L (Section 1) and L_S (Eq. spca).  FP32 arithmetic; the error is
// that of a backward-stable reduction, about k * 6e-8 relative at worst.
#pragma once

#include <cuda_runtime.h>

namespace slista {
namespace eig {

struct WarpGroup {
    static constexpr int size = 32;
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static void sync() { __syncwarp(); }
    // sum over the group; scratch unused
    __device__ static float sum(float v, float *) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    __device__ static bool any(bool p) { return __any_sync(0xffffffffu, p); }
    // smallest rank whose predicate is true (size if none)
    __device__ static int first_true(bool p, int *) {
        const unsigned b = __ballot_sync(0xffffffffu, p);
        return b ? __ffs(b) - 1 : size;
    }
};

template <int NT>
struct CtaGroup {
    static constexpr int size = NT;
    __device__ static int rank() { return threadIdx.x; }
    __device__ static void sync() { __syncthreads(); }
    // scratch: NT/32 floats
    __device__ static float sum(float v, float *scratch) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
        __syncthreads();
        float s = 0.0f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += scratch[w];
        return s;
    }
    __device__ static bool any(bool p) { return __syncthreads_or(p) != 0; }
    __device__ static int first_true(bool p, int *scratch) {
        const unsigned b = __ballot_sync(0xffffffffu, p);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = b ? (threadIdx.x & ~31) + __ffs(b) - 1 : NT;
        __syncthreads();
        int r = NT;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) r = min(r, scratch[w]);
        return r;
    }
};

// Odd leading dimension for a k x k matrix (conflict-free column walks).
__host__ __device__ constexpr int odd_ld(int k) { return (k & 1) ? k : k + 1; }

// Leading dimension >= k with lda % 8 == 4: rows start on 16-byte boundaries
// and the 16-byte loads of 8 lanes at one offset of 8 consecutive rows fall
// in distinct bank groups (row stride an odd number of 16-byte units).
__host__ __device__ constexpr int vec_ld(int k) { return 4 * (((k + 3) >> 2) | 1); }

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
__device__ inline int sturm_count(const float *d, const float *e2, int k, float x, float pivmin)
{
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.0f;
    for (int i = 1; i < k; ++i) {
        q = d[i] - x - __fdividef(e2[i - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.0f;
    }
    return c;
}

// Largest eigenvalue of the k x k symmetric matrix A (leading dimension lda,
// both triangles stored; destroyed).  v, p, d, e, e2: k floats each of group-
// shared scratch; red: CtaGroup reduction scratch (NT/32 floats and ints).
// Must be called by every thread of the group with identical arguments.
template <class G>
__device__ double max_eig_sym(float *A, int lda, int k, float *v, float *p, float *d, float *e, float *e2,
                              float *redf, int *redi)
{
    const int r0 = G::rank();
    if (k == 1) return (double)A[0];
    for (int j = 0; j + 2 < k; ++j) {
        float s = 0.0f;
        for (int i = j + 1 + r0; i < k; i += G::size) {
            const float x = A[i * lda + j];
            s = fmaf(x, x, s);
        }
        s = G::sum(s, redf);
        const float x0 = A[(j + 1) * lda + j];
        if (s == 0.0f) {
            if (r0 == 0) e[j] = 0.0f;
            G::sync();
            continue;
        }
        const float nrm = sqrtf(s);
        const float alpha = x0 >= 0.0f ? -nrm : nrm;
        for (int i = j + 1 + r0; i < k; i += G::size) v[i] = (i == j + 1) ? x0 - alpha : A[i * lda + j];
        const float vtv = 2.0f * (s - alpha * x0);
        const float beta = 2.0f / vtv;
        G::sync();
        float pv = 0.0f;
        for (int i = j + 1 + r0; i < k; i += G::size) {
            const float *row = A + i * lda;
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
            int l = j + 1;
            for (; l + 3 < k; l += 4) {
                a0 = fmaf(row[l], v[l], a0);
                a1 = fmaf(row[l + 1], v[l + 1], a1);
                a2 = fmaf(row[l + 2], v[l + 2], a2);
                a3 = fmaf(row[l + 3], v[l + 3], a3);
            }
            for (; l < k; ++l) a0 = fmaf(row[l], v[l], a0);
            const float acc = beta * ((a0 + a1) + (a2 + a3));
            p[i] = acc;
            pv = fmaf(acc, v[i], pv);
        }
        pv = G::sum(pv, redf);
        const float Kc = 0.5f * beta * pv;
        for (int i = j + 1 + r0; i < k; i += G::size) p[i] = fmaf(-Kc, v[i], p[i]);
        G::sync();
        for (int i = j + 1 + r0; i < k; i += G::size) {
            float *row = A + i * lda;
            const float vi = v[i], qi = p[i];
#pragma unroll 4
            for (int l = j + 1; l < k; ++l) row[l] = fmaf(-vi, p[l], fmaf(-qi, v[l], row[l]));
        }
        if (r0 == 0) e[j] = alpha;
        G::sync();
    }
    for (int i = r0; i < k; i += G::size) {
        d[i] = A[i * lda + i];
        if (i == k - 2) e[i] = A[(k - 1) * lda + (k - 2)];
    }
    G::sync();
    for (int i = r0; i + 1 < k; i += G::size) e2[i] = e[i] * e[i];
    G::sync();
    // Gershgorin bracket: max d_i <= lambda_max <= max(d_i + |e_{i-1}| + |e_i|)
    float lo = -INFINITY, hi = -INFINITY, scale = 0.0f;
    for (int i = 0; i < k; ++i) {
        const float r = (i > 0 ? fabsf(e[i - 1]) : 0.0f) + (i + 1 < k ? fabsf(e[i]) : 0.0f);
        lo = fmaxf(lo, d[i]);
        hi = fmaxf(hi, d[i] + r);
        scale = fmaxf(scale, fabsf(d[i]) + r);
    }
    const float pivmin = fmaxf(scale * 1e-30f, 1e-37f);
    hi = hi + 2e-7f * scale;  // round-off margin: the bracket must contain lambda_max
    for (int round = 0; round < 8 && hi - lo > 1.2e-7f * scale; ++round) {
        const float x = lo + (hi - lo) * (float)(r0 + 1) / (float)(G::size + 1);
        const bool above_all = sturm_count(d, e2, k, x, pivmin) == k;  // every eigenvalue < x
        const int f = G::first_true(above_all, redi);
        const float nhi = f < G::size ? lo + (hi - lo) * (float)(f + 1) / (float)(G::size + 1) : hi;
        const float nlo = f > 0 ? lo + (hi - lo) * (float)f / (float)(G::size + 1) : lo;
        lo = nlo;
        hi = nhi;
    }
    return (double)hi;
}


// Entry a of the start vector of the Krylov / power iterations: the
// golden-ratio sequence 0.5 + frac((a + 1) * 0.618...), in [0.5, 1.5).
__host__ __device__ inline float start_vector(int a)
{
    const float x = (float)(a + 1) * 0.6180339887f;
    return 0.5f + (x - floorf(x));
}

// Upper end of a bracket of the largest eigenvalue of the symmetric
// tridiagonal matrix (d[0..k-1], e[0..k-2]) by Sturm multisection over one
// warp (33 trial points per round).  e2 receives e^2.
// With a lower bound `ref` of that eigenvalue (e.g. the lower end of the
// bracket for a leading principal submatrix, whose largest eigenvalue is never
// above it: Cauchy interlacing) and a trial upper end `top`, the first round
// tests the 32 points of (ref, top] instead: if no eigenvalue lies above
// `top`, the bracket found there is final and *within = true (one round
// instead of a full multisection).  *lo_out (if given) receives the lower end
// of the final bracket.
__device__ inline float tridiag_max_eig_warp(const float *d, const float *e, float *e2, int k,
                                             float ref = -INFINITY, float top = -INFINITY, bool *within = nullptr,
                                             float *lo_out = nullptr)
{
    const int lane = threadIdx.x & 31;
    // Gershgorin bracket of the spectrum, one row per lane, then max over the warp
    float lo = -INFINITY, hi = -INFINITY, scale = 0.0f;
    for (int i = lane; i < k; i += 32) {
        if (i + 1 < k) e2[i] = e[i] * e[i];
        const float r = (i > 0 ? fabsf(e[i - 1]) : 0.0f) + (i + 1 < k ? fabsf(e[i]) : 0.0f);
        lo = fmaxf(lo, d[i]);
        hi = fmaxf(hi, d[i] + r);
        scale = fmaxf(scale, fabsf(d[i]) + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmaxf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        scale = fmaxf(scale, __shfl_xor_sync(0xffffffffu, scale, o));
    }
    __syncwarp();
    const float pivmin = fmaxf(scale * 1e-30f, 1e-37f);
    hi = hi + 2e-7f * scale;
    if (within) *within = false;
    lo = fmaxf(lo, ref);
    if (top > lo && top < hi) {
        const float x = lo + (top - lo) * (float)(lane + 1) / 32.0f;
        const bool above_all = sturm_count(d, e2, k, x, pivmin) == k;
        const unsigned b = __ballot_sync(0xffffffffu, above_all);
        if (b) {
            const int f = __ffs(b) - 1;
            hi = lo + (top - lo) * (float)(f + 1) / 32.0f;
            lo = f > 0 ? lo + (top - lo) * (float)f / 32.0f : lo;
            if (within) *within = true;
            if (lo_out) *lo_out = lo;
            return hi;
        }
        lo = top;  // an eigenvalue lies above the tested interval
    }
    for (int round = 0; round < 8 && hi - lo > 1.2e-7f * scale; ++round) {
        const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
        const bool above_all = sturm_count(d, e2, k, x, pivmin) == k;
        const unsigned b = __ballot_sync(0xffffffffu, above_all);
        const int f = b ? __ffs(b) - 1 : 32;
        const float nhi = f < 32 ? lo + (hi - lo) * (float)(f + 1) / 33.0f : hi;
        const float nlo = f > 0 ? lo + (hi - lo) * (float)f / 33.0f : lo;
        lo = nlo;
        hi = nhi;
    }
    if (lo_out) *lo_out = lo;
    return hi;
}

// Largest eigenvalue of a k x k symmetric matrix by Lanczos (one warp).
// The three-term recurrence  beta_j q_{j+1} = A q_j - alpha_j q_j - beta_{j-1} q_{j-1}
// builds the tridiagonal T_J whose largest eigenvalue (the top Ritz value)
// converges to that of A from below; in finite precision the extreme Ritz
// values stay accurate without reorthogonalisation (Paige).  J = k steps are
// run when k <= LANCZOS_J0 (T_k is then similar to A); otherwise the top
// Ritz value is bracketed after LANCZOS_J0 steps and then every
// LANCZOS_DJ more, up to min(k, LANCZOS_JMAX), until it has moved by less
// than 2e-7 (relative) since the previous check: that test is one
// multisection round over the interval just above the previous bracket,
// and only when it fails is the new Ritz value bracketed in full.  (On the
// supports of the 64 x 256 workload - |S| = 11 .. 160, B_SS or D_S D_S^T -
// the top Ritz value is within 1e-8 of lambda_max (FP64 model) when the rule
// stops, at 12 - 14 steps on average.)  A is in shared memory with leading
// dimension lda; with lda = vec_ld(k) and 16-byte aligned A and q the rows
// are read as 16-byte vectors, and columns k .. 4 ceil(k/4) - 1 of A must then
// hold finite values (zeros).  j0 replaces LANCZOS_J0 (j0 >= k: the full
// dimension, at most LANCZOS_JMAX steps).
// q, qp: 4 ceil(k/4) floats; al, be, e2: LANCZOS_JMAX floats of warp scratch.
// RPL = rows per lane (>= ceil(k / 32)).
constexpr int LANCZOS_J0 = 10;
constexpr int LANCZOS_DJ = 2;
constexpr int LANCZOS_JMAX = 64;

template <int RPL>
__device__ double lanczos_max_eig_warp(const float *A, int lda, int k, float *q, float *qp, float *al, float *be,
                                       float *e2, int j0 = LANCZOS_J0)
{
    constexpr int JMAX = LANCZOS_JMAX;
    const int lane = threadIdx.x & 31;
    // generic start vector (a structured one such as all-ones can be exactly
    // orthogonal to the top eigenvector, e.g. [[1, c], [c, 1]] with c < 0)
    float nrm0 = 0.0f;
    for (int a = lane; a < k; a += 32) {
        const float v = start_vector(a);
        nrm0 = fmaf(v, v, nrm0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm0 += __shfl_xor_sync(0xffffffffu, nrm0, o);
    const float inv = rsqrtf(nrm0);
    for (int a = lane; a < k; a += 32) {
        q[a] = start_vector(a) * inv;
        qp[a] = 0.0f;
    }
    // rows as 16-byte vectors when the layout allows (vec_ld); q is then
    // zero-padded to a multiple of 4 entries, so the pad columns of A (which
    // the caller zeroes) contribute nothing
    const bool vec = (lda & 7) == 4 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(q) & 15) == 0;
    const int ku = (k + 3) >> 2;
    if (vec && lane < 4 * ku - k) q[k + lane] = 0.0f;
    __syncwarp();
    float beta_prev = 0.0f;
    float ref = -INFINITY, theta = -INFINITY;
    int j = 0;
    int target = min(min(k, j0), JMAX);
    bool done = false;
#pragma unroll 1
    for (;;) {
#pragma unroll 1
        for (; j < target; ++j) {
            float w[RPL];
            float dot = 0.0f;
            if (vec) {
                // the rows of this lane side by side (one pass over the
                // Lanczos vector, independent FMA chains per row)
                const float4 *q4 = reinterpret_cast<const float4 *>(q);
                float acc[RPL][4];
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) acc[rr][0] = acc[rr][1] = acc[rr][2] = acc[rr][3] = 0.0f;
                for (int u = 0; u < ku; ++u) {
                    const float4 y = q4[u];
#pragma unroll
                    for (int rr = 0; rr < RPL; ++rr) {
                        const int a = lane + 32 * rr;
                        if (a < k) {
                            const float4 x = reinterpret_cast<const float4 *>(A + a * lda)[u];
                            acc[rr][0] = fmaf(x.x, y.x, acc[rr][0]);
                            acc[rr][1] = fmaf(x.y, y.y, acc[rr][1]);
                            acc[rr][2] = fmaf(x.z, y.z, acc[rr][2]);
                            acc[rr][3] = fmaf(x.w, y.w, acc[rr][3]);
                        }
                    }
                }
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    const int a = lane + 32 * rr;
                    const float sv = (acc[rr][0] + acc[rr][1]) + (acc[rr][2] + acc[rr][3]);
                    w[rr] = a < k ? sv : 0.0f;
                    if (a < k) dot = fmaf(sv, q[a], dot);
                }
            } else {
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    const int a = lane + 32 * rr;
                    float sv = 0.0f;
                    if (a < k) {
                        const float *row = A + a * lda;
                        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
                        int b = 0;
                        for (; b + 3 < k; b += 4) {
                            s0 = fmaf(row[b], q[b], s0);
                            s1 = fmaf(row[b + 1], q[b + 1], s1);
                            s2 = fmaf(row[b + 2], q[b + 2], s2);
                            s3 = fmaf(row[b + 3], q[b + 3], s3);
                        }
                        for (; b < k; ++b) s0 = fmaf(row[b], q[b], s0);
                        sv = (s0 + s1) + (s2 + s3);
                        dot = fmaf(sv, q[a], dot);
                    }
                    w[rr] = sv;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            const float alpha = dot;
            float nrm = 0.0f;
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                const int a = lane + 32 * rr;
                if (a < k) {
                    w[rr] = w[rr] - alpha * q[a] - beta_prev * qp[a];
                    nrm = fmaf(w[rr], w[rr], nrm);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
            const float beta = sqrtf(nrm);
            if (lane == 0) {
                al[j] = alpha;
                be[j] = beta;
            }
            __syncwarp();
            if (beta <= 1e-6f * fabsf(alpha) || j + 1 == k) {  // invariant subspace or full dimension
                ++j;
                done = true;
                break;
            }
            const float ib = 1.0f / beta;
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                const int a = lane + 32 * rr;
                if (a < k) {
                    qp[a] = q[a];
                    q[a] = w[rr] * ib;
                }
            }
            __syncwarp();
            beta_prev = beta;
        }
        bool conv = false;
        theta = tridiag_max_eig_warp(al, be, e2, j, ref, theta + 2e-7f * fabsf(theta), &conv, &ref);
        if (done || conv) break;  // exhausted, or moved by less than 2e-7 since the last check
        if (j >= JMAX || j >= k) break;
        target = min(min(j + LANCZOS_DJ, k), JMAX);
    }
    return (double)theta;
}

// Upper end of a bracket of the largest eigenvalue of the symmetric
// tridiagonal (d, e) by Sturm multisection over a whole CTA (NT + 1 points
// per round).  e2: k floats (written).  redi: NT/32 ints of scratch.
template <int NT>
__device__ float tridiag_max_eig_cta(const float *d, const float *e, float *e2, int k, int *redi)
{
    for (int i = threadIdx.x; i + 1 < k; i += NT) e2[i] = e[i] * e[i];
    __syncthreads();
    float lo = -INFINITY, hi = -INFINITY, scale = 0.0f;
    for (int i = 0; i < k; ++i) {
        const float r = (i > 0 ? fabsf(e[i - 1]) : 0.0f) + (i + 1 < k ? fabsf(e[i]) : 0.0f);
        lo = fmaxf(lo, d[i]);
        hi = fmaxf(hi, d[i] + r);
        scale = fmaxf(scale, fabsf(d[i]) + r);
    }
    const float pivmin = fmaxf(scale * 1e-30f, 1e-37f);
    hi = hi + 2e-7f * scale;
    for (int round = 0; round < 6 && hi - lo > 1.2e-7f * scale; ++round) {
        const float x = lo + (hi - lo) * (float)(threadIdx.x + 1) / (float)(NT + 1);
        const bool above_all = sturm_count(d, e2, k, x, pivmin) == k;
        const int f = CtaGroup<NT>::first_true(above_all, redi);
        const float nhi = f < NT ? lo + (hi - lo) * (float)(f + 1) / (float)(NT + 1) : hi;
        const float nlo = f > 0 ? lo + (hi - lo) * (float)f / (float)(NT + 1) : lo;
        lo = nlo;
        hi = nhi;
    }
    return hi;
}

// Lanczos as in lanczos_max_eig_warp, with every product spread over a CTA:
// row a of the matrix-vector product is summed by TPR = 2^floor(log2(NT/k))
// threads (strided columns, shuffle-combined).  q, qp, w: k floats; al, be,
// e2: LANCZOS_JMAX floats; redf: NT/32 floats, redi: NT/32 ints (scratch).
template <int NT>
__device__ double lanczos_max_eig_cta(const float *A, int lda, int k, float *q, float *qp, float *w, float *al,
                                      float *be, float *e2, float *redf, int *redi)
{
    constexpr int JMAX = LANCZOS_JMAX;
    int tpr = 1;
    while (tpr < 32 && tpr * 2 * k <= NT) tpr *= 2;
    const int row = threadIdx.x / tpr, col0 = threadIdx.x % tpr;
    const bool has_row = row < k;
    float nrm0 = 0.0f;
    for (int a = threadIdx.x; a < k; a += NT) {
        const float v = start_vector(a);
        nrm0 = fmaf(v, v, nrm0);
    }
    nrm0 = CtaGroup<NT>::sum(nrm0, redf);
    const float inv = rsqrtf(nrm0);
    for (int a = threadIdx.x; a < k; a += NT) {
        q[a] = start_vector(a) * inv;
        qp[a] = 0.0f;
    }
    __syncthreads();
    float beta_prev = 0.0f, theta_prev = -INFINITY, theta = 0.0f;
    int j = 0, target = k <= 32 ? k : 32;
    bool done = false;
#pragma unroll 1
    for (;;) {
#pragma unroll 1
        for (; j < target; ++j) {
            float s = 0.0f;
            if (has_row) {
                const float *r = A + row * lda;
                float s0 = 0.0f, s1 = 0.0f;
                int b = col0;
                for (; b + tpr < k; b += 2 * tpr) {
                    s0 = fmaf(r[b], q[b], s0);
                    s1 = fmaf(r[b + tpr], q[b + tpr], s1);
                }
                if (b < k) s0 = fmaf(r[b], q[b], s0);
                s = s0 + s1;
            }
            for (int o = tpr / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const bool lead = has_row && col0 == 0;
            const float alpha = CtaGroup<NT>::sum(lead ? s * q[row] : 0.0f, redf);
            float wv = 0.0f;
            if (lead) wv = s - alpha * q[row] - beta_prev * qp[row];
            const float beta = sqrtf(CtaGroup<NT>::sum(lead ? wv * wv : 0.0f, redf));
            if (threadIdx.x == 0) {
                al[j] = alpha;
                be[j] = beta;
            }
            if (beta <= 1e-6f * fabsf(alpha) || j + 1 == k) {
                ++j;
                done = true;
                break;
            }
            if (lead) w[row] = wv / beta;
            __syncthreads();
            for (int a = threadIdx.x; a < k; a += NT) {
                qp[a] = q[a];
                q[a] = w[a];
            }
            __syncthreads();
            beta_prev = beta;
        }
        __syncthreads();
        theta = tridiag_max_eig_cta<NT>(al, be, e2, j, redi);
        if (done) break;
        if (theta - theta_prev <= 2e-7f * fabsf(theta)) break;
        if (j >= JMAX || j >= k) break;
        theta_prev = theta;
        target = min(min(j + 16, k), JMAX);
    }
    return (double)theta;
}

}  // namespace eig
}  // namespace slista
