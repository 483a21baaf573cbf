// Largest eigenvalue of a small symmetric matrix by one warp: Lanczos (the
// three-term recurrence builds a tridiagonal T_j similar, in the limit, to
// the matrix restricted to the Krylov space) and Sturm-sequence
// multisection on T_j: each lane counts the eigenvalues below its own trial
// point (LDL^T pivots), so every round shrinks the bracket of the largest
// eigenvalue by a factor 33.  The upper end of the final bracket is
// returned, so the result does not underestimate the largest eigenvalue of
// T_j.  Used for L (Section 1) and L_S (Eq. spca).  FP32 arithmetic.
#pragma once

#include <cuda_runtime.h>

namespace slista {
namespace eig {

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
// dimension, at most LANCZOS_JMAX steps) and dj LANCZOS_DJ.
// q, qp: 4 ceil(k/4) floats; al, be, e2: LANCZOS_JMAX floats of warp scratch.
// RPL = rows per lane (>= ceil(k / 32)).
constexpr int LANCZOS_J0 = 10;
constexpr int LANCZOS_DJ = 2;
constexpr int LANCZOS_JMAX = 64;

template <int RPL>
__device__ double lanczos_max_eig_warp(const float *A, int lda, int k, float *q, float *qp, float *al, float *be,
                                       float *e2, int j0 = LANCZOS_J0, int dj = LANCZOS_DJ)
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
#pragma unroll 4
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
        target = min(min(j + dj, k), JMAX);
    }
    return (double)theta;
}

}  // namespace eig
}  // namespace slista
