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

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
__device__ inline int sturm_count(const float *d, const float *e2, int k, float x, float pivmin)
{
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.0f;
    for (int i = 1; i < k; ++i) {
        q = d[i] - x - e2[i - 1] / q;
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
            float acc = 0.0f;
            for (int l = j + 1; l < k; ++l) acc = fmaf(row[l], v[l], acc);
            acc *= beta;
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
            for (int l = j + 1; l < k; ++l) row[l] = row[l] - vi * p[l] - qi * v[l];
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

}  // namespace eig
}  // namespace slista
