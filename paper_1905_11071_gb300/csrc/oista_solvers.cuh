// Warp-level solvers for L_S = lambda_max(B_SS) (Eq. spca) used by the
// Oracle-ISTA kernels: support index lists, B_SS gathered into a warp's
// shared buffer or held one row per lane in registers, D_S D_S^T for large
// supports, Lanczos with the stopping rule of eig.cuh.
#pragma once
#include "common.cuh"
#include "eig.cuh"

namespace slista {
namespace simt {
namespace {

constexpr int KMAX = 64;  // largest matrix a warp solves in its own buffer
constexpr int JM = eig::LANCZOS_JMAX;
// The solve kernel's block: A_WARPS warps with a shared-memory buffer for
// B_SS or D_S D_S^T (supports of more than SMALL_K indices first, then the
// small ones), and S_WARPS warps that solve supports of at most SMALL_K
// indices with the matrix in registers (one row per lane).
constexpr int A_WARPS = 8;
constexpr int S_WARPS = 8;
constexpr int SMALL_K = 32;
constexpr int NCLS = 3;  // list classes: |S| > KMAX, SMALL_K < |S| <= KMAX, |S| <= SMALL_K
// (the tensor-core step kernel files samples into the same classes: 64 / 32)
static_assert(KMAX == 64 && SMALL_K == 32 && NCLS == 3, "list classes of the tensor-core step");

constexpr int GCOLS = 8;  // D_S columns staged per round in gram_ds

struct alignas(16) WarpEig {
    static constexpr int LDA = eig::vec_ld(KMAX);
    float A[KMAX * LDA];
    float q[256], qp[256], al[JM], be[JM], e2[JM];
    float col[GCOLS * KMAX];
    int idx[256];
};

// Index list of a support given by its words (one warp); returns |S|.  The
// W <= 32 words are loaded at once, one per lane.
__device__ int support_indices(const uint32_t *words, int W, int *idx)
{
    const int lane = threadIdx.x & 31;
    const uint32_t mine = lane < W ? words[lane] : 0u;
    int k = 0;
    for (int w = 0; w < W; ++w) {
        const uint32_t bits = __shfl_sync(0xffffffffu, mine, w);
        const bool has = (bits >> lane) & 1u;
        if (has) idx[k + __popc(bits & ((1u << lane) - 1u))] = w * 32 + lane;
        k += __popc(bits);
    }
    __syncwarp();
    return k;
}

// B_SS into A (leading dimension lda >= 4 ceil(k/4), k <= 64), columns
// k .. 4 ceil(k/4) - 1 zeroed; returns whether an off-diagonal entry is
// non-zero.  Lane l gathers columns l and l + 32 of RG rows at a time (2 RG
// loads in flight).
template <int RG = 8>
__device__ bool gather_bss(const float *__restrict__ B, int m, const int *idx, int k, float *A, int lda)
{
    const int lane = threadIdx.x & 31;
    const int kp = (k + 3) & ~3;
    const int c0 = lane, c1 = lane + 32;
    const int j0 = c0 < k ? idx[c0] : 0, j1 = c1 < k ? idx[c1] : 0;
    bool off = false;
#pragma unroll 1
    for (int a0 = 0; a0 < k; a0 += RG) {
        float x0[RG], x1[RG];
#pragma unroll
        for (int u = 0; u < RG; ++u) {
            const int a = a0 + u;
            const float *row = B + (size_t)(a < k ? idx[a] : 0) * m;
            x0[u] = (a < k && c0 < k) ? __ldg(row + j0) : 0.0f;
            x1[u] = (a < k && c1 < k) ? __ldg(row + j1) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < RG; ++u) {
            const int a = a0 + u;
            if (a < k) {
                if (c0 < kp) A[a * lda + c0] = x0[u];
                if (c1 < kp) A[a * lda + c1] = x1[u];
                off |= (a != c0 && x0[u] != 0.0f) || (a != c1 && x1[u] != 0.0f);
            }
        }
    }
    __syncwarp();
    return __any_sync(0xffffffffu, off);
}

// G = D_S D_S^T (n x n, n <= KMAX) into A (leading dimension lda), columns
// n .. 4 ceil(n/4) - 1 zeroed; Dt is D transposed, so column j of D is the
// contiguous row j of Dt.  Lane a owns rows a and a + 32.  Two passes over
// the support columns (staged GCOLS at a time in col): columns 0..31 for
// rows < 32, then columns 32..63 for all rows; the block of rows >= 32 x
// columns < 32 is the transpose of the one computed for rows < 32.
__device__ void gram_ds(const float *__restrict__ Dt, int n, const int *idx, int k, float *A, int lda, float *col)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int b0 = 32 * h;
        if (b0 >= n) break;
        float acc0[32], acc1[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) acc0[b] = acc1[b] = 0.0f;
#pragma unroll 1
        for (int s0 = 0; s0 < k; s0 += GCOLS) {
            float x[GCOLS][KMAX / 32];
#pragma unroll
            for (int c = 0; c < GCOLS; ++c)
#pragma unroll
                for (int r = 0; r < KMAX / 32; ++r) {
                    const int a = lane + 32 * r;
                    x[c][r] = (s0 + c < k && a < n) ? __ldg(Dt + (size_t)idx[s0 + c] * n + a) : 0.0f;
                }
            __syncwarp();
#pragma unroll
            for (int c = 0; c < GCOLS; ++c)
#pragma unroll
                for (int r = 0; r < KMAX / 32; ++r) col[c * KMAX + lane + 32 * r] = x[c][r];
            __syncwarp();
#pragma unroll
            for (int c = 0; c < GCOLS; ++c) {
                const float d0 = col[c * KMAX + lane], d1 = col[c * KMAX + lane + 32];
                const float4 *cb = reinterpret_cast<const float4 *>(col + c * KMAX + b0);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 v = cb[u];
                    acc0[4 * u] = fmaf(d0, v.x, acc0[4 * u]);
                    acc0[4 * u + 1] = fmaf(d0, v.y, acc0[4 * u + 1]);
                    acc0[4 * u + 2] = fmaf(d0, v.z, acc0[4 * u + 2]);
                    acc0[4 * u + 3] = fmaf(d0, v.w, acc0[4 * u + 3]);
                    if (h == 1) {
                        acc1[4 * u] = fmaf(d1, v.x, acc1[4 * u]);
                        acc1[4 * u + 1] = fmaf(d1, v.y, acc1[4 * u + 1]);
                        acc1[4 * u + 2] = fmaf(d1, v.z, acc1[4 * u + 2]);
                        acc1[4 * u + 3] = fmaf(d1, v.w, acc1[4 * u + 3]);
                    }
                }
            }
        }
        if (lane < n)
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (b0 + b < n) A[lane * lda + b0 + b] = acc0[b];
        if (h == 1 && lane + 32 < n)
#pragma unroll
            for (int b = 0; b < 32; ++b)
                if (b0 + b < n) A[(lane + 32) * lda + b0 + b] = acc1[b];
    }
    __syncwarp();
    // rows 32.. x columns 0..31 by symmetry; zero pad columns
    for (int a = 32; a < n; ++a)
        if (lane < n) A[a * lda + lane] = A[lane * lda + a];
    const int np = (n + 3) & ~3;
    for (int a = lane; a < n; a += 32)
        for (int b = n; b < np; ++b) A[a * lda + b] = 0.0f;
    __syncwarp();
}

// Lanczos with the matrix-vector products read from global memory, for the
// rare supports too large for the shared buffer when D is not given.
__device__ double lanczos_global(const float *__restrict__ B, int m, const int *idx, int k, WarpEig &we)
{
    const int lane = threadIdx.x & 31;
    float *q = we.q, *qp = we.qp;
    float nrm0 = 0.0f;
    for (int a = lane; a < k; a += 32) nrm0 = fmaf(eig::start_vector(a), eig::start_vector(a), nrm0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm0 += __shfl_xor_sync(0xffffffffu, nrm0, o);
    const float inv = rsqrtf(nrm0);
    for (int a = lane; a < k; a += 32) {
        q[a] = eig::start_vector(a) * inv;
        qp[a] = 0.0f;
    }
    __syncwarp();
    float beta_prev = 0.0f, theta_prev = -INFINITY;
    int j = 0;
    const int J = k < JM ? k : JM;
#pragma unroll 1
    for (; j < J; ++j) {
        float w[8];  // k <= 256 rows over 32 lanes
        float dot = 0.0f;
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int a = lane + 32 * rr;
            float s = 0.0f;
            if (a < k) {
                const float *row = B + (size_t)idx[a] * m;
                for (int b = 0; b < k; ++b) s = fmaf(__ldg(row + idx[b]), q[b], s);
                dot = fmaf(s, q[a], dot);
            }
            w[rr] = s;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        float nrm = 0.0f;
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int a = lane + 32 * rr;
            if (a < k) {
                w[rr] = w[rr] - dot * q[a] - beta_prev * qp[a];
                nrm = fmaf(w[rr], w[rr], nrm);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        const float beta = sqrtf(nrm);
        if (lane == 0) {
            we.al[j] = dot;
            we.be[j] = beta;
        }
        __syncwarp();
        if (beta <= 1e-6f * fabsf(dot)) {
            ++j;
            break;
        }
        if ((j + 1) % 16 == 0) {
            const float theta = eig::tridiag_max_eig_warp(we.al, we.be, we.e2, j + 1);
            if (theta - theta_prev <= 2e-7f * fabsf(theta)) {
                ++j;
                break;
            }
            theta_prev = theta;
        }
        const float ib = 1.0f / beta;
        __syncwarp();
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int a = lane + 32 * rr;
            if (a < k) {
                qp[a] = q[a];
                q[a] = w[rr] * ib;
            }
        }
        __syncwarp();
        beta_prev = beta;
    }
    return (double)eig::tridiag_max_eig_warp(we.al, we.be, we.e2, j);
}

__device__ inline float max_diag(const float *A, int lda, int k)
{
    float v = A[0];
    for (int a = 1; a < k; ++a) v = fmaxf(v, A[a * lda + a]);
    return v;
}

// ---------------------------------------------------------------------------
// Register-resident solver for 2 <= |S| <= SMALL_K: lane a holds row a of
// B_SS (ar[]) and entry a of the Lanczos vectors; the three-term recurrence
// and the stopping rule of eig::lanczos_max_eig_warp (all k steps, T_k
// similar to B_SS, when k <= LANCZOS_J0), the largest eigenvalue of the
// tridiagonal bracketed by Sturm multisection.  A diagonal B_SS gives its
// largest entry exactly.
// ---------------------------------------------------------------------------
struct WarpEigS {
    float al[SMALL_K], be[SMALL_K], e2[SMALL_K];
    int idx[SMALL_K];
};

__device__ double solve_small(const float *__restrict__ B, int m, const int *idx, int k, float *al, float *be,
                              float *e2, int j0 = eig::LANCZOS_J0, int dj = eig::LANCZOS_DJ)
{
    const int lane = threadIdx.x & 31;
    const bool on = lane < k;
    float ar[SMALL_K];
    const float *brow = B + (size_t)idx[on ? lane : 0] * m;
#pragma unroll
    for (int b = 0; b < SMALL_K; ++b) ar[b] = (on && b < k) ? __ldg(brow + idx[b]) : 0.0f;
    bool off = false;
#pragma unroll
    for (int b = 0; b < SMALL_K; ++b) off |= (b != lane) && (ar[b] != 0.0f);
    if (!__any_sync(0xffffffffu, off)) {
        float d = -INFINITY;
#pragma unroll
        for (int b = 0; b < SMALL_K; ++b)
            if (b == lane && on) d = ar[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
        return (double)d;
    }
    float q = on ? eig::start_vector(lane) : 0.0f;
    float nrm = q * q;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    q *= rsqrtf(nrm);
    float qp = 0.0f, beta_prev = 0.0f;
    float ref = -INFINITY, theta = -INFINITY;
    int j = 0;
    int target = k <= j0 ? k : j0;
#pragma unroll 1
    for (;;) {
        bool done = false;
#pragma unroll 1
        for (; j < target; ++j) {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
            for (int b = 0; b < SMALL_K; b += 4) {
                s0 = fmaf(ar[b], __shfl_sync(0xffffffffu, q, b), s0);
                s1 = fmaf(ar[b + 1], __shfl_sync(0xffffffffu, q, b + 1), s1);
                s2 = fmaf(ar[b + 2], __shfl_sync(0xffffffffu, q, b + 2), s2);
                s3 = fmaf(ar[b + 3], __shfl_sync(0xffffffffu, q, b + 3), s3);
            }
            const float sv = (s0 + s1) + (s2 + s3);
            float alpha = sv * q;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) alpha += __shfl_xor_sync(0xffffffffu, alpha, o);
            const float w = on ? sv - alpha * q - beta_prev * qp : 0.0f;
            float bb = w * w;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bb += __shfl_xor_sync(0xffffffffu, bb, o);
            const float beta = sqrtf(bb);
            if (lane == 0) {
                al[j] = alpha;
                be[j] = beta;
            }
            if (beta <= 1e-6f * fabsf(alpha) || j + 1 == k) {  // invariant subspace or full dimension
                ++j;
                done = true;
                break;
            }
            qp = q;
            q = w * (1.0f / beta);
            beta_prev = beta;
        }
        __syncwarp();
        // the stopping rule of eig::lanczos_max_eig_warp
        bool conv = false;
        theta = eig::tridiag_max_eig_warp(al, be, e2, j, ref, theta + 2e-7f * fabsf(theta), &conv, &ref);
        if (done || conv) break;
        target = min(j + dj, k);
    }
    return (double)theta;
}

}  // namespace
}  // namespace simt
}  // namespace slista
