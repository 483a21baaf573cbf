// Gram quantities of the Lasso and the Lipschitz constant L.
//
//   C = X D        (row i = (D^T x_i)^T, the D^T x term of Eq. ista's gradient)
//   xsq_i = ||x_i||^2
//   B = D^T D      (behind W_z = Id - D^T D / L, Section 4)
//   L = largest eigenvalue of D^T D (Section 1)
//
// C and xsq come from the SIMT tile engine (the sample tile X_b in shared
// memory, D streamed through it); B from a direct per-entry kernel whose
// summation order makes B exactly symmetric; L from the smaller of D D^T and
// D^T D by a single-CTA Lanczos / Sturm eigen-solver (eig.cuh).
#include "common.cuh"
#include "eig.cuh"
#include "kernels.h"
#include "simt.cuh"

namespace slista {
namespace gram {

using simt::NT;

template <int MP, int NB>
__global__ void __launch_bounds__(NT) xd_kernel(const float *__restrict__ X, const float *__restrict__ D,
                                                int n, int m, int N, int lda, float *__restrict__ C,
                                                double *__restrict__ xsq)
{
    using TL = simt::Tile<MP, NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    float *B_s = A_s + NB * lda;
    const int row0 = blockIdx.x * NB;
    const int kp = lda - 4;  // n rounded up to 16
    for (int e = threadIdx.x; e < NB * kp; e += NT) {
        const int r = e / kp, k = e % kp;
        A_s[r * lda + k] = (row0 + r < N && k < n) ? __ldg(X + (size_t)(row0 + r) * n + k) : 0.0f;
    }
    __syncthreads();
    // ||x_i||^2 in FP64: one warp per row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < NB; r += NT / 32) {
        double s = 0.0;
        for (int k = lane; k < n; k += 32) {
            const double v = (double)A_s[r * lda + k];
            s = fma(v, v, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && row0 + r < N) xsq[row0 + r] = s;
    }
    float acc[TL::RM][TL::RN];
#pragma unroll
    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) acc[i][j] = 0.0f;
    simt::gemm_acc<TL>(acc, A_s, lda, D, n, m < MP ? m : MP, m, B_s);
    simt::store_rows<TL>(C, acc, row0, N, m < MP ? m : MP, m);
    // wider dictionaries: the remaining column blocks of MP columns
#pragma unroll 1
    for (int c0 = MP; c0 < m; c0 += MP) {
        const int nc = m - c0 < MP ? m - c0 : MP;
#pragma unroll
        for (int i = 0; i < TL::RM; ++i)
#pragma unroll
            for (int j = 0; j < TL::RN; ++j) acc[i][j] = 0.0f;
        simt::gemm_acc<TL>(acc, A_s, lda, D + c0, n, nc, m, B_s);
        simt::store_rows<TL>(C + c0, acc, row0, N, nc, m);
    }
}

// B[a][b] = sum_i D[i][a] D[i][b]; identical arithmetic for (a,b) and (b,a).
__global__ void dtd_kernel(const float *__restrict__ D, int n, int m, float *__restrict__ B)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y * blockDim.y + threadIdx.y;
    if (a >= m || b >= m) return;
    float s = 0.0f;
    for (int i = 0; i < n; ++i) s = fmaf(__ldg(D + (size_t)i * m + a), __ldg(D + (size_t)i * m + b), s);
    B[(size_t)a * m + b] = s;
}

// ---------------------------------------------------------------------------
// Largest eigenvalue of a k x k symmetric PSD matrix K.  For k <= KL_SMEM the
// matrix is formed in shared memory (from a shared copy of D when it fits) and
// solved by one warp with Lanczos and Sturm multisection on the tridiagonal,
// with the stopping rule of eig::lanczos_max_eig_warp (eig.cuh).  Larger matrices fall back to power iteration on K in
// global memory (FP32 products, FP64 Rayleigh quotients), which keeps the
// largest quotient seen and stops after 400 iterations without progress.
// ---------------------------------------------------------------------------
constexpr int KL_SMEM = 128;
constexpr int PI_NT = 256;
constexpr int L_STAGE_FLOATS = 32768;  // D (n x m) staged in shared memory up to 128 KiB

// mode 0: K = Kg (k x k, global);  mode 1: K = D D^T (k = n);  mode 2: K = D^T D (k = m).
__global__ void __launch_bounds__(PI_NT) lipschitz_kernel(const float *__restrict__ Kg,
                                                          const float *__restrict__ D, int n, int m,
                                                          int mode, int k, double *__restrict__ L)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ double redd[3][PI_NT / 32];
    if (k <= KL_SMEM) {
        const int lda = eig::odd_ld(k);
        float *Ks = sm;
        float *vec = Ks + k * lda;            // q, qp (k each), al, be, e2 (JMAX each)
        float *Ds = vec + 2 * k + 3 * eig::LANCZOS_JMAX;
        const int ldd_s = m | 1;  // odd row stride: lanes reading different rows hit different banks
        const bool stage = mode != 0 && (size_t)n * ldd_s <= (size_t)L_STAGE_FLOATS;
        const float *Dsrc = D;
        int ldd = m;
        if (stage) {  // coalesced copy of D; the Gram entries then read shared memory
            for (int e = threadIdx.x; e < n * m; e += PI_NT) Ds[(e / m) * ldd_s + e % m] = __ldg(D + e);
            __syncthreads();
            Dsrc = Ds;
            ldd = ldd_s;
        }
        bool off = false;
        for (int e = threadIdx.x; e < k * k; e += PI_NT) {
            const int a = e / k, b = e % k;
            float s;
            if (mode == 0) {
                s = __ldg(Kg + (size_t)a * k + b);
            } else if (mode == 1) {  // (D D^T)_ab = sum_j D_aj D_bj
                s = 0.0f;
                for (int j = 0; j < m; ++j) s = fmaf(Dsrc[(size_t)a * ldd + j], Dsrc[(size_t)b * ldd + j], s);
            } else {  // (D^T D)_ab = sum_i D_ia D_ib
                s = 0.0f;
                for (int i = 0; i < n; ++i) s = fmaf(Dsrc[(size_t)i * ldd + a], Dsrc[(size_t)i * ldd + b], s);
            }
            Ks[a * lda + b] = s;
            off |= (a != b) && (s != 0.0f);
        }
        if (!__syncthreads_or(off)) {  // diagonal (orthonormal D): the largest entry, exactly
            if (threadIdx.x == 0) {
                float v = Ks[0];
                for (int a = 1; a < k; ++a) v = fmaxf(v, Ks[a * lda + a]);
                *L = (double)v;
            }
            return;
        }
        if (threadIdx.x < 32) {
            const double v = eig::lanczos_max_eig_warp<(KL_SMEM + 31) / 32>(
                Ks, lda, k, vec, vec + k, vec + 2 * k, vec + 2 * k + eig::LANCZOS_JMAX,
                vec + 2 * k + 2 * eig::LANCZOS_JMAX);
            if (threadIdx.x == 0) *L = v;
        }
        return;
    }
    // power iteration fallback (mode 0 only)
    float *v = sm;
    for (int a = threadIdx.x; a < k; a += PI_NT) v[a] = eig::start_vector(a);
    __syncthreads();
    double best = 0.0;
    int stall = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int it = 0; it < 20000 && stall < 400; ++it) {
        double vw = 0.0, vv = 0.0, ww = 0.0;
        float wl[4];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int a = threadIdx.x + rr * PI_NT;
            float s = 0.0f;
            if (a < k) {
                const float *row = Kg + (size_t)a * k;
                for (int b = 0; b < k; ++b) s = fmaf(__ldg(row + b), v[b], s);
                const double va = (double)v[a];
                vw += va * (double)s;
                vv += va * va;
                ww += (double)s * (double)s;
            }
            wl[rr] = s;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vw += __shfl_xor_sync(0xffffffffu, vw, o);
            vv += __shfl_xor_sync(0xffffffffu, vv, o);
            ww += __shfl_xor_sync(0xffffffffu, ww, o);
        }
        if (lane == 0) {
            redd[0][warp] = vw;
            redd[1][warp] = vv;
            redd[2][warp] = ww;
        }
        __syncthreads();
        vw = vv = ww = 0.0;
#pragma unroll
        for (int w = 0; w < PI_NT / 32; ++w) {
            vw += redd[0][w];
            vv += redd[1][w];
            ww += redd[2][w];
        }
        const double rq = vw / vv;
        if (rq > best * (1.0 + 1e-9)) {
            best = rq;
            stall = 0;
        } else {
            ++stall;
        }
        const float inv = (float)(1.0 / sqrt(ww));
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int a = threadIdx.x + rr * PI_NT;
            if (a < k) v[a] = wl[rr] * inv;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *L = best;
}

namespace {

template <int MP>
int launch_xd(const float *D, int n, int m, const float *X, int N, float *C, double *xsq, cudaStream_t st)
{
    constexpr int NB = 32;
    const int kp = ((n + 15) / 16) * 16;
    const int lda = kp + 4;
    const size_t smem = sizeof(float) * ((size_t)NB * lda + simt::Tile<MP, NB>::BS_FLOATS);
    if (smem > 227 * 1024) return fail(SLISTA_ERR_UNSUPPORTED, "lasso_gram: n = %d too large", n);
    auto k = xd_kernel<MP, NB>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    const int grid = ceil_div(N, NB);
    if (grid == 0) return SLISTA_OK;
    k<<<grid, NT, smem, st>>>(X, D, n, m, N, lda, C, xsq);
    return check_launch("xd_kernel");
}

int launch_power(const float *Kg, const float *D, int n, int m, int mode, int k, double *L, cudaStream_t st)
{
    const bool staged = k <= KL_SMEM;
    const bool stage_d = mode != 0 && (size_t)n * (m | 1) <= (size_t)L_STAGE_FLOATS;
    const size_t smem = sizeof(float) * (staged ? (size_t)k * eig::odd_ld(k) + 2 * (size_t)k +
                                                      3 * (size_t)eig::LANCZOS_JMAX + (stage_d ? (size_t)n * (m | 1) : 0)
                                                : (size_t)k);
    if (!staged && (k > 4 * PI_NT || mode != 0))
        return fail(SLISTA_ERR_UNSUPPORTED, "Lipschitz kernel supports k <= %d (got %d)", 4 * PI_NT, k);
    SLISTA_CUDA_TRY(allow_smem(lipschitz_kernel, smem));
    lipschitz_kernel<<<1, PI_NT, smem, st>>>(Kg, D, n, m, mode, k, L);
    return check_launch("lipschitz_kernel");
}

}  // namespace

int launch_gram(const float *D, int n, int m, const float *X, int N, float *B, float *C, double *xsq,
                cudaStream_t st)
{
    dim3 blk(32, 8);
    dim3 grd(ceil_div(m, 32), ceil_div(m, 8));
    dtd_kernel<<<grd, blk, 0, st>>>(D, n, m, B);
    int rc = check_launch("dtd_kernel");
    if (rc) return rc;
    switch (simt::padded_mp(m)) {
        case 32: return launch_xd<32>(D, n, m, X, N, C, xsq, st);
        case 64: return launch_xd<64>(D, n, m, X, N, C, xsq, st);
        case 128: return launch_xd<128>(D, n, m, X, N, C, xsq, st);
        case 256: return launch_xd<256>(D, n, m, X, N, C, xsq, st);
    }
    if (m <= 1024) return launch_xd<256>(D, n, m, X, N, C, xsq, st);  // column blocks of 256
    return fail(SLISTA_ERR_UNSUPPORTED, "lasso_gram supports m <= 1024 (got %d)", m);
}

int launch_lipschitz_from_D(const float *D, int n, int m, double *L, cudaStream_t st)
{
    // D D^T (n x n) and D^T D (m x m) share their non-zero spectrum: use the smaller.
    if (n <= m && n <= KL_SMEM) return launch_power(nullptr, D, n, m, 1, n, L, st);
    if (m < n && m <= KL_SMEM) return launch_power(nullptr, D, n, m, 2, m, L, st);
    return fail(SLISTA_ERR_UNSUPPORTED, "L from D needs min(n, m) <= %d; use lasso_lipschitz(B)", KL_SMEM);
}

int launch_lipschitz_from_B(const float *B, int m, double *L, cudaStream_t st)
{
    return launch_power(B, nullptr, 0, m, 0, m, L, st);
}

}  // namespace gram
}  // namespace slista
