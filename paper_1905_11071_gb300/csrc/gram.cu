// The Lipschitz constant of the Lasso, L = largest eigenvalue of D^T D
// (Section 1), from the smaller of D D^T and D^T D by a single-CTA Lanczos /
// Sturm eigen-solver (eig.cuh).  (B = D^T D, C = X D and ||x||^2 are the
// tensor-core products of tc_gemm.cu.)
#include "common.cuh"
#include "eig.cuh"
#include "kernels.h"
#include "simt.cuh"

namespace slista {
namespace gram {

// ---------------------------------------------------------------------------
// Largest eigenvalue of a k x k symmetric PSD matrix K.  For k <= KL_SMEM the
// matrix is formed in shared memory and solved by one warp with Lanczos and
// Sturm multisection on the tridiagonal (eig.cuh), the top Ritz value checked
// after 16 steps and then every 8.  K = D D^T or D^T D is accumulated by the
// whole CTA in 4 x 4 register tiles (upper triangle, mirrored, so K is
// exactly symmetric) over chunks of the summation index staged in shared
// memory, each tile reading two 16-byte vectors per 16 products.  Larger
// matrices fall back to power iteration on K in global memory (FP32
// products, FP64 Rayleigh quotients), which keeps the largest quotient seen
// and stops after 400 iterations without progress.
// ---------------------------------------------------------------------------
constexpr int KL_SMEM = 128;
constexpr int PI_NT = 512;
constexpr int L_CHUNK = 64;  // summation indices staged per round

// Shared-memory floats of the k <= KL_SMEM path: K (k x vec_ld(k)), the
// Lanczos vectors and tridiagonal, and one staged chunk (L_CHUNK x (4 ceil(k/4) + 4)).
__host__ __device__ inline int lip_smem_floats(int k)
{
    const int kp = (k + 3) & ~3;
    return k * eig::vec_ld(k) + 2 * kp + 3 * eig::LANCZOS_JMAX + L_CHUNK * (kp + 4);
}

// mode 0: K = Kg (k x k, global);  mode 1: K = D D^T (k = n);  mode 2: K = D^T D (k = m).
__global__ void __launch_bounds__(PI_NT) lipschitz_kernel(const float *__restrict__ Kg,
                                                          const float *__restrict__ D, int n, int m,
                                                          int mode, int k, double *__restrict__ L)
{
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ double redd[3][PI_NT / 32];
    if (k <= KL_SMEM) {
        const int lda = eig::vec_ld(k);
        const int kp = (k + 3) & ~3;
        float *Ks = sm;
        float *vec = Ks + k * lda;  // q, qp (kp each), al, be, e2 (JMAX each)
        float *St = vec + 2 * kp + 3 * eig::LANCZOS_JMAX;
        const int lds = kp + 4;
        if (mode == 0) {
            for (int e = threadIdx.x; e < k * lda; e += PI_NT) {
                const int a = e / lda, b = e % lda;
                Ks[e] = b < k ? __ldg(Kg + (size_t)a * k + b) : 0.0f;
            }
        } else {
            // K_ab = sum_r S[r][a] S[r][b], S = D^T (mode 1, r < m) or D (mode 2, r < n)
            const int R = mode == 1 ? m : n;
            const int nt = kp / 4;  // tiles per side
            const int ntile = nt * (nt + 1) / 2;
            float acc[2][16];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[u][e] = 0.0f;
#pragma unroll 1
            for (int r0 = 0; r0 < R; r0 += L_CHUNK) {
                const int rc = R - r0 < L_CHUNK ? R - r0 : L_CHUNK;
                __syncthreads();
                for (int e = threadIdx.x; e < L_CHUNK * kp; e += PI_NT) {
                    // consecutive threads read consecutive addresses of D
                    const int r = mode == 1 ? e % L_CHUNK : e / kp, c = mode == 1 ? e / L_CHUNK : e % kp;
                    float v = 0.0f;
                    if (r < rc && c < k)
                        v = mode == 1 ? __ldg(D + (size_t)c * m + r0 + r) : __ldg(D + (size_t)(r0 + r) * m + c);
                    St[r * lds + c] = v;
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int t = threadIdx.x + u * PI_NT;
                    if (t >= ntile) continue;
                    int ta = 0, rem = t;  // upper-triangle tile (ta, tb), tb >= ta
                    while (rem >= nt - ta) {
                        rem -= nt - ta;
                        ++ta;
                    }
                    const int tb = ta + rem;
#pragma unroll 4
                    for (int r = 0; r < rc; ++r) {
                        const float4 x = *reinterpret_cast<const float4 *>(St + r * lds + 4 * ta);
                        const float4 y = *reinterpret_cast<const float4 *>(St + r * lds + 4 * tb);
                        const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc[u][4 * i + j] = fmaf(xa[i], yb[j], acc[u][4 * i + j]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int t = threadIdx.x + u * PI_NT;
                if (t >= ntile) continue;
                int ta = 0, rem = t;
                while (rem >= nt - ta) {
                    rem -= nt - ta;
                    ++ta;
                }
                const int tb = ta + rem;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int a = 4 * ta + i, b = 4 * tb + j;
                        if (a < kp && b < kp) {
                            const float v = (a < k && b < k) ? acc[u][4 * i + j] : 0.0f;
                            if (a < k) Ks[a * lda + b] = v;
                            if (b < k) Ks[b * lda + a] = v;
                        }
                    }
            }
        }
        __syncthreads();
        bool off = false;
        for (int e = threadIdx.x; e < k * k; e += PI_NT) {
            const int a = e / k, b = e % k;
            off |= (a != b) && (Ks[a * lda + b] != 0.0f);
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
                Ks, lda, k, vec, vec + kp, vec + 2 * kp, vec + 2 * kp + eig::LANCZOS_JMAX,
                vec + 2 * kp + 2 * eig::LANCZOS_JMAX, 16, 8);
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
        float wl[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
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
        for (int rr = 0; rr < 2; ++rr) {
            const int a = threadIdx.x + rr * PI_NT;
            if (a < k) v[a] = wl[rr] * inv;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *L = best;
}

namespace {

int launch_power(const float *Kg, const float *D, int n, int m, int mode, int k, double *L, cudaStream_t st)
{
    const bool staged = k <= KL_SMEM;
    const size_t smem = sizeof(float) * (staged ? (size_t)lip_smem_floats(k) : (size_t)k);
    if (!staged && (k > 2 * PI_NT || mode != 0))
        return fail(SLISTA_ERR_UNSUPPORTED, "Lipschitz kernel supports k <= %d (got %d)", 2 * PI_NT, k);
    SLISTA_CUDA_TRY(allow_smem(lipschitz_kernel, smem));
    lipschitz_kernel<<<1, PI_NT, smem, st>>>(Kg, D, n, m, mode, k, L);
    return check_launch("lipschitz_kernel");
}

}  // namespace

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
