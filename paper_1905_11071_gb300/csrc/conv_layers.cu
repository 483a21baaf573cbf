// Unfolded proximal-gradient layers on a 1-D convolutional dictionary: the
// structured dictionaries of Section 6, where the product with B = D^T D is
// replaced by the fast operator z -> D^T (D z).
//
// D holds K filters d_k of length Lf; a code has K maps z_k of P = n - Lf + 1
// entries (valid positions) and
//     (D z)[i]      = sum_k sum_l d_k[l] z_k[i - l]          (i < n)
//     (D^T r)_k[j]  = sum_l d_k[l] r[j + l]                   (j < P)
// so a layer z <- ST(z - alpha_t D^T (D z - x), alpha_t lam) (Eq. pgd, with
// the steps of Eq. steprec, or 1/L for ISTA) costs 2 K P Lf multiply-adds per
// sample instead of the (K P)^2 of the dense product.  One CTA works on one
// sample at a time with the filters, x, the residual r and the codes in shared
// memory; FP32 arithmetic on the CUDA cores.
#include "common.cuh"
#include "kernels.h"

namespace slista {
namespace conv {

namespace {

constexpr int NT = 256;

// tpi threads per output position of D z (a power of two <= 32 dividing the
// warp), each summing the filters k = sub, sub + tpi, ...
__global__ void __launch_bounds__(NT) conv_pgd_kernel(const float *__restrict__ F, int K, int Lf,
                                                      const float *__restrict__ X, int N, int n, float lam,
                                                      const float *__restrict__ alpha, const double *__restrict__ Lp,
                                                      int T, int tpi, float *__restrict__ Z)
{
    extern __shared__ float sm[];
    const int P = n - Lf + 1, m = K * P;
    float *d = sm;           // K x Lf
    float *x = d + K * Lf;   // n
    float *r = x + n;        // n: D z - x
    float *z = r + n;        // m: codes, map k at [k P, (k + 1) P)
    const int tid = threadIdx.x;
    for (int e = tid; e < K * Lf; e += NT) d[e] = __ldg(F + e);
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
    const int item = tid / tpi, sub = tid % tpi, per = NT / tpi;
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        __syncthreads();  // the previous sample's codes are stored
        for (int e = tid; e < n; e += NT) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < m; e += NT) z[e] = 0.0f;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            // r = D z - x
#pragma unroll 1
            for (int i0 = 0; i0 < n; i0 += per) {
                const int i = i0 + item;
                float acc = 0.0f;
                if (i < n) {
                    const int l0 = i - P + 1 > 0 ? i - P + 1 : 0, l1 = i < Lf - 1 ? i : Lf - 1;
                    for (int k = sub; k < K; k += tpi) {
                        const float *dk = d + k * Lf;
                        const float *zk = z + k * P + i;
                        for (int l = l0; l <= l1; ++l) acc = fmaf(dk[l], zk[-l], acc);
                    }
                }
                for (int o = tpi >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (sub == 0 && i < n) r[i] = acc - x[i];
            }
            __syncthreads();
            // z = ST(z - a D^T r, a lam)
#pragma unroll 1
            for (int e = tid; e < m; e += NT) {
                const int k = e / P, j = e - k * P;
                const float *dk = d + k * Lf;
                const float *rj = r + j;
                float g = 0.0f;
                for (int l = 0; l < Lf; ++l) g = fmaf(dk[l], rj[l], g);
                const float u = fmaf(-a, g, z[e]);
                z[e] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
            }
            __syncthreads();
        }
        for (int e = tid; e < m; e += NT) Z[(size_t)s * m + e] = z[e];
    }
}

// The same layers with register blocking, for filters of at most LF taps
// (zero-padded to LF, LF a multiple of 4): a work item is J = 4 consecutive
// outputs of one filter, computed from a window of inputs read as 16-byte
// vectors (conflict-free: the items of a warp read one contiguous segment)
// and the taps of its filter.  Each code map lives in shared memory with LF
// zeros on its left and at least LF - 1 on its right, the residual with
// zeros after it, so no item needs bounds checks.  Per layer:
//   1. y_k[i] = sum_l d_k[l] z_k[i - l] for every filter and i < n  (items k, i-block)
//   2. r[i] = sum_k y_k[i] - x[i]                                    (fixed order over k)
//   3. z_k[j] = ST(z_k[j] - a sum_l d_k[l] r[j + l], a lam)          (items k, j-block)
__host__ __device__ constexpr int up4(int v) { return (v + 3) & ~3; }

template <int LF>
struct Blk {
    static_assert(LF % 4 == 0, "taps in 16-byte units");
    static constexpr int J = 4;
    static constexpr int WV = LF / 4 + 1;  // 16-byte units of a window
    int P, XS, RS, YS, PS;                  // positions; strides of x, r, y, the padded maps
    __host__ __device__ Blk(int K, int Lf, int n)
    {
        P = n - Lf + 1;
        XS = up4(n);
        RS = up4(n + LF + J);
        YS = up4(n + J);
        PS = up4(LF + P + LF);
        (void)K;
    }
    // floats: taps, x, r, y, maps, and one window past the last map
    __host__ __device__ size_t floats(int K) const
    {
        return (size_t)K * LF + XS + RS + (size_t)K * YS + (size_t)K * PS + 4 * WV;
    }
};

template <int LF>
__global__ void __launch_bounds__(NT) conv_pgd_blk_kernel(const float *__restrict__ F, int K, int Lf,
                                                          const float *__restrict__ X, int N, int n, float lam,
                                                          const float *__restrict__ alpha,
                                                          const double *__restrict__ Lp, int T, float *__restrict__ Z)
{
    constexpr int J = 4, WV = Blk<LF>::WV;
    const Blk<LF> bl(K, Lf, n);
    const int P = bl.P, m = K * P, PS = bl.PS, YS = bl.YS;
    extern __shared__ float4 sm4[];
    float *d = reinterpret_cast<float *>(sm4);  // K x LF taps (zero past Lf)
    float *x = d + K * LF;                      // n
    float *r = x + bl.XS;                       // n, then zeros
    float *y = r + bl.RS;                       // K x YS: per-filter partial sums of D z
    float *z = y + (size_t)K * YS;              // K x PS: map k at [k PS + LF, k PS + LF + P)
    const int nb = (n + J - 1) / J;             // output blocks of D z per filter
    const int pb = (P + J - 1) / J;             // output blocks of D^T r per filter
    const int tid = threadIdx.x;
    for (int e = tid; e < K * LF; e += NT) {
        const int k = e / LF, l = e - k * LF;
        d[e] = l < Lf ? __ldg(F + k * Lf + l) : 0.0f;
    }
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        __syncthreads();  // the previous sample's codes are stored
        for (int e = tid; e < n; e += NT) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < bl.RS; e += NT) r[e] = 0.0f;
        for (int e = tid; e < K * PS + 4 * WV; e += NT) z[e] = 0.0f;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            // 1. y_k = d_k * z_k: window zpad[i0 .. i0 + LF + 3]; z_k[i0 + jj - l] = w[LF + jj - l]
#pragma unroll 1
            for (int it = tid; it < K * nb; it += NT) {
                const int k = it / nb, i0 = (it - k * nb) * J;
                const float *dk = d + k * LF;
                const float4 *zw = reinterpret_cast<const float4 *>(z + (size_t)k * PS + i0);
                float w[4 * WV];
#pragma unroll
                for (int u = 0; u < WV; ++u) {
                    const float4 v = zw[u];
                    w[4 * u] = v.x;
                    w[4 * u + 1] = v.y;
                    w[4 * u + 2] = v.z;
                    w[4 * u + 3] = v.w;
                }
                float acc[J] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int l = 0; l < LF; ++l) {
                    const float dl = dk[l];
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) acc[jj] = fmaf(dl, w[LF + jj - l], acc[jj]);
                }
                *reinterpret_cast<float4 *>(y + (size_t)k * YS + i0) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            }
            __syncthreads();
            // 2. r = sum_k y_k - x
            for (int i = tid; i < n; i += NT) {
                float acc = 0.0f;
                for (int k = 0; k < K; ++k) acc += y[(size_t)k * YS + i];
                r[i] = acc - x[i];
            }
            __syncthreads();
            // 3. the step on the codes: window r[j0 .. j0 + LF + 3]
#pragma unroll 1
            for (int it = tid; it < K * pb; it += NT) {
                const int k = it / pb, j0 = (it - k * pb) * J;
                const float *dk = d + k * LF;
                const float4 *rw = reinterpret_cast<const float4 *>(r + j0);
                float w[4 * WV];
#pragma unroll
                for (int u = 0; u < WV; ++u) {
                    const float4 v = rw[u];
                    w[4 * u] = v.x;
                    w[4 * u + 1] = v.y;
                    w[4 * u + 2] = v.z;
                    w[4 * u + 3] = v.w;
                }
                float g[J] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int l = 0; l < LF; ++l) {
                    const float dl = dk[l];
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) g[jj] = fmaf(dl, w[jj + l], g[jj]);
                }
                float *zk = z + (size_t)k * PS + LF + j0;
                if (j0 + J <= P) {
                    float4 v = *reinterpret_cast<const float4 *>(zk);
                    float zz[J] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int jj = 0; jj < J; ++jj) {
                        const float u = fmaf(-a, g[jj], zz[jj]);
                        zz[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                    }
                    *reinterpret_cast<float4 *>(zk) = make_float4(zz[0], zz[1], zz[2], zz[3]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < J; ++jj)
                        if (j0 + jj < P) {
                            const float u = fmaf(-a, g[jj], zk[jj]);
                            zk[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                        }
                }
            }
            __syncthreads();
        }
        for (int e = tid; e < m; e += NT) {
            const int k = e / P, j = e - k * P;
            Z[(size_t)s * m + e] = z[(size_t)k * PS + LF + j];
        }
    }
}

template <int LF>
size_t blk_smem_bytes(int K, int Lf, int n)
{
    return sizeof(float) * Blk<LF>(K, Lf, n).floats(K);
}

template <int LF>
int launch_blk(const ConvArgs &a, cudaStream_t st)
{
    const size_t smem = blk_smem_bytes<LF>(a.K, a.Lf, a.n);
    auto k = conv_pgd_blk_kernel<LF>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    int per_sm = 0;
    SLISTA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
    const long long want = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(a.N < want ? a.N : want);
    k<<<grid, NT, smem, st>>>(a.F, a.K, a.Lf, a.X, a.N, a.n, a.lam, a.alpha, a.L, a.T, a.Z);
    return check_launch("conv_pgd_blk_kernel");
}

}  // namespace

size_t smem_bytes(int K, int Lf, int n) { return sizeof(float) * ((size_t)K * Lf + 2 * (size_t)n + (size_t)K * (n - Lf + 1)); }

bool supported(int K, int Lf, int n)
{
    return K >= 1 && Lf >= 1 && n >= Lf && n <= 8192 && (long long)K * Lf <= 8192 &&
           smem_bytes(K, Lf, n) <= 200 * 1024;
}

int launch_forward(const ConvArgs &a, cudaStream_t st)
{
    const int P = a.n - a.Lf + 1, m = a.K * P;
    if (a.N == 0) return SLISTA_OK;
    if (a.T == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(float) * (size_t)a.N * m, st));
        return SLISTA_OK;
    }
    // register-blocked kernel for filters of up to 32 taps when its padded
    // buffers fit, the plain one otherwise
    if (a.Lf <= 8 && blk_smem_bytes<8>(a.K, a.Lf, a.n) <= 200 * 1024) return launch_blk<8>(a, st);
    if (a.Lf <= 16 && blk_smem_bytes<16>(a.K, a.Lf, a.n) <= 200 * 1024) return launch_blk<16>(a, st);
    if (a.Lf <= 32 && blk_smem_bytes<32>(a.K, a.Lf, a.n) <= 200 * 1024) return launch_blk<32>(a, st);
    int tpi = 1;
    while (tpi < 32 && tpi * 2 <= a.K && (long long)tpi * 2 * a.n <= NT) tpi *= 2;
    const size_t smem = smem_bytes(a.K, a.Lf, a.n);
    SLISTA_CUDA_TRY(allow_smem(conv_pgd_kernel, smem));
    // one CTA per sample at a time, as many resident as shared memory allows
    int per_sm = 0;
    SLISTA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_pgd_kernel, NT, smem));
    const long long want = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(a.N < want ? a.N : want);
    conv_pgd_kernel<<<grid, NT, smem, st>>>(a.F, a.K, a.Lf, a.X, a.N, a.n, a.lam, a.alpha, a.L, a.T, tpi, a.Z);
    return check_launch("conv_pgd_kernel");
}

}  // namespace conv
}  // namespace slista
