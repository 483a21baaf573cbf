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
#include "tc_ptx.cuh"

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
// (zero-padded to LF, LF a multiple of 4), in CTAs of NB threads: a work item
// is JB consecutive outputs of one filter, computed from a window of inputs
// read as 16-byte vectors (conflict-free: the items of a warp read one
// contiguous segment) and the taps of its filter (16-byte vectors, the same
// for the whole warp).  Each code map lives in shared memory with LF zeros on
// its left and at least LF on its right, the residual with zeros after it,
// so no item needs bounds checks.  Per layer:
//   1. y_k[i] = sum_l d_k[l] z_k[i - l] for every filter and i < n  (items k, i-block)
//   2. r[i] = sum_k y_k[i] - x[i]                                    (fixed order over k)
//   3. z_k[j] = ST(z_k[j] - a sum_l d_k[l] r[j + l], a lam)          (items k, j-block)
constexpr int NB = 128;  // threads of a blocked CTA
constexpr int JB = 8;    // outputs of a work item
__host__ __device__ constexpr int up4(int v) { return (v + 3) & ~3; }

template <int LF>
struct Blk {
    static_assert(LF % 4 == 0 && JB % 4 == 0 && JB <= LF + 2, "16-byte units; windows within the zero pads");
    static constexpr int WV = (LF + JB) / 4;  // 16-byte units of a window
    int P, XS, RS, YS, PS;                     // positions; strides of x, r, y, the padded maps
    __host__ __device__ Blk(int K, int Lf, int n)
    {
        P = n - Lf + 1;
        XS = up4(n);
        RS = up4(n + LF + JB);
        YS = up4(n + JB);
        PS = up4(LF + P + LF);
        (void)K;
    }
    // floats: taps, x, r, y, maps, and one window past the last map
    __host__ __device__ size_t floats(int K) const
    {
        return (size_t)K * LF + XS + RS + (size_t)K * YS + (size_t)K * PS + 4 * WV;
    }
};

// n floats (a multiple of 4) from 16-byte aligned shared memory into registers
template <int NV>
__device__ __forceinline__ void load_vec(const float *src, float (&w)[4 * NV])
{
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        const float4 v = reinterpret_cast<const float4 *>(src)[u];
        w[4 * u] = v.x;
        w[4 * u + 1] = v.y;
        w[4 * u + 2] = v.z;
        w[4 * u + 3] = v.w;
    }
}

struct Outs {
    float v[JB];
};

// 1. y_k = d_k * u_k for the padded maps u (map k at u + k PS, data from LF)
template <int LF>
__device__ __forceinline__ void phase_dz(const float *d, const float *u, float *y, int K, int nb, int PS, int YS)
{
    constexpr int WV = Blk<LF>::WV;
#pragma unroll 1
    for (int it = threadIdx.x; it < K * nb; it += NB) {
        const int k = it / nb, i0 = (it - k * nb) * JB;
        float dk[LF], w[4 * WV];
        load_vec<LF / 4>(d + k * LF, dk);
        load_vec<WV>(u + (size_t)k * PS + i0, w);  // u_k[i0 + jj - l] = w[LF + jj - l]
        float acc[JB];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) acc[jj] = 0.0f;
#pragma unroll
        for (int l = 0; l < LF; ++l)
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) acc[jj] = fmaf(dk[l], w[LF + jj - l], acc[jj]);
        float4 *yo = reinterpret_cast<float4 *>(y + (size_t)k * YS + i0);
#pragma unroll
        for (int q = 0; q < JB / 4; ++q) yo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
}

// 2. r = sum_k y_k (- x, when given), the filters in a fixed order
__device__ __forceinline__ void phase_sum(const float *y, const float *x, float *r, int K, int n, int YS)
{
    for (int i = threadIdx.x; i < n; i += NB) {
        float acc = 0.0f;
        for (int k = 0; k < K; ++k) acc += y[(size_t)k * YS + i];
        r[i] = x ? acc - x[i] : acc;
    }
}

// 3. (D^T r)_k[j0 .. j0 + JB - 1] for each item, handed to f(k, j0, g)
// (g.v[jj] valid for j0 + jj < P)
template <int LF, class Fn>
__device__ __forceinline__ void phase_dtr(const float *d, const float *r, int K, int pb, Fn f)
{
    constexpr int WV = Blk<LF>::WV;
#pragma unroll 1
    for (int it = threadIdx.x; it < K * pb; it += NB) {
        const int k = it / pb, j0 = (it - k * pb) * JB;
        float dk[LF], w[4 * WV];
        load_vec<LF / 4>(d + k * LF, dk);
        load_vec<WV>(r + j0, w);
        Outs g;
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) g.v[jj] = 0.0f;
#pragma unroll
        for (int l = 0; l < LF; ++l)
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) g.v[jj] = fmaf(dk[l], w[jj + l], g.v[jj]);
        f(k, j0, g);
    }
}

// Forward; with traj, z^(t+1) of every layer t is written to traj (sample
// s, layer t at (s T + t) m), the input of the adjoint below.
template <int LF, bool TRAJ>
__global__ void __launch_bounds__(NB) conv_pgd_blk_kernel(const float *__restrict__ F, int K, int Lf,
                                                          const float *__restrict__ X, int N, int n, float lam,
                                                          const float *__restrict__ alpha,
                                                          const double *__restrict__ Lp, int T, float *__restrict__ Z,
                                                          float *__restrict__ traj)
{
    constexpr int WV = Blk<LF>::WV;
    const Blk<LF> bl(K, Lf, n);
    const int P = bl.P, m = K * P, PS = bl.PS, YS = bl.YS;
    extern __shared__ float4 sm4[];
    float *d = reinterpret_cast<float *>(sm4);  // K x LF taps (zero past Lf)
    float *x = d + K * LF;                      // n
    float *r = x + bl.XS;                       // n, then zeros
    float *y = r + bl.RS;                       // K x YS: per-filter partial sums of D z
    float *z = y + (size_t)K * YS;              // K x PS: map k at [k PS + LF, k PS + LF + P)
    const int nb = (n + JB - 1) / JB;           // output blocks of D z per filter
    const int pb = (P + JB - 1) / JB;           // output blocks of D^T r per filter
    const int tid = threadIdx.x;
    for (int e = tid; e < K * LF; e += NB) {
        const int k = e / LF, l = e - k * LF;
        d[e] = l < Lf ? __ldg(F + k * Lf + l) : 0.0f;
    }
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        __syncthreads();  // the previous sample's codes are stored
        for (int e = tid; e < n; e += NB) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < bl.RS; e += NB) r[e] = 0.0f;
        for (int e = tid; e < K * PS + 4 * WV; e += NB) z[e] = 0.0f;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            phase_dz<LF>(d, z, y, K, nb, PS, YS);
            __syncthreads();
            phase_sum(y, x, r, K, n, YS);
            __syncthreads();
            phase_dtr<LF>(d, r, K, pb, [&](int k, int j0, Outs g) {
                float *zk = z + (size_t)k * PS + LF + j0;
                if (j0 + JB <= P) {
#pragma unroll
                    for (int q = 0; q < JB / 4; ++q) {
                        const float4 v = reinterpret_cast<const float4 *>(zk)[q];
                        float zz[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const float u = fmaf(-a, g.v[4 * q + jj], zz[jj]);
                            zz[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                        }
                        reinterpret_cast<float4 *>(zk)[q] = make_float4(zz[0], zz[1], zz[2], zz[3]);
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < JB; ++jj)
                        if (j0 + jj < P) {
                            const float u = fmaf(-a, g.v[jj], zk[jj]);
                            zk[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                        }
                }
            });
            __syncthreads();
            if (TRAJ)
                for (int e = tid; e < m; e += NB) {
                    const int k = e / P, j = e - k * P;
                    traj[((size_t)s * T + t) * m + e] = z[(size_t)k * PS + LF + j];
                }
        }
        for (int e = tid; e < m; e += NB) {
            const int k = e / P, j = e - k * P;
            Z[(size_t)s * m + e] = z[(size_t)k * PS + LF + j];
        }
    }
}

// Adjoint of the forward (Eq. steprec), from its trajectory: per sample,
//   G = dF/dz^(T) = D^T (D z^(T) - x) + lam sign(z^(T)), then for t = T-1 .. 0
//   h = G * [z^(t+1) != 0];  dalpha_t += <h, z^(t+1) - z^(t)> / alpha_t;
//   G = h - alpha_t D^T (D h)
// (on the support of z^(t+1), dz^(t+1)/dalpha_t = (z^(t+1) - z^(t)) / alpha_t).
// The CTA's per-layer sums of <h, z^(t+1) - z^(t)> over its samples go to
// partial[t gridDim.x + block]; the division by alpha_t is left to the reduction.
template <int LF>
__global__ void __launch_bounds__(NB, 8) conv_adjoint_blk_kernel(const float *__restrict__ F, int K, int Lf,
                                                              const float *__restrict__ X, int N, int n, float lam,
                                                              const float *__restrict__ alpha, int T,
                                                              const float *__restrict__ traj,
                                                              float *__restrict__ partial)
{
    constexpr int WV = Blk<LF>::WV;
    const Blk<LF> bl(K, Lf, n);
    const int P = bl.P, m = K * P, PS = bl.PS, YS = bl.YS;
    extern __shared__ float4 sm4[];
    float *d = reinterpret_cast<float *>(sm4);  // K x LF taps
    float *x = d + K * LF;                      // n
    float *r = x + bl.XS;                       // n, then zeros
    float *y = r + bl.RS;                       // K x YS
    float *u = y + (size_t)K * YS;              // K x PS: padded maps (z^(T), then h)
    float *G = u + (size_t)K * PS + 4 * WV;     // m: the adjoint state
    float *zn = G + up4(m);                     // three rotating code buffers: z^(t+1),
    float *zo = zn + up4(m);                    // z^(t),
    float *zp = zo + up4(m);                    // and z^(t-1) arriving (cp.async)
    float *acc = zp + up4(m);                   // NB / 32 x T: each warp's sums of alpha_t dalpha_t
    const int nb = (n + JB - 1) / JB, pb = (P + JB - 1) / JB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < K * LF; e += NB) {
        const int k = e / LF, l = e - k * LF;
        d[e] = l < Lf ? __ldg(F + k * Lf + l) : 0.0f;
    }
    for (int e = tid; e < (NB / 32) * T; e += NB) acc[e] = 0.0f;
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        const float *ts = traj + (size_t)s * T * m;
        __syncthreads();
        for (int e = tid; e < n; e += NB) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < bl.RS; e += NB) r[e] = 0.0f;
        for (int e = tid; e < K * PS + 4 * WV; e += NB) u[e] = 0.0f;
        __syncthreads();
        for (int e = tid; e < m; e += NB) {
            const int k = e / P, j = e - k * P;
            const float v = __ldg(ts + (size_t)(T - 1) * m + e);
            zn[e] = v;
            u[(size_t)k * PS + LF + j] = v;
            zo[e] = T >= 2 ? __ldg(ts + (size_t)(T - 2) * m + e) : 0.0f;
        }
        __syncthreads();
        // G = D^T (D z^(T) - x) + lam sign(z^(T))
        phase_dz<LF>(d, u, y, K, nb, PS, YS);
        __syncthreads();
        phase_sum(y, x, r, K, n, YS);
        __syncthreads();
        phase_dtr<LF>(d, r, K, pb, [&](int k, int j0, Outs g) {
#pragma unroll
            for (int jj = 0; jj < JB; ++jj)
                if (j0 + jj < P) {
                    const int e = k * P + j0 + jj;
                    const float z = zn[e];
                    G[e] = g.v[jj] + lam * (float)((z > 0.0f) - (z < 0.0f));
                }
        });
        __syncthreads();
#pragma unroll 1
        for (int t = T - 1; t >= 0; --t) {
            // h = G on the support of z^(t+1), into the padded maps; <h, z^(t+1) - z^(t)>
            float part = 0.0f;
            for (int e = tid; e < m; e += NB) {
                const int k = e / P, j = e - k * P;
                const float h = zn[e] != 0.0f ? G[e] : 0.0f;
                part = fmaf(h, zn[e] - zo[e], part);
                u[(size_t)k * PS + LF + j] = h;
                G[e] = h;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) acc[warp * T + t] += part;
            if (t == 0) break;  // G^(0) is not needed
            // z^(t-1) into the free buffer while the products run (zero for t = 1)
            if (t >= 2) {
                for (int e = tid; e < m; e += NB) tc::cp_async4(tc::smem_u32(zp + e), ts + (size_t)(t - 2) * m + e);
                tc::cp_async_commit();
            } else {
                for (int e = tid; e < m; e += NB) zp[e] = 0.0f;
            }
            __syncthreads();
            // G = h - a D^T (D h)
            const float a = __ldg(alpha + t);
            phase_dz<LF>(d, u, y, K, nb, PS, YS);
            __syncthreads();
            phase_sum(y, nullptr, r, K, n, YS);
            __syncthreads();
            phase_dtr<LF>(d, r, K, pb, [&](int k, int j0, Outs g) {
#pragma unroll
                for (int jj = 0; jj < JB; ++jj)
                    if (j0 + jj < P) {
                        const int e = k * P + j0 + jj;
                        G[e] = fmaf(-a, g.v[jj], G[e]);
                    }
            });
            tc::cp_async_wait_all();
            __syncthreads();
            float *const fr = zn;  // z^(t+1) <- z^(t), z^(t) <- z^(t-1)
            zn = zo;
            zo = zp;
            zp = fr;
        }
    }
    __syncthreads();
    for (int t = tid; t < T; t += NB) {
        float sum = 0.0f;
        for (int w = 0; w < NB / 32; ++w) sum += acc[w * T + t];
        partial[(size_t)t * gridDim.x + blockIdx.x] = sum;
    }
}

// dalpha[t] = sum over blocks of partial[t][b] / alpha[t], in FP64, in a fixed order
__global__ void conv_reduce_kernel(const float *__restrict__ partial, int nblk, const float *__restrict__ alpha, int T,
                                   float *__restrict__ dalpha)
{
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= T) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += (double)partial[(size_t)t * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dalpha[t] = (float)(s / (double)alpha[t]);
}

template <int LF>
size_t blk_smem_bytes(int K, int Lf, int n)
{
    return sizeof(float) * Blk<LF>(K, Lf, n).floats(K);
}

template <int LF>
size_t adj_smem_bytes(int K, int Lf, int n, int T)
{
    const int m = K * (n - Lf + 1);
    return blk_smem_bytes<LF>(K, Lf, n) + sizeof(float) * (4 * (size_t)up4(m) + (size_t)(NB / 32) * T);
}

template <int LF, bool TRAJ>
int launch_blk(const ConvArgs &a, float *traj, cudaStream_t st)
{
    const size_t smem = blk_smem_bytes<LF>(a.K, a.Lf, a.n);
    auto k = conv_pgd_blk_kernel<LF, TRAJ>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    int per_sm = 0;
    SLISTA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NB, smem));
    const long long want = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(a.N < want ? a.N : want);
    k<<<grid, NB, smem, st>>>(a.F, a.K, a.Lf, a.X, a.N, a.n, a.lam, a.alpha, a.L, a.T, a.Z, traj);
    return check_launch("conv_pgd_blk_kernel");
}

// LF: the smallest of 8, 16, 32 that holds the filters and whose buffers fit
// (0: none - the plain kernel, no trajectory)
int pick_lf(int K, int Lf, int n, int T, bool adjoint)
{
    const size_t lim = 200 * 1024;
    if (Lf <= 8 && (adjoint ? adj_smem_bytes<8>(K, Lf, n, T) : blk_smem_bytes<8>(K, Lf, n)) <= lim) return 8;
    if (Lf <= 16 && (adjoint ? adj_smem_bytes<16>(K, Lf, n, T) : blk_smem_bytes<16>(K, Lf, n)) <= lim) return 16;
    if (Lf <= 32 && (adjoint ? adj_smem_bytes<32>(K, Lf, n, T) : blk_smem_bytes<32>(K, Lf, n)) <= lim) return 32;
    return 0;
}

template <int LF>
int adj_grid(int K, int Lf, int n, int T, int N)
{
    const size_t smem = adj_smem_bytes<LF>(K, Lf, n, T);
    auto k = conv_adjoint_blk_kernel<LF>;
    int per_sm = 0;
    if (allow_smem(k, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NB, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long want = (long long)num_sms() * per_sm;
    return (int)(N < want ? N : want);
}

// CTAs of the adjoint: as many as are resident at once, at most one per sample
int grid_for_adjoint(int K, int Lf, int n, int T, int N)
{
    switch (pick_lf(K, Lf, n, T, true)) {
        case 8: return adj_grid<8>(K, Lf, n, T, N);
        case 16: return adj_grid<16>(K, Lf, n, T, N);
        case 32: return adj_grid<32>(K, Lf, n, T, N);
        default: return 1;
    }
}

template <int LF>
int launch_adj(const ConvArgs &a, const float *traj, float *dalpha, void *ws, cudaStream_t st)
{
    const size_t smem = adj_smem_bytes<LF>(a.K, a.Lf, a.n, a.T);
    auto k = conv_adjoint_blk_kernel<LF>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    const int grid = grid_for_adjoint(a.K, a.Lf, a.n, a.T, a.N);
    float *partial = reinterpret_cast<float *>(ws);
    k<<<grid, NB, smem, st>>>(a.F, a.K, a.Lf, a.X, a.N, a.n, a.lam, a.alpha, a.T, traj, partial);
    int rc = check_launch("conv_adjoint_blk_kernel");
    if (rc) return rc;
    conv_reduce_kernel<<<ceil_div(a.T, 8), 256, 0, st>>>(partial, grid, a.alpha, a.T, dalpha);
    return check_launch("conv_reduce_kernel");
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
    switch (pick_lf(a.K, a.Lf, a.n, a.T, false)) {
        case 8: return launch_blk<8, false>(a, nullptr, st);
        case 16: return launch_blk<16, false>(a, nullptr, st);
        case 32: return launch_blk<32, false>(a, nullptr, st);
        default: break;
    }
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

bool traj_supported(int K, int Lf, int n, int T) { return T >= 1 && pick_lf(K, Lf, n, T, true) != 0; }

size_t backward_ws_bytes(int K, int Lf, int n, int N, int T)
{
    return sizeof(float) * (size_t)T * (size_t)grid_for_adjoint(K, Lf, n, T, N > 0 ? N : 1) + 256;
}

int launch_forward_traj(const ConvArgs &a, float *traj, cudaStream_t st)
{
    if (a.N == 0) return SLISTA_OK;
    switch (pick_lf(a.K, a.Lf, a.n, a.T, true)) {
        case 8: return launch_blk<8, true>(a, traj, st);
        case 16: return launch_blk<16, true>(a, traj, st);
        case 32: return launch_blk<32, true>(a, traj, st);
        default: return fail(SLISTA_ERR_UNSUPPORTED, "conv_slista_forward_traj: filters of at most 32 taps");
    }
}

int launch_backward(const ConvArgs &a, const float *traj, float *dalpha, void *ws, cudaStream_t st)
{
    if (a.N == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(dalpha, 0, sizeof(float) * a.T, st));
        return SLISTA_OK;
    }
    switch (pick_lf(a.K, a.Lf, a.n, a.T, true)) {
        case 8: return launch_adj<8>(a, traj, dalpha, ws, st);
        case 16: return launch_adj<16>(a, traj, dalpha, ws, st);
        case 32: return launch_adj<32>(a, traj, dalpha, ws, st);
        default: return fail(SLISTA_ERR_UNSUPPORTED, "conv_slista_backward: filters of at most 32 taps");
    }
}

}  // namespace conv
}  // namespace slista
