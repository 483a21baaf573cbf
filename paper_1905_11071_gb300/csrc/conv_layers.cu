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

// The same layers on a 2-D convolutional dictionary: K filters of Lh x Lw
// taps on H x W images, codes of K maps of Ph x Pw = (H - Lh + 1) x
// (W - Lw + 1) valid positions (images and maps row-major), so that
//   (D z)[i, j]      = sum_k sum_{a, b} d_k[a, b] z_k[i - a, j - b]
//   (D^T r)_k[p, q]  = sum_{a, b} d_k[a, b] r[p + a, q + b]
// One CTA per image at a time with the filters, the image, the residual and
// the codes in shared memory; a thread per pixel of D z (the filters summed
// in order, the taps limited to valid code positions) and per code of
// D^T r.  Consecutive threads take consecutive pixels or codes, so their
// shared-memory reads are consecutive words.
__global__ void __launch_bounds__(NT) conv2d_pgd_kernel(const float *__restrict__ F, int K, int Lh, int Lw,
                                                        const float *__restrict__ X, int N, int H, int W, float lam,
                                                        const float *__restrict__ alpha,
                                                        const double *__restrict__ Lp, int T, float *__restrict__ Z)
{
    extern __shared__ float sm[];
    const int Ph = H - Lh + 1, Pw = W - Lw + 1, PP = Ph * Pw, m = K * PP, n = H * W, LL = Lh * Lw;
    float *d = sm;          // K x Lh x Lw
    float *x = d + K * LL;  // H x W
    float *r = x + n;       // H x W: D z - x
    float *z = r + n;       // K x Ph x Pw
    const int tid = threadIdx.x;
    for (int e = tid; e < K * LL; e += NT) d[e] = __ldg(F + e);
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        __syncthreads();  // the previous image's codes are stored
        for (int e = tid; e < n; e += NT) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < m; e += NT) z[e] = 0.0f;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            // r = D z - x
#pragma unroll 1
            for (int e = tid; e < n; e += NT) {
                const int i = e / W, j = e - i * W;
                const int a0 = max(0, i - Ph + 1), a1 = min(Lh - 1, i);
                const int b0 = max(0, j - Pw + 1), b1 = min(Lw - 1, j);
                float acc = 0.0f;
                for (int k = 0; k < K; ++k) {
                    const float *dk = d + k * LL;
                    const float *zk = z + k * PP;
                    for (int ta = a0; ta <= a1; ++ta)
                        for (int tb = b0; tb <= b1; ++tb)
                            acc = fmaf(dk[ta * Lw + tb], zk[(i - ta) * Pw + (j - tb)], acc);
                }
                r[e] = acc - x[e];
            }
            __syncthreads();
            // z = ST(z - a D^T r, a lam)
#pragma unroll 1
            for (int e = tid; e < m; e += NT) {
                const int k = e / PP, pq = e - k * PP, p = pq / Pw, q = pq - p * Pw;
                const float *dk = d + k * LL;
                const float *rp = r + p * W + q;
                float g = 0.0f;
                for (int ta = 0; ta < Lh; ++ta)
                    for (int tb = 0; tb < Lw; ++tb) g = fmaf(dk[ta * Lw + tb], rp[ta * W + tb], g);
                const float u = fmaf(-a, g, z[e]);
                z[e] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
            }
            __syncthreads();
        }
        for (int e = tid; e < m; e += NT) Z[(size_t)s * m + e] = z[e];
    }
}

// The same layers with register blocking, for filters of at most LF taps
// (zero-padded to LF, LF a multiple of 4), in CTAs of NB threads.  The
// filters are taken in groups of KG (K rounded up with all-zero filters); a
// work item is JB = 4 consecutive outputs for one group, computed from
// windows of inputs read as 16-byte vectors (conflict-free: the items of a
// warp read one contiguous segment) and the group's taps (16-byte vectors,
// the same for the whole warp).  Each code map lives in shared memory with
// LF zeros on its left and at least LF on its right, the residual with zeros
// after it, so no item needs bounds checks.  Per layer:
//   1. y_g[i] = sum_{k in g} sum_l d_k[l] z_k[i - l], i < n   (items g, i-block; k in order)
//   2. r[i] = sum_g y_g[i] - x[i]                              (fixed order over g)
//   3. z_k[j] = ST(z_k[j] - a sum_l d_k[l] r[j + l], a lam)    (items g, j-block: one window of r
//                                                                for the group's filters)
constexpr int NB = 128;  // threads of a blocked CTA
constexpr int JB = 4;    // outputs of a work item
constexpr int KG = 2;    // filters of a work item
__host__ __device__ constexpr int up4(int v) { return (v + 3) & ~3; }

template <int LF>
struct Blk {
    static_assert(LF % 4 == 0, "taps in 16-byte units");
    static constexpr int WV = (LF + JB) / 4;  // 16-byte units of a window
    int P, Kp, NG;                             // positions; filters rounded up to groups; groups
    int XS, RS, YS, PS;                        // strides of x, r, y, the padded maps
    __host__ __device__ Blk(int K, int Lf, int n)
    {
        P = n - Lf + 1;
        Kp = (K + KG - 1) / KG * KG;
        NG = Kp / KG;
        XS = up4(n);
        RS = up4(n + LF + JB);
        YS = up4(n + JB);
        PS = up4(LF + P + LF);
    }
    // floats: taps, x, r, y, maps, and one window past the last map
    __host__ __device__ size_t floats() const
    {
        return (size_t)Kp * LF + XS + RS + (size_t)NG * YS + (size_t)Kp * PS + 4 * WV;
    }
};

// 4 NV floats from 16-byte aligned shared memory into registers
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

// taps of the Kp padded filters (zero past Lf and for k >= K)
template <int LF>
__device__ __forceinline__ void load_taps(const float *F, int K, int Kp, int Lf, float *d)
{
    for (int e = threadIdx.x; e < Kp * LF; e += NB) {
        const int k = e / LF, l = e - k * LF;
        d[e] = (k < K && l < Lf) ? __ldg(F + k * Lf + l) : 0.0f;
    }
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

// A thread's work items are it = tid, tid + NB, ... of NG x nb; (g, b) of the
// first comes from the caller (one division per kernel), the next by stepping.
struct Item {
    int g, b, dg, db;  // current item; the step NB = dg nb + db
    __device__ Item(int it, int nb) : g(it / nb), b(it % nb), dg(NB / nb), db(NB % nb) {}
    __device__ __forceinline__ void next(int nb)
    {
        g += dg;
        b += db;
        if (b >= nb) b -= nb, ++g;
    }
};

// 1. y_g = sum_{k in g} d_k * u_k for the padded maps u (map k at u + k PS, data from LF)
template <int LF>
__device__ __forceinline__ void phase_dz(const float *d, const float *u, float *y, int NG, int nb, Item c, int PS,
                                         int YS)
{
    constexpr int WV = Blk<LF>::WV;
#pragma unroll 1
    for (; c.g < NG; c.next(nb)) {
        const int g = c.g, i0 = c.b * JB;
        float acc[JB] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < KG; ++q) {
            const int k = g * KG + q;
            float dk[LF], w[4 * WV];
            load_vec<LF / 4>(d + k * LF, dk);
            load_vec<WV>(u + (k * PS + i0), w);  // u_k[i0 + jj - l] = w[LF + jj - l]
#pragma unroll
            for (int l = 0; l < LF; ++l)
#pragma unroll
                for (int jj = 0; jj < JB; ++jj) acc[jj] = fmaf(dk[l], w[LF + jj - l], acc[jj]);
        }
        *reinterpret_cast<float4 *>(y + (g * YS + i0)) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    }
}

// 2. r = sum_g y_g (- x, when given), the groups in a fixed order
__device__ __forceinline__ void phase_sum(const float *y, const float *x, float *r, int NG, int n, int YS)
{
    for (int i = threadIdx.x; i < n; i += NB) {
        float acc = 0.0f;
        for (int g = 0; g < NG; ++g) acc += y[g * YS + i];
        r[i] = x ? acc - x[i] : acc;
    }
}

// 3. (D^T r)_k[j0 .. j0 + 3] for each filter k of each item, handed to
// f(k, j0, g) as a float4 (component jj valid for j0 + jj < P; k may be a
// padding filter, k >= K)
template <int LF, class Fn>
__device__ __forceinline__ void phase_dtr(const float *d, const float *r, int NG, int pb, Item c, Fn f)
{
    constexpr int WV = Blk<LF>::WV;
#pragma unroll 1
    for (; c.g < NG; c.next(pb)) {
        const int g = c.g, j0 = c.b * JB;
        float w[4 * WV];
        load_vec<WV>(r + j0, w);
#pragma unroll
        for (int q = 0; q < KG; ++q) {
            const int k = g * KG + q;
            float dk[LF];
            load_vec<LF / 4>(d + k * LF, dk);
            float o[JB] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int l = 0; l < LF; ++l)
#pragma unroll
                for (int jj = 0; jj < JB; ++jj) o[jj] = fmaf(dk[l], w[jj + l], o[jj]);
            f(k, j0, make_float4(o[0], o[1], o[2], o[3]));
        }
    }
}

// Forward; with traj, z^(t+1) of every layer t is written to traj, the input
// of the adjoint below: sample s, layer t, map k at ((s T + t) K + k) PQ, PQ =
// P rounded up to a multiple of 4 (entries past P zero), so that every item
// stores 16 bytes and the adjoint loads 16 bytes at a time.
template <int LF, bool TRAJ>
__global__ void __launch_bounds__(NB, LF >= 32 ? 7 : 10) conv_pgd_blk_kernel(const float *__restrict__ F, int K, int Lf,
                                                          const float *__restrict__ X, int N, int n, float lam,
                                                          const float *__restrict__ alpha,
                                                          const double *__restrict__ Lp, int T, float *__restrict__ Z,
                                                          float *__restrict__ traj)
{
    constexpr int WV = Blk<LF>::WV;
    const Blk<LF> bl(K, Lf, n);
    const int P = bl.P, m = K * P, PS = bl.PS, YS = bl.YS, NG = bl.NG;
    extern __shared__ float4 sm4[];
    float *d = reinterpret_cast<float *>(sm4);  // Kp x LF taps
    float *x = d + bl.Kp * LF;                  // n
    float *r = x + bl.XS;                       // n, then zeros
    float *y = r + bl.RS;                       // NG x YS: per-group partial sums of D z
    float *z = y + (size_t)NG * YS;             // Kp x PS: map k at [k PS + LF, k PS + LF + P)
    const int nb = (n + JB - 1) / JB;           // output blocks of D z
    const int pb = (P + JB - 1) / JB;           // output blocks of D^T r
    const int tid = threadIdx.x;
    const Item it_dz(tid, nb), it_dtr(tid, pb);
    const size_t mq = (size_t)K * up4(P);       // floats of one layer in traj
    load_taps<LF>(F, K, bl.Kp, Lf, d);
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        __syncthreads();  // the previous sample's codes are stored
        for (int e = tid; e < n; e += NB) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < bl.RS; e += NB) r[e] = 0.0f;
        for (int e = tid; e < bl.Kp * PS + 4 * WV; e += NB) z[e] = 0.0f;
        __syncthreads();
#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            phase_dz<LF>(d, z, y, NG, nb, it_dz, PS, YS);
            __syncthreads();
            phase_sum(y, x, r, NG, n, YS);
            __syncthreads();
            // the step; with TRAJ the new codes also go to traj (16-byte stores)
            float *zt = TRAJ ? traj + ((size_t)s * T + t) * mq : nullptr;
            phase_dtr<LF>(d, r, NG, pb, it_dtr, [&](int k, int j0, float4 g4) {
                if (k >= K) return;
                const float g[JB] = {g4.x, g4.y, g4.z, g4.w};
                float *zk = z + (k * PS + LF + j0);
                float zz[JB];
                if (j0 + JB <= P) {
                    const float4 v = *reinterpret_cast<const float4 *>(zk);
                    zz[0] = v.x, zz[1] = v.y, zz[2] = v.z, zz[3] = v.w;
#pragma unroll
                    for (int jj = 0; jj < JB; ++jj) {
                        const float u = fmaf(-a, g[jj], zz[jj]);
                        zz[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                    }
                    *reinterpret_cast<float4 *>(zk) = make_float4(zz[0], zz[1], zz[2], zz[3]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < JB; ++jj) {
                        zz[jj] = 0.0f;
                        if (j0 + jj < P) {
                            const float u = fmaf(-a, g[jj], zk[jj]);
                            zz[jj] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                            zk[jj] = zz[jj];
                        }
                    }
                }
                if (TRAJ)
                    *reinterpret_cast<float4 *>(zt + (k * up4(P) + j0)) = make_float4(zz[0], zz[1], zz[2], zz[3]);
            });
            __syncthreads();
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
// The masking and the dot product of layer t - 1 are done in the epilogue of
// layer t's D^T product, so each layer is one pass of the three phases.  The
// adjoint state and two code vectors (z^(t), z^(t-1), the next arriving by
// cp.async while the products run) are kept per map with a 16-byte aligned
// stride PQ.  The CTA's per-layer sums of <h, z^(t+1) - z^(t)> over its
// samples go to partial[t gridDim.x + block]; the division by alpha_t is left
// to the reduction.
template <int LF>
__global__ void __launch_bounds__(NB, LF == 16 ? 9 : (LF >= 32 ? 7 : 8)) conv_adjoint_blk_kernel(const float *__restrict__ F, int K, int Lf,
                                                              const float *__restrict__ X, int N, int n, float lam,
                                                              const float *__restrict__ alpha, int T,
                                                              const float *__restrict__ traj,
                                                              float *__restrict__ partial)
{
    constexpr int WV = Blk<LF>::WV;
    const Blk<LF> bl(K, Lf, n);
    const int P = bl.P, PS = bl.PS, YS = bl.YS, NG = bl.NG, PQ = up4(P);
    const int mq = K * PQ;                      // floats of one layer in traj
    extern __shared__ float4 sm4[];
    float *d = reinterpret_cast<float *>(sm4);  // Kp x LF taps
    float *x = d + bl.Kp * LF;                  // n
    float *r = x + bl.XS;                       // n, then zeros
    float *y = r + bl.RS;                       // NG x YS
    float *u = y + (size_t)NG * YS;             // Kp x PS: padded maps (z^(T), then h)
    float *G = u + (size_t)bl.Kp * PS + 4 * WV; // K x PQ: the adjoint state
    float *zc = G + (size_t)K * PQ;             // K x PQ: z^(t)
    float *zp = zc + (size_t)K * PQ;            // K x PQ: z^(t-1)
    float *acc = zp + (size_t)K * PQ;           // NB / 32 x T: each warp's sums of alpha_t dalpha_t
    const int nb = (n + JB - 1) / JB, pb = (P + JB - 1) / JB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Item it_dz(tid, nb), it_dtr(tid, pb);
    load_taps<LF>(F, K, bl.Kp, Lf, d);
    for (int e = tid; e < (NB / 32) * T; e += NB) acc[e] = 0.0f;
    // the dot product of layer tt: this thread's part, summed over the warp
    auto add_part = [&](float part, int tt) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) acc[warp * T + tt] += part;
    };
    // layer tt's mask and dot product for codes (k, j0 .. j0 + 3) given the new
    // adjoint state gv: h = gv on the support of znew; part += <h, znew - zold>;
    // h to the padded maps and to G
    auto mask_step = [&](int k, int j0, const float (&gv)[JB], const float *znew, const float *zold, float &part) {
        const int q = k * PQ + j0;
        float zn4[JB], zo4[JB], h[JB];
        load_vec<1>(znew + q, zn4);
        load_vec<1>(zold + q, zo4);
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {  // past P the codes are zero, so h is too
            h[jj] = zn4[jj] != 0.0f ? gv[jj] : 0.0f;
            part = fmaf(h[jj], zn4[jj] - zo4[jj], part);
        }
        const float4 h4 = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(G + q) = h4;
        *reinterpret_cast<float4 *>(u + (k * PS + LF + j0)) = h4;  // zeros past P keep the pad
    };
    // codes of layer tt of this sample (z^(tt+1), K x PQ; zeros for tt < 0), 16 bytes at a time
    auto fetch = [&](const float *ts, int tt, float *dst, bool async) {
        const float *src = ts + (size_t)tt * mq;
        for (int e = 4 * tid; e < mq; e += 4 * NB) {
            if (tt < 0)
                *reinterpret_cast<float4 *>(dst + e) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            else if (async)
                cp_async16(dst + e, src + e);
            else
                *reinterpret_cast<float4 *>(dst + e) = __ldg(reinterpret_cast<const float4 *>(src + e));
        }
    };
#pragma unroll 1
    for (int s = blockIdx.x; s < N; s += gridDim.x) {
        const float *ts = traj + (size_t)s * T * mq;
        __syncthreads();
        for (int e = tid; e < n; e += NB) x[e] = __ldg(X + (size_t)s * n + e);
        for (int e = tid; e < bl.RS; e += NB) r[e] = 0.0f;
        for (int e = tid; e < bl.Kp * PS + 4 * WV; e += NB) u[e] = 0.0f;
        fetch(ts, T - 1, zc, false);  // z^(T)
        fetch(ts, T - 2, zp, false);  // z^(T-1)
        __syncthreads();
        // z^(T) into the padded maps (16 bytes at a time: the entries past P are zero)
        for (int e = 4 * tid; e < mq; e += 4 * NB) {
            const int k = e / PQ, j = e - k * PQ;
            *reinterpret_cast<float4 *>(u + (size_t)k * PS + LF + j) = *reinterpret_cast<const float4 *>(zc + e);
        }
        __syncthreads();
        // G = D^T (D z^(T) - x) + lam sign(z^(T)), then layer T-1's mask and dot product
        phase_dz<LF>(d, u, y, NG, nb, it_dz, PS, YS);
        __syncthreads();
        phase_sum(y, x, r, NG, n, YS);
        __syncthreads();
        float part = 0.0f;
        phase_dtr<LF>(d, r, NG, pb, it_dtr, [&](int k, int j0, float4 g4) {
            if (k >= K) return;
            const float g[JB] = {g4.x, g4.y, g4.z, g4.w};
            float gv[JB];
            const float *zk = zc + (k * PQ + j0);
#pragma unroll
            for (int jj = 0; jj < JB; ++jj) gv[jj] = g[jj] + lam * (float)((zk[jj] > 0.0f) - (zk[jj] < 0.0f));
            mask_step(k, j0, gv, zc, zp, part);
        });
        add_part(part, T - 1);
#pragma unroll 1
        for (int t = T - 1; t >= 1; --t) {
            // here G = h of layer t (also in the padded maps), zc = z^(t+1), zp = z^(t)
            float *const zq = zc;  // z^(t+1) is no longer needed: z^(t-1) arrives there
            zc = zp;
            zp = zq;
            __syncthreads();
            fetch(ts, t - 2, zp, true);
            tc::cp_async_commit();
            // G = h - a D^T (D h), then layer t-1's mask and dot product
            const float a = __ldg(alpha + t);
            phase_dz<LF>(d, u, y, NG, nb, it_dz, PS, YS);
            __syncthreads();
            phase_sum(y, nullptr, r, NG, n, YS);
            tc::cp_async_wait_all();
            __syncthreads();
            part = 0.0f;
            phase_dtr<LF>(d, r, NG, pb, it_dtr, [&](int k, int j0, float4 g4) {
                if (k >= K) return;
                const float g[JB] = {g4.x, g4.y, g4.z, g4.w};
                float gv[JB], gk[JB];
                load_vec<1>(G + (k * PQ + j0), gk);
#pragma unroll
                for (int jj = 0; jj < JB; ++jj) gv[jj] = fmaf(-a, g[jj], gk[jj]);
                mask_step(k, j0, gv, zc, zp, part);
            });
            add_part(part, t - 1);
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
    return sizeof(float) * Blk<LF>(K, Lf, n).floats();
}

template <int LF>
size_t adj_smem_bytes(int K, int Lf, int n, int T)
{
    return blk_smem_bytes<LF>(K, Lf, n) + sizeof(float) * (3 * (size_t)K * up4(n - Lf + 1) + (size_t)(NB / 32) * T);
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

size_t smem2d_bytes(int K, int Lh, int Lw, int H, int W)
{
    return sizeof(float) * ((size_t)K * Lh * Lw + 2 * (size_t)H * W + (size_t)K * (H - Lh + 1) * (W - Lw + 1));
}

bool supported2d(int K, int Lh, int Lw, int H, int W)
{
    return K >= 1 && Lh >= 1 && Lw >= 1 && H >= Lh && W >= Lw && (long long)H * W <= 16384 &&
           (long long)K * Lh * Lw <= 8192 && smem2d_bytes(K, Lh, Lw, H, W) <= 200 * 1024;
}

int launch_forward2d(const Conv2dArgs &a, cudaStream_t st)
{
    const size_t m = (size_t)a.K * (a.H - a.Lh + 1) * (a.W - a.Lw + 1);
    if (a.N == 0) return SLISTA_OK;
    if (a.T == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(float) * (size_t)a.N * m, st));
        return SLISTA_OK;
    }
    const size_t smem = smem2d_bytes(a.K, a.Lh, a.Lw, a.H, a.W);
    SLISTA_CUDA_TRY(allow_smem(conv2d_pgd_kernel, smem));
    int per_sm = 0;
    SLISTA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv2d_pgd_kernel, NT, smem));
    const long long want = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(a.N < want ? a.N : want);
    conv2d_pgd_kernel<<<grid, NT, smem, st>>>(a.F, a.K, a.Lh, a.Lw, a.X, a.N, a.H, a.W, a.lam, a.alpha, a.L, a.T,
                                              a.Z);
    return check_launch("conv2d_pgd_kernel");
}

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

size_t traj_floats(int K, int Lf, int n, int N, int T)
{
    return (size_t)N * (size_t)T * (size_t)K * (size_t)up4(n - Lf + 1);
}

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
