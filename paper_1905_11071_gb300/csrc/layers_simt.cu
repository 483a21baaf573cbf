// FP32 CUDA-core kernels for the unfolded proximal-gradient layers
// (Eq. pgd / Eq. steprec), their adjoint and the Lasso objective.
//
// State per sample lives in registers for all T layers: the code z and the
// residual correlation g = c - B z (the negative gradient of the smooth part
// of F_x).  A layer is
//     u = z + alpha_t g,  z' = ST(u, alpha_t lam),  g' = g - B (z' - z)
// which is Eq. pgd with D^T(Dz - x) = B z - c kept up to date incrementally:
// only the step d = z - z' goes through the contraction (g' = g + d B, B
// symmetric), so C is read once and no per-layer HBM traffic remains.
#include "common.cuh"
#include "simt.cuh"
#include "kernels.h"

namespace slista {
namespace simt {

// ---------------------------------------------------------------------------
// Forward: ISTA (alpha == nullptr, step 1/L from *Lp) or SLISTA (alpha[t]).
// ---------------------------------------------------------------------------
template <int MP, int NB>
__global__ void __launch_bounds__(NT) pgd_forward_kernel(
    const float *__restrict__ B, const float *__restrict__ C, int m, int N, float lam,
    const float *__restrict__ alpha, const double *__restrict__ Lp, int T,
    float *__restrict__ Z, uint32_t *__restrict__ masks, float *__restrict__ ckpt, int K)
{
    using TL = Tile<MP, NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    float *B_s = A_s + TL::A_FLOATS;
    const int row0 = blockIdx.x * NB;
    const int W = (m + 31) / 32;
    const size_t plane = (size_t)N * m;

    float g[TL::RM][TL::RN], z[TL::RM][TL::RN], d[TL::RM][TL::RN];
    load_rows<TL>(g, C, row0, N, m, m);
#pragma unroll
    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) z[i][j] = 0.0f;
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));

#pragma unroll 1
    for (int t = 0; t < T; ++t) {
        if (ckpt && t > 0 && t % K == 0) {
            float *base = ckpt + (size_t)(t / K - 1) * 2 * plane;
            store_rows<TL>(base, z, row0, N, m, m);
            store_rows<TL>(base + plane, g, row0, N, m, m);
        }
        const float a = alpha ? __ldg(alpha + t) : a_const;
        const float thr = __fmul_rn(a, lam);
#pragma unroll
        for (int i = 0; i < TL::RM; ++i)
#pragma unroll
            for (int j = 0; j < TL::RN; ++j) {
                float zn = soft_threshold(fmaf(a, g[i][j], z[i][j]), thr);
                d[i][j] = z[i][j] - zn;
                z[i][j] = zn;
            }
        if (masks) store_support_words<TL>(masks + (size_t)t * N * W, z, row0, N, W);
        if (t == T - 1) break;
        store_tile<TL>(A_s, d);
        gemm_acc<TL>(g, A_s, TL::LDA, B, m, m, m, B_s);
    }
    store_rows<TL>(Z, z, row0, N, m, m);
}

// ---------------------------------------------------------------------------
// Adjoint of Step-LISTA (Eq. steprec), recomputing between checkpoints.
//
// Per tile and segment [t0, t1) (walked last to first): reload (z, g) at t0
// from the checkpoint (or z = 0, g = c at t0 = 0), recompute the layers with
// the forward's arithmetic while storing q_t = g^(t) - lam sign(z^(t+1)) to
// the workspace, then walk the segment backwards:
//     h = G * mask_t,  dalpha_t += <h, q_t>,  G = h - alpha_t B h.
// Per-CTA partial sums of dalpha_t go to partial[t * gridDim.x + block].
// ---------------------------------------------------------------------------
template <int MP, int NB>
__global__ void __launch_bounds__(NT) slista_backward_kernel(
    const float *__restrict__ B, const float *__restrict__ C, int m, int N, float lam,
    const float *__restrict__ alpha, int T, const uint32_t *__restrict__ masks,
    const float *__restrict__ ckpt, int K, const float *__restrict__ gZ,
    float *__restrict__ qbuf, float *__restrict__ partial)
{
    using TL = Tile<MP, NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    float *B_s = A_s + TL::A_FLOATS;
    __shared__ float red[NT / 32];
    const Idx<TL> ix;
    const int row0 = blockIdx.x * NB;
    const int W = (m + 31) / 32;
    const size_t plane = (size_t)N * m;
    const size_t npad = (size_t)gridDim.x * NB;
    const int nseg = (T + K - 1) / K;

    float G[TL::RM][TL::RN];
#pragma unroll 1
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int t0 = seg * K;
        const int t1 = min(T, t0 + K);
        const bool last = (seg == nseg - 1);
        {
            float z[TL::RM][TL::RN], g[TL::RM][TL::RN], d[TL::RM][TL::RN];
            if (seg == 0) {
                load_rows<TL>(g, C, row0, N, m, m);
#pragma unroll
                for (int i = 0; i < TL::RM; ++i)
#pragma unroll
                    for (int j = 0; j < TL::RN; ++j) z[i][j] = 0.0f;
            } else {
                const float *base = ckpt + (size_t)(seg - 1) * 2 * plane;
                load_rows<TL>(z, base, row0, N, m, m);
                load_rows<TL>(g, base + plane, row0, N, m, m);
            }
#pragma unroll 1
            for (int t = t0; t < t1; ++t) {
                const float a = __ldg(alpha + t);
                const float thr = __fmul_rn(a, lam);
                float *qt = qbuf + (size_t)(t - t0) * npad * MP;
#pragma unroll
                for (int i = 0; i < TL::RM; ++i) {
                    const size_t r = (size_t)row0 + ix.row(i);
#pragma unroll
                    for (int q = 0; q < TL::GPT; ++q) {
                        float qv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = q * 4 + e;
                            float zn = soft_threshold(fmaf(a, g[i][j], z[i][j]), thr);
                            qv[e] = g[i][j] - lam * signf(zn);
                            d[i][j] = z[i][j] - zn;
                            z[i][j] = zn;
                        }
                        *reinterpret_cast<float4 *>(qt + r * MP + ix.col(q, 0)) =
                            make_float4(qv[0], qv[1], qv[2], qv[3]);
                    }
                }
                const bool need_next = (t + 1 < t1) || (last && t == T - 1 && gZ == nullptr);
                if (need_next) {
                    store_tile<TL>(A_s, d);
                    gemm_acc<TL>(g, A_s, TL::LDA, B, m, m, m, B_s);
                }
            }
            if (last) {
                if (gZ) {
                    load_rows<TL>(G, gZ, row0, N, m, m);
                } else {
                    // dF/dz^(T) = B z - c + lam sign(z) = -g + lam sign(z)
#pragma unroll
                    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
                        for (int j = 0; j < TL::RN; ++j) G[i][j] = -g[i][j] + lam * signf(z[i][j]);
                }
            }
        }
#pragma unroll 1
        for (int t = t1 - 1; t >= t0; --t) {
            const uint32_t *mk = masks + (size_t)t * N * W;
            const float *qt = qbuf + (size_t)(t - t0) * npad * MP;
            float part = 0.0f;
#pragma unroll
            for (int i = 0; i < TL::RM; ++i) {
                const int r = row0 + ix.row(i);
#pragma unroll
                for (int q = 0; q < TL::GPT; ++q) {
                    const int c0 = ix.col(q, 0);
                    uint32_t word = (r < N && c0 < m) ? __ldg(mk + (size_t)r * W + (c0 >> 5)) : 0u;
                    float4 qv = *reinterpret_cast<const float4 *>(qt + (size_t)r * MP + c0);
                    const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = q * 4 + e;
                        const bool on = (word >> ((c0 + e) & 31)) & 1u;
                        G[i][j] = on ? G[i][j] : 0.0f;  // h = G * mask_t
                        part = fmaf(G[i][j], qa[e], part);
                    }
                }
            }
            // block reduction of part -> partial[t][block]
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                float s = 0.0f;
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) s += red[w];
                partial[(size_t)t * gridDim.x + blockIdx.x] = s;
            }
            if (t == 0) break;
            const float a = __ldg(alpha + t);
            float acc[TL::RM][TL::RN];
#pragma unroll
            for (int i = 0; i < TL::RM; ++i)
#pragma unroll
                for (int j = 0; j < TL::RN; ++j) acc[i][j] = 0.0f;
            store_tile<TL>(A_s, G);
            gemm_acc<TL>(acc, A_s, TL::LDA, B, m, m, m, B_s);  // B h (B symmetric)
#pragma unroll
            for (int i = 0; i < TL::RM; ++i)
#pragma unroll
                for (int j = 0; j < TL::RN; ++j) G[i][j] = fmaf(-a, acc[i][j], G[i][j]);
        }
    }
}

// dalpha[t] = sum over blocks of partial[t][b], in FP64, fixed order.
__global__ void reduce_partials_kernel(const float *__restrict__ partial, int nblk, int T,
                                       float *__restrict__ dalpha)
{
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= T) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += (double)partial[(size_t)t * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dalpha[t] = (float)s;
}

// ---------------------------------------------------------------------------
// Objective and duality gap from (B, c, xsq): per row, with w = B z,
//   F = xsq/2 - c.z + z.w/2 + lam |z|_1,  r2 = xsq - 2 c.z + z.w,
//   xr = xsq - c.z,  s = min(1, lam / |c - w|_inf),  gap = F - (s xr - s^2 r2 / 2).
// ---------------------------------------------------------------------------

// Objective and gap for wide dictionaries (256 < m <= 1024): the sample
// rows z (all m codes) sit in A_s, w = z B is formed 256 columns at a time
// by the tile engine, and the per-row sums (c.z, z.w, |z|_1, |c - w|_inf) accumulate
// over the column blocks in registers.
template <int NB>
__global__ void __launch_bounds__(NT) objective_wide_kernel(
    const float *__restrict__ B, const float *__restrict__ C, const double *__restrict__ xsq,
    const float *__restrict__ Z, int m, int N, int lda, float lam, double *__restrict__ F,
    double *__restrict__ gap)
{
    using TL = Tile<256, NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    float *B_s = A_s + (size_t)NB * lda;
    const Idx<TL> ix;
    const int row0 = blockIdx.x * NB;
    const int kp = lda - 4;  // m rounded up to 16
    for (int e = threadIdx.x; e < NB * kp; e += NT) {
        const int r = e / kp, k = e % kp;
        A_s[r * lda + k] = (row0 + r < N && k < m) ? __ldg(Z + (size_t)(row0 + r) * m + k) : 0.0f;
    }
    double cz[TL::RM], zw[TL::RM], l1[TL::RM];
    float cinf[TL::RM];
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        cz[i] = zw[i] = l1[i] = 0.0;
        cinf[i] = 0.0f;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < m; c0 += 256) {
        const int nc = m - c0 < 256 ? m - c0 : 256;
        float w[TL::RM][TL::RN], c[TL::RM][TL::RN];
#pragma unroll
        for (int i = 0; i < TL::RM; ++i)
#pragma unroll
            for (int j = 0; j < TL::RN; ++j) w[i][j] = 0.0f;
        gemm_acc<TL>(w, A_s, lda, B + c0, m, nc, m, B_s);
        load_rows<TL>(c, C + c0, row0, N, nc, m);
#pragma unroll
        for (int i = 0; i < TL::RM; ++i)
#pragma unroll
            for (int q = 0; q < TL::GPT; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int col = ix.col(q, e);
                    if (col >= nc) continue;
                    const float zv = A_s[ix.row(i) * lda + c0 + col];
                    const float wv = w[i][q * 4 + e], cv = c[i][q * 4 + e];
                    cz[i] = fma((double)cv, (double)zv, cz[i]);
                    zw[i] = fma((double)zv, (double)wv, zw[i]);
                    l1[i] += (double)fabsf(zv);
                    cinf[i] = fmaxf(cinf[i], fabsf(cv - wv));
                }
    }
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
#pragma unroll
        for (int o = TL::TXN / 2; o > 0; o >>= 1) {
            cz[i] += __shfl_xor_sync(0xffffffffu, cz[i], o);
            zw[i] += __shfl_xor_sync(0xffffffffu, zw[i], o);
            l1[i] += __shfl_xor_sync(0xffffffffu, l1[i], o);
            cinf[i] = fmaxf(cinf[i], __shfl_xor_sync(0xffffffffu, cinf[i], o));
        }
        const int r = row0 + ix.row(i);
        if (ix.tx == 0 && r < N) {
            const double xx = xsq[r];
            const double Fv = 0.5 * xx - cz[i] + 0.5 * zw[i] + (double)lam * l1[i];
            F[r] = Fv;
            if (gap) {
                const double r2 = xx - 2.0 * cz[i] + zw[i];
                const double xr = xx - cz[i];
                const double sc = (double)cinf[i] > (double)lam ? (double)lam / (double)cinf[i] : 1.0;
                gap[r] = Fv - (sc * xr - 0.5 * sc * sc * r2);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
namespace {

template <int MP>
struct Choice;
template <> struct Choice<32> { static constexpr int NB = 64; };
template <> struct Choice<64> { static constexpr int NB = 64; };
template <> struct Choice<128> { static constexpr int NB = 64; };
template <> struct Choice<256> { static constexpr int NB = 32; };

template <int MP>
int launch_forward_mp(const PgdArgs &a, cudaStream_t st)
{
    constexpr int NB = Choice<MP>::NB;
    using TL = Tile<MP, NB>;
    const size_t smem = (size_t)TL::SMEM_FLOATS * sizeof(float);
    auto k = pgd_forward_kernel<MP, NB>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    const int grid = ceil_div(a.N, NB);
    if (grid == 0) return SLISTA_OK;
    k<<<grid, NT, smem, st>>>(a.B, a.C, a.m, a.N, a.lam, a.alpha, a.L, a.T, a.Z, a.masks, a.ckpt,
                              a.ckpt_every);
    return check_launch("pgd_forward_kernel");
}

template <int MP>
int launch_backward_mp(const BwdArgs &a, void *ws, cudaStream_t st)
{
    constexpr int NB = Choice<MP>::NB;
    using TL = Tile<MP, NB>;
    const size_t smem = (size_t)TL::SMEM_FLOATS * sizeof(float);
    auto k = slista_backward_kernel<MP, NB>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    const int grid = ceil_div(a.N, NB);
    float *qbuf = reinterpret_cast<float *>(ws);
    float *partial = qbuf + (size_t)a.ckpt_every * grid * NB * MP;
    if (grid > 0) {
        k<<<grid, NT, smem, st>>>(a.B, a.C, a.m, a.N, a.lam, a.alpha, a.T, a.masks, a.ckpt, a.ckpt_every,
                                  a.gZ, qbuf, partial);
        int rc = check_launch("slista_backward_kernel");
        if (rc) return rc;
        reduce_partials_kernel<<<ceil_div(a.T, 8), 256, 0, st>>>(partial, grid, a.T, a.dalpha);
    } else {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.dalpha, 0, sizeof(float) * a.T, st));
    }
    return check_launch("reduce_partials_kernel");
}

template <int MP>
size_t backward_ws_mp(int N, int T, int K)
{
    constexpr int NB = Choice<MP>::NB;
    const size_t grid = (size_t)ceil_div(N, NB);
    return sizeof(float) * ((size_t)K * grid * NB * MP + (size_t)T * grid);
}


}  // namespace

int padded_mp(int m)
{
    if (m <= 32) return 32;
    if (m <= 64) return 64;
    if (m <= 128) return 128;
    if (m <= 256) return 256;
    return 0;
}

int launch_forward(const PgdArgs &a, cudaStream_t st)
{
    switch (padded_mp(a.m)) {
        case 32: return launch_forward_mp<32>(a, st);
        case 64: return launch_forward_mp<64>(a, st);
        case 128: return launch_forward_mp<128>(a, st);
        case 256: return launch_forward_mp<256>(a, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "FP32 layer kernel supports m <= 256 (got %d)", a.m);
}

int launch_backward(const BwdArgs &a, void *ws, cudaStream_t st)
{
    switch (padded_mp(a.m)) {
        case 32: return launch_backward_mp<32>(a, ws, st);
        case 64: return launch_backward_mp<64>(a, ws, st);
        case 128: return launch_backward_mp<128>(a, ws, st);
        case 256: return launch_backward_mp<256>(a, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "FP32 adjoint kernel supports m <= 256 (got %d)", a.m);
}

size_t backward_ws_bytes(int m, int N, int T, int K)
{
    switch (padded_mp(m)) {
        case 32: return backward_ws_mp<32>(N, T, K);
        case 64: return backward_ws_mp<64>(N, T, K);
        case 128: return backward_ws_mp<128>(N, T, K);
        case 256: return backward_ws_mp<256>(N, T, K);
    }
    return 0;
}

// The objective for wide dictionaries (256 < m <= 1024); narrower ones run on
// the tensor cores (tc_gemm.cu).
int launch_objective(const ObjArgs &a, cudaStream_t st)
{
    if (a.m <= 1024) {
        constexpr int NB = 32;
        const int lda = ((a.m + 15) / 16) * 16 + 4;
        const size_t smem = sizeof(float) * ((size_t)NB * lda + Tile<256, NB>::BS_FLOATS);
        auto k = objective_wide_kernel<NB>;
        SLISTA_CUDA_TRY(allow_smem(k, smem));
        const int grid = ceil_div(a.N, NB);
        if (grid == 0) return SLISTA_OK;
        k<<<grid, NT, smem, st>>>(a.B, a.C, a.xsq, a.Z, a.m, a.N, lda, a.lam, a.F, a.gap);
        return check_launch("objective_wide_kernel");
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "objective kernel supports m <= 1024 (got %d)", a.m);
}

}  // namespace simt
}  // namespace slista
