// Oracle-ISTA (Algorithm 1, Section 3) on the CUDA cores.
//
// One CTA owns NB samples for all T layers (state z and g = c - B z in
// registers, as in the forward kernel).  Per layer t, with S = supp(z^(t)):
//
//   (star)  The candidate y = ST(z + g / L_S, lam / L_S) has y_j = 0 for
//           every j outside S iff |g_j| <= lam there (z_j = 0 off S, so both
//           the argument and the threshold scale with 1 / L_S).  Condition
//           (star) is therefore decided first, without L_S.
//   L_S     Only samples whose step is accepted need L_S = lambda_max(B_SS)
//           (Eq. spca); it is recomputed only when S differs from the support
//           it was last computed for (L_empty = L, |S| = 1 gives B_jj).  One
//           warp gathers B_SS into shared memory and runs Lanczos with a Sturm
//           multisection on the Lanczos tridiagonal (eig.cuh); larger
//           supports are gathered by the whole block into a shared buffer.
//   step    z^(t+1) = ST(z + a g, a lam) with a = 1/L_S if (star) holds,
//           else a = 1/L (the ISTA fallback of Algorithm 1);
//   update  g <- g + (z^(t) - z^(t+1)) B, as in the forward kernel.
// The result is Algorithm 1 exactly (up to rounding); only the order in
// which L_S and (star) are evaluated differs from the listing.
#include "common.cuh"
#include "eig.cuh"
#include "kernels.h"
#include "simt.cuh"

namespace slista {
namespace simt {

namespace {

constexpr int KMAX = 64;  // largest |S| solved by one warp in its own buffer

constexpr int JM = eig::LANCZOS_JMAX;

template <int MP>
struct WarpEig {
    static constexpr int LDA = eig::odd_ld(KMAX);
    float A[KMAX * LDA];
    float q[KMAX], qp[KMAX], al[JM], be[JM], e2[JM];
    int idx[MP];
};

// Largest k whose k x odd_ld(k) matrix, three k-vectors, the Lanczos scratch
// and MP indices fit in the eight warps' buffers together.
template <int MP>
__host__ __device__ constexpr int kbig()
{
    constexpr int words = (int)(sizeof(WarpEig<MP>) / 4) * (NT / 32);
    int k = MP;
    while (k > KMAX && k * eig::odd_ld(k) + 3 * k + 3 * JM + MP > words) --k;
    return k;
}

template <int MP, int NB>
struct OistaSmem {
    static constexpr int WP = MP / 32;
    static constexpr size_t tile_bytes = sizeof(float) * (size_t)Tile<MP, NB>::SMEM_FLOATS;
    static constexpr size_t eig_bytes = sizeof(WarpEig<MP>) * (NT / 32);
    static constexpr size_t words_bytes = sizeof(uint32_t) * 2 * NB * WP;
    static constexpr size_t misc_bytes = sizeof(double) * NB + sizeof(int) * (3 * NB + 8);
    static constexpr size_t total = tile_bytes + eig_bytes + words_bytes + misc_bytes;
    static_assert(total <= 227 * 1024, "OISTA shared memory exceeds the per-CTA limit");
};

// Gathers B_SS (k x k, indices idx) into A with leading dimension lda.
// Returns whether B_SS has a non-zero off-diagonal entry (group-uniform).
template <class G>
__device__ bool gather_bss(const float *__restrict__ B, int m, const int *idx, int k, float *A, int lda)
{
    const int kk = k * k;
    bool off = false;
    int e = G::rank();
    for (; e + 3 * G::size < kk; e += 4 * G::size) {
        float x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = e + u * G::size;
            x[u] = __ldg(B + (size_t)idx[q / k] * m + idx[q % k]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = e + u * G::size;
            const int a = q / k, b = q % k;
            A[a * lda + b] = x[u];
            off |= (a != b) && (x[u] != 0.0f);
        }
    }
    for (; e < kk; e += G::size) {
        const int a = e / k, b = e % k;
        const float x = __ldg(B + (size_t)idx[a] * m + idx[b]);
        A[a * lda + b] = x;
        off |= (a != b) && (x != 0.0f);
    }
    G::sync();
    return G::any(off);
}

// Largest diagonal entry of A (the largest eigenvalue when A is diagonal,
// e.g. B_SS of an orthogonal D_S, where it is exact).
__device__ inline float max_diag(const float *A, int lda, int k)
{
    float v = A[0];
    for (int a = 1; a < k; ++a) v = fmaxf(v, A[a * lda + a]);
    return v;
}

// Fallback for supports too large for shared memory: power iteration on B_SS
// read from global memory, FP32 products and FP64 Rayleigh quotients; keeps
// the largest quotient seen and stops after 400 iterations without progress.
template <int MP>
__device__ double power_iteration_global(const float *__restrict__ B, int m, const int *idx, int k, float *v)
{
    const int lane = threadIdx.x & 31;
    for (int a = lane; a < k; a += 32) v[a] = eig::start_vector(a);
    __syncwarp();
    double best = 0.0;
    int stall = 0;
#pragma unroll 1
    for (int it = 0; it < 20000 && stall < 400; ++it) {
        float wl[MP / 32];
        double vw = 0.0, ww = 0.0, vv = 0.0;
#pragma unroll
        for (int rr = 0; rr < MP / 32; ++rr) {
            const int a = lane + 32 * rr;
            float s = 0.0f;
            if (a < k) {
                const float *row = B + (size_t)idx[a] * m;
                for (int b = 0; b < k; ++b) s = fmaf(__ldg(row + idx[b]), v[b], s);
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
        const double rq = vw / vv;
        if (rq > best * (1.0 + 1e-9)) {
            best = rq;
            stall = 0;
        } else {
            ++stall;
        }
        const float inv = (float)(1.0 / sqrt(ww));
        __syncwarp();
#pragma unroll
        for (int rr = 0; rr < MP / 32; ++rr) {
            const int a = lane + 32 * rr;
            if (a < k) v[a] = wl[rr] * inv;
        }
        __syncwarp();
    }
    return best;
}

// Index list of the support words of one row (by one warp); returns |S|.
__device__ int support_indices(const uint32_t *words, int WP, int *idx)
{
    const int lane = threadIdx.x & 31;
    int k = 0;
    for (int w = 0; w < WP; ++w) {
        const uint32_t bits = words[w];
        const bool has = (bits >> lane) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, has);
        if (has) idx[k + __popc(bal & ((1u << lane) - 1u))] = w * 32 + lane;
        k += __popc(bal);
    }
    __syncwarp();
    return k;
}

template <int MP, int NB>
__global__ void __launch_bounds__(NT) oista_kernel(
    const float *__restrict__ B, const float *__restrict__ C, int m, int N, float lam,
    const double *__restrict__ Lp, int T, float *__restrict__ Z, double *__restrict__ LS_out,
    int *__restrict__ accepted)
{
    using TL = Tile<MP, NB>;
    using SM = OistaSmem<MP, NB>;
    constexpr int WP = SM::WP;
    constexpr int KBIG = kbig<MP>();
    extern __shared__ float4 smem4[];
    char *base = reinterpret_cast<char *>(smem4);
    float *A_s = reinterpret_cast<float *>(base);
    float *B_s = A_s + TL::A_FLOATS;
    WarpEig<MP> *eigw = reinterpret_cast<WarpEig<MP> *>(base + SM::tile_bytes);
    float *big = reinterpret_cast<float *>(eigw);  // all warps' buffers, for one large support
    uint32_t *Scur = reinterpret_cast<uint32_t *>(base + SM::tile_bytes + SM::eig_bytes);
    uint32_t *Sprev = Scur + NB * WP;
    double *LSrow = reinterpret_cast<double *>(Sprev + NB * WP);
    int *flag = reinterpret_cast<int *>(LSrow + NB);  // 1: condition (star) fails
    int *valid = flag + NB;                           // LSrow[r] holds L_{Sprev[r]}
    int *deferred = valid + NB;                       // rows whose support is too large for a warp
    int *ctr = deferred + NB;                         // [0] queue, [1] accepted, [2] #deferred, [4] |S|
    __shared__ float redf[NT / 32];
    __shared__ int redi[NT / 32];

    const Idx<TL> ix;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.x * NB;
    const double L = __ldg(Lp);
    const float aL = (float)(1.0 / L);

    float g[TL::RM][TL::RN], z[TL::RM][TL::RN], d[TL::RM][TL::RN];
    load_rows<TL>(g, C, row0, N, m, m);
#pragma unroll
    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) z[i][j] = 0.0f;
    for (int r = threadIdx.x; r < NB; r += NT) {
        valid[r] = 0;
        flag[r] = 0;
        LSrow[r] = L;
    }
    if (threadIdx.x < 8) ctr[threadIdx.x] = 0;
    __syncthreads();

#pragma unroll 1
    for (int t = 0; t < T; ++t) {
        const bool want_ls_out = (LS_out != nullptr) && (t == T - 1);
        // 1. S = supp(z^(t)) and condition (star): |g_j| <= lam wherever z_j = 0
        store_support_words<TL>(Scur, z, 0, NB, WP);
#pragma unroll
        for (int i = 0; i < TL::RM; ++i) {
            bool bad = false;
#pragma unroll
            for (int j = 0; j < TL::RN; ++j) bad |= (z[i][j] == 0.0f) && (fabsf(g[i][j]) > lam);
            if (bad) flag[ix.row(i)] = 1;
        }
        __syncthreads();
        // 2. L_S for accepted samples whose support changed (dynamic row queue)
#pragma unroll 1
        for (;;) {
            int lr = 0;
            if (lane == 0) lr = atomicAdd(&ctr[0], 1);
            lr = __shfl_sync(0xffffffffu, lr, 0);
            if (lr >= NB) break;
            if (row0 + lr >= N) continue;
            if (flag[lr] && !want_ls_out) continue;
            bool changed = valid[lr] == 0;
            for (int w = 0; w < WP; ++w) changed |= (Scur[lr * WP + w] != Sprev[lr * WP + w]);
            if (!changed) continue;
            WarpEig<MP> &we = eigw[warp];
            const int k = support_indices(Scur + lr * WP, WP, we.idx);
            double LS;
            if (k == 0) {
                LS = L;
            } else if (k == 1) {
                LS = (double)__ldg(B + (size_t)we.idx[0] * m + we.idx[0]);
            } else if (k <= KMAX) {
                const int lda = eig::odd_ld(k);
                if (gather_bss<eig::WarpGroup>(B, m, we.idx, k, we.A, lda))
                    LS = eig::lanczos_max_eig_warp<(KMAX + 31) / 32>(we.A, lda, k, we.q, we.qp, we.al, we.be,
                                                                     we.e2);
                else
                    LS = (double)max_diag(we.A, lda, k);
            } else {
                if (lane == 0) deferred[atomicAdd(&ctr[2], 1)] = lr;
                continue;
            }
            __syncwarp();
            if (lane == 0) {
                LSrow[lr] = LS;
                valid[lr] = 1;
            }
            for (int w = lane; w < WP; w += 32) Sprev[lr * WP + w] = Scur[lr * WP + w];
        }
        __syncthreads();
        // 3. large supports: the whole block on every warp's buffer, one at a time
        const int ndef = ctr[2];
#pragma unroll 1
        for (int q = 0; q < ndef; ++q) {
            const int lr = deferred[q];
            int *idx = reinterpret_cast<int *>(big);
            int *kp = ctr + 4;
            if (warp == 0) {
                const int k = support_indices(Scur + lr * WP, WP, idx);
                if (lane == 0) *kp = k;
            }
            __syncthreads();
            const int k = *kp;
            double LS;
            if (k <= KBIG) {
                const int lda = eig::odd_ld(k);
                float *A = big + MP;
                float *vv = A + k * lda;
                const bool off = gather_bss<eig::CtaGroup<NT>>(B, m, idx, k, A, lda);
                LS = off ? eig::lanczos_max_eig_cta<NT>(A, lda, k, vv, vv + k, vv + 2 * k, vv + 3 * k,
                                                        vv + 3 * k + JM, vv + 3 * k + 2 * JM, redf, redi)
                         : (double)max_diag(A, lda, k);
            } else {
                LS = 0.0;
                if (warp == 0) LS = power_iteration_global<MP>(B, m, idx, k, big + MP);
            }
            if (threadIdx.x == 0) {
                LSrow[lr] = LS;
                valid[lr] = 1;
            }
            for (int w = threadIdx.x; w < WP; w += NT) Sprev[lr * WP + w] = Scur[lr * WP + w];
            __syncthreads();
        }
        // 4. the step: 1/L_S if (star) holds, else the ISTA step 1/L
#pragma unroll
        for (int i = 0; i < TL::RM; ++i) {
            const bool ok = flag[ix.row(i)] == 0;
            const float a = ok ? (float)(1.0 / LSrow[ix.row(i)]) : aL;
            const float thr = a * lam;
#pragma unroll
            for (int j = 0; j < TL::RN; ++j) {
                const float zn = soft_threshold(fmaf(a, g[i][j], z[i][j]), thr);
                d[i][j] = z[i][j] - zn;
                z[i][j] = zn;
            }
            if (ix.tx == 0 && row0 + ix.row(i) < N && ok) atomicAdd(&ctr[1], 1);
        }
        if (want_ls_out)
            for (int r = threadIdx.x; r < NB; r += NT)
                if (row0 + r < N) LS_out[row0 + r] = LSrow[r];
        store_tile<TL>(A_s, d);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (accepted) atomicAdd(accepted + t, ctr[1]);
            ctr[0] = ctr[1] = ctr[2] = 0;
        }
        for (int r = threadIdx.x; r < NB; r += NT) flag[r] = 0;
        if (t == T - 1) break;
        // 5. g <- g + (z^(t) - z^(t+1)) B  (gemm_acc starts with a barrier)
        gemm_acc<TL>(g, A_s, TL::LDA, B, m, m, m, B_s);
    }
    store_rows<TL>(Z, z, row0, N, m, m);
}

template <int MP>
int launch_oista_mp(const OistaArgs &a, cudaStream_t st)
{
    constexpr int NB = 32;
    const size_t smem = OistaSmem<MP, NB>::total;
    auto k = oista_kernel<MP, NB>;
    SLISTA_CUDA_TRY(allow_smem(k, smem));
    if (a.accepted && a.T > 0) SLISTA_CUDA_TRY(cudaMemsetAsync(a.accepted, 0, sizeof(int) * a.T, st));
    const int grid = ceil_div(a.N, NB);
    if (grid == 0) return SLISTA_OK;
    k<<<grid, NT, smem, st>>>(a.B, a.C, a.m, a.N, a.lam, a.L, a.T, a.Z, a.LS, a.accepted);
    return check_launch("oista_kernel");
}

}  // namespace

int launch_oista(const OistaArgs &a, void *, cudaStream_t st)
{
    switch (padded_mp(a.m)) {
        case 32: return launch_oista_mp<32>(a, st);
        case 64: return launch_oista_mp<64>(a, st);
        case 128: return launch_oista_mp<128>(a, st);
        case 256: return launch_oista_mp<256>(a, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "OISTA kernel supports m <= 256 (got %d)", a.m);
}

size_t oista_ws_bytes(int, int) { return 0; }

}  // namespace simt
}  // namespace slista
