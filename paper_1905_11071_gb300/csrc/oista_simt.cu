// Oracle-ISTA (Algorithm 1, Section 3).
//
// Per layer t, with S = supp(z^(t)):
//   (star)  The candidate y = ST(z + g / L_S, lam / L_S) has y_j = 0 for every
//           j outside S iff |g_j| <= lam there (z_j = 0 off S, so argument and
//           threshold both scale with 1 / L_S): condition (star) is decided
//           without L_S.
//   L_S     Only samples whose step is accepted need L_S = lambda_max(B_SS)
//           (Eq. spca), and only when S differs from the support it was last
//           computed for (L_empty = L; |S| = 1 gives B_jj).
//   step    z^(t+1) = ST(z + a g, a lam), a = 1/L_S if (star) holds, else 1/L
//           (the ISTA fallback); then g <- g + (z^(t) - z^(t+1)) B.
// The result is Algorithm 1 (up to rounding); only the order in which L_S and
// (star) are evaluated differs from the listing.
//
// The layers run as two kernels each, with the per-sample state (z, g, the
// support words, the cached L_S) in the workspace:
//   oista_solve_kernel  every warp of the grid takes samples from the layer's
//                       list of required L_S and computes them by Lanczos on
//                       B_SS gathered into its shared buffer (|S| <= 64), or on
//                       the n x n matrix D_S D_S^T (same non-zero spectrum) for
//                       larger supports when D is given;
//   oista_step_kernel   the layer for a tile of samples (FP32, the tile engine
//                       of the forward kernel), fused with the next layer's
//                       preparation: S, condition (star) and the list of
//                       samples that need a new L_S.
// Splitting the eigen-solves from the layer balances them over the whole GPU.
#include "common.cuh"
#include "eig.cuh"
#include "oista_solvers.cuh"
#include "kernels.h"
#include "simt.cuh"

namespace slista {
namespace simt {

namespace {

constexpr int STEP_NB = 32;

// Per-sample state of the layer loop, carved out of the workspace.
struct OistaWs {
    double *LSv;              // N: cached L_S
    float *Zs, *Gs;           // N x m each: z^(t), g^(t) = c - B z^(t)
    uint32_t *Scur, *Sprev;   // N x W: supp(z^(t)), support of the cached L_S
    int *flag;                // N: 1 if condition (star) fails at the current layer
    int *valid;               // N: LSv holds L_{Sprev}
    int *list;                // 2 x NCLS x N: samples needing L_S, [layer parity][class]
    int *counter;             // 2 x NCLS: list lengths, same indexing
    int *qpos;                // T x NCLS: queue positions of the solve kernels
    float *Dt;                // m x n: D transposed (columns of D contiguous), when D is given
    uint8_t *tiles;           // split B for the tensor-core layers (after Dt)
    int N, W;

    // Every array starts on a 256-byte boundary (the layer kernels read rows
    // of Zs, Gs and Dt with 16-byte vector loads).
    static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
    static size_t bytes(int m, int N, int T)
    {
        const size_t W = (size_t)(m + 31) / 32;
        return a256(sizeof(double) * (size_t)N) + 2 * a256(sizeof(float) * (size_t)N * m) +
               2 * a256(sizeof(uint32_t) * N * W) + 2 * a256(sizeof(int) * (size_t)N) +
               a256(sizeof(int) * 2 * NCLS * (size_t)N) + a256(sizeof(int) * (2 * NCLS + NCLS * (size_t)T)) +
               a256(sizeof(float) * (size_t)m * 256) + 256;
    }
    static OistaWs carve(void *ws, int m, int N, int T)
    {
        const size_t W = (size_t)(m + 31) / 32;
        char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255);
        auto take = [&p](size_t b) {
            char *q = p;
            p += a256(b);
            return q;
        };
        OistaWs o;
        o.LSv = reinterpret_cast<double *>(take(sizeof(double) * (size_t)N));
        o.Zs = reinterpret_cast<float *>(take(sizeof(float) * (size_t)N * m));
        o.Gs = reinterpret_cast<float *>(take(sizeof(float) * (size_t)N * m));
        o.Scur = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)N * W));
        o.Sprev = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (size_t)N * W));
        o.flag = reinterpret_cast<int *>(take(sizeof(int) * (size_t)N));
        o.valid = reinterpret_cast<int *>(take(sizeof(int) * (size_t)N));
        o.list = reinterpret_cast<int *>(take(sizeof(int) * 2 * NCLS * (size_t)N));
        // counter and qpos adjacent: one memset clears both at the start of a call
        o.counter = reinterpret_cast<int *>(take(sizeof(int) * (2 * NCLS + NCLS * (size_t)T)));
        o.qpos = o.counter + 2 * NCLS;
        o.Dt = reinterpret_cast<float *>(take(sizeof(float) * (size_t)m * 256));
        o.tiles = reinterpret_cast<uint8_t *>(p);
        o.N = N;
        o.W = (int)W;
        return o;
    }
};

// Takes the next sample of list class cls of layer t (one warp); -1 when empty.
// The queue position is read before it is incremented, so that the warps of
// the grid stop taking atomics on the three queue counters once a list is
// exhausted (a stale read only costs one atomic, whose result decides).
__device__ __forceinline__ int next_sample(const OistaWs &ws, int t, int cls)
{
    const int lane = threadIdx.x & 31;
    const int par = t & 1;
    int q = 0, n = 0;
    if (lane == 0) {
        n = ws.counter[NCLS * par + cls];
        int *qp = ws.qpos + NCLS * t + cls;
        q = *reinterpret_cast<volatile int *>(qp) >= n ? n : atomicAdd(qp, 1);
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    n = __shfl_sync(0xffffffffu, n, 0);
    if (q >= n) return -1;
    return ws.list[(size_t)(NCLS * par + cls) * ws.N + q];
}

__device__ __forceinline__ void publish(const OistaWs &ws, int i, const uint32_t *words, double LS)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        ws.LSv[i] = LS;
        ws.valid[i] = 1;
    }
    for (int w = lane; w < ws.W; w += 32) ws.Sprev[(size_t)i * ws.W + w] = words[w];
    __syncwarp();
}

// ---------------------------------------------------------------------------
// L_S for the samples listed for layer t.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__((A_WARPS + S_WARPS) * 32, 1) oista_solve_kernel(
    const float *__restrict__ B, bool have_D, int n, int m, const double *__restrict__ Lp, OistaWs ws, int t)
{
    extern __shared__ float4 smem4[];
    const int warp = threadIdx.x >> 5;
    const int par = t & 1;
    // launched as a programmatic dependent of the previous layer's kernel:
    // nothing of it is read or written before this
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (blockIdx.x == 0 && threadIdx.x < NCLS) ws.counter[NCLS * (par ^ 1) + threadIdx.x] = 0;  // next layer's lists
    const double L = __ldg(Lp);
    if (warp >= A_WARPS) {
        // small supports, matrix in registers
        WarpEigS &we = reinterpret_cast<WarpEigS *>(reinterpret_cast<WarpEig *>(smem4) + A_WARPS)[warp - A_WARPS];
#pragma unroll 1
        for (;;) {
            const int i = next_sample(ws, t, 2);
            if (i < 0) break;
            const uint32_t *words = ws.Scur + (size_t)i * ws.W;
            const int k = support_indices(words, ws.W, we.idx);
            const double LS = k == 0 ? L : k == 1 ? (double)__ldg(B + (size_t)we.idx[0] * m + we.idx[0])
                                                  : solve_small(B, m, we.idx, k, we.al, we.be, we.e2);
            publish(ws, i, words, LS);
        }
        return;
    }
    WarpEig &we = reinterpret_cast<WarpEig *>(smem4)[warp];
#pragma unroll 1
    for (int cls = 0; cls < NCLS; ++cls) {  // large supports first: they set the kernel's tail
#pragma unroll 1
        for (;;) {
            const int i = next_sample(ws, t, cls);
            if (i < 0) break;
            const uint32_t *words = ws.Scur + (size_t)i * ws.W;
            const int k = support_indices(words, ws.W, we.idx);
            double LS;
            if (k == 0) {
                LS = L;
            } else if (k == 1) {
                LS = (double)__ldg(B + (size_t)we.idx[0] * m + we.idx[0]);
            } else if (k <= SMALL_K) {
                LS = solve_small(B, m, we.idx, k, we.al, we.be, we.e2);
            } else if (k <= KMAX) {
                const int lda = eig::vec_ld(k);
                if (gather_bss(B, m, we.idx, k, we.A, lda))
                    LS = eig::lanczos_max_eig_warp<KMAX / 32>(we.A, lda, k, we.q, we.qp, we.al, we.be, we.e2);
                else
                    LS = (double)max_diag(we.A, lda, k);
            } else if (have_D && n <= KMAX) {
                const int lda = eig::vec_ld(n);
                gram_ds(ws.Dt, n, we.idx, k, we.A, lda, we.col);
                LS = eig::lanczos_max_eig_warp<KMAX / 32>(we.A, lda, n, we.q, we.qp, we.al, we.be, we.e2);
            } else {
                LS = lanczos_global(B, m, we.idx, k, we);
            }
            __syncwarp();
            publish(ws, i, words, LS);
        }
    }
}

// Dt = D^T (m x n).
__global__ void transpose_kernel(const float *__restrict__ D, int n, int m, float *__restrict__ Dt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * m) {
        const int i = e / m, j = e % m;
        Dt[(size_t)j * n + i] = __ldg(D + e);
    }
}

// ---------------------------------------------------------------------------
// Shared preparation of layer t+1 for one tile: S, condition (star), the list.
// ---------------------------------------------------------------------------
template <class TL>
__device__ void prepare_next(const float (&z)[TL::RM][TL::RN], const float (&g)[TL::RM][TL::RN], float lam,
                             int row0, int N, OistaWs ws, int next, bool want_ls, uint32_t *Sw, int *rowflag)
{
    const Idx<TL> ix;
    for (int r = threadIdx.x; r < TL::NB; r += NT) rowflag[r] = 0;
    __syncthreads();
    store_support_words<TL>(Sw, z, 0, TL::NB, ws.W);
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        bool bad = false;
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) bad |= (z[i][j] == 0.0f) && (fabsf(g[i][j]) > lam);
        if (bad) rowflag[ix.row(i)] = 1;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < TL::NB; r += NT) {
        const int gr = row0 + r;
        if (gr >= N) continue;
        const int f = rowflag[r];
        ws.flag[gr] = f;
        bool changed = ws.valid[gr] == 0;
        for (int w = 0; w < ws.W; ++w) {
            const uint32_t s = Sw[r * ws.W + w];
            ws.Scur[(size_t)gr * ws.W + w] = s;
            changed |= s != ws.Sprev[(size_t)gr * ws.W + w];
        }
        if ((f == 0 || want_ls) && changed) {
            int k = 0;
            for (int w = 0; w < ws.W; ++w) k += __popc(Sw[r * ws.W + w]);
            const int cls = (k > KMAX) ? 0 : (k > SMALL_K) ? 1 : 2;
            const int li = NCLS * (next & 1) + cls;
            const int pos = atomicAdd(ws.counter + li, 1);
            ws.list[(size_t)li * ws.N + pos] = gr;
        }
    }
}

template <int MP>
struct StepSmem {
    using TL = Tile<MP, STEP_NB>;
    static constexpr size_t bytes =
        sizeof(float) * TL::SMEM_FLOATS + sizeof(uint32_t) * STEP_NB * (MP / 32) + sizeof(int) * (STEP_NB + 4);
};

// z^(0) = 0, g^(0) = c, S = empty (L_S = L), and condition (star) for layer 0.
template <int MP>
__global__ void __launch_bounds__(NT) oista_init_kernel(const float *__restrict__ C, int m, int N, float lam,
                                                        const double *__restrict__ Lp, OistaWs ws, bool want_ls)
{
    using TL = Tile<MP, STEP_NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    uint32_t *Sw = reinterpret_cast<uint32_t *>(A_s + TL::SMEM_FLOATS);
    int *rowflag = reinterpret_cast<int *>(Sw + STEP_NB * (MP / 32));
    const int row0 = blockIdx.x * STEP_NB;
    float g[TL::RM][TL::RN], z[TL::RM][TL::RN];
    load_rows<TL>(g, C, row0, N, m, m);
#pragma unroll
    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) z[i][j] = 0.0f;
    store_rows<TL>(ws.Gs, g, row0, N, m, m);
    store_rows<TL>(ws.Zs, z, row0, N, m, m);
    const double L = __ldg(Lp);
    for (int r = threadIdx.x; r < STEP_NB; r += NT) {
        const int gr = row0 + r;
        if (gr >= N) continue;
        ws.LSv[gr] = L;  // L_empty = L
        ws.valid[gr] = 1;
        for (int w = 0; w < ws.W; ++w) ws.Sprev[(size_t)gr * ws.W + w] = 0u;
    }
    __syncthreads();
    prepare_next<TL>(z, g, lam, row0, N, ws, 0, want_ls, Sw, rowflag);
}

// Layer t for one tile, then the preparation of layer t+1.
template <int MP>
__global__ void __launch_bounds__(NT) oista_step_kernel(const float *__restrict__ B, int m, int N, float lam,
                                                        const double *__restrict__ Lp, OistaWs ws, int t, int T,
                                                        bool want_ls_next, float *__restrict__ Z,
                                                        double *__restrict__ LS_out, int *__restrict__ accepted)
{
    using TL = Tile<MP, STEP_NB>;
    extern __shared__ float4 smem4[];
    float *A_s = reinterpret_cast<float *>(smem4);
    float *B_s = A_s + TL::A_FLOATS;
    uint32_t *Sw = reinterpret_cast<uint32_t *>(A_s + TL::SMEM_FLOATS);
    int *rowflag = reinterpret_cast<int *>(Sw + STEP_NB * (MP / 32));
    int *cnt = rowflag + STEP_NB;
    const Idx<TL> ix;
    const int row0 = blockIdx.x * STEP_NB;
    if (threadIdx.x == 0) *cnt = 0;
    float g[TL::RM][TL::RN], z[TL::RM][TL::RN], d[TL::RM][TL::RN];
    load_rows<TL>(z, ws.Zs, row0, N, m, m);
    load_rows<TL>(g, ws.Gs, row0, N, m, m);
    const float aL = (float)(1.0 / __ldg(Lp));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        const int r = row0 + ix.row(i);
        const bool live = r < N;
        const bool ok = live && ws.flag[r] == 0;
        const float a = ok ? (float)(1.0 / ws.LSv[r]) : aL;
        const float thr = __fmul_rn(a, lam);
#pragma unroll
        for (int j = 0; j < TL::RN; ++j) {
            const float zn = soft_threshold(fmaf(a, g[i][j], z[i][j]), thr);
            d[i][j] = z[i][j] - zn;
            z[i][j] = zn;
        }
        if (ix.tx == 0 && ok) atomicAdd(cnt, 1);
    }
    if (t == T - 1) {
        store_rows<TL>(Z, z, row0, N, m, m);
        if (LS_out)
            for (int r = threadIdx.x; r < STEP_NB; r += NT)
                if (row0 + r < N) LS_out[row0 + r] = ws.LSv[row0 + r];
    } else {
        store_tile<TL>(A_s, d);
        gemm_acc<TL>(g, A_s, TL::LDA, B, m, m, m, B_s);  // g <- g + (z^(t) - z^(t+1)) B
        store_rows<TL>(ws.Zs, z, row0, N, m, m);
        store_rows<TL>(ws.Gs, g, row0, N, m, m);
        prepare_next<TL>(z, g, lam, row0, N, ws, t + 1, want_ls_next, Sw, rowflag);
    }
    __syncthreads();
    if (threadIdx.x == 0 && accepted && *cnt) atomicAdd(accepted + t, *cnt);
}

template <int MP>
int launch_oista_mp(const OistaArgs &a, void *wsp, cudaStream_t st)
{
    const OistaWs ws = OistaWs::carve(wsp, a.m, a.N, a.T);
    if (a.accepted && a.T > 0) SLISTA_CUDA_TRY(cudaMemsetAsync(a.accepted, 0, sizeof(int) * a.T, st));
    if (a.N == 0) return SLISTA_OK;
    if (a.T == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(float) * (size_t)a.N * a.m, st));
        return SLISTA_OK;
    }
    SLISTA_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, sizeof(int) * (2 * NCLS + NCLS * (size_t)a.T), st));  // counters, qpos
    const bool have_D = a.D != nullptr && a.n >= 1 && a.n <= KMAX;
    if (have_D) {
        transpose_kernel<<<ceil_div((long long)a.n * a.m, 256), 256, 0, st>>>(a.D, a.n, a.m, ws.Dt);
        int rc0 = check_launch("transpose_kernel");
        if (rc0) return rc0;
    }
    const size_t step_smem = StepSmem<MP>::bytes;
    const size_t solve_smem = sizeof(WarpEig) * A_WARPS + sizeof(WarpEigS) * S_WARPS;
    auto kinit = oista_init_kernel<MP>;
    auto kstep = oista_step_kernel<MP>;
    SLISTA_CUDA_TRY(allow_smem(kinit, step_smem));
    SLISTA_CUDA_TRY(allow_smem(kstep, step_smem));
    SLISTA_CUDA_TRY(allow_smem(oista_solve_kernel, solve_smem));
    const bool tc = a.prec == SLISTA_PREC_BF16 || a.prec == SLISTA_PREC_BF16X3;
    if (tc) {
        int rc1 = tcw::oista_split(a.B, a.m, ws.tiles, st);
        if (rc1) return rc1;
    }
    const int grid = ceil_div(a.N, STEP_NB);
    const bool want_ls = a.LS != nullptr;
    kinit<<<grid, NT, step_smem, st>>>(a.C, a.m, a.N, a.lam, a.L, ws, want_ls && a.T == 1);
    int rc = check_launch("oista_init_kernel");
    if (rc) return rc;
    const int solve_grid = num_sms();
    for (int t = 0; t < a.T; ++t) {
        if (tc) {  // may start while the previous layer's kernel finishes (griddepcontrol.wait inside)
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(solve_grid);
            cfg.blockDim = dim3((A_WARPS + S_WARPS) * 32);
            cfg.dynamicSmemBytes = solve_smem;
            cfg.stream = st;
            cudaLaunchAttribute attr{};
            attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr.val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            SLISTA_CUDA_TRY(cudaLaunchKernelEx(&cfg, oista_solve_kernel, a.B, have_D, a.n, a.m, a.L, ws, t));
        } else {
            oista_solve_kernel<<<solve_grid, (A_WARPS + S_WARPS) * 32, solve_smem, st>>>(a.B, have_D, a.n, a.m, a.L,
                                                                                           ws, t);
        }
        rc = check_launch("oista_solve_kernel");
        if (rc) return rc;
        if (tc) {
            tcw::OistaStep o{};
            o.tiles = ws.tiles;
            o.C = a.C;
            o.Zs = ws.Zs;
            o.Gs = ws.Gs;
            o.Zfinal = a.Z;
            o.L = a.L;
            o.LSv = ws.LSv;
            o.flag = ws.flag;
            o.Scur = ws.Scur;
            o.Sprev = ws.Sprev;
            o.valid = ws.valid;
            o.list = ws.list + (size_t)NCLS * ((t + 1) & 1) * a.N;
            o.counter = ws.counter + NCLS * ((t + 1) & 1);
            o.listN = a.N;
            o.accepted = a.accepted ? a.accepted + t : nullptr;
            o.LS_out = a.LS;
            o.m = a.m;
            o.N = a.N;
            o.t = t;
            o.T = a.T;
            o.want_ls = want_ls && t + 2 == a.T;
            o.lam = a.lam;
            rc = tcw::launch_oista_step(o, a.prec, st);
        } else {
            kstep<<<grid, NT, step_smem, st>>>(a.B, a.m, a.N, a.lam, a.L, ws, t, a.T, want_ls && t + 2 == a.T, a.Z,
                                               a.LS, a.accepted);
            rc = check_launch("oista_step_kernel");
        }
        if (rc) return rc;
    }
    return SLISTA_OK;
}

// Files sample i of a standalone L_S call into the solve kernel's list of its
// class (|S| > KMAX, SMALL_K < |S| <= KMAX, |S| <= SMALL_K), copying its
// support words with the bits of codes >= m cleared (the solvers index B by
// them).
__global__ void __launch_bounds__(256) support_classify_kernel(const uint32_t *__restrict__ S, int m, OistaWs ws)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ws.N) return;
    int k = 0;
    for (int w = 0; w < ws.W; ++w) {
        const int rem = m - 32 * w;
        const uint32_t keep = rem >= 32 ? 0xffffffffu : (1u << rem) - 1u;
        const uint32_t bits = __ldg(S + (size_t)i * ws.W + w) & keep;
        ws.Scur[(size_t)i * ws.W + w] = bits;
        k += __popc(bits);
    }
    const int cls = k > KMAX ? 0 : k > SMALL_K ? 1 : 2;
    ws.list[(size_t)cls * ws.N + atomicAdd(ws.counter + cls, 1)] = i;
}

// Workspace of a standalone L_S call: copied supports, the solve kernel's
// scratch (published supports, flags, class lists, counters and queue
// positions) and D^T, each on a 256-byte boundary.
size_t support_ls_layout(int m, int N, void *wsp, OistaWs *out)
{
    const size_t W = (size_t)(m + 31) / 32;
    const size_t sizes[7] = {sizeof(uint32_t) * N * W, sizeof(uint32_t) * N * W, sizeof(int) * (size_t)N,
                             sizeof(int) * 2 * NCLS * (size_t)N, sizeof(int) * 3 * NCLS,
                             sizeof(float) * (size_t)m * KMAX, 0};
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(wsp) + 255) & ~(uintptr_t)255);
    char *ptr[7];
    size_t off = 0;
    for (int s = 0; s < 7; ++s) {
        ptr[s] = base + off;
        off += OistaWs::a256(sizes[s]);
    }
    if (out) {
        OistaWs &o = *out;
        o = OistaWs{};
        o.Scur = reinterpret_cast<uint32_t *>(ptr[0]);
        o.Sprev = reinterpret_cast<uint32_t *>(ptr[1]);
        o.valid = reinterpret_cast<int *>(ptr[2]);
        o.list = reinterpret_cast<int *>(ptr[3]);
        o.counter = reinterpret_cast<int *>(ptr[4]);  // 2 x NCLS counters, then NCLS queue positions
        o.qpos = o.counter + 2 * NCLS;
        o.Dt = reinterpret_cast<float *>(ptr[5]);
        o.N = N;
        o.W = (int)W;
    }
    return off + 256;
}

}  // namespace

size_t support_ls_ws_bytes(int m, int N) { return support_ls_layout(m, N, nullptr, nullptr); }

int launch_support_lipschitz(const SupportLsArgs &a, void *wsp, cudaStream_t st)
{
    if (a.N == 0) return SLISTA_OK;
    OistaWs ws;
    support_ls_layout(a.m, a.N, wsp, &ws);
    ws.LSv = a.LS;
    SLISTA_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, sizeof(int) * 3 * NCLS, st));
    const bool have_D = a.D != nullptr && a.n >= 1 && a.n <= KMAX;
    if (have_D) {
        transpose_kernel<<<ceil_div((long long)a.n * a.m, 256), 256, 0, st>>>(a.D, a.n, a.m, ws.Dt);
        int rc = check_launch("transpose_kernel");
        if (rc) return rc;
    }
    support_classify_kernel<<<ceil_div(a.N, 256), 256, 0, st>>>(a.S, a.m, ws);
    int rc = check_launch("support_classify_kernel");
    if (rc) return rc;
    const size_t solve_smem = sizeof(WarpEig) * A_WARPS + sizeof(WarpEigS) * S_WARPS;
    SLISTA_CUDA_TRY(allow_smem(oista_solve_kernel, solve_smem));
    oista_solve_kernel<<<num_sms(), (A_WARPS + S_WARPS) * 32, solve_smem, st>>>(a.B, have_D, a.n, a.m, a.L, ws, 0);
    return check_launch("oista_solve_kernel");
}

int launch_oista(const OistaArgs &a, void *ws, cudaStream_t st)
{
    switch (padded_mp(a.m)) {
        case 32: return launch_oista_mp<32>(a, ws, st);
        case 64: return launch_oista_mp<64>(a, ws, st);
        case 128: return launch_oista_mp<128>(a, ws, st);
        case 256: return launch_oista_mp<256>(a, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "OISTA kernel supports m <= 256 (got %d)", a.m);
}

size_t oista_ws_bytes(int m, int N, int T, int prec)
{
    const bool tc = prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3;
    return OistaWs::bytes(m, N, T) + 64 + (tc ? tcw::oista_tiles_bytes(m) + 256 : 0);
}

}  // namespace simt
}  // namespace slista
