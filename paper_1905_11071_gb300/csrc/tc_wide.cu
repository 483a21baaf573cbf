// Tensor-core layers for wide dictionaries (256 < m <= 1024), and for
// batches of problems of any width: one launch per layer.
//
// For m > 256 neither B (m x m) nor the accumulator of a full sample row fits
// on chip, so the state (z, g = c - B z) of layer t lives in HBM and a layer
//   z' = ST(z + alpha_t g, alpha_t lam),   g' = g + (z - z') B     (Eq. pgd / Eq. steprec)
// is one GEMM-shaped launch: CTA (row tile r, column block b) computes the
// 128 x 256 block [r, b] of (z - z') B on the tensor cores and finishes its
// block of g' and z' in the epilogue.  Per K-chunk of 64 codes:
//   * all 16 warps build the A operand (z - z') of the chunk from z and g
//     (FP32 soft-threshold, split into BF16 hi / lo) straight into shared
//     memory in the K-major 128-byte-swizzled layout;
//   * thread 0 streams the chunk's B tile (hi and lo, pre-split and
//     pre-swizzled) from L2 with one bulk copy, and issues
//       BF16X3: a_hi b_hi + a_lo b_hi + a_hi b_lo      BF16: a_hi b_hi
//     as tcgen05.mma (A and B from shared memory, FP32 accumulator in tensor
//     memory), two stages deep.
// Every REFRESH layers (at the checkpoints when checkpoints are kept) the
// A operand is -z' and the epilogue adds C instead of g, so g' = c - B z' is
// rebuilt from scratch (the drift bound of the resident kernel).
// The adjoint layer has the same shape: A = h = G * mask_t, and the epilogue
// forms G' = h - alpha_t (B h) and the block's share of
// dalpha_t = <h, g^(t) - lam sign z^(t+1)>.
// Work items (problem, row tile, column block) come from a table in the
// launch parameters, so a ragged batch of problems is one launch per layer.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace slista {
namespace tcw {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int NT = 512;                          // 16 warps
constexpr int TILE_A = BM * BK * 2;              // one BF16 A chunk (16 KB)
constexpr int TILE_B = BN * BK * 2;              // one BF16 B tile (32 KB)
constexpr int TILE_PAIR = 2 * TILE_B;            // hi then lo, as stored in the workspace
constexpr int REFRESH = 8;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);
constexpr int SW = 128;       // epilogue slice: columns staged through shared memory at a time
constexpr int EPI_SMEM = 2 * BM * SW * 4;  // the z and g slices

enum Mode { FWD = 0, ADJ = 1, OIS = 2 };

template <bool SPLIT>
struct WCfg {
    static constexpr int OFF_B = SPLIT ? 2 * TILE_A : TILE_A;
    static constexpr int STAGE = OFF_B + (SPLIT ? 2 * TILE_B : TILE_B);
    static constexpr uint32_t BBYTES = SPLIT ? 2 * TILE_B : TILE_B;
    static constexpr int SMEM = (2 * STAGE > EPI_SMEM ? 2 * STAGE : EPI_SMEM) + 1024;
};

int read_and_clear_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "a wide-layer kernel's bounded wait expired (device flag %d)", h);
    }
    return SLISTA_OK;
}

// One layer of one problem.
struct WLayer {
    const uint8_t *Bt;        // split B tiles [column block][K chunk] (hi, lo)
    const float *C;           // N x m
    const float *Zin, *Gin;   // FWD: state at layer t (Zin == nullptr: z = 0, g = C); ADJ: Gin = G
    float *Zout, *Gout;       // FWD: state at layer t+1 (either may be nullptr); ADJ: Gout = next G
    const uint32_t *mask_in;  // ADJ: support of z^(t+1)
    uint32_t *mask_out;       // FWD: support of z^(t+1) (nullable)
    const float *Zq, *Gq;     // ADJ: z^(t+1) and g^(t) of the forward trajectory (Gq == nullptr: C)
    float *partial;           // ADJ: per-item sums of dalpha_t (indexed by item within the problem)
    const float *alpha;       // step sizes (nullptr: 1 / L)
    const double *Lp;
    int t, m, N, refresh, skip_mma;
    int TR;                   // rows per tile (<= 128; 0: 128): smaller tiles spread a short batch over every SM
    float lam;
    // Oracle-ISTA step (MODE == OIS, m <= 256, state updated in place): the
    // step of sample i is 1 / L_S (cached for its support) when condition
    // (star) held for it at this layer (flag_i == 0), else 1 / L; the epilogue
    // prepares the next layer: supports, condition (star), the list of samples
    // that need a new L_S (Algorithm 1; see oista_simt.cu).
    const double *LSv;        // N: cached L_S
    int *flag;                // N: in: (star) failed at layer t; out: at layer t+1
    uint32_t *Scur;           // N x W: out: supp(z^(t+1))
    const uint32_t *Sprev;    // N x W: support of the cached L_S
    const int *valid;         // N: the cached L_S is valid
    int *list, *counter;      // next layer's lists: class c at list + c * listN, length counter[c]
    int *accepted;            // accepted steps at this layer (nullable)
    double *LS_out;           // last layer: L_S per sample (nullable)
    int want_ls, listN, last;
    int coherent;             // the state was written by this launch: load it through L2 only
};

template <int NP>
struct WBatch {
    int nprob;
    int base[NP + 1];  // first work item of each problem; base[nprob] = total
    WLayer L[NP];
};

__host__ __device__ inline int n_colblocks(int m) { return (m + BN - 1) / BN; }
__host__ __device__ inline int n_kchunks(int m) { return (m + BK - 1) / BK; }
inline int n_items(int m, int N, int TR = 0) { return ceil_div(N, TR > 0 ? TR : BM) * n_colblocks(m); }

// Loads through the read-only path, or (coh) through L2 only: state written
// earlier by the same launch (the persistent batch kernels) must not come
// from the non-coherent cache.
__device__ __forceinline__ float4 ld4(const float4 *p, bool coh) { return coh ? __ldcg(p) : __ldg(p); }
__device__ __forceinline__ float ld1(const float *p, bool coh) { return coh ? __ldcg(p) : __ldg(p); }

// 16 consecutive entries (columns k0..k0+15) of row `row` of an N x m FP32
// matrix, zero outside the matrix or when M is null.
__device__ __forceinline__ void load16(const float *__restrict__ M, int row, bool ok, int m, int k0, float (&v)[16],
                                       bool coh = false)
{
    if (M != nullptr && ok && (m & 3) == 0 && (reinterpret_cast<uintptr_t>(M) & 15) == 0) {
        const float4 *src = reinterpret_cast<const float4 *>(M + (size_t)row * m + k0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 x = k0 + 4 * q < m ? ld4(src + q, coh) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * q + 0] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = (M != nullptr && ok && k0 + j < m) ? ld1(M + (size_t)row * m + k0 + j, coh) : 0.0f;
    }
}

// 16 bits of a support mask (columns k0..k0+15, k0 a multiple of 16), zero past m.
__device__ __forceinline__ uint32_t mask16(const uint32_t *__restrict__ words, int row, bool ok, int m, int k0)
{
    if (!ok || k0 >= m) return 0u;
    const int W = (m + 31) / 32;
    uint32_t b = (__ldg(words + (size_t)row * W + (k0 >> 5)) >> (k0 & 31)) & 0xffffu;
    if (k0 + 16 > m) b &= (1u << (m - k0)) - 1u;
    return b;
}

// Row `row` (0..127), codes kl..kl+15 (kl a multiple of 16) of an A chunk in
// the K-major 128-byte-swizzled layout: two 16-byte units per part.
template <bool SPLIT>
__device__ __forceinline__ void store_a16(uint8_t *stage, int row, int kl, const float (&v)[16])
{
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        hi[j] = *reinterpret_cast<const uint32_t *>(&h2);
        if (SPLIT) {
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
            lo[j] = *reinterpret_cast<const uint32_t *>(&l2);
        }
    }
    const int rbase = (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int unit = (kl >> 3) + u;
        const int off = rbase + ((unit ^ (row & 7)) << 4);
        *reinterpret_cast<uint4 *>(stage + off) = make_uint4(hi[4 * u], hi[4 * u + 1], hi[4 * u + 2], hi[4 * u + 3]);
        if (SPLIT)
            *reinterpret_cast<uint4 *>(stage + TILE_A + off) =
                make_uint4(lo[4 * u], lo[4 * u + 1], lo[4 * u + 2], lo[4 * u + 3]);
    }
}

// A staged slice holds rows 0..BM-1 x columns 0..SW-1 of the block, row r
// at r * SW, its 16-byte units (4 columns) permuted by XOR with r % 8: a
// warp's 16-byte accesses to one row (global side) or to 8 consecutive rows
// at one unit (epilogue side) are then free of bank conflicts.
__device__ __forceinline__ int sidx(int r, int c) { return r * SW + ((((c >> 2) ^ (r & 7)) << 2) | (c & 3)); }

// Rows [row0, row0 + TR) x columns [cs, cs + SW) of the row-major N x m
// matrices M0 (and M1 when NM = 2) into the staged slices t0 (t1), zero
// outside the matrix or when the matrix is null.  With 16-byte aligned rows
// each warp moves one 512-byte row segment per instruction and a thread
// issues all of its loads before its first shared-memory store.
constexpr int SV = SW / 4;           // 16-byte units per slice row
constexpr int SPER = BM * SV / NT;   // units per thread and matrix

template <int NM>
__device__ __forceinline__ bool stage_vec(const float *M0, const float *M1, int m)
{
    return (m & 3) == 0 && (reinterpret_cast<uintptr_t>(M0) & 15) == 0 &&
           (NM == 1 || (reinterpret_cast<uintptr_t>(M1) & 15) == 0);
}

// The vector path of stage_in in two halves: the loads into registers, then
// the shared stores.
template <int NM>
__device__ __forceinline__ void stage_load(float4 (&x0)[SPER], float4 (&x1)[SPER], const float *__restrict__ M0,
                                           const float *__restrict__ M1, int row0, int cs, int m, int N, int TR,
                                           int tid, bool coh)
{
#pragma unroll
    for (int k = 0; k < SPER; ++k) {
        const int e = tid + k * NT, r = e / SV, c = (e % SV) * 4;
        const int gr = row0 + r, gc = cs + c;
        const bool ok = r < TR && gr < N && gc < m;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        x0[k] = (ok && M0 != nullptr) ? ld4(reinterpret_cast<const float4 *>(M0 + (size_t)gr * m + gc), coh) : zero;
        if (NM == 2)
            x1[k] = (ok && M1 != nullptr) ? ld4(reinterpret_cast<const float4 *>(M1 + (size_t)gr * m + gc), coh) : zero;
    }
}

template <int NM>
__device__ __forceinline__ void stage_store(const float4 (&x0)[SPER], const float4 (&x1)[SPER], float *t0, float *t1,
                                            int tid)
{
#pragma unroll
    for (int k = 0; k < SPER; ++k) {
        const int e = tid + k * NT, r = e / SV, c = (e % SV) * 4;
        *reinterpret_cast<float4 *>(t0 + sidx(r, c)) = x0[k];
        if (NM == 2) *reinterpret_cast<float4 *>(t1 + sidx(r, c)) = x1[k];
    }
}

template <int NM>
__device__ __forceinline__ void stage_in(float *t0, const float *__restrict__ M0, float *t1,
                                         const float *__restrict__ M1, int row0, int cs, int m, int N, int TR, int tid,
                                         bool coh = false)
{
    if (stage_vec<NM>(M0, M1, m)) {
        float4 x0[SPER], x1[SPER];
        stage_load<NM>(x0, x1, M0, M1, row0, cs, m, N, TR, tid, coh);
        stage_store<NM>(x0, x1, t0, t1, tid);
        return;
    }
#pragma unroll 4
    for (int e = tid; e < BM * SW; e += NT) {
        const int r = e / SW, c = e % SW;
        const int gr = row0 + r, gc = cs + c;
        const bool ok = r < TR && gr < N && gc < m;
        t0[sidx(r, c)] = (ok && M0 != nullptr) ? ld1(M0 + (size_t)gr * m + gc, coh) : 0.0f;
        if (NM == 2) t1[sidx(r, c)] = (ok && M1 != nullptr) ? ld1(M1 + (size_t)gr * m + gc, coh) : 0.0f;
    }
}

// The reverse of stage_in for one matrix (rows r < TR inside N x m).
__device__ __forceinline__ void stage_out(const float *t, float *__restrict__ M, int row0, int cs, int m, int N,
                                          int TR, int tid)
{
    if ((m & 3) == 0 && (reinterpret_cast<uintptr_t>(M) & 15) == 0) {
        constexpr int V = SW / 4;
#pragma unroll 4
        for (int e = tid; e < BM * V; e += NT) {
            const int r = e / V, c = (e % V) * 4;
            const int gr = row0 + r, gc = cs + c;
            if (r < TR && gr < N && gc < m)
                *reinterpret_cast<float4 *>(M + (size_t)gr * m + gc) = *reinterpret_cast<const float4 *>(t + sidx(r, c));
        }
        return;
    }
#pragma unroll 4
    for (int e = tid; e < BM * SW; e += NT) {
        const int r = e / SW, c = e % SW;
        const int gr = row0 + r, gc = cs + c;
        if (r < TR && gr < N && gc < m) M[(size_t)gr * m + gc] = t[sidx(r, c)];
    }
}

__device__ __forceinline__ float st_f(float u, float thr) { return copysignf(fmaxf(fabsf(u) - thr, 0.0f), u); }

// ---------------------------------------------------------------------------
// Prep: B (m x m FP32) -> tiles [cb][kc] of BN x BK (B_hi, then B_lo), each
// K-major with the 128-byte swizzle; zero past m.
// ---------------------------------------------------------------------------
__global__ void split_tiles_kernel(const float *__restrict__ B, int m, uint8_t *__restrict__ out)
{
    const int ncb = n_colblocks(m), nkc = n_kchunks(m);
    const long long KP = (long long)nkc * BK;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ncb * BN * KP) return;
    const int n = (int)(idx / KP), k = (int)(idx % KP);
    const int cb = n / BN, nl = n % BN, kc = k / BK, kl = k % BK;
    const float v = (n < m && k < m) ? __ldg(B + (size_t)n * m + k) : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const uint32_t off = (uint32_t)((nl >> 3) * 1024 + (nl & 7) * 128 + (((kl >> 3) ^ (nl & 7)) << 4) + (kl & 7) * 2);
    uint8_t *tile = out + ((size_t)cb * nkc + kc) * TILE_PAIR;
    *reinterpret_cast<__nv_bfloat16 *>(tile + off) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(tile + TILE_B + off) = lo;
}

// ---------------------------------------------------------------------------
// The layer block: one (row tile, column block) of one layer.  A CTA may run
// many of them (the persistent batch kernels); the barriers, the tensor
// memory and the mbarrier phases persist across them in WRes.
// ---------------------------------------------------------------------------
struct WRes {
    uint8_t *smem;     // 1024-aligned dynamic shared memory (the two stages / epilogue slices)
    uint32_t sbase;    // its shared address
    uint32_t full0;    // full[2]: a stage's B tile landed
    uint32_t done0;    // done[2]: the MMAs reading a stage retired
    uint32_t tmem;     // the 128 x 256 FP32 accumulator
    uint32_t fph;      // thread 0: parity of the next phase of full[s] (bit s)
    uint32_t pend;     // thread 0: bulk copies into stage s not waited for (bit s)
    uint32_t dph;      // every thread: parity of the next phase of done[s] (bit s)
};

// Barriers and tensor memory of a CTA (every thread).
__device__ __forceinline__ void wres_init(WRes &R, uint8_t *smem_raw, uint64_t *bars, uint32_t *tmem_slot)
{
    const int tid = threadIdx.x;
    R.smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    R.sbase = smem_u32(R.smem);
    R.full0 = smem_u32(&bars[0]);
    R.done0 = smem_u32(&bars[2]);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&bars[i]), 1);
        fence_mbar_init();
    }
    if ((tid >> 5) == 0) tmem_alloc(tmem_slot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    R.tmem = *tmem_slot;
    R.fph = R.pend = R.dph = 0u;
}

// Drain pending bulk copies, release tensor memory (every thread).
__device__ __forceinline__ void wres_finish(WRes &R)
{
    if (threadIdx.x == 0)
        for (int s = 0; s < 2; ++s)
            if ((R.pend >> s) & 1u) {
                mbar_wait(R.full0 + 8 * s, (R.fph >> s) & 1u, 24);
                R.fph ^= 1u << s;
            }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(R.tmem, BN);
}

// Runs block `local` (row tile local / ncb, column block local % ncb) of
// layer L; returns false (uniformly) if a bounded wait expired.
template <bool SPLIT, int MODE>
__device__ __forceinline__ bool layer_block(const WLayer &L, int local, WRes &R)
{
    using CF = WCfg<SPLIT>;
    __shared__ float red[NT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = L.m, N = L.N;
    const int ncb = n_colblocks(m), nkc = n_kchunks(m);
    const int TR = L.TR > 0 ? L.TR : BM;  // rows of this tile that are real (the MMA always spans 128)
    const int row0 = (local / ncb) * TR, col0 = (local % ncb) * BN;
    const bool do_mma = !L.skip_mma;
    uint8_t *smem = R.smem;
    const uint32_t sbase = R.sbase, full0 = R.full0, done0 = R.done0, tmem = R.tmem;
    const uint8_t *Bcol = L.Bt + (size_t)(col0 / BN) * nkc * TILE_PAIR;
    const float *Zs = L.Zin;
    const float *Gs = (MODE == FWD && L.Zin == nullptr) ? L.C : L.Gin;
    const bool coh = L.coherent != 0;

    bool bad = false;     // thread 0: a wait for a B tile expired (folded into `failed` at the next barrier)
    bool failed = false;  // uniform over the CTA
    auto issue_b = [&](int kc) {
        const int s = kc & 1;
        mbar_arrive_expect_tx(full0 + 8 * s, CF::BBYTES);
        bulk_g2s(sbase + s * CF::STAGE + CF::OFF_B, Bcol + (size_t)kc * TILE_PAIR, CF::BBYTES, full0 + 8 * s);
        R.pend |= 1u << s;
    };
    auto wait_b = [&](int s, int code) {
        const bool ok = mbar_wait(full0 + 8 * s, (R.fph >> s) & 1u, code);
        R.fph ^= 1u << s;
        R.pend &= ~(1u << s);
        return ok;
    };
    // The first two B tiles are in flight before the wait below: the tiles
    // are written once, before the layers.  Oracle-ISTA layers are launched
    // as programmatic dependents of the solve kernel: nothing else of the
    // previous kernels is read or written before the wait.
    if (do_mma && tid == 0) {
        issue_b(0);
        if (nkc > 1) issue_b(1);
    }
    grid_dependency_wait();
    grid_dependents_launch();
    const float a = L.alpha ? __ldg(L.alpha + L.t) : (float)(1.0 / __ldg(L.Lp));

    // epilogue rows: warp w reads TMEM lanes 32 (w % 4).. (the tile rows)
    const int q = warp & 3, cg = warp >> 2;
    const int erow = row0 + 32 * q + lane;
    const bool eok = 32 * q + lane < TR && erow < N;
    const int W = (m + 31) / 32;
    // Oracle-ISTA: the rows' inputs from the previous kernels (condition
    // (star) flag, cached L_S, its validity and support words), all loaded at
    // once before the products and kept in shared memory: step s_ea (1 / L_S
    // or 1 / L), s_flag, s_valid, and s_sp[slice][column group][row].
    static_assert(BN / SW == 2, "two epilogue slices");
    __shared__ float s_ea[BM];
    __shared__ int s_flag[BM], s_valid[BM];
    __shared__ uint32_t s_sp[BN / SW][NT / 128][BM];
    int pf_flag = 1, pf_valid = 1;
    double pf_ls = 1.0;
    uint32_t pf_sp0 = 0u, pf_sp1 = 0u;
    if (MODE == OIS && eok) {
        if (cg == 0) {
            pf_flag = __ldg(L.flag + erow);
            pf_ls = __ldg(L.LSv + erow);
            pf_valid = __ldg(L.valid + erow);
        }
        const int c0 = col0 + cg * 32;
        if (!L.last && c0 < m) pf_sp0 = __ldg(L.Sprev + (size_t)erow * W + (c0 >> 5));
        if (!L.last && c0 + SW < m) pf_sp1 = __ldg(L.Sprev + (size_t)erow * W + ((c0 + SW) >> 5));
    }
    auto publish_rows = [&]() {
        const int r = 32 * q + lane;
        if (cg == 0) {
            s_ea[r] = (eok && pf_flag == 0) ? (float)(1.0 / pf_ls) : a;
            s_flag[r] = pf_flag;
            s_valid[r] = pf_valid;
        }
        s_sp[0][cg][r] = pf_sp0;
        s_sp[1][cg][r] = pf_sp1;
    };
    const int prow = tid >> 2, pk = (tid & 3) * 16;  // producer: one row, 16 codes of the chunk
    const int grow = row0 + prow;
    const bool rok = prow < TR && grow < N;
    // the loads of chunk kc + 1 are issued before chunk kc's barrier and
    // MMA issue, so their latency overlaps the tensor-core work
    float nz[16], ng[16];
    if (do_mma) {
        if (MODE != ADJ) {
            load16(Zs, grow, rok, m, pk, nz, coh);
            load16(Gs, grow, rok, m, pk, ng, coh && Gs != L.C);
        } else {
            load16(L.Gin, grow, rok, m, pk, ng, coh);
        }
    }
    if (MODE == OIS) {  // (waits for the row inputs while chunk 0 loads)
        publish_rows();
        __syncthreads();
    }
    if (do_mma) {
        const float pa = (MODE == OIS && rok) ? s_ea[prow] : a;
        const float pthr = __fmul_rn(pa, L.lam);
#pragma unroll 1
        for (int kc = 0; kc < nkc; ++kc) {
            const int s = kc & 1;
            uint8_t *stage = smem + s * CF::STAGE;
            if (kc >= 2) {  // stage s is free once the MMAs of chunk kc - 2 have retired
                const bool ok = mbar_wait(done0 + 8 * s, (R.dph >> s) & 1u, 21);
                R.dph ^= 1u << s;
                failed = __syncthreads_or(!ok || bad) != 0;
                if (failed) break;
                tc_fence_after();
                if (tid == 0) issue_b(kc);
            }
            // --- A operand of chunk kc: 16 codes of row prow
            const int k0 = kc * BK + pk;
            float v[16];
            if (MODE != ADJ) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float zn = st_f(fmaf(pa, ng[j], nz[j]), pthr);
                    v[j] = L.refresh ? -zn : nz[j] - zn;
                }
            } else {
                const uint32_t bits = mask16(L.mask_in, grow, rok, m, k0);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = ((bits >> j) & 1u) ? ng[j] : 0.0f;
            }
            if (kc + 1 < nkc) {
                if (MODE != ADJ) {
                    load16(Zs, grow, rok, m, k0 + BK, nz, coh);
                    load16(Gs, grow, rok, m, k0 + BK, ng, coh && Gs != L.C);
                } else {
                    load16(L.Gin, grow, rok, m, k0 + BK, ng, coh);
                }
            }
            store_a16<SPLIT>(stage, prow, pk, v);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                bad |= !wait_b(s, 22);
                tc_fence_after();
                const uint32_t a_base = sbase + s * CF::STAGE, b_base = a_base + CF::OFF_B;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(a_base + kk * 32);
                    const uint64_t bd = sdesc_sw128(b_base + kk * 32);
                    mma_ss(tmem, ad, bd, IDESC, (kc | kk) ? 1u : 0u);
                    if (SPLIT) {
                        mma_ss(tmem, sdesc_sw128(a_base + TILE_A + kk * 32), bd, IDESC, 1u);
                        mma_ss(tmem, ad, sdesc_sw128(b_base + TILE_B + kk * 32), IDESC, 1u);
                    }
                }
                mma_commit(done0 + 8 * s);
            }
        }
        if (!failed) {  // the last commit fires once every MMA issued before it has retired
            const int kl = nkc - 1;
            const bool ok = mbar_wait(done0 + 8 * (kl & 1), (R.dph >> (kl & 1)) & 1u, 23);
            R.dph ^= 1u << (kl & 1);
            // the other stage's last commit (chunk nkc - 2) has fired as well
            if (nkc >= 2) R.dph ^= 1u << ((kl - 1) & 1);
            failed = __syncthreads_or(!ok || bad) != 0;
        }
        tc_fence_after();
    }

    // --- epilogue
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    const float ea = MODE == OIS ? s_ea[32 * q + lane] : a;
    const float ethr = __fmul_rn(ea, L.lam);
    float part = 0.0f;
    bool obad = false, ochg = false;  // OIS: (star) fails for the next layer; support changed
    int ok_cnt = 0;                   // OIS: support size
    if (MODE != ADJ && !failed) {
        // z, g of the block pass through shared memory in two slices of 128
        // columns, so that every global load and store is a coalesced row
        // segment; thread (q, cg) finishes columns [32 cg, 32 cg + 32) of
        // the slice for its row.
        float *zt = reinterpret_cast<float *>(smem);
        float *gt = zt + BM * SW;
#pragma unroll 1
        for (int sl = 0; sl < BN / SW; ++sl) {
            const int cs = col0 + sl * SW;
            if (cs >= m) break;  // uniform
            stage_in<2>(zt, Zs, gt, Gs, row0, cs, m, N, TR, tid, coh);
            __syncthreads();
            float acc[32];
            if (do_mma) {
                float h0[16], h1[16];
                tmem_ld16(tq + sl * SW + cg * 32, h0);
                tmem_ld16(tq + sl * SW + cg * 32 + 16, h1);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    acc[j] = h0[j];
                    acc[16 + j] = h1[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
            }
            const int r = 32 * q + lane;
            uint32_t word = 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float4 *zp = reinterpret_cast<float4 *>(zt + sidx(r, cg * 32 + 4 * u));
                const float4 g4 = *reinterpret_cast<const float4 *>(gt + sidx(r, cg * 32 + 4 * u));
                float4 z4 = *zp;
                z4.x = st_f(fmaf(ea, g4.x, z4.x), ethr);
                z4.y = st_f(fmaf(ea, g4.y, z4.y), ethr);
                z4.z = st_f(fmaf(ea, g4.z, z4.z), ethr);
                z4.w = st_f(fmaf(ea, g4.w, z4.w), ethr);
                *zp = z4;
                word |= ((uint32_t)(z4.x != 0.0f) | (uint32_t)(z4.y != 0.0f) << 1 | (uint32_t)(z4.z != 0.0f) << 2 |
                         (uint32_t)(z4.w != 0.0f) << 3)
                        << (4 * u);
            }
            const int c0 = cs + cg * 32;  // first code of this thread's word
            if (c0 + 32 > m) word &= c0 < m ? (1u << (m - c0)) - 1u : 0u;
            if (L.refresh && L.Gout) {  // g' = c + (-z') B: the slice of C replaces g
                __syncthreads();
                stage_in<1>(gt, L.C, nullptr, nullptr, row0, cs, m, N, TR, tid);
                __syncthreads();
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float4 *gp = reinterpret_cast<float4 *>(gt + sidx(r, cg * 32 + 4 * u));
                float4 g4 = *gp;
                g4.x += acc[4 * u];
                g4.y += acc[4 * u + 1];
                g4.z += acc[4 * u + 2];
                g4.w += acc[4 * u + 3];
                *gp = g4;
                if (MODE == OIS) {
                    const float4 z4 = *reinterpret_cast<const float4 *>(zt + sidx(r, cg * 32 + 4 * u));
                    const int c = c0 + 4 * u;
                    obad |= (c < m) && (z4.x == 0.0f) && (fabsf(g4.x) > L.lam);
                    obad |= (c + 1 < m) && (z4.y == 0.0f) && (fabsf(g4.y) > L.lam);
                    obad |= (c + 2 < m) && (z4.z == 0.0f) && (fabsf(g4.z) > L.lam);
                    obad |= (c + 3 < m) && (z4.w == 0.0f) && (fabsf(g4.w) > L.lam);
                }
            }
            if (eok && c0 < m) {
                const int wi = c0 >> 5;
                if (L.mask_out) L.mask_out[(size_t)erow * W + wi] = word;
                if (MODE == OIS && !L.last) {
                    L.Scur[(size_t)erow * W + wi] = word;
                    ochg |= word != s_sp[sl][cg][32 * q + lane];
                    ok_cnt += __popc(word);
                }
            }
            __syncthreads();
            if (L.Zout) stage_out(zt, L.Zout, row0, cs, m, N, TR, tid);
            if (L.Gout) stage_out(gt, L.Gout, row0, cs, m, N, TR, tid);
            __syncthreads();
        }
    }
    if (MODE == ADJ) {
        // columns 64 (w / 4).. of the block, 16 at a time
        const uint32_t tl = tq + (uint32_t)(cg * 64);
#pragma unroll 1
        for (int pc = 0; pc < 4; ++pc) {
            const int c = col0 + cg * 64 + pc * 16;
            float acc[16];
            if (do_mma && !failed) {
                tmem_ld16(tl + pc * 16, acc);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
            }
            if (failed || !eok || c >= m) continue;
            float G[16], gq[16], zq[16];
            load16(L.Gin, erow, true, m, c, G, coh);
            load16(L.Gq ? L.Gq : L.C, erow, true, m, c, gq, coh && L.Gq != nullptr);
            load16(L.Zq, erow, true, m, c, zq, coh);
            const uint32_t bits = mask16(L.mask_in, erow, true, m, c);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float h = ((bits >> j) & 1u) ? G[j] : 0.0f;
                const float qv = gq[j] - L.lam * (float)((zq[j] > 0.0f) - (zq[j] < 0.0f));
                part = fmaf(h, qv, part);
                G[j] = fmaf(-a, acc[j], h);
            }
            if (L.Gout)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c + j < m) L.Gout[(size_t)erow * m + c + j] = G[j];
        }
    }
    if (MODE == OIS) {
        // combine the four column groups of each row, then one thread per row
        // prepares the next layer (condition (star), the L_S list)
        __shared__ int rbad[BM], rchg[BM], rk[BM], nacc;
        for (int r = tid; r < BM; r += NT) rbad[r] = rchg[r] = rk[r] = 0;
        if (tid == 0) nacc = 0;
        __syncthreads();
        if (eok && !failed) {
            if (obad) atomicOr(&rbad[32 * q + lane], 1);
            if (ochg) atomicOr(&rchg[32 * q + lane], 1);
            if (ok_cnt) atomicAdd(&rk[32 * q + lane], ok_cnt);
        }
        __syncthreads();
        if (cg == 0 && eok && !failed) {
            if (s_flag[32 * q + lane] == 0) atomicAdd(&nacc, 1);
            if (L.last) {
                if (L.LS_out) L.LS_out[erow] = __ldg(L.LSv + erow);
            }
        }
        __syncthreads();  // every read of flag[] precedes its update
        if (cg == 0 && eok && !failed && !L.last) {
            const int r = 32 * q + lane;
            const int f = rbad[r];
            L.flag[erow] = f;
            const bool changed = rchg[r] != 0 || s_valid[r] == 0;
            if ((f == 0 || L.want_ls) && changed) {
                const int k = rk[r];
                const int cls = k > 64 ? 0 : k > 32 ? 1 : 2;
                const int pos = atomicAdd(L.counter + cls, 1);
                L.list[(size_t)cls * L.listN + pos] = erow;
            }
        }
        if (tid == 0 && L.accepted && nacc) atomicAdd(L.accepted, nacc);
    }
    if (MODE == ADJ) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (tid == 0) {
            float sum = 0.0f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) sum += red[w];
            L.partial[local] = sum;
        }
    }

    // the accumulator and the stages are free for the next block (whose bulk
    // copies overwrite, through the async proxy, what the epilogue staged)
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return !failed;
}

// One layer (or Oracle-ISTA step) of up to NP problems: one block per CTA.
template <bool SPLIT, int MODE, int NP>
__global__ void __launch_bounds__(NT, 1) tcw_layer_kernel(const __grid_constant__ WBatch<NP> P)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[4];  // full[2] (B tile landed), done[2] (MMAs of the stage retired)
    __shared__ uint32_t tmem_slot;
    int p = 0;
    while (p + 1 < P.nprob && (int)blockIdx.x >= P.base[p + 1]) ++p;
    WRes R;
    wres_init(R, smem_raw, bars, &tmem_slot);
    layer_block<SPLIT, MODE>(P.L[p], (int)blockIdx.x - P.base[p], R);
    wres_finish(R);
}

// G_T = gZ (if given) or dF/dz^(T) = B z - c + lam sign(z) = -g^(T) + lam sign(z^(T)).
__global__ void adjoint_seed_kernel(const float *__restrict__ ZT, const float *__restrict__ GT,
                                    const float *__restrict__ gZ, size_t n, float lam, float *__restrict__ G)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (gZ) {
        G[i] = __ldg(gZ + i);
    } else {
        const float z = __ldg(ZT + i);
        G[i] = -__ldg(GT + i) + lam * (float)((z > 0.0f) - (z < 0.0f));
    }
}

// dalpha[t] = sum of partial[t][0..nitem), FP64, fixed order (one warp per layer).
__global__ void reduce_items_kernel(const float *__restrict__ partial, int nitem, int T, float *__restrict__ dalpha)
{
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= T) return;
    double s = 0.0;
    for (int b = lane; b < nitem; b += 32) s += (double)partial[(size_t)t * nitem + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dalpha[t] = (float)s;
}

// ---------------------------------------------------------------------------
// Persistent batch kernels (ragged batches): every CTA takes items - a row
// tile of one problem - from a queue in the workspace and runs all of the
// item's layers, column block after column block, before taking the next.
// An item's layers depend only on its own rows, so no CTA ever waits for
// another; the state between layers lives in the workspace (read back
// through L2: it was written by this launch).  Items are queued largest
// problem first.
// ---------------------------------------------------------------------------
constexpr int PMAXP = 64;
// Sample rows of a persistent item (the MMA's M: items of 64 rows, whose
// states in flight would fit in L2 up to m = 512, measured slower - 102 against
// 79 ms on the 64-problem ragged batch - with the MMAs half filled).
constexpr int PTR = BM;

struct PProb {
    const uint8_t *Bt;        // split B tiles
    const float *C;
    int m, N;
    float lam;
    const float *alpha;
    const double *Lp;
    float *Z;                 // forward: z^(T)
    uint32_t *masks;
    float *ckpt;
    const float *gZ;          // backward
    float *dalpha;            // backward: T (out)
    float *buf[4];            // forward: (z, g) ping-pong; backward: (G, G) ping-pong in buf[0], buf[1]
    uint8_t *seg;             // backward: 2 K + 2 states of the recomputed segment
    size_t state;             // bytes of one N x m state
    float *partial;           // backward: T x nitem per-block sums of dalpha
    int nitem;                // backward: blocks (row tiles x column blocks)
};

struct PBatch {
    int nprob, T, K;
    int base[PMAXP + 1];      // first item of each problem; base[nprob] = total
    int *queue;               // the next item (zeroed before the launch)
    PProb q[PMAXP];
};

// The next item for this CTA (-1 when none are left).
__device__ __forceinline__ int next_item(const PBatch &P, int *s_item)
{
    if (threadIdx.x == 0) *s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    return it < P.base[P.nprob] ? it : -1;
}

__device__ __forceinline__ int item_problem(const PBatch &P, int it)
{
    int p = 0;
    while (p + 1 < P.nprob && it >= P.base[p + 1]) ++p;
    return p;
}

// The layer-t descriptor of the forward of problem q (the buffers of
// forward_batch: checkpoints every K layers, else the ping-pong; Z last).
__device__ __forceinline__ WLayer fwd_layer(const PProb &q, int t, int T, int K, bool ck, const float *Zc,
                                            const float *Gc, int &pp)
{
    WLayer L{};
    L.Bt = q.Bt;
    L.C = q.C;
    L.Zin = Zc;
    L.Gin = Gc;
    L.alpha = q.alpha;
    L.Lp = q.Lp;
    L.t = t;
    L.m = q.m;
    L.N = q.N;
    L.lam = q.lam;
    L.coherent = 1;
    L.TR = PTR;
    L.refresh = (ck && K < T) ? ((t + 1) % K == 0) : ((t + 1) % REFRESH == 0);
    const int W = (q.m + 31) / 32;
    L.mask_out = q.masks ? q.masks + (size_t)t * q.N * W : nullptr;
    if (t == T - 1) {
        L.Zout = q.Z;
        L.Gout = nullptr;
        L.skip_mma = 1;  // g^(T) is not needed
    } else if (ck && (t + 1) % K == 0) {
        float *slot = q.ckpt + (size_t)((t + 1) / K - 1) * 2 * q.N * q.m;
        L.Zout = slot;
        L.Gout = slot + (size_t)q.N * q.m;
    } else {
        L.Zout = q.buf[2 * pp];
        L.Gout = q.buf[2 * pp + 1];
        pp ^= 1;
    }
    return L;
}

template <bool SPLIT>
__global__ void __launch_bounds__(NT, 1) tcw_persist_fwd_kernel(const __grid_constant__ PBatch P)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[4];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_item;
    WRes R;
    wres_init(R, smem_raw, bars, &tmem_slot);
    bool ok = true;
    for (int it = next_item(P, &s_item); it >= 0 && ok; it = next_item(P, &s_item)) {
        const PProb &q = P.q[item_problem(P, it)];
        const int tile = it - P.base[item_problem(P, it)];
        const int ncb = n_colblocks(q.m);
        const bool ck = q.ckpt != nullptr && P.K >= 1 && P.K < P.T;
        const float *Zc = nullptr, *Gc = nullptr;
        int pp = 0;
        for (int t = 0; t < P.T && ok; ++t) {
            const WLayer L = fwd_layer(q, t, P.T, P.K, ck, Zc, Gc, pp);
            // (each block ends with a CTA barrier: its state is visible to the next layer)
            for (int cb = 0; cb < ncb && ok; ++cb) ok = layer_block<SPLIT, FWD>(L, tile * ncb + cb, R);
            Zc = L.Zout;
            Gc = L.Gout;
        }
    }
    wres_finish(R);
}

template <bool SPLIT>
__global__ void __launch_bounds__(NT, 1) tcw_persist_bwd_kernel(const __grid_constant__ PBatch P)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[4];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_item;
    WRes R;
    wres_init(R, smem_raw, bars, &tmem_slot);
    const int T = P.T, K = P.K < P.T ? P.K : P.T;
    const bool ck = K < T;
    const int nseg = (T + K - 1) / K;
    bool ok = true;
    for (int it = next_item(P, &s_item); it >= 0 && ok; it = next_item(P, &s_item)) {
        const int pi = item_problem(P, it);
        const PProb &q = P.q[pi];
        const int tile = it - P.base[pi];
        const int ncb = n_colblocks(q.m);
        const int W = (q.m + 31) / 32;
        const size_t nm = (size_t)q.N * q.m;
        auto segZ = [&](int i) { return reinterpret_cast<float *>(q.seg + (size_t)(2 * i) * q.state); };
        auto segG = [&](int i) { return reinterpret_cast<float *>(q.seg + (size_t)(2 * i + 1) * q.state); };
        int gcur = 0;
        for (int sg = nseg - 1; sg >= 0 && ok; --sg) {
            const int t0 = sg * K, t1 = t0 + K < T ? t0 + K : T;
            const bool lastseg = sg == nseg - 1;
            const float *Z0 = t0 > 0 ? q.ckpt + (size_t)(t0 / K - 1) * 2 * nm : nullptr;
            const float *G0 = t0 > 0 ? Z0 + nm : nullptr;
            // recompute layers t0 .. t1-1 of this item's rows with the forward's arithmetic
            for (int t = t0; t < t1 && ok; ++t) {
                const int j = t - t0;
                WLayer L{};
                L.Bt = q.Bt;
                L.C = q.C;
                L.Zin = j == 0 ? Z0 : segZ(j);
                L.Gin = j == 0 ? G0 : segG(j);
                L.Zout = segZ(j + 1);
                const bool need_g = (t + 1 < t1) || (lastseg && t + 1 == T);
                L.Gout = need_g ? segG(j + 1) : nullptr;
                L.skip_mma = need_g ? 0 : 1;
                L.alpha = q.alpha;
                L.t = t;
                L.m = q.m;
                L.N = q.N;
                L.lam = q.lam;
                L.coherent = 1;
                L.TR = PTR;
                L.refresh = ck ? ((t + 1) % K == 0) : ((t + 1) % REFRESH == 0);
                for (int cb = 0; cb < ncb && ok; ++cb) ok = layer_block<SPLIT, FWD>(L, tile * ncb + cb, R);
            }
            if (!ok) break;
            if (lastseg) {
                // G_T = gZ, or dF/dz^(T) = -g^(T) + lam sign(z^(T)), on this item's rows
                const int n = t1 - t0;
                const float *ZT = segZ(n), *GT = segG(n);
                const size_t r0 = (size_t)tile * PTR, r1 = r0 + PTR < (size_t)q.N ? r0 + PTR : (size_t)q.N;
                for (size_t e = r0 * q.m + threadIdx.x; e < r1 * q.m; e += NT) {
                    float g;
                    if (q.gZ) {
                        g = __ldg(q.gZ + e);
                    } else {
                        const float z = __ldcg(ZT + e);
                        g = -__ldcg(GT + e) + q.lam * (float)((z > 0.0f) - (z < 0.0f));
                    }
                    q.buf[gcur][e] = g;
                }
                __syncthreads();
            }
            for (int t = t1 - 1; t >= t0 && ok; --t) {
                const int j = t - t0;
                WLayer L{};
                L.Bt = q.Bt;
                L.C = q.C;
                L.Gin = q.buf[gcur];
                L.Gout = t > 0 ? q.buf[gcur ^ 1] : nullptr;
                L.skip_mma = t > 0 ? 0 : 1;
                L.mask_in = q.masks + (size_t)t * q.N * W;
                L.Zq = segZ(j + 1);
                L.Gq = j == 0 ? G0 : segG(j);  // nullptr at t = 0: g^(0) = c
                L.partial = q.partial + (size_t)t * q.nitem;
                L.alpha = q.alpha;
                L.t = t;
                L.m = q.m;
                L.N = q.N;
                L.lam = q.lam;
                L.coherent = 1;
                L.TR = PTR;
                for (int cb = 0; cb < ncb && ok; ++cb) ok = layer_block<SPLIT, ADJ>(L, tile * ncb + cb, R);
                gcur ^= 1;
            }
        }
    }
    wres_finish(R);
}

// dalpha of every problem of a persistent batch: one warp per (problem, layer).
__global__ void reduce_batch_kernel(const __grid_constant__ PBatch P)
{
    const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const int p = w / P.T, t = w % P.T;
    if (p >= P.nprob) return;
    const PProb &q = P.q[p];
    double s = 0.0;
    for (int b = lane; b < q.nitem; b += 32) s += (double)q.partial[(size_t)t * q.nitem + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && q.N > 0) q.dalpha[t] = (float)s;
}

// ---------------------------------------------------------------------------
// Host side: every entry point runs a batch of problems (one problem is a
// batch of one); per layer, one launch covers the work items of up to MAXP
// problems.
// ---------------------------------------------------------------------------
namespace {

constexpr int MAXP = 64;

size_t tiles_bytes(int m) { return (size_t)n_colblocks(m) * n_kchunks(m) * TILE_PAIR; }
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
size_t state_bytes(int m, int N) { return align256(sizeof(float) * (size_t)N * m); }

int split_tiles(const float *B, int m, uint8_t *out, cudaStream_t st)
{
    const long long total = (long long)n_colblocks(m) * BN * n_kchunks(m) * BK;
    split_tiles_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(B, m, out);
    return check_launch("split_tiles_kernel");
}

template <bool SPLIT, int MODE, int NP>
int launch_chunk(const WLayer *Ls, int count, cudaStream_t st, bool dependent = false)
{
    WBatch<NP> P{};
    P.nprob = count;
    P.base[0] = 0;
    for (int i = 0; i < count; ++i) {
        P.L[i] = Ls[i];
        P.base[i + 1] = P.base[i] + n_items(Ls[i].m, Ls[i].N, Ls[i].TR);
    }
    if (P.base[count] == 0) return SLISTA_OK;
    auto k = tcw_layer_kernel<SPLIT, MODE, NP>;
    SLISTA_CUDA_TRY(allow_smem(k, WCfg<SPLIT>::SMEM));
    if (dependent) {  // may start while the previous kernel in the stream finishes (see grid_dependency_wait)
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(P.base[count]);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = WCfg<SPLIT>::SMEM;
        cfg.stream = st;
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr.val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        SLISTA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, P));
    } else {
        k<<<P.base[count], NT, WCfg<SPLIT>::SMEM, st>>>(P);
    }
    return check_launch(MODE == FWD   ? "tcw_layer_kernel (forward)"
                        : MODE == ADJ ? "tcw_layer_kernel (adjoint)"
                                      : "tcw_layer_kernel (Oracle-ISTA step)");
}

// One layer for every problem of the batch: launches of at most MAXP problems.
template <int MODE>
int launch_layers(const std::vector<WLayer> &Ls, bool split, cudaStream_t st)
{
    for (size_t i = 0; i < Ls.size(); i += MAXP) {
        const int c = (int)std::min(Ls.size() - i, (size_t)MAXP);
        int rc;
        if (c == 1)
            rc = split ? launch_chunk<true, MODE, 1>(&Ls[i], 1, st) : launch_chunk<false, MODE, 1>(&Ls[i], 1, st);
        else
            rc = split ? launch_chunk<true, MODE, MAXP>(&Ls[i], c, st)
                       : launch_chunk<false, MODE, MAXP>(&Ls[i], c, st);
        if (rc) return rc;
    }
    return SLISTA_OK;
}

bool refresh_at(int t, int T, int K, bool ckpt)
{
    return (ckpt && K < T) ? ((t + 1) % K == 0) : ((t + 1) % REFRESH == 0);
}

size_t fwd_bytes_one(int m, int N) { return align256(tiles_bytes(m)) + 4 * state_bytes(m, N); }

size_t bwd_bytes_one(int m, int N, int T, int K)
{
    return align256(tiles_bytes(m)) + (size_t)(2 * K + 4) * state_bytes(m, N) +
           align256(sizeof(float) * (size_t)T * n_items(m, N));
}

}  // namespace

bool supported(int m) { return m >= 1 && m <= 1024; }

size_t forward_ws_bytes(int m, int N) { return fwd_bytes_one(m, N); }

size_t backward_ws_bytes(int m, int N, int T, int K) { return bwd_bytes_one(m, N, T, K); }

size_t forward_batch_ws_bytes(const Problem *P, int count)
{
    size_t b = 0;
    for (int i = 0; i < count; ++i) b += fwd_bytes_one(P[i].m, P[i].N);
    return b;
}

size_t backward_batch_ws_bytes(const Problem *P, int count, int T, int K)
{
    size_t b = 0;
    for (int i = 0; i < count; ++i) b += bwd_bytes_one(P[i].m, P[i].N, T, K < T ? K : T);
    return b;
}

int forward_batch(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    struct Buf {
        uint8_t *tiles;
        float *buf[4];
        const float *Zc, *Gc;
        int pp;
        bool ck;
    };
    std::vector<Buf> bb(count);
    uint8_t *cur = reinterpret_cast<uint8_t *>(ws);
    for (int i = 0; i < count; ++i) {
        Buf &b = bb[i];
        b.tiles = cur;
        cur += align256(tiles_bytes(P[i].m));
        for (int j = 0; j < 4; ++j) {
            b.buf[j] = reinterpret_cast<float *>(cur);
            cur += state_bytes(P[i].m, P[i].N);
        }
        b.Zc = b.Gc = nullptr;
        b.pp = 0;
        b.ck = P[i].ckpt != nullptr && K >= 1 && K < T;
        int rc = split_tiles(P[i].B, P[i].m, b.tiles, st);
        if (rc) return rc;
        if (T == 0 && P[i].N > 0)
            SLISTA_CUDA_TRY(cudaMemsetAsync(P[i].Z, 0, sizeof(float) * (size_t)P[i].N * P[i].m, st));
    }
    std::vector<WLayer> Ls;
    for (int t = 0; t < T; ++t) {
        Ls.clear();
        for (int i = 0; i < count; ++i) {
            const Problem &q = P[i];
            if (q.N == 0) continue;
            Buf &b = bb[i];
            const int W = (q.m + 31) / 32;
            WLayer L{};
            L.Bt = b.tiles;
            L.C = q.C;
            L.Zin = b.Zc;
            L.Gin = b.Gc;
            L.alpha = q.alpha;
            L.Lp = q.L;
            L.t = t;
            L.m = q.m;
            L.N = q.N;
            L.lam = q.lam;
            L.refresh = refresh_at(t, T, K, b.ck);
            L.mask_out = q.masks ? q.masks + (size_t)t * q.N * W : nullptr;
            if (t == T - 1) {
                L.Zout = q.Z;
                L.Gout = nullptr;
                L.skip_mma = 1;  // g^(T) is not needed
            } else if (b.ck && (t + 1) % K == 0) {
                float *slot = q.ckpt + (size_t)((t + 1) / K - 1) * 2 * q.N * q.m;
                L.Zout = slot;
                L.Gout = slot + (size_t)q.N * q.m;
            } else {
                L.Zout = b.buf[2 * b.pp];
                L.Gout = b.buf[2 * b.pp + 1];
                b.pp ^= 1;
            }
            b.Zc = L.Zout;
            b.Gc = L.Gout;
            Ls.push_back(L);
        }
        int rc = launch_layers<FWD>(Ls, split, st);
        if (rc) return rc;
    }
    return SLISTA_OK;
}

int backward_batch(const Problem *P, int count, int T, int Kin, int prec, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    const int K = Kin < T ? Kin : T;
    const bool ck = K < T;
    struct Buf {
        uint8_t *tiles, *seg;
        float *Gb[2];
        float *partial;
        size_t state;
        int nitem, gcur;
        float *segZ(int i) const { return reinterpret_cast<float *>(seg + (size_t)(2 * i) * state); }
        float *segG(int i) const { return reinterpret_cast<float *>(seg + (size_t)(2 * i + 1) * state); }
    };
    std::vector<Buf> bb(count);
    uint8_t *cur = reinterpret_cast<uint8_t *>(ws);
    for (int i = 0; i < count; ++i) {
        Buf &b = bb[i];
        const Problem &q = P[i];
        b.state = state_bytes(q.m, q.N);
        b.tiles = cur;
        cur += align256(tiles_bytes(q.m));
        b.seg = cur;
        cur += (size_t)(2 * K + 2) * b.state;
        b.Gb[0] = reinterpret_cast<float *>(cur);
        b.Gb[1] = reinterpret_cast<float *>(cur + b.state);
        cur += 2 * b.state;
        b.partial = reinterpret_cast<float *>(cur);
        b.nitem = n_items(q.m, q.N);
        cur += align256(sizeof(float) * (size_t)T * b.nitem);
        b.gcur = 0;
        int rc = split_tiles(q.B, q.m, b.tiles, st);
        if (rc) return rc;
        if (q.N == 0) SLISTA_CUDA_TRY(cudaMemsetAsync(q.dalpha, 0, sizeof(float) * T, st));
    }
    const int nseg = ceil_div(T, K);
    std::vector<WLayer> Ls;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int t0 = sg * K, t1 = t0 + K < T ? t0 + K : T;
        const bool lastseg = sg == nseg - 1;
        auto Z0 = [&](int i) -> const float * {
            return t0 > 0 ? P[i].ckpt + (size_t)(t0 / K - 1) * 2 * P[i].N * P[i].m : nullptr;
        };
        auto G0 = [&](int i) -> const float * {
            return t0 > 0 ? P[i].ckpt + (size_t)(t0 / K - 1) * 2 * P[i].N * P[i].m + (size_t)P[i].N * P[i].m
                          : nullptr;
        };
        // recompute layers t0 .. t1-1 with the forward's arithmetic
        for (int t = t0; t < t1; ++t) {
            const int j = t - t0;
            Ls.clear();
            for (int i = 0; i < count; ++i) {
                const Problem &q = P[i];
                if (q.N == 0) continue;
                const Buf &b = bb[i];
                WLayer L{};
                L.Bt = b.tiles;
                L.C = q.C;
                L.Zin = j == 0 ? Z0(i) : b.segZ(j);
                L.Gin = j == 0 ? G0(i) : b.segG(j);
                L.Zout = b.segZ(j + 1);
                const bool need_g = (t + 1 < t1) || (lastseg && t + 1 == T);
                L.Gout = need_g ? b.segG(j + 1) : nullptr;
                L.skip_mma = need_g ? 0 : 1;
                L.alpha = q.alpha;
                L.t = t;
                L.m = q.m;
                L.N = q.N;
                L.lam = q.lam;
                L.refresh = refresh_at(t, T, K, ck);
                Ls.push_back(L);
            }
            int rc = launch_layers<FWD>(Ls, split, st);
            if (rc) return rc;
        }
        if (lastseg) {
            const int n = t1 - t0;
            for (int i = 0; i < count; ++i) {
                const Problem &q = P[i];
                if (q.N == 0) continue;
                Buf &b = bb[i];
                const size_t nm = (size_t)q.N * q.m;
                adjoint_seed_kernel<<<(unsigned)ceil_div((long long)nm, 256), 256, 0, st>>>(
                    b.segZ(n), b.segG(n), q.gZ, nm, q.lam, b.Gb[b.gcur]);
                int rc = check_launch("adjoint_seed_kernel");
                if (rc) return rc;
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const int j = t - t0;
            Ls.clear();
            for (int i = 0; i < count; ++i) {
                const Problem &q = P[i];
                if (q.N == 0) continue;
                Buf &b = bb[i];
                const int W = (q.m + 31) / 32;
                WLayer L{};
                L.Bt = b.tiles;
                L.C = q.C;
                L.Gin = b.Gb[b.gcur];
                L.Gout = t > 0 ? b.Gb[b.gcur ^ 1] : nullptr;
                L.skip_mma = t > 0 ? 0 : 1;
                L.mask_in = q.masks + (size_t)t * q.N * W;
                L.Zq = b.segZ(j + 1);
                L.Gq = j == 0 ? G0(i) : b.segG(j);  // nullptr at t = 0: g^(0) = c
                L.partial = b.partial + (size_t)t * b.nitem;
                L.alpha = q.alpha;
                L.t = t;
                L.m = q.m;
                L.N = q.N;
                L.lam = q.lam;
                Ls.push_back(L);
                b.gcur ^= 1;
            }
            int rc = launch_layers<ADJ>(Ls, split, st);
            if (rc) return rc;
        }
    }
    for (int i = 0; i < count; ++i) {
        if (P[i].N == 0) continue;
        reduce_items_kernel<<<ceil_div(T, 8), 256, 0, st>>>(bb[i].partial, bb[i].nitem, T, P[i].dalpha);
        int rc = check_launch("reduce_items_kernel");
        if (rc) return rc;
    }
    return SLISTA_OK;
}

// ---------------------------------------------------------------------------
// Ragged batches through the persistent kernels: one launch for the forward
// (and one plus a reduction for the backward) per PMAXP problems.
// ---------------------------------------------------------------------------
namespace {

// Problems by decreasing work (rows x m^2), so that the queue hands out the
// largest items first.
std::vector<int> by_cost(const Problem *P, int count)
{
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return (double)P[a].N * P[a].m * P[a].m > (double)P[b].N * P[b].m * P[b].m;
    });
    return idx;
}

template <bool SPLIT, bool BWD>
int launch_persist(const PBatch &B, cudaStream_t st)
{
    const int total = B.base[B.nprob];
    if (total == 0) return SLISTA_OK;
    SLISTA_CUDA_TRY(cudaMemsetAsync(B.queue, 0, sizeof(int), st));
    const int grid = total < num_sms() ? total : num_sms();
    if (BWD) {
        auto k = tcw_persist_bwd_kernel<SPLIT>;
        SLISTA_CUDA_TRY(allow_smem(k, WCfg<SPLIT>::SMEM));
        k<<<grid, NT, WCfg<SPLIT>::SMEM, st>>>(B);
        int rc = check_launch("tcw_persist_bwd_kernel");
        if (rc) return rc;
        reduce_batch_kernel<<<ceil_div((long long)B.nprob * B.T, 8), 256, 0, st>>>(B);
        return check_launch("reduce_batch_kernel");
    }
    auto k = tcw_persist_fwd_kernel<SPLIT>;
    SLISTA_CUDA_TRY(allow_smem(k, WCfg<SPLIT>::SMEM));
    k<<<grid, NT, WCfg<SPLIT>::SMEM, st>>>(B);
    return check_launch("tcw_persist_fwd_kernel");
}

}  // namespace

size_t persist_forward_ws_bytes(const Problem *P, int count) { return 256 + forward_batch_ws_bytes(P, count); }

size_t persist_backward_ws_bytes(const Problem *P, int count, int T, int K)
{
    // the layout of backward_batch_persist: tiles, 2 K + 2 segment states, two
    // adjoint states and T partial sums per item
    const int Kc = K < T ? K : T;
    size_t b = 256;
    for (int i = 0; i < count; ++i)
        b += align256(tiles_bytes(P[i].m)) + (size_t)(2 * Kc + 4) * state_bytes(P[i].m, P[i].N) +
             align256(sizeof(float) * (size_t)T * n_items(P[i].m, P[i].N, PTR));
    return b;
}

int forward_batch_persist(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    int *queue = reinterpret_cast<int *>(ws);
    uint8_t *cur = reinterpret_cast<uint8_t *>(ws) + 256;
    std::vector<PProb> qs(count);
    for (int i = 0; i < count; ++i) {
        PProb &q = qs[i];
        q = PProb{};
        q.Bt = cur;
        cur += align256(tiles_bytes(P[i].m));
        for (int j = 0; j < 4; ++j) {
            q.buf[j] = reinterpret_cast<float *>(cur);
            cur += state_bytes(P[i].m, P[i].N);
        }
        q.C = P[i].C;
        q.m = P[i].m;
        q.N = P[i].N;
        q.lam = P[i].lam;
        q.alpha = P[i].alpha;
        q.Lp = P[i].L;
        q.Z = P[i].Z;
        q.masks = P[i].masks;
        q.ckpt = P[i].ckpt;
        int rc = split_tiles(P[i].B, P[i].m, const_cast<uint8_t *>(q.Bt), st);
        if (rc) return rc;
        if (T == 0 && P[i].N > 0)
            SLISTA_CUDA_TRY(cudaMemsetAsync(P[i].Z, 0, sizeof(float) * (size_t)P[i].N * P[i].m, st));
    }
    if (T == 0) return SLISTA_OK;
    const std::vector<int> order = by_cost(P, count);
    for (size_t c0 = 0; c0 < order.size(); c0 += PMAXP) {
        PBatch B{};
        B.T = T;
        B.K = K;
        B.queue = queue;
        B.base[0] = 0;
        for (size_t c = c0; c < order.size() && B.nprob < PMAXP; ++c) {
            const PProb &q = qs[order[c]];
            B.q[B.nprob] = q;
            B.base[B.nprob + 1] = B.base[B.nprob] + ceil_div(q.N, PTR);
            ++B.nprob;
        }
        int rc = split ? launch_persist<true, false>(B, st) : launch_persist<false, false>(B, st);
        if (rc) return rc;
    }
    return SLISTA_OK;
}

int backward_batch_persist(const Problem *P, int count, int T, int Kin, int prec, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    const int K = Kin < T ? Kin : T;
    int *queue = reinterpret_cast<int *>(ws);
    uint8_t *cur = reinterpret_cast<uint8_t *>(ws) + 256;
    std::vector<PProb> qs(count);
    for (int i = 0; i < count; ++i) {
        PProb &q = qs[i];
        const Problem &p = P[i];
        q = PProb{};
        q.state = state_bytes(p.m, p.N);
        q.Bt = cur;
        cur += align256(tiles_bytes(p.m));
        q.seg = cur;
        cur += (size_t)(2 * K + 2) * q.state;
        q.buf[0] = reinterpret_cast<float *>(cur);
        q.buf[1] = reinterpret_cast<float *>(cur + q.state);
        cur += 2 * q.state;
        q.partial = reinterpret_cast<float *>(cur);
        q.nitem = n_items(p.m, p.N, PTR);
        cur += align256(sizeof(float) * (size_t)T * q.nitem);
        q.C = p.C;
        q.m = p.m;
        q.N = p.N;
        q.lam = p.lam;
        q.alpha = p.alpha;
        q.masks = p.masks;
        q.ckpt = p.ckpt;
        q.gZ = p.gZ;
        q.dalpha = p.dalpha;
        int rc = split_tiles(p.B, p.m, const_cast<uint8_t *>(q.Bt), st);
        if (rc) return rc;
        if (p.N == 0) SLISTA_CUDA_TRY(cudaMemsetAsync(p.dalpha, 0, sizeof(float) * T, st));
    }
    const std::vector<int> order = by_cost(P, count);
    for (size_t c0 = 0; c0 < order.size(); c0 += PMAXP) {
        PBatch B{};
        B.T = T;
        B.K = K;
        B.queue = queue;
        B.base[0] = 0;
        for (size_t c = c0; c < order.size() && B.nprob < PMAXP; ++c) {
            const PProb &q = qs[order[c]];
            B.q[B.nprob] = q;
            B.base[B.nprob + 1] = B.base[B.nprob] + ceil_div(q.N, PTR);
            ++B.nprob;
        }
        int rc = split ? launch_persist<true, true>(B, st) : launch_persist<false, true>(B, st);
        if (rc) return rc;
    }
    return SLISTA_OK;
}

size_t oista_tiles_bytes(int m) { return align256(tiles_bytes(m)); }

int oista_split(const float *B, int m, uint8_t *tiles, cudaStream_t st) { return split_tiles(B, m, tiles, st); }

int launch_oista_step(const OistaStep &o, int prec, cudaStream_t st)
{
    WLayer L{};
    L.Bt = o.tiles;
    L.C = o.C;
    L.Zin = o.Zs;
    L.Gin = o.Gs;
    const bool last = o.t == o.T - 1;
    L.Zout = last ? o.Zfinal : o.Zs;
    L.Gout = last ? nullptr : o.Gs;
    L.skip_mma = last ? 1 : 0;
    L.alpha = nullptr;
    L.Lp = o.L;
    L.t = o.t;
    L.m = o.m;
    L.N = o.N;
    L.lam = o.lam;
    L.refresh = refresh_at(o.t, o.T, 0, false);
    L.LSv = o.LSv;
    L.flag = o.flag;
    L.Scur = o.Scur;
    L.Sprev = o.Sprev;
    L.valid = o.valid;
    L.list = o.list;
    L.counter = o.counter;
    L.listN = o.listN;
    L.accepted = o.accepted;
    L.LS_out = o.LS_out;
    L.want_ls = o.want_ls;
    L.last = last ? 1 : 0;
    // one column block per row tile: spread the rows evenly over the SMs
    const int sms = num_sms();
    const int rounds = ceil_div(ceil_div(o.N, BM), sms);
    L.TR = o.N > 0 ? ceil_div(o.N, (long long)rounds * sms) : BM;
    const bool split = prec == SLISTA_PREC_BF16X3;
    return split ? launch_chunk<true, OIS, 1>(&L, 1, st, true) : launch_chunk<false, OIS, 1>(&L, 1, st, true);
}

int launch_forward(const PgdArgs &a, int prec, void *ws, cudaStream_t st)
{
    Problem q{};
    q.B = a.B;
    q.C = a.C;
    q.m = a.m;
    q.N = a.N;
    q.lam = a.lam;
    q.alpha = a.alpha;
    q.L = a.L;
    q.Z = a.Z;
    q.masks = a.masks;
    q.ckpt = a.ckpt;
    return forward_batch(&q, 1, a.T, a.ckpt_every, prec, ws, st);
}

int launch_backward(const BwdArgs &a, int prec, void *ws, cudaStream_t st)
{
    Problem q{};
    q.B = a.B;
    q.C = a.C;
    q.m = a.m;
    q.N = a.N;
    q.lam = a.lam;
    q.alpha = a.alpha;
    q.masks = const_cast<uint32_t *>(a.masks);
    q.ckpt = const_cast<float *>(a.ckpt);
    q.gZ = a.gZ;
    q.dalpha = a.dalpha;
    return backward_batch(&q, 1, a.T, a.ckpt_every, prec, ws, st);
}

}  // namespace tcw
}  // namespace slista
