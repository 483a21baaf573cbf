// tcgen05 products of the Gram quantities and of the objective (sm_103a):
//
//   GRAM_C :  C = X D          (rows: samples, K = n, columns: codes; also ||x_i||^2)
//   GRAM_B :  B = D^T D        (rows and columns: codes, K = n; written symmetric)
//   OBJ    :  W = Z B          (rows: samples, K = m, columns: codes), finished into
//             F_i and the duality gap in the epilogue (Eq. lasso)
//   RESID  :  R = Z D^T - X    (rows: samples, K = m, columns: atoms), the residual
//             D z - x of a coupled LISTA layer (Eq. lista_layer)
//   LSTEP  :  V = R W          (rows: samples, K = n, columns: codes), finished into
//             z <- ST(z - alpha V, beta lam) in place (Eq. lista_layer)
//
// These products feed every layer (C), define the layers (B) or are the
// final reductions (objective), so they are held to FP32 accuracy: each FP32
// operand v is split into three BF16 parts v = hi + mid + lo (hi = RN(v),
// mid = RN(v - hi), lo = RN(v - hi - mid); the differences are exact in FP32)
// and the six products whose order is at most 2^-16 relative are kept,
//   hi.hi + hi.mid + mid.hi + hi.lo + mid.mid + lo.hi,
// about 2^-24 relative per product term, like an FP32 product (the dropped
// ones are 2^-24 and below).  The tensor cores' FP32 accumulator loses up to
// an ulp of its own magnitude per accumulating MMA, so hi.hi goes into one
// accumulator (K/16 additions) and the five correction products, 2^-8
// smaller, into a second one; the epilogue adds the two (for K = 256 the
// single-accumulator form was 2e-6 off, the split one matches FP32).
//
// Both operands are split on the fly from the caller's FP32 arrays, so no
// workspace is needed:
//   A (a 128-row tile, one K chunk of 64) : every thread splits 16 values of
//       its row into tensor memory (tcgen05.st), the MMA's A operand;
//   B (256 output columns x 64 K)         : every thread splits 4 units of 8
//       K values into shared memory in the K-major 128-byte-swizzled layout.
// A CTA owns a tile of up to 128 rows and 256 output columns, done as two
// halves of 128 columns (the two accumulators of a half fill 256 tensor
// memory columns; the double-buffered A operand takes 192 more).  Chunks are
// double-buffered: while the tensor cores multiply chunk c, the threads split
// chunk c + 1.  One thread issues the 24 MMAs of a chunk (4 K-steps x 6
// products, M = 128, N = 128).  Every mbarrier wait is bounded; on expiry the
// kernel raises the device flag and exits after releasing its tensor memory.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace slista {
namespace tcg {

int read_and_clear_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, tc::tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(tc::tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "a Gram / objective kernel's bounded wait expired (device flag %d)", h);
    }
    return SLISTA_OK;
}

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int BH = 128;                       // output columns per half
constexpr int NT = 512;                       // 16 warps
constexpr int PART_B = BH * BK * 2;           // one BF16 part of a B chunk: 16 KB
constexpr int STAGE_B = 3 * PART_B;           // hi, mid, lo: 48 KB
constexpr int SMEM = 2 * STAGE_B + 1024;      // two stages (+ alignment)
constexpr int T_P = 0;                        // hi.hi accumulator: columns [0, 128)
constexpr int T_Q = 128;                      // correction accumulator: [128, 256)
constexpr int T_A = 256;                      // A buffer b, part p: [T_A + 96 b + 32 p, + 32)
constexpr int TMEM_COLS = 512;
constexpr uint32_t IDESC = idesc_bf16(BM, BH);

enum Mode { GRAM_C = 0, GRAM_B = 1, OBJ = 2, RESID = 3, LSTEP = 4 };

// Operand layouts: A(r, k) is row-major (rows x K) except for GRAM_B (A = D^T);
// Bop(j, k) is row-major (ncol x K) for OBJ and RESID, else column access of
// a K x ncol matrix.
__host__ __device__ constexpr bool b_rowmajor(int mode) { return mode == OBJ || mode == RESID; }

struct Params {
    const float *A;       // GRAM_C: X (rows x K); GRAM_B: D (K x rows, A(a, k) = D[k][a]); OBJ: Z (rows x K)
    const float *Bsrc;    // GRAM_*: D (K x ncol, Bop(j, k) = D[k][j]); OBJ: B (ncol x K, Bop(j, k) = B[j][k])
    int rows, K, ncol;
    int TR;               // rows per tile (<= 128)
    float *out;           // GRAM_C: C (rows x ncol); GRAM_B: B (ncol x ncol)
    double *xsq;          // GRAM_C: ||x_i||^2 (written by column block 0)
    const float *C;       // OBJ: correlations (rows x ncol)
    const double *xsq_in; // OBJ
    float lam;            // OBJ, LSTEP
    double *F, *gap;      // OBJ (gap nullable)
    const float *Xsub;    // RESID: X (rows x ncol), subtracted
    float *Zio;           // LSTEP: codes (rows x ncol), updated in place
    const float *alpha;   // LSTEP: alpha_t = alpha[t], threshold beta[t] lam (device)
    const float *beta;
    int t;
};

// Compensated FP32 accumulation (an unevaluated sum hi + lo): the product
// a b is split exactly into p + e with an FMA and p is added by Knuth's
// two-sum; the result carries about 48 significant bits, as an FP64
// accumulator would.
struct Acc2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = hi + v;
        const float bb = t - hi;
        lo += (hi - (t - bb)) + (v - bb);
        hi = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        add(p);
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// v = hi + mid + lo in BF16 (round to nearest at each step; the residuals
// v - hi and v - hi - mid are exact in FP32).
__device__ __forceinline__ void split3(float v0, float v1, uint32_t &h, uint32_t &m, uint32_t &l)
{
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h2);
    const float r0 = v0 - hf.x, r1 = v1 - hf.y;
    const __nv_bfloat162 m2 = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(m2);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    h = *reinterpret_cast<const uint32_t *>(&h2);
    m = *reinterpret_cast<const uint32_t *>(&m2);
    l = *reinterpret_cast<const uint32_t *>(&l2);
}

// A of chunk c: 16 values of this thread's row (K positions k0 .. k0 + 15),
// loaded one chunk ahead (load_a) and split into tensor memory at column ta
// (+ 32 per part) when their chunk comes (store_a).
template <int MODE>
__device__ __forceinline__ void load_a(const Params &p, int row, bool rok, int k0, float (&v)[16])
{
    if (MODE == GRAM_B) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = (rok && k0 + j < p.K) ? __ldg(p.A + (size_t)(k0 + j) * p.rows + row) : 0.0f;
    } else {
        const float *src = p.A + (size_t)row * p.K + k0;
        if (rok && k0 + 16 <= p.K && (p.K & 3) == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 x = __ldg(reinterpret_cast<const float4 *>(src) + u);
                v[4 * u] = x.x;
                v[4 * u + 1] = x.y;
                v[4 * u + 2] = x.z;
                v[4 * u + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (rok && k0 + j < p.K) ? __ldg(src + j) : 0.0f;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void store_a(const float (&v)[16], uint32_t ta, Acc2 *xx)
{
    if (MODE == GRAM_C && xx)
#pragma unroll
        for (int j = 0; j < 16; ++j) xx->add_prod(v[j], v[j]);
    uint32_t h[8], mi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split3(v[2 * j], v[2 * j + 1], h[j], mi[j], lo[j]);
    tmem_st8(ta, h);
    tmem_st8(ta + 32, mi);
    tmem_st8(ta + 64, lo);
}

// B of chunk c for output columns hc0 .. hc0 + BH - 1: units of 8 K values of
// one column (unit u = tid + NT i), loaded one chunk ahead (load_b) and split
// into the three parts of stage `stage` when their chunk comes (store_b).
constexpr int BUNITS = BH * BK / 8 / NT;  // units per thread
static_assert(BUNITS * NT * 8 == BH * BK, "B units");

template <int MODE>
__device__ __forceinline__ void unit_pos(int u, int &jr, int &ku)
{
    if (b_rowmajor(MODE)) {  // Bop(j, k) = B[j][k]: eight threads share a 256-byte row segment
        jr = u >> 3;
        ku = u & 7;
    } else {                 // Bop(j, k) = D[k][j]: a warp reads 32 consecutive columns per row
        jr = u & (BH - 1);
        ku = u / BH;
    }
}

template <int MODE>
__device__ __forceinline__ void load_b(const Params &p, int hc0, int kc0, int tid, float (&v)[BUNITS][8])
{
#pragma unroll
    for (int i = 0; i < BUNITS; ++i) {
        int jr, ku;
        unit_pos<MODE>(tid + NT * i, jr, ku);
        const int j = hc0 + jr, k = kc0 + 8 * ku;
        if (b_rowmajor(MODE)) {
            const float *src = p.Bsrc + (size_t)j * p.K + k;
            if (j < p.ncol && k + 8 <= p.K && (p.K & 3) == 0 && (reinterpret_cast<uintptr_t>(p.Bsrc) & 15) == 0) {
                const float4 x0 = __ldg(reinterpret_cast<const float4 *>(src));
                const float4 x1 = __ldg(reinterpret_cast<const float4 *>(src) + 1);
                v[i][0] = x0.x; v[i][1] = x0.y; v[i][2] = x0.z; v[i][3] = x0.w;
                v[i][4] = x1.x; v[i][5] = x1.y; v[i][6] = x1.z; v[i][7] = x1.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[i][e] = (j < p.ncol && k + e < p.K) ? __ldg(src + e) : 0.0f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                v[i][e] = (j < p.ncol && k + e < p.K) ? __ldg(p.Bsrc + (size_t)(k + e) * p.ncol + j) : 0.0f;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void store_b(const float (&v)[BUNITS][8], uint8_t *stage, int tid)
{
#pragma unroll
    for (int i = 0; i < BUNITS; ++i) {
        int jr, ku;
        unit_pos<MODE>(tid + NT * i, jr, ku);
        uint32_t h[4], mi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split3(v[i][2 * e], v[i][2 * e + 1], h[e], mi[e], lo[e]);
        const uint32_t off = sw128_offset(BH, jr, 8 * ku);
        *reinterpret_cast<uint4 *>(stage + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(stage + PART_B + off) = make_uint4(mi[0], mi[1], mi[2], mi[3]);
        *reinterpret_cast<uint4 *>(stage + 2 * PART_B + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// One output tile (block `blk` of the mode's grid) of the kernels below.
template <int MODE>
__device__ __forceinline__ void gemm_block(const Params &p, int blk)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2];  // done[b]: the MMAs of the chunk in buffer b retired
    __shared__ uint32_t tmem_slot;
    __shared__ double red[4][4][BM];            // per-row partial sums of the four column groups
    __shared__ float redf[4][BM];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, cg = warp >> 2;     // TMEM lane quadrant, column group
    const int ncb = (p.ncol + BN - 1) / BN;
    const int tile = blk / ncb, cb = blk % ncb;
    const int row0 = tile * p.TR, col0 = cb * BN;
    const int rl = 32 * q + lane;               // tile row of this thread (TMEM lane)
    const int row = row0 + rl;
    const bool rok = rl < p.TR && row < p.rows;
    const int nkc = (p.K + BK - 1) / BK;
    const int ncols = p.ncol - col0 < BN ? p.ncol - col0 : BN;
    const int nh = (ncols + BH - 1) / BH;       // halves of this column block

    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sb = smem_u32(smem);
    const uint32_t done0 = smem_u32(&bars[0]);
    if (tid == 0) {
        mbar_init(done0, 1);
        mbar_init(done0 + 8, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);

    Acc2 xx;               // GRAM_C: ||x||^2 of this thread's share of the row
    Acc2 cz, zw, l1;       // OBJ: c.z, z.(Bz), ||z||_1 of this thread's columns
    float cinf = 0.0f;     // OBJ: max |c - Bz| of this thread's columns
    bool failed = false;
    int it = 0;            // chunk iterations so far: buffer it & 1
    // the operands of the first chunk; each iteration loads the next one's
    // before it issues its products, so the loads' latency overlaps them
    float va[16], vb[BUNITS][8];
    load_a<MODE>(p, row, rok, 16 * cg, va);
    load_b<MODE>(p, col0, 0, tid, vb);
#pragma unroll 1
    for (int h = 0; h < nh && !failed; ++h) {
        const int hc0 = col0 + h * BH;
#pragma unroll 1
        for (int c = 0; c < nkc; ++c, ++it) {
            const int b = it & 1;
            if (it >= 2) {  // buffer b is free once the MMAs of iteration it - 2 have retired
                const bool ok = mbar_wait(done0 + 8 * b, ((it >> 1) - 1) & 1, 31);
                failed = __syncthreads_or(!ok) != 0;
                if (failed) break;
                tc_fence_after();
            }
            // the A operand does not depend on the half: the first half's ||x||^2 only
            store_a<MODE>(va, tlane + T_A + 96 * b + 8 * cg, h == 0 ? &xx : nullptr);
            store_b<MODE>(vb, smem + b * STAGE_B, tid);
            {
                const bool more_c = c + 1 < nkc;
                if (more_c || h + 1 < nh) {
                    const int cn = more_c ? c + 1 : 0, hn = more_c ? hc0 : hc0 + BH;
                    load_a<MODE>(p, row, rok, cn * BK + 16 * cg, va);
                    load_b<MODE>(p, hn, cn * BK, tid, vb);
                }
            }
            tmem_st_wait();
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t bst = sb + b * STAGE_B;
                // (A part, B part) of the six kept products: hi.hi into P, the rest into Q
                const int pa[6] = {0, 0, 1, 0, 1, 2};
                const int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
#pragma unroll
                    for (int r = 0; r < 6; ++r) {
                        const uint32_t acc = r == 0 ? ((c | kk) ? 1u : 0u) : ((c | kk | (r > 1)) ? 1u : 0u);
                        mma_ts(tmem + (r == 0 ? T_P : T_Q), tmem + T_A + 96 * b + 32 * pa[r] + 8 * kk,
                               sdesc_sw128(bst + pb[r] * PART_B + kk * 32), IDESC, acc);
                    }
                mma_commit(done0 + 8 * b);
            }
        }
        if (failed) break;
        {  // the last commit of the half fires once every MMA issued before it has retired
            const int il = it - 1;
            const bool ok = mbar_wait(done0 + 8 * (il & 1), (il >> 1) & 1, 32);
            failed = __syncthreads_or(!ok) != 0;
            if (failed) break;
        }
        tc_fence_after();
        // --- epilogue of the half: columns [32 cg, 32 cg + 32) of this thread's row
#pragma unroll 1
        for (int pc = 0; pc < 2; ++pc) {
            float w[16], wq[16];
            tmem_ld16(tlane + T_P + 32 * cg + 16 * pc, w);
            tmem_ld16(tlane + T_Q + 32 * cg + 16 * pc, wq);
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] += wq[j];
            const int j0 = hc0 + 32 * cg + 16 * pc;
            if (MODE == RESID && rok) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j0 + j < p.ncol) w[j] -= __ldg(p.Xsub + (size_t)row * p.ncol + j0 + j);
            }
            if (MODE == LSTEP) {
                if (rok) {
                    const float step = __ldg(p.alpha + p.t), thr = __fmul_rn(__ldg(p.beta + p.t), p.lam);
                    float *zp = p.Zio + (size_t)row * p.ncol + j0;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j0 + j < p.ncol) {
                            const float u = fmaf(-step, w[j], zp[j]);
                            zp[j] = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                        }
                }
            } else if (MODE == GRAM_C || MODE == RESID) {
                if (rok) {
                    float *dst = p.out + (size_t)row * p.ncol + j0;
                    if (j0 + 16 <= p.ncol && (p.ncol & 3) == 0 && (reinterpret_cast<uintptr_t>(p.out) & 15) == 0) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            reinterpret_cast<float4 *>(dst)[u] =
                                make_float4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (j0 + j < p.ncol) dst[j] = w[j];
                    }
                }
            } else if (MODE == GRAM_B) {
                // B is symmetric: entry (a, b) with b >= a is written to both
                // places from this one value, so B == B^T exactly
                if (rok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int bcol = j0 + j;
                        if (bcol < p.ncol && bcol >= row) {
                            p.out[(size_t)row * p.ncol + bcol] = w[j];
                            p.out[(size_t)bcol * p.ncol + row] = w[j];
                        }
                    }
                }
            } else {  // OBJ
                float zr[16], cr[16];
                const float *zs = p.A + (size_t)row * p.K + j0;
                const float *cs = p.C + (size_t)row * p.ncol + j0;
                if (rok && j0 + 16 <= p.ncol && (p.ncol & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(p.A) | reinterpret_cast<uintptr_t>(p.C)) & 15) == 0) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 a4 = __ldg(reinterpret_cast<const float4 *>(zs) + u);
                        const float4 c4 = __ldg(reinterpret_cast<const float4 *>(cs) + u);
                        zr[4 * u] = a4.x; zr[4 * u + 1] = a4.y; zr[4 * u + 2] = a4.z; zr[4 * u + 3] = a4.w;
                        cr[4 * u] = c4.x; cr[4 * u + 1] = c4.y; cr[4 * u + 2] = c4.z; cr[4 * u + 3] = c4.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const bool ok = rok && j0 + j < p.ncol;
                        zr[j] = ok ? __ldg(zs + j) : 0.0f;
                        cr[j] = ok ? __ldg(cs + j) : 0.0f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const bool ok = rok && j0 + j < p.ncol;
                    const float z = zr[j], cc = cr[j];
                    cz.add_prod(cc, z);
                    zw.add_prod(z, w[j]);
                    l1.add(fabsf(z));
                    if (ok) cinf = fmaxf(cinf, fabsf(cc - w[j]));
                }
            }
        }
        // the next half's products overwrite the accumulators
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    if (!failed) {
        if (MODE == GRAM_C && cb == 0) {  // ||x_i||^2: the four column groups' shares, in a fixed order
            red[0][cg][rl] = (double)xx.hi;
            red[1][cg][rl] = (double)xx.lo;
            __syncthreads();
            if (cg == 0 && rok) {
                double s = 0.0;
#pragma unroll
                for (int g = 0; g < 4; ++g) s += red[0][g][rl] + red[1][g][rl];
                p.xsq[row] = s;
            }
        } else if (MODE == OBJ) {  // F_i = 1/2 xsq - c^T z + 1/2 z^T (B z) + lam ||z||_1; gap from ||c - Bz||_inf
            red[0][cg][rl] = cz.value();
            red[1][cg][rl] = zw.value();
            red[2][cg][rl] = l1.value();
            redf[cg][rl] = cinf;
            __syncthreads();
            if (cg == 0 && rok) {
                double scz = 0.0, szw = 0.0, sl1 = 0.0;
                float ci = 0.0f;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    scz += red[0][g][rl];
                    szw += red[1][g][rl];
                    sl1 += red[2][g][rl];
                    ci = fmaxf(ci, redf[g][rl]);
                }
                const double xv = p.xsq_in[row];
                const double Fv = 0.5 * xv - scz + 0.5 * szw + (double)p.lam * sl1;
                p.F[row] = Fv;
                if (p.gap) {
                    const double r2 = xv - 2.0 * scz + szw;
                    const double xr = xv - scz;
                    const double s = (double)ci > (double)p.lam ? (double)p.lam / (double)ci : 1.0;
                    p.gap[row] = Fv - (s * xr - 0.5 * s * s * r2);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <int MODE>
__global__ void __launch_bounds__(NT, 1) tc6_gemm_kernel(const Params p)
{
    gemm_block<MODE>(p, (int)blockIdx.x);
}

// B = D^T D and C = X D (with ||x||^2) in one launch: blocks [0, nb) form B,
// the others C.
__global__ void __launch_bounds__(NT, 1) tc6_gram_kernel(const Params pb, const Params pc, int nb)
{
    if ((int)blockIdx.x < nb)
        gemm_block<GRAM_B>(pb, (int)blockIdx.x);
    else
        gemm_block<GRAM_C>(pc, (int)blockIdx.x - nb);
}

namespace {

// Rows per tile: a tile costs the same MMA time for any number of rows up to
// 128, so the rows are spread evenly over rounds x SMs tiles (x column blocks).
int rows_per_tile(int rows, int ncb)
{
    const int sms = num_sms();
    const int per_round = sms / (ncb < sms ? ncb : sms);
    const int rounds = ceil_div(ceil_div(rows, BM), per_round > 0 ? per_round : 1);
    const int tr = ceil_div(rows, (long long)rounds * (per_round > 0 ? per_round : 1));
    return tr < 1 ? 1 : (tr > BM ? BM : tr);
}

// Sets p.TR; returns the number of blocks of the mode's grid.
int grid_of(Params &p)
{
    if (p.rows <= 0 || p.ncol <= 0) return 0;
    const int ncb = ceil_div(p.ncol, BN);
    p.TR = rows_per_tile(p.rows, ncb);
    return ceil_div(p.rows, p.TR) * ncb;
}

template <int MODE>
int launch(const Params &p0, cudaStream_t st, const char *name)
{
    if (p0.rows <= 0 || p0.ncol <= 0) return SLISTA_OK;
    Params p = p0;
    const int ncb = ceil_div(p.ncol, BN);
    p.TR = rows_per_tile(p.rows, ncb);
    const int ntiles = ceil_div(p.rows, p.TR);
    auto k = tc6_gemm_kernel<MODE>;
    SLISTA_CUDA_TRY(allow_smem(k, SMEM));
    k<<<ntiles * ncb, NT, SMEM, st>>>(p);
    return check_launch(name);
}

}  // namespace

int launch_gram(const float *D, int n, int m, const float *X, int N, float *B, float *C, double *xsq, cudaStream_t st)
{
    Params pb{};
    pb.A = D;
    pb.Bsrc = D;
    pb.rows = m;
    pb.K = n;
    pb.ncol = m;
    pb.out = B;
    Params pc{};
    pc.A = X;
    pc.Bsrc = D;
    pc.rows = N;
    pc.K = n;
    pc.ncol = m;
    pc.out = C;
    pc.xsq = xsq;
    const int nb = grid_of(pb), nc = grid_of(pc);
    if (nb + nc == 0) return SLISTA_OK;
    SLISTA_CUDA_TRY(allow_smem(tc6_gram_kernel, SMEM));
    tc6_gram_kernel<<<nb + nc, NT, SMEM, st>>>(pb, pc, nb);
    return check_launch("tc6_gram_kernel");
}

bool objective_supported(int m) { return m >= 1 && m <= BN; }

int launch_objective(const ObjArgs &a, cudaStream_t st)
{
    Params p{};
    p.A = a.Z;
    p.Bsrc = a.B;
    p.rows = a.N;
    p.K = a.m;
    p.ncol = a.m;
    p.C = a.C;
    p.xsq_in = a.xsq;
    p.lam = a.lam;
    p.F = a.F;
    p.gap = a.gap;
    return launch<OBJ>(p, st, "tc6_gemm_kernel (objective)");
}

size_t lista_ws_bytes(int n, int N) { return N > 0 ? (size_t)N * n * sizeof(float) + 256 : 0; }

int launch_lista(const ListaArgs &a, void *ws, cudaStream_t st)
{
    if (a.N == 0) return SLISTA_OK;
    SLISTA_CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(float) * (size_t)a.N * a.m, st));  // z^(0) = 0
    float *R = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255);
    for (int t = 0; t < a.T; ++t) {
        Params pr{};  // R = Z D^T - X  (the residual D z - x of every sample)
        pr.A = a.Z;
        pr.Bsrc = a.D;
        pr.rows = a.N;
        pr.K = a.m;
        pr.ncol = a.n;
        pr.out = R;
        pr.Xsub = a.X;
        int rc = launch<RESID>(pr, st, "tc6_gemm_kernel (LISTA residual)");
        if (rc) return rc;
        Params pl{};  // z <- ST(z - alpha_t (R W_t), beta_t lam)
        pl.A = R;
        pl.Bsrc = a.W + (size_t)t * a.n * a.m;
        pl.rows = a.N;
        pl.K = a.n;
        pl.ncol = a.m;
        pl.Zio = a.Z;
        pl.alpha = a.alpha;
        pl.beta = a.beta;
        pl.lam = a.lam;
        pl.t = t;
        rc = launch<LSTEP>(pl, st, "tc6_gemm_kernel (LISTA step)");
        if (rc) return rc;
    }
    return SLISTA_OK;
}

}  // namespace tcg
}  // namespace slista
