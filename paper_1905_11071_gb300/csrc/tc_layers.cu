// tcgen05 (sm_103a tensor core) forward kernel for the unfolded
// proximal-gradient layers (Eq. pgd / Eq. steprec): ISTA and Step-LISTA.
//
// Per CTA: a tile of up to 128 samples (MMA M = 128), all T layers, persistent
// over tiles.  The per-sample state is
//   g = c - B z   in tensor memory, as the FP32 accumulator of the MMA, and
//   z             in registers (thread = one sample row, one half of the codes).
// A layer is the epilogue
//   u = z + alpha_t g,  z' = ST(u, alpha_t lam),  a = z - z'   (FP32)
// followed by the contraction g <- g + a B (B symmetric), issued as
//   tcgen05.mma  D[tmem] += A[tmem] x B[smem]    (kind::f16, BF16 in, FP32 acc)
// with a split into BF16 parts a = a_hi + a_lo and B = B_hi + B_lo:
//   BF16   : a_hi B_hi
//   BF16X3 : a_hi B_hi + a_lo B_hi + a_hi B_lo   (a_lo B_lo dropped)
// Every REFRESH layers the same products rebuild g from scratch instead:
// the accumulator is reloaded with c and the A operand is -z', so the MMAs
// produce g = c - B z' (bounded rounding drift, same MMA count).
// The epilogue writes a_hi / a_lo straight into tensor memory as the MMA's
// A operand (tcgen05.st); B_hi (and B_lo for m <= 128) stay resident in
// shared memory in the K-major 128-byte-swizzled layout; for m = 256 B_lo is
// streamed per layer from L2 through a two-stage ring of bulk copies.
// C is read once per tile and Z written once: no per-layer HBM traffic.
//
// Tensor-memory columns: [0, MP) g;  [MP, MP + MP/2) a_hi;  [MP + MP/2, 2 MP) a_lo.
// Every wait on an mbarrier is bounded (about one second); on expiry the
// kernel raises the library's device flag, stops issuing work and exits after
// releasing its tensor memory.
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc_engine.cuh"
#include "tc_ptx.cuh"

namespace slista {

int read_and_clear_device_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, tc::tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(tc::tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "a kernel's bounded wait expired (device flag %d)", h);
    }
    int rc = tcw::read_and_clear_flag(st);
    int rc2 = tcg::read_and_clear_flag(st);
    int rc3 = tco::read_and_clear_flag(st);
    return rc ? rc : rc2 ? rc2 : rc3;
}

namespace tc {

// Failure-detection check: one thread waits, with the kernels' bounded wait,
// on an mbarrier that nothing arrives at, so the wait expires after
// `limit` cycles and raises the device flag exactly as an expired wait of a
// layer kernel does (code 7).  No copy, MMA or tensor memory is involved.
__global__ void wait_probe_kernel(long long limit)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
        mbar_wait(smem_u32(&bar), 0, 7, limit);  // phase 0 never completes
    }
}

int launch_wait_probe(long long limit_cycles, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(limit_cycles);
    return check_launch("wait_probe_kernel");
}

// ---------------------------------------------------------------------------
// Prep: B (m x m FP32) -> B_hi, B_lo (BF16, zero-padded to MP, swizzled).
// ---------------------------------------------------------------------------
__global__ void split_b_kernel(const float *__restrict__ B, int m, int MP, uint8_t *__restrict__ out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= MP * MP) return;
    const int n = idx / MP, k = idx % MP;
    const float v = (n < m && k < m) ? __ldg(B + (size_t)n * m + k) : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const uint32_t off = sw128_offset(MP, n, k);
    *reinterpret_cast<__nv_bfloat16 *>(out + off) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(out + (size_t)MP * MP * 2 + off) = lo;
}

template <int MP>
__device__ __forceinline__ size_t lane_index(int s, int ntiles, int tile, int quad, int col, int lane)
{
    return ((((size_t)s * ntiles + tile) * 4 + quad) * MP + col) * 32 + lane;
}

struct TcParams {
    const uint8_t *Bsplit;
    const float *C;
    int m, N;
    float lam;
    const float *alpha;   // T steps, or nullptr: 1/L
    const double *Lp;
    int T;
    float *Z;
    uint32_t *masks;
    float *ckpt;          // forward: written; recompute / adjoint: read (const)
    int K;                // checkpoint spacing
    int TR;               // rows per tile
    // recompute and adjoint
    int t0, t1;           // layer range [t0, t1)
    float *qbuf;          // (t1 - t0) layers of g^(t) - lam sign(z^(t+1)), tile layout (lane_index)
    float *Gbuf;          // adjoint state G, tile layout (lane_index)
    int ntiles;           // tiles of the batch (the tile layout's extent)
    const float *gZ;      // nullable upstream gradient
    int want_gT;          // recompute: form G_T after the last layer
    float *partial;       // T x gridDim.x per-CTA sums of dalpha
    const float *Ginit;   // adjoint: initial G row-major (N x m) instead of Gbuf (nullable)
    int traj_steps;       // adjoint over a trajectory: slot t holds a_t unless layer t refreshed
};

// ---------------------------------------------------------------------------
// Kernel modes (KM):
// Forward (KM_FWD): T layers from z = 0, g = c, writing Z, masks and
// checkpoints.  Forward with trajectory (KM_TRAJ): the same, without
// checkpoints, also writing q_t of every layer into slot t of qbuf and, after
// one more contraction, dF/dz^(T) = -g^(T) + lam sign(z^(T)) into slot T (the
// inputs of the adjoint, which then needs no recompute).
// Recompute (KM_RECOMP): layers [t0, t1) from the
// checkpoint at t0 with the forward's arithmetic, writing q_t per layer and,
// for the last segment, G_T = gZ or dF/dz^(T) = -g^(T) + lam sign(z^(T)).
// Thread (warp w, lane l): tile row 32*(w%4) + l, code columns
// [CW*(w/4), CW*(w/4) + CW), z of those columns in registers.
// ---------------------------------------------------------------------------
enum { KM_FWD = 0, KM_RECOMP = 1, KM_TRAJ = 2 };

template <int MP, bool SPLIT, int KM>
__global__ void __launch_bounds__(Cfg<MP, SPLIT>::NT, 1) tc_pgd_forward_kernel(const TcParams p)
{
    constexpr bool RECOMP = KM == KM_RECOMP;
    constexpr bool WRITE_Q = KM != KM_FWD;
    using CF = Cfg<MP, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cbase = (warp >> 2) * CF::CW;
    const int N = p.N, m = p.m, TR = p.TR;
    const int ntiles = (N + TR - 1) / TR;  // TR <= 128 rows per tile (lanes >= TR idle)
    const int W = (m + 31) / 32;
    const float lam = p.lam;
    const float *__restrict__ Cg = p.C;
    const float *__restrict__ alpha = p.alpha;
    float *__restrict__ ckpt = p.ckpt;
    TcEngine<MP, SPLIT> E;
    E.init(smem_raw, p.Bsplit, blockIdx.x < ntiles);
    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(p.Lp));
    const int tb = RECOMP ? p.t0 : 0, te = RECOMP ? p.t1 : p.T;

#pragma unroll 1
    for (int tile = blockIdx.x; tile < ntiles && !E.failed; tile += gridDim.x) {
        const int row = tile * TR + quad * 32 + lane;
        const bool row_ok = (quad * 32 + lane < TR) && row < N;
        float z[CF::CW];
        if (!RECOMP || tb == 0) {  // g <- c, z <- 0
#pragma unroll 1
            for (int pc = 0; pc < CF::NPC; ++pc)
                row16_to_tmem(E, Cg, row, row_ok, m, cbase + 16 * pc, CF::T_G + cbase + 16 * pc);
#pragma unroll
            for (int j = 0; j < CF::CW; ++j) z[j] = 0.0f;
        } else {  // (z, g) from the checkpoint at layer tb
            const float *ck = ckpt + (size_t)(tb / p.K - 1) * 2 * N * m;
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                const int col0 = cbase + 16 * pc;
                row16_to_tmem(E, ck + (size_t)N * m, row, row_ok, m, col0, CF::T_G + col0);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    z[16 * pc + j] = (row_ok && col0 + j < m) ? __ldg(ck + (size_t)row * m + col0 + j) : 0.0f;
            }
        }
        tmem_st_wait();

#pragma unroll 1
        for (int t = tb; t < te; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = __fmul_rn(a, lam);
            if constexpr (!RECOMP) {
                if (ckpt && t > 0 && t % p.K == 0) {
                    // checkpoint (z^(t), g^(t)) every K layers, layout of slista_forward
                    float *ck = ckpt + (size_t)(t / p.K - 1) * 2 * N * m;
                    float *wbuf = E.warp_stage();
                    const int rbase = tile * TR + quad * 32;
                    const int nrow = max(0, min(min(32, TR - quad * 32), N - rbase));
#pragma unroll
                    for (int pc = 0; pc < CF::NPC; ++pc) {
                        const int col0 = cbase + 16 * pc;
                        float gv[16];
                        tmem_ld16(E.taddr(CF::T_G + col0), gv);
                        stage_put(wbuf, gv);
                        stage_to_global(wbuf, ck + (size_t)N * m, rbase, nrow, m, col0);
#pragma unroll
                        for (int j = 0; j < 16; ++j) gv[j] = z[16 * pc + j];
                        stage_put(wbuf, gv);
                        stage_to_global(wbuf, ck, rbase, nrow, m, col0);
                    }
                }
            }
            const bool last = (t == te - 1);
            const bool contract_after = !last || KM == KM_TRAJ || (RECOMP && p.want_gT);
            // --- epilogue: z update and the split step a = z - z' into tensor memory
            // (a = -z' on refresh layers, whose accumulator is reloaded with c)
            const bool refresh = ckpt ? ((t + 1) % p.K == 0) : ((t + 1) % REFRESH == 0);
            uint32_t word = 0u;
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                const int col0 = cbase + 16 * pc;
                float gv[16];
                tmem_ld16(E.taddr(CF::T_G + col0), gv);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float zo = z[16 * pc + j];
                    const float u = fmaf(a, gv[j], zo);
                    const float zn = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                    gv[j] = refresh ? -zn : zo - zn;  // the MMA's A operand
                    z[16 * pc + j] = zn;
                    word |= (uint32_t)(zn != 0.0f) << (16 * (pc & 1) + j);
                }
                store_split16(E, col0, gv);
                if constexpr (!RECOMP) {
                    if ((pc & 1) && p.masks && row_ok && ((col0 - 16) >> 5) < W)
                        p.masks[((size_t)t * N + row) * W + ((col0 - 16) >> 5)] = word;
                }
                if (pc & 1) word = 0u;
            }
            // trajectory slot t (KM_TRAJ): on layers without a refresh the step
            // a_t = z^(t) - z^(t+1), read back from the A operand while the
            // products run (on the support of z^(t+1), q_t = -a_t / alpha_t);
            // on refresh layers, and in the recompute, q_t itself, before them
            const bool step_slot = KM == KM_TRAJ && !refresh;
            if (WRITE_Q && !step_slot) {
                // q_t = g^(t) - lam sign(z^(t+1)) in a second pass over the
                // accumulator (still g^(t)), off the first pass's register
                // budget; every lane takes part in the (warp-wide) loads
                float *qt = p.qbuf + lane_index<MP>(t - tb, p.ntiles, tile, quad, 0, lane);
#pragma unroll
                for (int pc = 0; pc < CF::NPC; ++pc) {
                    const int col0 = cbase + 16 * pc;
                    float gv[16];
                    tmem_ld16(E.taddr(CF::T_G + col0), gv);
                    if (row_ok)
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float zn = z[16 * pc + j];
                            // the adjoint reads q_t only on the support of z^(t+1)
                            if (col0 + j < m && zn != 0.0f)
                                qt[(size_t)(col0 + j) * 32] = gv[j] - lam * (float)((zn > 0.0f) - (zn < 0.0f));
                        }
                }
            }
            if (refresh && contract_after) {
#pragma unroll 1
                for (int pc = 0; pc < CF::NPC; ++pc)
                    row16_to_tmem(E, Cg, row, row_ok, m, cbase + 16 * pc, CF::T_G + cbase + 16 * pc);
            }
            tmem_st_wait();
            if (!contract_after) break;
            // --- contraction g += a B on the tensor cores
            E.contract_issue(false);
            if (step_slot) {
                // only codes in the support of z^(t+1) are written: the adjoint reads no others
                float *qt = p.qbuf + lane_index<MP>(t - tb, p.ntiles, tile, quad, 0, lane);
#pragma unroll 1
                for (int pc = 0; pc < CF::NPC; ++pc) {
                    const int col0 = cbase + 16 * pc;
                    // support bits of these codes: the mask word this thread just stored
                    // (read back through the coherent path, off the register budget)
                    uint32_t wd = 0u;
                    if (row_ok && col0 < m) wd = p.masks[((size_t)t * N + row) * W + (col0 >> 5)] >> (col0 & 31);
                    uint32_t hv[8], lv[8];
                    tmem_ld8(E.taddr(CF::T_AHI + col0 / 2), hv);
                    if (SPLIT) tmem_ld8(E.taddr(CF::T_ALO + col0 / 2), lv);
                    if (row_ok)
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const float2 h = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hv[jj]));
                            float2 a2 = h;
                            if (SPLIT) {
                                const float2 l = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lv[jj]));
                                a2.x += l.x;
                                a2.y += l.y;
                            }
                            if ((wd >> (2 * jj)) & 1u) qt[(size_t)(col0 + 2 * jj) * 32] = a2.x;
                            if ((wd >> (2 * jj + 1)) & 1u) qt[(size_t)(col0 + 2 * jj + 1) * 32] = a2.y;
                        }
                }
            }
            {
                // this tile's rows of C into L2 before a refresh layer reloads them
                const bool refresh_next = ckpt ? ((t + 2) % p.K == 0) : ((t + 2) % REFRESH == 0);
                if (refresh_next && row_ok && !last)
#pragma unroll
                    for (int c = 0; c < CF::CW; c += 32)
                        if (cbase + c < m) prefetch_l2(Cg + (size_t)row * m + cbase + c);
            }
            if (!E.contract_wait()) break;
            if constexpr (WRITE_Q) {
                if (last) {
                    // G_T = gZ, or dF/dz^(T) = B z - c + lam sign(z) = -g + lam sign(z); the
                    // trajectory keeps the latter in slot T of qbuf
                    float *gt = RECOMP ? p.Gbuf + lane_index<MP>(0, p.ntiles, tile, quad, 0, lane)
                                       : p.qbuf + lane_index<MP>(te - tb, p.ntiles, tile, quad, 0, lane);
                    const float *gz = RECOMP ? p.gZ : nullptr;
#pragma unroll
                    for (int pc = 0; pc < CF::NPC; ++pc) {
                        const int col0 = cbase + 16 * pc;
                        float gv[16];
                        tmem_ld16(E.taddr(CF::T_G + col0), gv);
                        if (row_ok)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (col0 + j < m) {
                                    const size_t o = (size_t)row * m + col0 + j;
                                    const float zj = z[16 * pc + j];
                                    gt[(size_t)(col0 + j) * 32] =
                                        gz ? __ldg(gz + o) : -gv[j] + lam * (float)((zj > 0.0f) - (zj < 0.0f));
                                }
                    }
                }
            }
        }
        if (E.failed) break;
        if constexpr (!RECOMP) {
            float *wbuf = E.warp_stage();
            const int rbase = tile * TR + quad * 32;
            const int nrow = max(0, min(min(32, TR - quad * 32), N - rbase));
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = z[16 * pc + j];
                stage_put(wbuf, v);
                stage_to_global(wbuf, p.Z, rbase, nrow, m, cbase + 16 * pc);
            }
        }
        E.tile_done();
    }
    E.finish();
}

// ---------------------------------------------------------------------------
// Adjoint of Eq. steprec over the layers [t0, t1), walked backwards, for the
// state G in Gbuf (updated in place):
//   h = G * mask_t;  dalpha_t += <h, q_t>;  G = h - alpha_t B h
// with B h on the tensor cores (split products into a fresh accumulator).
// Per-CTA sums of dalpha_t go to partial[t * gridDim.x + block].
// ---------------------------------------------------------------------------
template <int MP, bool SPLIT>
__global__ void __launch_bounds__(Cfg<MP, SPLIT>::NT, 1) tc_adjoint_kernel(const TcParams p)
{
    using CF = Cfg<MP, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    // per-warp sums of dalpha_t over this CTA's tiles, reduced once at the end
    // (a warp writes only its own column: no barrier per layer)
    __shared__ float part_w[ADJ_KMAX][CF::NT / 32];
    // this thread's support words of the next layer, copied in (cp.async) while
    // the current layer's products run; double-buffered by layer parity
    constexpr int NW = CF::CW / 32;
    __shared__ uint32_t s_mw[2][CF::NT][NW];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cbase = (warp >> 2) * CF::CW;
    const int N = p.N, m = p.m, TR = p.TR;
    const int ntiles = (N + TR - 1) / TR;
    const int W = (m + 31) / 32;
    const float *__restrict__ alpha = p.alpha;
    const uint32_t *__restrict__ masks = p.masks;
    const float *__restrict__ qbuf = p.qbuf;  // q_t, or (trajectory) the step a_t on layers without a refresh
    float *__restrict__ Gbuf = p.Gbuf;
    TcEngine<MP, SPLIT> E;
    E.init(smem_raw, p.Bsplit, blockIdx.x < ntiles);
    if (lane == 0)
        for (int t = 0; t < p.t1 - p.t0; ++t) part_w[t][warp] = 0.0f;

#pragma unroll 1
    for (int tile = blockIdx.x; tile < ntiles && !E.failed; tile += gridDim.x) {
        const int row = tile * TR + quad * 32 + lane;
        const bool row_ok = (quad * 32 + lane < TR) && row < N;
        // the warp's q lines are worth prefetching when at least 8 of its 32
        // rows hold samples: a prefetch brings the whole 128-byte line of a
        // code, the demand loads of a few rows only their 32-byte sectors (a
        // 66-row tile's third quad has 2 rows: prefetching its lines read
        // 16 times the bytes it uses)
        const int quad_rows = min(min(TR, N - tile * TR) - quad * 32, 32);
        const bool quad_live = quad_rows >= 8;
        auto fetch_masks = [&](int tt) {
            if (row_ok) {
#pragma unroll
                for (int i = 0; i < NW; ++i)
                    if (cbase + 32 * i < m)
                        cp_async4(smem_u32(&s_mw[tt & 1][tid][i]), masks + ((size_t)tt * N + row) * W + ((cbase >> 5) + i));
            }
            cp_async_commit();
        };
        fetch_masks(p.t1 - 1);
        float G[CF::CW];
        if (p.Ginit) {
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                uint32_t v[16];
                load_c16(p.Ginit, row, row_ok, m, cbase + 16 * pc, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) G[16 * pc + j] = __uint_as_float(v[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < CF::CW; ++j)
                G[j] = (row_ok && cbase + j < m) ? Gbuf[lane_index<MP>(0, p.ntiles, tile, quad, cbase + j, lane)]
                                                 : 0.0f;
        }
#pragma unroll 1
        for (int t = p.t1 - 1; t >= p.t0; --t) {
            const float a = __ldg(alpha + t);
            const float *qt = qbuf + lane_index<MP>(t - p.t0, p.ntiles, tile, quad, 0, lane);  // + 32 per code
            float part = 0.0f;
            cp_async_wait_all();  // this layer's support words have landed
            uint32_t wd[NW];  // this row's support bits of the thread's code columns (zero past m and N)
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const int col0 = cbase + 32 * i;
                const uint32_t valid = col0 + 32 <= m ? 0xffffffffu : col0 < m ? (1u << (m - col0)) - 1u : 0u;
                wd[i] = row_ok ? s_mw[t & 1][tid][i] & valid : 0u;
            }
            if (t - 1 >= p.t0) fetch_masks(t - 1);  // in flight during this layer
            // h = G * mask_t, split into tensor memory as the products' A operand
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                const int col0 = cbase + 16 * pc;
                const uint32_t word = wd[pc >> 1] >> (16 * (pc & 1));
                float hv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    G[16 * pc + j] = ((word >> j) & 1u) ? G[16 * pc + j] : 0.0f;
                    hv[j] = G[16 * pc + j];
                }
                store_split16(E, col0, hv);
            }
            tmem_st_wait();
            if (t > 0) {
                if (t - 1 >= p.t0 && quad_live) {
                    // q_{t-1} of this warp's codes into L2 while the products run
                    // (one 128-byte line per code: the warp's 32 rows)
                    const float *qn = qbuf + lane_index<MP>(t - 1 - p.t0, p.ntiles, tile, quad, 0, 0);
#pragma unroll
                    for (int c = lane; c < CF::CW; c += 32) prefetch_l2(qn + (size_t)(cbase + c) * 32);
                }
                // --- B h on the tensor cores (G = h - alpha_t B h below)
                E.contract_issue(true);
            }
            // <h, q_t> while the products run, 16 codes at a time (the compiler
            // barrier keeps a batch's loads from being hoisted into the one before:
            // 16 loads in flight per thread, no spills); q_t of one code is 32
            // consecutive floats over the warp's rows, read only on the support
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                const int col0 = cbase + 16 * pc;
                const uint32_t word = wd[pc >> 1] >> (16 * (pc & 1));
                float qv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) qv[j] = ((word >> j) & 1u) ? __ldg(qt + (size_t)(col0 + j) * 32) : 0.0f;
#pragma unroll
                for (int j = 0; j < 16; ++j) part = fmaf(G[16 * pc + j], qv[j], part);
                asm volatile("" ::: "memory");
            }
            // dalpha_t partial: warp sum into this warp's slot
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            // a trajectory slot holding the step a_t: q_t = -a_t / alpha_t on the support
            const bool step_slot = p.traj_steps && (t + 1) % REFRESH != 0;
            if (lane == 0) part_w[t - p.t0][warp] += step_slot ? -part / a : part;
            if (t == 0) break;  // G^(0) is not needed
            if (!E.contract_wait()) break;
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                float bh[16];
                tmem_ld16(E.taddr(CF::T_G + cbase + 16 * pc), bh);
#pragma unroll
                for (int j = 0; j < 16; ++j) G[16 * pc + j] = fmaf(-a, bh[j], G[16 * pc + j]);
            }
        }
        if (E.failed) break;
        if (p.t0 > 0 && row_ok) {
#pragma unroll
            for (int j = 0; j < CF::CW; ++j)
                if (cbase + j < m) Gbuf[lane_index<MP>(0, p.ntiles, tile, quad, cbase + j, lane)] = G[j];
        }
        E.tile_done();
    }
    __syncthreads();
    for (int t = p.t0 + tid; t < p.t1; t += CF::NT) {
        float sum = 0.0f;  // the warps' sums in a fixed order
#pragma unroll
        for (int w = 0; w < CF::NT / 32; ++w) sum += part_w[t - p.t0][w];
        p.partial[(size_t)t * gridDim.x + blockIdx.x] = sum;
    }
    E.finish();
}

// dalpha[t] = sum over blocks of partial[t][b], in FP64, fixed order.
__global__ void tc_reduce_partials_kernel(const float *__restrict__ partial, int nblk, int T, float *__restrict__ dalpha)
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

std::atomic<int> g_tile_rows{0};

namespace {

int mp_for(int m)
{
    if (m <= 64) return 64;
    if (m <= 128) return 128;
    if (m <= 256) return 256;
    return 0;
}

// Tiles sized to keep every SM busy: a layer costs the same for a partial
// tile as for 128 rows, so rows are spread evenly over rounds x SMs tiles.
// (rows per tile chosen by slista_set_tile_rows, 0: the even spread above)
void tiling(int N, int *TR, int *grid)
{
    const int sms = num_sms();
    const int fixed = g_tile_rows.load(std::memory_order_relaxed);
    if (fixed > 0) {
        *TR = fixed;
    } else {
        const int rounds = ceil_div(ceil_div(N, 128), sms);
        *TR = N > 0 ? ceil_div(N, (long long)rounds * sms) : 128;
    }
    const int ntiles = N > 0 ? ceil_div(N, *TR) : 0;
    *grid = ntiles < sms ? ntiles : sms;
}

template <int MP, bool SPLIT>
int split_b(const float *B, int m, uint8_t *bsplit, cudaStream_t st)
{
    split_b_kernel<<<ceil_div(MP * MP, 256), 256, 0, st>>>(B, m, MP, bsplit);
    return check_launch("split_b_kernel");
}

template <int MP, bool SPLIT>
int launch_mp(const PgdArgs &a, void *ws, cudaStream_t st)
{
    using CF = Cfg<MP, SPLIT>;
    uint8_t *bsplit = reinterpret_cast<uint8_t *>(ws);
    int rc = split_b<MP, SPLIT>(a.B, a.m, bsplit, st);
    if (rc) return rc;
    if (a.N == 0) return SLISTA_OK;
    TcParams p{};
    p.Bsplit = bsplit;
    p.C = a.C;
    p.m = a.m;
    p.N = a.N;
    p.lam = a.lam;
    p.alpha = a.alpha;
    p.Lp = a.L;
    p.T = a.T;
    p.Z = a.Z;
    p.masks = a.masks;
    // A checkpoint buffer is only written when ckpt_every < T; the layers
    // then refresh the accumulator at every checkpoint, else every REFRESH.
    p.ckpt = a.ckpt_every < a.T ? a.ckpt : nullptr;
    p.K = a.ckpt_every;
    int grid = 0;
    tiling(a.N, &p.TR, &grid);
    auto k = tc_pgd_forward_kernel<MP, SPLIT, KM_FWD>;
    SLISTA_CUDA_TRY(allow_smem(k, CF::SMEM_STAGED));
    k<<<grid, CF::NT, CF::SMEM_STAGED, st>>>(p);
    return check_launch("tc_pgd_forward_kernel");
}

size_t backward_ws_mp(int MP, int m, int N, int T, int K)
{
    int TR = 0, grid = 0;
    tiling(N, &TR, &grid);
    const size_t bsplit = (size_t)MP * MP * 4;
    const int ntiles = N > 0 ? ceil_div(N, TR) : 0;
    const size_t tileset = (size_t)ntiles * 128 * MP;  // tile layout: 4 quadrants x MP codes x 32 lanes
    const size_t q = sizeof(float) * (size_t)K * tileset;
    const size_t G = sizeof(float) * tileset;
    const size_t part = sizeof(float) * (size_t)T * (grid > 0 ? grid : 1);
    return bsplit + q + G + part + 256;
}

template <int MP, bool SPLIT>
int launch_backward_mp(const BwdArgs &a, void *ws, cudaStream_t st)
{
    using CF = Cfg<MP, SPLIT>;
    uint8_t *base = reinterpret_cast<uint8_t *>(ws);
    uint8_t *bsplit = base;
    int TRt = 0, gridt = 0;
    tiling(a.N, &TRt, &gridt);
    const int ntiles = a.N > 0 ? ceil_div(a.N, TRt) : 0;
    const size_t tileset = (size_t)ntiles * 128 * MP;
    float *qbuf = reinterpret_cast<float *>(base + (size_t)MP * MP * 4);
    float *Gbuf = qbuf + (size_t)a.ckpt_every * tileset;
    float *partial = Gbuf + tileset;
    int rc = split_b<MP, SPLIT>(a.B, a.m, bsplit, st);
    if (rc) return rc;
    if (a.N == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.dalpha, 0, sizeof(float) * a.T, st));
        return SLISTA_OK;
    }
    TcParams p{};
    p.Bsplit = bsplit;
    p.C = a.C;
    p.m = a.m;
    p.N = a.N;
    p.lam = a.lam;
    p.alpha = a.alpha;
    p.Lp = nullptr;
    p.T = a.T;
    p.masks = const_cast<uint32_t *>(a.masks);
    // the forward's refresh schedule: at checkpoints when there are any
    p.ckpt = a.ckpt_every < a.T ? const_cast<float *>(a.ckpt) : nullptr;
    p.K = a.ckpt_every;
    p.qbuf = qbuf;
    p.Gbuf = Gbuf;
    p.ntiles = ntiles;
    p.gZ = a.gZ;
    p.partial = partial;
    int grid = 0;
    tiling(a.N, &p.TR, &grid);
    auto kr = tc_pgd_forward_kernel<MP, SPLIT, KM_RECOMP>;
    auto ka = tc_adjoint_kernel<MP, SPLIT>;
    SLISTA_CUDA_TRY(allow_smem(kr, CF::SMEM));
    SLISTA_CUDA_TRY(allow_smem(ka, CF::SMEM));
    const int K = a.ckpt_every;
    const int nseg = ceil_div(a.T, K);
    for (int seg = nseg - 1; seg >= 0; --seg) {
        p.t0 = seg * K;
        p.t1 = p.t0 + K < a.T ? p.t0 + K : a.T;
        p.want_gT = (seg == nseg - 1);
        kr<<<grid, CF::NT, CF::SMEM, st>>>(p);
        rc = check_launch("tc_pgd_forward_kernel (recompute)");
        if (rc) return rc;
        ka<<<grid, CF::NT, CF::SMEM, st>>>(p);
        rc = check_launch("tc_adjoint_kernel");
        if (rc) return rc;
    }
    tc_reduce_partials_kernel<<<ceil_div(a.T, 8), 256, 0, st>>>(partial, grid, a.T, a.dalpha);
    return check_launch("tc_reduce_partials_kernel");
}

// Trajectory of the one-pass backward: (T + 1) slots of the tile layout
// (lane_index): q_t for t < T, dF/dz^(T) in slot T.
size_t traj_floats_mp(int MP, int N, int T)
{
    int TR = 0, grid = 0;
    tiling(N, &TR, &grid);
    const size_t ntiles = N > 0 ? (size_t)ceil_div(N, TR) : 0;
    return (size_t)(T + 1) * ntiles * 128 * MP;
}

template <int MP, bool SPLIT>
int launch_traj_mp(const PgdArgs &a, float *traj, void *ws, cudaStream_t st)
{
    using CF = Cfg<MP, SPLIT>;
    uint8_t *bsplit = reinterpret_cast<uint8_t *>(ws);
    int rc = split_b<MP, SPLIT>(a.B, a.m, bsplit, st);
    if (rc) return rc;
    if (a.N == 0) return SLISTA_OK;
    TcParams p{};
    p.Bsplit = bsplit;
    p.C = a.C;
    p.m = a.m;
    p.N = a.N;
    p.lam = a.lam;
    p.alpha = a.alpha;
    p.Lp = a.L;
    p.T = a.T;
    p.Z = a.Z;
    p.masks = a.masks;
    p.ckpt = nullptr;
    p.K = a.T;
    p.qbuf = traj;
    int grid = 0;
    tiling(a.N, &p.TR, &grid);
    p.ntiles = ceil_div(a.N, p.TR);
    auto k = tc_pgd_forward_kernel<MP, SPLIT, KM_TRAJ>;
    SLISTA_CUDA_TRY(allow_smem(k, CF::SMEM_STAGED));
    k<<<grid, CF::NT, CF::SMEM_STAGED, st>>>(p);
    return check_launch("tc_pgd_forward_kernel (trajectory)");
}

size_t backward_traj_ws_mp(int MP, int N, int T)
{
    int TR = 0, grid = 0;
    tiling(N, &TR, &grid);
    return (size_t)MP * MP * 4 + sizeof(float) * (size_t)T * (grid > 0 ? grid : 1) + 256;
}

template <int MP, bool SPLIT>
int launch_backward_traj_mp(const BwdArgs &a, const float *traj, void *ws, cudaStream_t st)
{
    using CF = Cfg<MP, SPLIT>;
    uint8_t *bsplit = reinterpret_cast<uint8_t *>(ws);
    float *partial = reinterpret_cast<float *>(bsplit + (size_t)MP * MP * 4);
    int rc = split_b<MP, SPLIT>(a.B, a.m, bsplit, st);
    if (rc) return rc;
    if (a.N == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.dalpha, 0, sizeof(float) * a.T, st));
        return SLISTA_OK;
    }
    TcParams p{};
    p.Bsplit = bsplit;
    p.m = a.m;
    p.N = a.N;
    p.lam = a.lam;
    p.alpha = a.alpha;
    p.T = a.T;
    p.masks = const_cast<uint32_t *>(a.masks);
    int grid = 0;
    tiling(a.N, &p.TR, &grid);
    p.ntiles = ceil_div(a.N, p.TR);
    const size_t tileset = (size_t)p.ntiles * 128 * MP;
    p.qbuf = const_cast<float *>(traj);
    p.Gbuf = const_cast<float *>(traj) + (size_t)a.T * tileset;  // read only: one segment
    p.Ginit = a.gZ;
    p.partial = partial;
    p.traj_steps = 1;
    p.t0 = 0;
    p.t1 = a.T;
    auto ka = tc_adjoint_kernel<MP, SPLIT>;
    SLISTA_CUDA_TRY(allow_smem(ka, CF::SMEM));
    ka<<<grid, CF::NT, CF::SMEM, st>>>(p);
    rc = check_launch("tc_adjoint_kernel (trajectory)");
    if (rc) return rc;
    tc_reduce_partials_kernel<<<ceil_div(a.T, 8), 256, 0, st>>>(partial, grid, a.T, a.dalpha);
    return check_launch("tc_reduce_partials_kernel");
}

}  // namespace

bool supported(int m) { return mp_for(m) != 0; }

size_t forward_ws_bytes(int m)
{
    const int MP = mp_for(m);
    return (size_t)MP * MP * 2 * 2;
}

size_t backward_ws_bytes(int m, int N, int T, int K)
{
    const int MP = mp_for(m);
    if (MP == 0) return 0;
    return backward_ws_mp(MP, m, N, T, K);
}

int launch_forward(const PgdArgs &a, int prec, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    switch (mp_for(a.m)) {
        case 64: return split ? launch_mp<64, true>(a, ws, st) : launch_mp<64, false>(a, ws, st);
        case 128: return split ? launch_mp<128, true>(a, ws, st) : launch_mp<128, false>(a, ws, st);
        case 256: return split ? launch_mp<256, true>(a, ws, st) : launch_mp<256, false>(a, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "tensor-core path supports m <= 256 (got %d)", a.m);
}

int launch_backward(const BwdArgs &a, int prec, void *ws, cudaStream_t st)
{
    if (a.ckpt_every > ADJ_KMAX)
        return fail(SLISTA_ERR_UNSUPPORTED, "tensor-core adjoint: at most %d layers between checkpoints", ADJ_KMAX);
    const bool split = prec == SLISTA_PREC_BF16X3;
    switch (mp_for(a.m)) {
        case 64: return split ? launch_backward_mp<64, true>(a, ws, st) : launch_backward_mp<64, false>(a, ws, st);
        case 128: return split ? launch_backward_mp<128, true>(a, ws, st) : launch_backward_mp<128, false>(a, ws, st);
        case 256: return split ? launch_backward_mp<256, true>(a, ws, st) : launch_backward_mp<256, false>(a, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "tensor-core path supports m <= 256 (got %d)", a.m);
}

size_t traj_floats(int m, int N, int T)
{
    const int MP = mp_for(m);
    if (MP == 0 || T < 1 || T > ADJ_KMAX || N < 0) return 0;
    return traj_floats_mp(MP, N, T);
}

size_t backward_traj_ws_bytes(int m, int N, int T)
{
    const int MP = mp_for(m);
    if (MP == 0) return 0;
    return backward_traj_ws_mp(MP, N, T);
}

int launch_forward_traj(const PgdArgs &a, int prec, float *traj, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    switch (mp_for(a.m)) {
        case 64: return split ? launch_traj_mp<64, true>(a, traj, ws, st) : launch_traj_mp<64, false>(a, traj, ws, st);
        case 128:
            return split ? launch_traj_mp<128, true>(a, traj, ws, st) : launch_traj_mp<128, false>(a, traj, ws, st);
        case 256:
            return split ? launch_traj_mp<256, true>(a, traj, ws, st) : launch_traj_mp<256, false>(a, traj, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "trajectory forward supports m <= 256 (got %d)", a.m);
}

int launch_backward_traj(const BwdArgs &a, int prec, const float *traj, void *ws, cudaStream_t st)
{
    const bool split = prec == SLISTA_PREC_BF16X3;
    switch (mp_for(a.m)) {
        case 64:
            return split ? launch_backward_traj_mp<64, true>(a, traj, ws, st)
                         : launch_backward_traj_mp<64, false>(a, traj, ws, st);
        case 128:
            return split ? launch_backward_traj_mp<128, true>(a, traj, ws, st)
                         : launch_backward_traj_mp<128, false>(a, traj, ws, st);
        case 256:
            return split ? launch_backward_traj_mp<256, true>(a, traj, ws, st)
                         : launch_backward_traj_mp<256, false>(a, traj, ws, st);
    }
    return fail(SLISTA_ERR_UNSUPPORTED, "trajectory backward supports m <= 256 (got %d)", a.m);
}

// ---------------------------------------------------------------------------
// Allocation-free variant (slista_forward_noalloc): the only scratch of the
// tensor-core forward is the split copy of B (B_hi and B_lo, BF16, swizzled),
// held here in a file-scope device array sized for m <= NOALLOC_MAX_M.  The
// array exists once per device for the life of the process; every call
// rewrites all of it before the layer kernel reads it, so nothing needs
// clearing, but two calls whose work overlaps on the GPU would race on it.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_MAX_M = 256;
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX_M * NOALLOC_MAX_M * 2 * 2;  // 256 KiB
static __device__ __align__(256) uint8_t g_noalloc_bsplit[NOALLOC_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

int noalloc_max_m() { return NOALLOC_MAX_M; }

int split_operands(const float *B, int m, int MP, uint8_t *out, cudaStream_t st)
{
    split_b_kernel<<<ceil_div((long long)MP * MP, 256), 256, 0, st>>>(B, m, MP, out);
    return check_launch("split_b_kernel");
}

int set_tile_rows(int rows)
{
    g_tile_rows.store(rows, std::memory_order_relaxed);
    return SLISTA_OK;
}

int tile_rows() { return g_tile_rows.load(std::memory_order_relaxed); }

int launch_forward_noalloc(const PgdArgs &a, int prec, cudaStream_t st)
{
    if (mp_for(a.m) == 0 || forward_ws_bytes(a.m) > NOALLOC_BYTES)
        return fail(SLISTA_ERR_UNSUPPORTED, "slista_forward_noalloc: m = %d exceeds the static scratch limit m <= %d",
                    a.m, NOALLOC_MAX_M);
    int dev = 0;
    SLISTA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(SLISTA_ERR_UNSUPPORTED, "slista_forward_noalloc: device %d out of range", dev);
    void *scratch = nullptr;
    {
        // once per device, with that device current: the device address of
        // the array (its host-side name is not a device address)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (g_noalloc_ptr[dev] == nullptr) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_bsplit);
            if (e != cudaSuccess)
                return fail(SLISTA_ERR_CUDA, "slista_forward_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    return launch_forward(a, prec, scratch, st);
}

}  // namespace tc
}  // namespace slista
