// The tensor-core engine of the layer kernels for m <= 256 (shared by the
// ISTA / Step-LISTA kernels and the fused Oracle-ISTA kernel): B_hi (and B_lo
// for m <= 128) resident in shared memory, B_lo streamed from L2 for m = 256,
// the MMA accumulator g and the split A operand in tensor memory, and the
// contraction D (+)= A x B with bounded waits.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace slista {
namespace tc {

// Every REFRESH layers (at the checkpoint layers instead when checkpoints are
// written) the accumulator is rebuilt as g = c - B z rather than updated by the
// step, which bounds the drift the split products accumulate (about 2e-6
// relative per layer, growing like t^0.8 without refreshes).
constexpr int REFRESH = 8;

// 16 consecutive entries of row `row` of C (columns col0..col0+15, zero
// outside N x m), as four 16-byte loads when the rows are 16-byte aligned.
__device__ __forceinline__ void load_c16(const float *__restrict__ C, int row, bool row_ok, int m, int col0,
                                         uint32_t (&v)[16])
{
    if (row_ok && (m & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0) {
        const float4 *src = reinterpret_cast<const float4 *>(C + (size_t)row * m + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 x = col0 + 4 * q < m ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * q + 0] = __float_as_uint(x.x);
            v[4 * q + 1] = __float_as_uint(x.y);
            v[4 * q + 2] = __float_as_uint(x.z);
            v[4 * q + 3] = __float_as_uint(x.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = __float_as_uint((row_ok && col0 + j < m) ? __ldg(C + (size_t)row * m + col0 + j) : 0.0f);
    }
}

// ---------------------------------------------------------------------------
// Engine shared by the layer kernels: resident operands, tensor memory, the
// contraction D (+)= A x B over all K with B_lo streamed when it does not
// fit, and the bounded waits.
// ---------------------------------------------------------------------------
template <int MP, bool SPLIT>
struct Cfg {
    static constexpr int KB = MP / 16;                // MMA K-steps per contraction
    static constexpr int CHUNK = MP * 128;            // bytes of one 64-wide K chunk of an operand
    static constexpr int OPER = MP * MP * 2;          // bytes of one BF16 operand
    static constexpr bool LO_RES = SPLIT && MP <= 128;
    static constexpr bool LO_STREAM = SPLIT && MP > 128;
    static constexpr int SMEM_OPER = OPER + (LO_RES ? OPER : 0) + (LO_STREAM ? 2 * CHUNK : 0);
    static constexpr int STAGE_OFF = SMEM_OPER + 64;  // after the barriers, tmem slot and B_lo address
    static constexpr int SMEM = STAGE_OFF + 1024 /*align*/;
    static constexpr int SMEM_STAGED = SMEM + 16 * 32 * 16 * 4;  // + per-warp staging (forward kernel)
    static constexpr int T_G = 0, T_AHI = MP, T_ALO = MP + MP / 2;
    static constexpr int COLS_USED = SPLIT ? 2 * MP : MP + MP / 2;
    static constexpr int TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                     : COLS_USED <= 256 ? 256 : 512;
    // Thread layout: warp w owns TMEM lanes 32*(w%4).. (tile rows) and the
    // column group w/4 of NG groups of CW code columns, worked in 16-column
    // pieces (NPC per thread).
    static constexpr int NG = MP / 32 < 4 ? MP / 32 : 4;
    static constexpr int NT = 128 * NG;               // threads per CTA
    static constexpr int CW = MP / NG;                // code columns per thread (>= 32)
    static constexpr int NPC = CW / 16;
    static constexpr uint32_t IDESC = idesc_bf16(128, MP);
    static_assert(MP % 64 == 0 && MP <= 256, "MP must be 64, 128 or 256");
    static_assert(NT > 96, "the issuing thread (96) must exist");
    static_assert(COLS_USED <= 512, "tensor memory");
};

constexpr int ADJ_KMAX = 256;  // layers per recompute segment of the adjoint

template <int MP, bool SPLIT>
struct TcEngine {
    using CF = Cfg<MP, SPLIT>;
    // The thread that initialises the barriers, streams B_lo and issues the
    // products: lane 0 of warp 3, whose TMEM lanes 96..127 hold tile rows
    // that are empty whenever a tile has at most 96 rows (the batch spread
    // over the SMs), so the issuing warp has the least epilogue work.
    static constexpr int ISSUER = 96;
    uint32_t tmem, lane_base, sB_u;  // sB_u: shared address of the operand area (1024-aligned)
    // producer state, one bit each: phase of bar_mma (0), of bar_full[s]
    // (1 + s) and bar_empty[s] (3 + s); a bulk copy into stage s not yet
    // waited for (5 + s)
    uint32_t bits;
    bool failed;

    __device__ __forceinline__ uint32_t bit(int i) const { return (bits >> i) & 1u; }
    __device__ __forceinline__ void flip(int i) { bits ^= 1u << i; }
    // global address of B_lo (read by the issuer only; kept in shared memory)
    __device__ __forceinline__ const uint8_t *lo_src() const
    {
        const uint8_t *g;
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(g) : "r"(bar(6)));
        return g;
    }

    __device__ __forceinline__ uint32_t sL_u() const { return sB_u + CF::OPER; }
    __device__ __forceinline__ uint32_t bar(int i) const { return sB_u + CF::SMEM_OPER + 8 * i; }
    __device__ __forceinline__ uint32_t bar_mma() const { return bar(0); }
    __device__ __forceinline__ uint32_t bar_full(int s) const { return bar(1 + s); }
    __device__ __forceinline__ uint32_t bar_empty(int s) const { return bar(3 + s); }
    // the operands copied back after a loan (reload); its phase is bit 7
    __device__ __forceinline__ uint32_t bar_reload() const { return bar(7); }

    // Barriers, tensor memory, resident operands; prefetch of the streamed
    // B_lo chunks 0 and 1 when `work` (the CTA has at least one tile).
    __device__ __forceinline__ void init(uint8_t *smem_raw, const uint8_t *Bsplit, bool work)
    {
        uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
        uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + CF::SMEM_OPER + 5 * 8);
        sB_u = smem_u32(smem);
        const int tid = threadIdx.x;
        if (tid == ISSUER) {
            for (int i = 0; i < 5; ++i) mbar_init(bar(i), 1);
            mbar_init(bar_reload(), 1);
            fence_mbar_init();
            const uint8_t *g = Bsplit + CF::OPER;
            asm volatile("st.shared.u64 [%0], %1;" ::"r"(bar(6)), "l"(g) : "memory");
        }
        if ((tid >> 5) == 0) tmem_alloc(tmem_slot, CF::TMEM_COLS);
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(Bsplit);
            uint4 *dst = reinterpret_cast<uint4 *>(smem);
            constexpr int n16 = (CF::OPER + (CF::LO_RES ? CF::OPER : 0)) / 16;
            for (int i = tid; i < n16; i += CF::NT) dst[i] = __ldg(src + i);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = *tmem_slot;
        lane_base = (uint32_t)(((tid >> 5) & 3) * 32) << 16;
        bits = 0u;
        failed = false;
        if (CF::LO_STREAM && tid == ISSUER && work) {
            load_stage(0, 0);
            load_stage(1, 1);
        }
    }

    __device__ __forceinline__ uint32_t taddr(int col) const { return tmem + lane_base + (uint32_t)col; }

    // this warp's 32 x 16-float staging area in shared memory
    __device__ __forceinline__ float *warp_stage() const
    {
        float *base = reinterpret_cast<float *>(__cvta_shared_to_generic((size_t)(sB_u + CF::STAGE_OFF)));
        return base + (threadIdx.x >> 5) * 32 * 16;
    }

    __device__ __forceinline__ void load_stage(int s, int chunk)
    {
        mbar_arrive_expect_tx(bar_full(s), CF::CHUNK);
        bulk_g2s(sL_u() + s * CF::CHUNK, lo_src() + chunk * CF::CHUNK, CF::CHUNK, bar_full(s));
        bits |= 1u << (5 + s);
    }

    __device__ __forceinline__ void wait_stage(int s, int code)
    {
        failed |= !mbar_wait(bar_full(s), bit(1 + s), code);
        flip(1 + s);
        bits &= ~(1u << (5 + s));
    }

    // Every thread: publish the A operand written to tensor memory, then
    // the issuer issues D = [D +] A x B over all K (fresh: the first product
    // overwrites D) and every thread waits for it.  Returns false, uniformly,
    // if a bounded wait expired.
    __device__ __forceinline__ bool contract(bool fresh)
    {
        contract_issue(fresh);
        return contract_wait();
    }

    // The two halves of contract(): every thread publishes the A operand and
    // the issuer issues the products; other work may run in between, as long as
    // it writes neither the accumulator nor the A operand.
    __device__ __forceinline__ void contract_issue(bool fresh)
    {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == ISSUER) {
            tc_fence_after();
            const uint32_t dG = tmem + CF::T_G;
            uint32_t acc = fresh ? 0u : 1u;
            if (CF::LO_STREAM) {
                // a_hi x B_lo on chunks 0 and 1 (prefetched)
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    wait_stage(s, 2);
#pragma unroll
                    for (int sub = 0; sub < 4; ++sub) {
                        mma_ts(dG, tmem + CF::T_AHI + (s * 4 + sub) * 8, sdesc_sw128(sL_u() + s * CF::CHUNK + sub * 32),
                               CF::IDESC, acc);
                        acc = 1u;
                    }
                    mma_commit(bar_empty(s));
                }
            }
#pragma unroll 1
            for (int kb = 0; kb < CF::KB; ++kb) {
                const uint64_t bd = sdesc_sw128(sB_u + (kb >> 2) * CF::CHUNK + (kb & 3) * 32);
                mma_ts(dG, tmem + CF::T_AHI + kb * 8, bd, CF::IDESC, acc);
                acc = 1u;
                if (SPLIT) mma_ts(dG, tmem + CF::T_ALO + kb * 8, bd, CF::IDESC, 1u);
                if (CF::LO_RES) {
                    const uint64_t ld = sdesc_sw128(sL_u() + (kb >> 2) * CF::CHUNK + (kb & 3) * 32);
                    mma_ts(dG, tmem + CF::T_AHI + kb * 8, ld, CF::IDESC, 1u);
                }
            }
            if (CF::LO_STREAM) {
                // refill both stages with chunks 2 and 3, then a_hi x B_lo on them
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    failed |= !mbar_wait(bar_empty(s), bit(3 + s), 3);
                    flip(3 + s);
                    load_stage(s, 2 + s);
                }
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    wait_stage(s, 4);
#pragma unroll
                    for (int sub = 0; sub < 4; ++sub)
                        mma_ts(dG, tmem + CF::T_AHI + ((2 + s) * 4 + sub) * 8,
                               sdesc_sw128(sL_u() + s * CF::CHUNK + sub * 32), CF::IDESC, 1u);
                }
            }
            mma_commit(bar_mma());
        }
    }

    __device__ __forceinline__ bool contract_wait()
    {
        const bool ok = mbar_wait(bar_mma(), bit(0), 1);
        flip(0);
        tc_fence_after();
        if (CF::LO_STREAM && threadIdx.x == ISSUER && ok && !failed) {
            // every product is done: both stages are free, prefetch chunks 0 and 1
            load_stage(0, 0);
            load_stage(1, 1);
        }
        failed = __syncthreads_or(!ok || failed) != 0;
        return !failed;
    }

    // The operand area on loan (the fused Oracle-ISTA kernel's eigen-solvers
    // use it between two contractions): quiesce() lets the streamed B_lo
    // copies land, reload() copies the operands back and re-issues the
    // stream's first two chunks.  Every thread calls both.
    __device__ __forceinline__ void quiesce()
    {
        if (CF::LO_STREAM && threadIdx.x == ISSUER)
            for (int s = 0; s < 2; ++s)
                if (bit(5 + s)) wait_stage(s, 6);
        failed = __syncthreads_or(failed) != 0;
    }

    __device__ __forceinline__ void reload(const uint8_t *Bsplit)
    {
        // the borrowers' generic stores come before the bulk copies that overwrite them
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == ISSUER) {
            constexpr int BYTES = CF::OPER + (CF::LO_RES ? CF::OPER : 0);
            constexpr int PIECE = 32768;
            mbar_arrive_expect_tx(bar_reload(), BYTES);
#pragma unroll 1
            for (int o = 0; o < BYTES; o += PIECE)
                bulk_g2s(sB_u + o, Bsplit + o, BYTES - o < PIECE ? BYTES - o : PIECE, bar_reload());
            if (CF::LO_STREAM) {
                load_stage(0, 0);
                load_stage(1, 1);
            }
            // the products read the operands only after the issuer has seen them land
            failed |= !mbar_wait(bar_reload(), bit(7), 8);
            flip(7);
        }
        failed = __syncthreads_or(failed) != 0;
    }

    // Tensor memory of the tile is no longer read.
    __device__ __forceinline__ void tile_done()
    {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    // Drain outstanding bulk copies, release tensor memory.
    __device__ __forceinline__ void finish()
    {
        if (CF::LO_STREAM && threadIdx.x == ISSUER)
            for (int s = 0; s < 2; ++s)
                if (bit(5 + s)) wait_stage(s, 5);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, CF::TMEM_COLS);
    }
};

// Writes the BF16 split of v (16 values of this thread's row, code columns
// col0..col0+15) as the A operand: 8 packed pairs per operand.
template <int MP, bool SPLIT>
__device__ __forceinline__ void store_split16(const TcEngine<MP, SPLIT> &E, int col0, const float (&v)[16])
{
    using CF = Cfg<MP, SPLIT>;
    uint32_t pk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        pk[j] = *reinterpret_cast<const uint32_t *>(&h2);
    }
    tmem_st8(E.taddr(CF::T_AHI + col0 / 2), pk);
    if (SPLIT) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162 *>(&pk[j]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
            pk[j] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        tmem_st8(E.taddr(CF::T_ALO + col0 / 2), pk);
    }
}

// Loads 16 consecutive columns (col0..) of row `row` of a row-major N x m
// FP32 matrix into this thread's tensor-memory lane at column tcol.
template <int MP, bool SPLIT>
__device__ __forceinline__ void row16_to_tmem(const TcEngine<MP, SPLIT> &E, const float *__restrict__ G, int row,
                                              bool row_ok, int m, int col0, int tcol)
{
    uint32_t v[16];
    load_c16(G, row, row_ok, m, col0, v);
    tmem_st16(E.taddr(tcol), v);
}

// Index of (layer s, tile, lane quadrant, code col, lane) in the adjoint's
// internal buffers: for one code the 32 rows of a warp are consecutive, so
// the row-per-lane accesses of the layer kernels are coalesced.
// Row-per-lane 16-code pieces made coalesced through a per-warp staging area
// of 32 rows x 16 floats in shared memory (column c of row r at
// r * 16 + (c ^ (r & 15))): a lane writes or reads its own row there, and the
// global side moves two 64-byte row segments per warp instruction.  Used for
// the checkpoint and Z stores of the forward, whose layout (sample-major rows)
// is the ABI's.
__device__ __forceinline__ void stage_put(float *buf, const float (&v)[16])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 16; ++c) buf[lane * 16 + (c ^ (lane & 15))] = v[c];
    __syncwarp();
}

// rows rbase .. rbase+31 (the first nrow real) x codes c0 .. c0+15 of a row-major N x m matrix
static __device__ __noinline__ void stage_to_global(const float *buf, float *M, int rbase, int nrow, int m, int c0)
{
    const int lane = threadIdx.x & 31;
    const int h = lane >> 4, c = lane & 15;
    if (c0 + c < m)
#pragma unroll 1
        for (int i = 0; i < 16; ++i) {
            const int r = 2 * i + h;
            if (r < nrow) M[(size_t)(rbase + r) * m + c0 + c] = buf[r * 16 + (c ^ (r & 15))];
        }
    __syncwarp();
}

}  // namespace tc
}  // namespace slista
