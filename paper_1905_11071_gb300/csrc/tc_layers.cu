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

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace slista {

__device__ int g_device_flag = 0;

int read_and_clear_device_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_device_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(g_device_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "a kernel's bounded wait expired (device flag %d)", h);
    }
    return SLISTA_OK;
}

namespace tc {

constexpr int NTHREADS = 256;   // warp w: TMEM lane quadrant (w & 3), code half (w >> 2)
// Every REFRESH layers (at the checkpoint layers instead when checkpoints are
// written) the accumulator is rebuilt as g = c - B z rather than updated by the
// step, which bounds the drift the split products accumulate (about 2e-6
// relative per layer, growing like t^0.8 without refreshes).
constexpr int REFRESH = 8;
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

// 16 consecutive entries of row `row` of C (columns col0..col0+15, zero
// outside N x m), as four 16-byte loads when the rows are 16-byte aligned.
__device__ __forceinline__ void load_c16(const float *__restrict__ C, int row, bool row_ok, int m, int col0,
                                         uint32_t (&v)[16])
{
    if (row_ok && (m & 3) == 0) {
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
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity`; false (and the device
// flag raised) if it does not complete within WAIT_LIMIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
            atomicExch(&g_device_flag, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[tmem] * B[smem descriptor]
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (ld + wait in one asm).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]),
          "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]),
          "=f"(v[16]), "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]),
          "=f"(v[24]), "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
        "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
        "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart (SBO); LBO unused for this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // LBO = 16 bytes (ignored)
    d |= (uint64_t)(1024 >> 4) << 32;     // SBO = 1024 bytes
    d |= (uint64_t)1 << 46;               // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (both K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (n, k) of an MP x MP operand stored as MP/64 chunks
// of 64 K-columns, each chunk MP rows x 128 bytes with the 128-byte swizzle:
// 16-byte unit c of row n sits at unit (c ^ (n % 8)) of that row.
__host__ __device__ inline uint32_t sw128_offset(int MP, int n, int k)
{
    const int kc = k >> 6, kin = k & 63;
    const int unit = kin >> 3, e = kin & 7;
    return (uint32_t)(kc * MP * 128 + (n >> 3) * 1024 + (n & 7) * 128 + ((unit ^ (n & 7)) << 4) + e * 2);
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

// ---------------------------------------------------------------------------
// The layer kernel
// ---------------------------------------------------------------------------
template <int MP, bool SPLIT>
struct Cfg {
    static constexpr int KB = MP / 16;                // MMA K-steps per layer
    static constexpr int CHUNK = MP * 128;            // bytes of one 64-wide K chunk of an operand
    static constexpr int OPER = MP * MP * 2;          // bytes of one BF16 operand
    static constexpr bool LO_RES = SPLIT && MP <= 128;
    static constexpr bool LO_STREAM = SPLIT && MP > 128;
    static constexpr int SMEM_OPER = OPER + (LO_RES ? OPER : 0) + (LO_STREAM ? 2 * CHUNK : 0);
    static constexpr int SMEM = SMEM_OPER + 1024 /*align*/ + 64 /*barriers*/;
    static constexpr int T_G = 0, T_AHI = MP, T_ALO = MP + MP / 2;
    static constexpr int COLS_USED = SPLIT ? 2 * MP : MP + MP / 2;
    static constexpr int TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                     : COLS_USED <= 256 ? 256 : 512;
    static constexpr int HALF = MP / 2;               // code columns per thread
    static constexpr int NCH = HALF / 32;             // 32-column chunks per thread
    static constexpr uint32_t IDESC = idesc_bf16(128, MP);
    static_assert(MP % 64 == 0 && MP <= 256, "MP must be 64, 128 or 256");
    static_assert(COLS_USED <= 512, "tensor memory");
};

template <int MP, bool SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1) tc_pgd_forward_kernel(
    const uint8_t *__restrict__ Bsplit, const float *__restrict__ C, int m, int N, float lam,
    const float *__restrict__ alpha, const double *__restrict__ Lp, int T, float *__restrict__ Z,
    uint32_t *__restrict__ masks, float *__restrict__ ckpt, int K, int TR)
{
    using CF = Cfg<MP, SPLIT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;                                 // B_hi (resident)
    uint8_t *sL = smem + CF::OPER;                      // B_lo: resident, or two streamed chunks
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + CF::SMEM_OPER);
    uint64_t *bar_mma = bars + 0;
    uint64_t *bar_full = bars + 1;                      // [2]
    uint64_t *bar_empty = bars + 3;                     // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 5);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int ntiles = (N + TR - 1) / TR;  // TR <= 128 rows per tile (lanes >= TR idle)
    const int W = (m + 31) / 32;
    const uint8_t *gLo = Bsplit + CF::OPER;

    // --- set-up: barriers, tensor memory, resident operands
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_full + 0, 1);
        mbar_init(bar_full + 1, 1);
        mbar_init(bar_empty + 0, 1);
        mbar_init(bar_empty + 1, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, CF::TMEM_COLS);
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(Bsplit);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        constexpr int n16 = (CF::OPER + (CF::LO_RES ? CF::OPER : 0)) / 16;
        for (int i = tid; i < n16; i += NTHREADS) dst[i] = __ldg(src + i);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;

    // producer state (thread 0)
    uint32_t ph_full[2] = {0u, 0u}, ph_empty[2] = {0u, 0u}, ph_mma = 0u;
    bool pending[2] = {false, false};  // a bulk copy into stage s has not been waited for
    bool failed = false;
    auto load_stage = [&](int s, int chunk) {
        mbar_arrive_expect_tx(bar_full + s, CF::CHUNK);
        bulk_g2s(sL + s * CF::CHUNK, gLo + chunk * CF::CHUNK, CF::CHUNK, bar_full + s);
        pending[s] = true;
    };
    auto wait_stage = [&](int s, int code) {
        failed |= !mbar_wait(bar_full + s, ph_full[s], code);
        ph_full[s] ^= 1u;
        pending[s] = false;
    };
    if (CF::LO_STREAM && tid == 0 && blockIdx.x < ntiles) {
        load_stage(0, 0);
        load_stage(1, 1);
    }

    const float a_const = alpha ? 0.0f : (float)(1.0 / __ldg(Lp));
    const uint32_t sB_u = smem_u32(sB), sL_u = smem_u32(sL);

#pragma unroll 1
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int row = tile * TR + quad * 32 + lane;
        const bool row_ok = (quad * 32 + lane < TR) && row < N;
        // g <- c, z <- 0
        float z[CF::HALF];
#pragma unroll
        for (int ch = 0; ch < CF::NCH; ++ch) {
            const int col0 = half * CF::HALF + ch * 32;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                uint32_t v[16];
                load_c16(C, row, row_ok, m, col0 + 16 * p, v);
                tmem_st16(tmem + lane_base + CF::T_G + col0 + 16 * p, v);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) z[ch * 32 + j] = 0.0f;
        }
        tmem_st_wait();

#pragma unroll 1
        for (int t = 0; t < T; ++t) {
            const float a = alpha ? __ldg(alpha + t) : a_const;
            const float thr = a * lam;
            if (ckpt && t > 0 && t % K == 0) {
                // checkpoint (z^(t), g^(t)) every K layers, layout of slista_forward
                float *ck = ckpt + (size_t)(t / K - 1) * 2 * N * m;
#pragma unroll
                for (int ch = 0; ch < CF::NCH; ++ch) {
                    const int col0 = half * CF::HALF + ch * 32;
                    float gv[32];
                    tmem_ld32(tmem + lane_base + CF::T_G + col0, gv);
                    if (row_ok)
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (col0 + j < m) {
                                ck[(size_t)row * m + col0 + j] = z[ch * 32 + j];
                                ck[(size_t)N * m + (size_t)row * m + col0 + j] = gv[j];
                            }
                }
            }
            // --- epilogue: z update and the split step a = z - z' into tensor memory
            // (a = -z' on refresh layers, whose accumulator is reloaded with c)
            const bool refresh = ckpt ? ((t + 1) % K == 0) : ((t + 1) % REFRESH == 0);
#pragma unroll
            for (int ch = 0; ch < CF::NCH; ++ch) {
                const int col0 = half * CF::HALF + ch * 32;
                float gv[32];
                tmem_ld32(tmem + lane_base + CF::T_G + col0, gv);
                uint32_t word = 0u;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float zo = z[ch * 32 + j];
                    const float u = fmaf(a, gv[j], zo);
                    const float zn = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                    gv[j] = refresh ? -zn : zo - zn;  // the MMA's A operand
                    z[ch * 32 + j] = zn;
                    word |= (uint32_t)(zn != 0.0f) << j;
                }
                uint32_t pk[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(gv[2 * j], gv[2 * j + 1]);
                    pk[j] = *reinterpret_cast<const uint32_t *>(&h2);
                }
                tmem_st16(tmem + lane_base + CF::T_AHI + col0 / 2, pk);
                if (SPLIT) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162 *>(&pk[j]);
                        const float2 hf = __bfloat1622float2(h2);
                        const __nv_bfloat162 l2 = __floats2bfloat162_rn(gv[2 * j] - hf.x, gv[2 * j + 1] - hf.y);
                        pk[j] = *reinterpret_cast<const uint32_t *>(&l2);
                    }
                    tmem_st16(tmem + lane_base + CF::T_ALO + col0 / 2, pk);
                }
                if (masks && row_ok && (col0 >> 5) < W) masks[((size_t)t * N + row) * W + (col0 >> 5)] = word;
            }
            if (refresh && t != T - 1) {
#pragma unroll
                for (int ch = 0; ch < CF::NCH; ++ch) {
                    const int col0 = half * CF::HALF + ch * 32;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        uint32_t cv[16];
                        load_c16(C, row, row_ok, m, col0 + 16 * p, cv);
                        tmem_st16(tmem + lane_base + CF::T_G + col0 + 16 * p, cv);
                    }
                }
            }
            tmem_st_wait();
            if (t == T - 1) break;
            tc_fence_before();
            __syncthreads();
            // --- contraction g += a B on the tensor cores (one thread issues)
            if (tid == 0) {
                tc_fence_after();
                const uint32_t dG = tmem + CF::T_G;
                if (CF::LO_STREAM) {
                    // a_hi x B_lo, chunks 0 and 1 (prefetched)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        wait_stage(s, 2);
#pragma unroll
                        for (int sub = 0; sub < 4; ++sub)
                            mma_ts(dG, tmem + CF::T_AHI + (s * 4 + sub) * 8, sdesc_sw128(sL_u + s * CF::CHUNK + sub * 32),
                                   CF::IDESC, 1u);
                        mma_commit(bar_empty + s);
                    }
                }
#pragma unroll 1
                for (int kb = 0; kb < CF::KB; ++kb) {
                    const uint64_t bd = sdesc_sw128(sB_u + (kb >> 2) * CF::CHUNK + (kb & 3) * 32);
                    mma_ts(dG, tmem + CF::T_AHI + kb * 8, bd, CF::IDESC, 1u);
                    if (SPLIT) mma_ts(dG, tmem + CF::T_ALO + kb * 8, bd, CF::IDESC, 1u);
                    if (CF::LO_RES) {
                        const uint64_t ld = sdesc_sw128(sL_u + (kb >> 2) * CF::CHUNK + (kb & 3) * 32);
                        mma_ts(dG, tmem + CF::T_AHI + kb * 8, ld, CF::IDESC, 1u);
                    }
                }
                if (CF::LO_STREAM) {
                    // refill the two stages with chunks 2 and 3, then a_hi x B_lo on them
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        failed |= !mbar_wait(bar_empty + s, ph_empty[s], 3);
                        ph_empty[s] ^= 1u;
                        load_stage(s, 2 + s);
                    }
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        wait_stage(s, 4);
#pragma unroll
                        for (int sub = 0; sub < 4; ++sub)
                            mma_ts(dG, tmem + CF::T_AHI + ((2 + s) * 4 + sub) * 8,
                                   sdesc_sw128(sL_u + s * CF::CHUNK + sub * 32), CF::IDESC, 1u);
                    }
                }
                mma_commit(bar_mma);
            }
            // --- wait for the contraction (every thread, bounded)
            bool ok = mbar_wait(bar_mma, ph_mma, 1);
            ph_mma ^= 1u;
            tc_fence_after();
            if (CF::LO_STREAM && tid == 0 && ok && !failed) {
                // all MMAs done: both stages are free, prefetch chunks 0 and 1 for the next layer
                load_stage(0, 0);
                load_stage(1, 1);
            }
            failed = __syncthreads_or(!ok || failed) != 0;
            if (failed) break;
        }
        if (failed) break;
        // z^(T) out
#pragma unroll
        for (int ch = 0; ch < CF::NCH; ++ch) {
            const int col0 = half * CF::HALF + ch * 32;
            if (row_ok)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (col0 + j < m) Z[(size_t)row * m + col0 + j] = z[ch * 32 + j];
        }
        tc_fence_before();
        __syncthreads();  // tensor memory of this tile is no longer read
        tc_fence_after();
    }
    // drain outstanding bulk copies before the shared memory goes away
    if (CF::LO_STREAM && tid == 0)
        for (int s = 0; s < 2; ++s)
            if (pending[s]) wait_stage(s, 5);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, CF::TMEM_COLS);
}

namespace {

int mp_for(int m)
{
    if (m <= 64) return 64;
    if (m <= 128) return 128;
    if (m <= 256) return 256;
    return 0;
}

template <int MP, bool SPLIT>
int launch_mp(const PgdArgs &a, void *ws, cudaStream_t st)
{
    using CF = Cfg<MP, SPLIT>;
    uint8_t *bsplit = reinterpret_cast<uint8_t *>(ws);
    split_b_kernel<<<ceil_div(MP * MP, 256), 256, 0, st>>>(a.B, a.m, MP, bsplit);
    int rc = check_launch("split_b_kernel");
    if (rc) return rc;
    if (a.N == 0) return SLISTA_OK;
    // A layer costs the same for a tile of 128 rows as for a partial one, so
    // tiles are sized to keep every SM busy: rounds = tiles per SM with full
    // tiles, then the rows are spread evenly over rounds x SMs tiles.
    const int sms = num_sms();
    const int rounds = ceil_div(ceil_div(a.N, 128), sms);
    const int TR = ceil_div(a.N, (long long)rounds * sms);
    const int ntiles = ceil_div(a.N, TR);
    auto k = tc_pgd_forward_kernel<MP, SPLIT>;
    SLISTA_CUDA_TRY(allow_smem(k, CF::SMEM));
    const int grid = ntiles < sms ? ntiles : sms;
    k<<<grid, NTHREADS, CF::SMEM, st>>>(bsplit, a.C, a.m, a.N, a.lam, a.alpha, a.L, a.T, a.Z, a.masks, a.ckpt,
                                        a.ckpt_every, TR);
    return check_launch("tc_pgd_forward_kernel");
}

}  // namespace

bool supported(int m) { return mp_for(m) != 0; }

size_t forward_ws_bytes(int m)
{
    const int MP = mp_for(m);
    return (size_t)MP * MP * 2 * 2;
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
