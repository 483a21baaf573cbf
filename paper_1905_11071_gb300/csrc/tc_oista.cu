// Oracle-ISTA (Algorithm 1, Section 3) as one cooperative kernel per call, for
// split BF16 products, 128 < m <= 256 and batches of at most 128 samples per
// SM (the eigen-solvers borrow the operand area that the split B_lo stream
// leaves at m = 256).
//
// Every CTA owns one tile of the batch for all T layers, with the state of
// the tensor-core forward: z in registers, g = c - B z as the MMA accumulator
// in tensor memory, B_hi resident in shared memory and B_lo streamed from L2.
// A layer t is three phases separated by grid-wide barriers:
//   (A) from z^(t), g^(t): S = supp(z^(t)); condition (star) - the candidate
//       y = ST(z + g / L_S, lam / L_S) stays inside S iff |g_j| <= lam off S
//       (z_j = 0 there, so argument and threshold both scale with 1 / L_S);
//       samples whose step is accepted and whose S differs from the support
//       of their cached L_S go to the layer's solve lists (by |S|);
//   (S) every warp of the grid takes samples from the lists and computes
//       L_S = lambda_max(B_SS) (Eq. spca) with the warp solvers of the
//       two-kernel path; when a list of supports larger than 32 is not empty
//       the CTA lends its operand area to those solvers (z is parked in the
//       tensor memory of the A operand, B is copied back afterwards);
//   (B) z^(t+1) = ST(z + a g, a lam) with a = 1 / L_S (accepted) or 1 / L
//       (the ISTA fallback), then g <- g + (z^(t) - z^(t+1)) B on the tensor
//       cores (split BF16; every REFRESH layers g is rebuilt from c).
// The result is Algorithm 1 up to rounding; only the order in which L_S and
// (star) are evaluated differs from the listing, as in the two-kernel path.
// The barriers and every mbarrier wait are bounded: on expiry the kernel
// raises the device flag, drains its copies, releases its tensor memory and
// returns; the other CTAs then give up at their next barrier.
#include <cuda_bf16.h>

#include "common.cuh"
#include "eig.cuh"
#include "kernels.h"
#include "oista_solvers.cuh"
#include "tc_engine.cuh"
#include "tc_ptx.cuh"

namespace slista {
namespace tco {

int read_and_clear_flag(cudaStream_t st)
{
    int h = 0;
    SLISTA_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, tc::tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        SLISTA_CUDA_TRY(cudaMemcpyToSymbolAsync(tc::tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
        return fail(SLISTA_ERR_TIMEOUT, "the Oracle-ISTA kernel's bounded wait expired (device flag %d)", h);
    }
    return SLISTA_OK;
}

namespace {

constexpr int MP = 256;
constexpr int NT = 512;
constexpr int NCLS = simt::NCLS;
constexpr int A_WARPS = simt::A_WARPS;  // warps with a solver buffer (when the operand area is lent)
static_assert(A_WARPS * sizeof(simt::WarpEig) <= tc::Cfg<MP, true>::SMEM_OPER, "solver buffers in the operand area");

struct OisParams {
    const uint8_t *Bsplit;  // B_hi, B_lo (the tensor-core engine's layout)
    const float *B;         // m x m, for the solvers' gathers
    const float *Dt;        // m x n (columns of D), or nullptr
    const float *C;
    int n, m, N, T, TR;
    float lam;
    const double *Lp;
    float *Z;
    double *LS_out;         // nullable
    int *accepted;          // nullable
    int want_ls;
    double *LSv;            // N: cached L_S
    uint32_t *Sprev;        // N x W: the support of the cached L_S
    uint32_t *Scur;         // N x W: supp(z^(t)) of listed samples (read by the solvers)
    int *list;              // 2 x NCLS x N, by layer parity
    int *counter;           // T x NCLS list lengths
    int *qpos;              // T x NCLS queue positions
    unsigned *gbar;         // grid barrier: arrivals, generation
};

// Per-CTA scratch in the engine's staging area (which only the final Z store
// uses): per tile row and column group, (star) failures, support changes and
// support sizes; the rows' steps; the register solvers' scratch.
struct OisShared {
    int bad[4][128];
    int chg[4][128];
    int k[4][128];
    float step[128];
    int nacc;
    int cnt[NCLS], base[NCLS];
    simt::WarpEigS small[NT / 32];
};
static_assert(sizeof(OisShared) <= 16 * 32 * 16 * 4, "per-CTA scratch in the staging area");

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of the cooperative launch (every thread calls it);
// false, uniformly within the CTA, if the wait expired.
__device__ bool grid_sync(unsigned *gbar, int code)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(gbar + 1);
        __threadfence();
        const unsigned arrived = atomicAdd(gbar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(gbar, 0u);
            __threadfence();
            atomicAdd(gbar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(gbar + 1) == gen) {
                if (clock64() - t0 > tc::WAIT_LIMIT_CYCLES) {
                    atomicExch(&tc::tc_flag, code);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Index list of a support (one warp), its words read through L2 (written by
// another CTA of this launch); returns |S|.
__device__ int support_indices_cg(const uint32_t *words, int W, int *idx)
{
    const int lane = threadIdx.x & 31;
    const uint32_t mine = lane < W ? __ldcg(words + lane) : 0u;
    int k = 0;
    for (int w = 0; w < W; ++w) {
        const uint32_t bits = __shfl_sync(0xffffffffu, mine, w);
        if ((bits >> lane) & 1u) idx[k + __popc(bits & ((1u << lane) - 1u))] = w * 32 + lane;
        k += __popc(bits);
    }
    __syncwarp();
    return k;
}

// The next sample of list cls of layer t (one warp); -1 when the list is done.
__device__ __forceinline__ int next_item(const OisParams &p, int t, int cls, int n)
{
    const int lane = threadIdx.x & 31;
    int q = n;
    if (lane == 0) {
        int *qp = p.qpos + NCLS * t + cls;
        q = *reinterpret_cast<volatile int *>(qp) >= n ? n : atomicAdd(qp, 1);
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n) return -1;
    return __ldcg(p.list + ((size_t)(t & 1) * NCLS + cls) * p.N + q);
}

__device__ __forceinline__ void publish(const OisParams &p, int i, int W, double LS)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) p.LSv[i] = LS;
    for (int w = lane; w < W; w += 32) p.Sprev[(size_t)i * W + w] = __ldcg(p.Scur + (size_t)i * W + w);
    __syncwarp();
}

template <bool SPLIT>
__global__ void __launch_bounds__(NT, 1) tc_oista_kernel(const __grid_constant__ OisParams p)
{
    using CF = tc::Cfg<MP, SPLIT>;
    static_assert(CF::NT == NT && CF::CW == 64 && CF::NPC == 4, "thread layout of the m = 256 engine");
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cg = warp >> 2, cbase = cg * CF::CW;
    const int N = p.N, m = p.m, TR = p.TR, W = (m + 31) / 32;
    const int r = quad * 32 + lane;  // tile row = tensor-memory lane
    const int row = blockIdx.x * TR + r;
    const bool row_ok = r < TR && row < N;
    const float lam = p.lam;
    const double L = __ldg(p.Lp);
    tc::TcEngine<MP, SPLIT> E;
    E.init(smem_raw, p.Bsplit, true);
    OisShared &sh = *reinterpret_cast<OisShared *>(E.warp_stage() - (size_t)warp * 32 * 16);
    uint8_t *oper = reinterpret_cast<uint8_t *>(__cvta_shared_to_generic((size_t)E.sB_u));

    // L_empty = L cached for the empty support; g = c, z = 0
    if (row_ok) {
        if (cg == 0) p.LSv[row] = L;
#pragma unroll
        for (int i = 0; i < 2; ++i)
            if ((cbase >> 5) + i < W) p.Sprev[(size_t)row * W + (cbase >> 5) + i] = 0u;
    }
#pragma unroll 1
    for (int pc = 0; pc < CF::NPC; ++pc)
        tc::row16_to_tmem(E, p.C, row, row_ok, m, cbase + 16 * pc, CF::T_G + cbase + 16 * pc);
    float z[CF::CW];
#pragma unroll
    for (int j = 0; j < CF::CW; ++j) z[j] = 0.0f;
    tc::tmem_st_wait();

    bool ok = true;
#pragma unroll 1
    for (int t = 0; t < p.T; ++t) {
        const bool last = t == p.T - 1;
        // ---- (A) condition (star), S and the solve lists of layer t
        {
            // the support words of the cached L_S first: their latency overlaps the rest
            uint32_t sp[2] = {0u, 0u};
            if (row_ok)
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    if ((cbase >> 5) + i < W) sp[i] = __ldcg(p.Sprev + (size_t)row * W + (cbase >> 5) + i);
            bool bad = false;
            uint32_t w[2] = {0u, 0u};
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                float gv[16];
                tc::tmem_ld16(E.taddr(CF::T_G + cbase + 16 * pc), gv);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = cbase + 16 * pc + j;
                    const bool nz = z[16 * pc + j] != 0.0f;
                    bad |= c < m && !nz && fabsf(gv[j]) > lam;
                    w[pc >> 1] |= (uint32_t)nz << (16 * (pc & 1) + j);
                }
            }
            int chg = 0;
            if (row_ok)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int wi = (cbase >> 5) + i;
                    if (wi < W) {
                        p.Scur[(size_t)row * W + wi] = w[i];
                        chg |= w[i] != sp[i];
                    }
                }
            sh.bad[cg][r] = bad;
            sh.chg[cg][r] = chg;
            sh.k[cg][r] = __popc(w[0]) + __popc(w[1]);
            if (tid == 0) sh.nacc = 0;
            if (tid < NCLS) sh.cnt[tid] = 0;
        }
        __syncthreads();
        // the CTA's rows for each list: one global atomic per list and CTA
        int cls = -1, lpos = 0;
        if (cg == 0) {
            const int bad = sh.bad[0][r] | sh.bad[1][r] | sh.bad[2][r] | sh.bad[3][r];
            const int chg = sh.chg[0][r] | sh.chg[1][r] | sh.chg[2][r] | sh.chg[3][r];
            const int k = sh.k[0][r] + sh.k[1][r] + sh.k[2][r] + sh.k[3][r];
            sh.bad[0][r] = bad;
            if (row_ok && chg && (!bad || (p.want_ls && last))) {
                cls = k > simt::KMAX ? 0 : k > simt::SMALL_K ? 1 : 2;
                lpos = atomicAdd(&sh.cnt[cls], 1);
            }
        }
        __syncthreads();
        if (tid < NCLS) sh.base[tid] = sh.cnt[tid] ? atomicAdd(p.counter + NCLS * t + tid, sh.cnt[tid]) : 0;
        __syncthreads();
        if (cls >= 0) p.list[((size_t)(t & 1) * NCLS + cls) * N + sh.base[cls] + lpos] = row;
        // ---- every list of layer t is complete
        if (!(ok = grid_sync(p.gbar, 31))) break;
        // ---- (S) the L_S solves of layer t, balanced over the grid
        const int n0 = __ldcg(p.counter + NCLS * t), n1 = __ldcg(p.counter + NCLS * t + 1),
                  n2 = __ldcg(p.counter + NCLS * t + 2);
        if (n0 + n1 + n2 > 0) {
            // supports of more than 32 codes need a warp's shared-memory buffer:
            // the first CTAs lend their operand area, as many as the buffered
            // warps that the layer's large supports can use (all when they
            // are many), the others solve only supports of at most 32 codes
            const int nbig = (n0 + n1 + A_WARPS - 1) / A_WARPS;
            const bool big = (int)blockIdx.x < nbig;
            // park z in the A operand's tensor memory (free between the layers)
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                uint32_t v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(z[16 * pc + j]);
                tc::tmem_st16(E.taddr(CF::T_AHI + cbase + 16 * pc), v);
            }
            tc::tmem_st_wait();
            if (big) E.quiesce();
            if (big && warp < A_WARPS) {
                simt::WarpEig &we = reinterpret_cast<simt::WarpEig *>(oper)[warp];
                const int nn[NCLS] = {n0, n1, n2};
#pragma unroll 1
                for (int cls = 0; cls < NCLS; ++cls) {  // large supports first: they set the tail
#pragma unroll 1
                    for (;;) {
                        const int i = next_item(p, t, cls, nn[cls]);
                        if (i < 0) break;
                        const int k = support_indices_cg(p.Scur + (size_t)i * W, W, we.idx);
                        double LS;
                        if (k == 0) {
                            LS = L;
                        } else if (k == 1) {
                            LS = (double)__ldg(p.B + (size_t)we.idx[0] * m + we.idx[0]);
                        } else if (k <= simt::SMALL_K) {
                            LS = simt::solve_small(p.B, m, we.idx, k, we.al, we.be, we.e2);
                        } else if (k <= simt::KMAX) {
                            const int lda = eig::vec_ld(k);
                            if (simt::gather_bss<32>(p.B, m, we.idx, k, we.A, lda))
                                LS = eig::lanczos_max_eig_warp<simt::KMAX / 32>(we.A, lda, k, we.q, we.qp, we.al,
                                                                                we.be, we.e2);
                            else
                                LS = (double)simt::max_diag(we.A, lda, k);
                        } else if (p.Dt != nullptr) {
                            const int lda = eig::vec_ld(p.n);
                            simt::gram_ds(p.Dt, p.n, we.idx, k, we.A, lda, we.col);
                            LS = eig::lanczos_max_eig_warp<simt::KMAX / 32>(we.A, lda, p.n, we.q, we.qp, we.al,
                                                                            we.be, we.e2);
                        } else {
                            LS = simt::lanczos_global(p.B, m, we.idx, k, we);
                        }
                        __syncwarp();
                        publish(p, i, W, LS);
                    }
                }
            } else {
                // supports of at most 32 codes, matrix in registers
                simt::WarpEigS &ws = sh.small[warp];
#pragma unroll 1
                for (;;) {
                    const int i = next_item(p, t, 2, n2);
                    if (i < 0) break;
                    const int k = support_indices_cg(p.Scur + (size_t)i * W, W, ws.idx);
                    const double LS = k == 0   ? L
                                      : k == 1 ? (double)__ldg(p.B + (size_t)ws.idx[0] * m + ws.idx[0])
                                               : simt::solve_small(p.B, m, ws.idx, k, ws.al, ws.be, ws.e2);
                    publish(p, i, W, LS);
                }
            }
            __syncthreads();
            if (big) E.reload(p.Bsplit);
#pragma unroll
            for (int pc = 0; pc < CF::NPC; ++pc) {
                float v[16];
                tc::tmem_ld16(E.taddr(CF::T_AHI + cbase + 16 * pc), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) z[16 * pc + j] = v[j];
            }
        }
        // ---- every L_S of layer t is published
        if (!(ok = grid_sync(p.gbar, 32))) break;
        // ---- (B) layer t
        if (cg == 0) {
            const bool acc = row_ok && sh.bad[0][r] == 0;
            float a = (float)(1.0 / L);
            if (acc) a = (float)(1.0 / __ldcg(p.LSv + row));
            sh.step[r] = a;
            if (last && row_ok && p.LS_out) p.LS_out[row] = __ldcg(p.LSv + row);
            const int cnt = __popc(__ballot_sync(0xffffffffu, acc));
            if (lane == 0 && cnt) atomicAdd(&sh.nacc, cnt);
        }
        __syncthreads();
        if (tid == 0 && p.accepted && sh.nacc) atomicAdd(p.accepted + t, sh.nacc);
        const float a = sh.step[r];
        const float thr = __fmul_rn(a, lam);
        const bool refresh = (t + 1) % tc::REFRESH == 0;
#pragma unroll
        for (int pc = 0; pc < CF::NPC; ++pc) {
            const int col0 = cbase + 16 * pc;
            float gv[16];
            tc::tmem_ld16(E.taddr(CF::T_G + col0), gv);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float zo = z[16 * pc + j];
                const float u = fmaf(a, gv[j], zo);
                const float zn = copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
                gv[j] = refresh ? -zn : zo - zn;  // the MMA's A operand
                z[16 * pc + j] = zn;
            }
            if (!last) tc::store_split16(E, col0, gv);
        }
        if (last) break;
        if (refresh)
#pragma unroll 1
            for (int pc = 0; pc < CF::NPC; ++pc)
                tc::row16_to_tmem(E, p.C, row, row_ok, m, cbase + 16 * pc, CF::T_G + cbase + 16 * pc);
        tc::tmem_st_wait();
        if (!(ok = E.contract(false))) break;
    }
    __syncthreads();  // the staging area held the per-row scratch
    if (ok) {
        float *wbuf = E.warp_stage();
        const int rbase = blockIdx.x * TR + quad * 32;
        const int nrow = max(0, min(min(32, TR - quad * 32), N - rbase));
#pragma unroll
        for (int pc = 0; pc < CF::NPC; ++pc) {
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = z[16 * pc + j];
            tc::stage_put(wbuf, v);
            tc::stage_to_global(wbuf, p.Z, rbase, nrow, m, cbase + 16 * pc);
        }
    }
    E.finish();
}

__global__ void transpose_kernel(const float *__restrict__ D, int n, int m, float *__restrict__ Dt)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * m) {
        const int i = e / m, j = e % m;
        Dt[(size_t)j * n + i] = __ldg(D + e);
    }
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace: split B, D^T, cached L_S, two support arrays, the lists, the
// counters, queue positions and the barrier.
struct OisWs {
    uint8_t *Bsplit;
    float *Dt;
    double *LSv;
    uint32_t *Sprev, *Scur;
    int *list, *counter, *qpos;
    unsigned *gbar;
    static size_t bytes(int m, int N, int T)
    {
        const size_t W = (size_t)(m + 31) / 32;
        return 256 + a256((size_t)MP * MP * 4) + a256(sizeof(float) * (size_t)m * simt::KMAX) +
               a256(sizeof(double) * (size_t)N) + 2 * a256(sizeof(uint32_t) * N * W) +
               a256(sizeof(int) * 2 * NCLS * (size_t)N) + a256(sizeof(int) * (2 * NCLS * (size_t)T + 2));
    }
    static OisWs carve(void *ws, int m, int N, int T)
    {
        const size_t W = (size_t)(m + 31) / 32;
        char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255);
        auto take = [&p](size_t b) {
            char *q = p;
            p += a256(b);
            return q;
        };
        OisWs o;
        o.Bsplit = reinterpret_cast<uint8_t *>(take((size_t)MP * MP * 4));
        o.Dt = reinterpret_cast<float *>(take(sizeof(float) * (size_t)m * simt::KMAX));
        o.LSv = reinterpret_cast<double *>(take(sizeof(double) * (size_t)N));
        o.Sprev = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * N * W));
        o.Scur = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * N * W));
        o.list = reinterpret_cast<int *>(take(sizeof(int) * 2 * NCLS * (size_t)N));
        // counters, queue positions and the barrier adjacent: one memset clears them
        o.counter = reinterpret_cast<int *>(take(sizeof(int) * (2 * NCLS * (size_t)T + 2)));
        o.qpos = o.counter + NCLS * (size_t)T;
        o.gbar = reinterpret_cast<unsigned *>(o.qpos + NCLS * (size_t)T);
        return o;
    }
};

int cooperative_ok()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return 0;
    return v;
}

}  // namespace

bool supported(int m, int N, int prec)
{
    return prec == SLISTA_PREC_BF16X3 && m > 128 && m <= MP && N >= 1 &&
           (long long)N <= 128LL * num_sms() && cooperative_ok();
}

size_t ws_bytes(int m, int N, int T) { return OisWs::bytes(m, N, T); }

int launch(const OistaArgs &a, void *wsp, cudaStream_t st)
{
    const OisWs w = OisWs::carve(wsp, a.m, a.N, a.T);
    if (a.accepted && a.T > 0) SLISTA_CUDA_TRY(cudaMemsetAsync(a.accepted, 0, sizeof(int) * a.T, st));
    if (a.T == 0) {
        SLISTA_CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(float) * (size_t)a.N * a.m, st));
        return SLISTA_OK;
    }
    SLISTA_CUDA_TRY(cudaMemsetAsync(w.counter, 0, sizeof(int) * (2 * NCLS * (size_t)a.T + 2), st));
    int rc = tc::split_operands(a.B, a.m, MP, w.Bsplit, st);
    if (rc) return rc;
    const bool have_D = a.D != nullptr && a.n >= 1 && a.n <= simt::KMAX;
    if (have_D) {
        transpose_kernel<<<ceil_div((long long)a.n * a.m, 256), 256, 0, st>>>(a.D, a.n, a.m, w.Dt);
        rc = check_launch("transpose_kernel (Oracle-ISTA)");
        if (rc) return rc;
    }
    OisParams p{};
    p.Bsplit = w.Bsplit;
    p.B = a.B;
    p.Dt = have_D ? w.Dt : nullptr;
    p.C = a.C;
    p.n = a.n;
    p.m = a.m;
    p.N = a.N;
    p.T = a.T;
    const int sms = num_sms();
    p.TR = ceil_div(a.N, sms);  // <= 128 (supported())
    p.lam = a.lam;
    p.Lp = a.L;
    p.Z = a.Z;
    p.LS_out = a.LS;
    p.accepted = a.accepted;
    p.want_ls = a.LS != nullptr;
    p.LSv = w.LSv;
    p.Sprev = w.Sprev;
    p.Scur = w.Scur;
    p.list = w.list;
    p.counter = w.counter;
    p.qpos = w.qpos;
    p.gbar = w.gbar;
    const int grid = ceil_div(a.N, p.TR);
    const size_t smem = tc::Cfg<MP, true>::SMEM_STAGED;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    SLISTA_CUDA_TRY(allow_smem(tc_oista_kernel<true>, smem));
    SLISTA_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_oista_kernel<true>, p));
    return check_launch("tc_oista_kernel");
}

}  // namespace tco
}  // namespace slista
