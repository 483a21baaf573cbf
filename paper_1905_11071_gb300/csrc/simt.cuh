// FP32 SIMT tile engine used by the CUDA-core kernels (the "plain FP32" path,
// the Gram/objective kernels, the adjoint and Oracle-ISTA).
//
// A CTA of 256 threads owns a tile of NB samples (rows) and all MP columns of
// the code (MP = m padded to a multiple of 32, zero padding).  Thread (ty, tx)
// owns RM consecutive rows and RN columns split into GPT groups of 4
// contiguous columns: column(q, e) = q*4*TXN + 4*tx + e.  Per-thread tile
// values live in registers (float v[RM][RN]).
//
// The contraction acc += A_s * Bg (A_s: NB x KP tile in shared memory, Bg: a
// KP x MP block of a row-major global matrix) streams Bg through a
// double-buffered shared-memory stage of KC rows; A_s rows are read as float4
// broadcasts and B_s rows as conflict-free float4 vectors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace slista {
namespace simt {

constexpr int NT = 256;  // threads per CTA

template <int MP_, int NB_>
struct Tile {
    static constexpr int MP = MP_;                 // output columns (padded)
    static constexpr int NB = NB_;                 // rows (samples) per CTA
    static constexpr int CG = MP / 4;              // float4 column groups
    static constexpr int TXN = CG < 32 ? CG : 32;  // threads along columns
    static constexpr int TYN = NT / TXN;           // threads along rows
    static constexpr int RM = NB / TYN;            // rows per thread
    static constexpr int GPT = CG / TXN;           // column groups per thread
    static constexpr int RN = 4 * GPT;             // columns per thread
    static constexpr int KC = 16;                  // rows of Bg per stage
    static constexpr int LDA = MP + 4;             // A_s row stride for square (K = MP) tiles
    static constexpr int A_FLOATS = NB * LDA;
    static constexpr int BS_FLOATS = 2 * KC * MP;
    static constexpr int SMEM_FLOATS = A_FLOATS + BS_FLOATS;
    static_assert(MP % 32 == 0, "MP must be a multiple of 32");
    static_assert(NB % TYN == 0 && RM >= 1, "NB must be a multiple of TYN");
    static_assert((KC * MP) % NT == 0, "stage must split evenly over threads");
    static_assert(TXN % 8 == 0, "mask packing needs 8-lane groups");
};

template <class TL>
struct Idx {
    int tx, ty;
    __device__ Idx() : tx(threadIdx.x % TL::TXN), ty(threadIdx.x / TL::TXN) {}
    __device__ int row(int i) const { return ty * TL::RM + i; }
    __device__ int col(int q, int e) const { return q * 4 * TL::TXN + 4 * tx + e; }
};

// Soft-thresholding ST(u, thr) = sign(u) max(|u| - thr, 0) (Section 1).
// A zero result may carry the sign of u (-0.0f); it compares equal to 0.
__device__ __forceinline__ float soft_threshold(float u, float thr)
{
    return copysignf(fmaxf(fabsf(u) - thr, 0.0f), u);
}

__device__ __forceinline__ float signf(float v) { return (float)((v > 0.0f) - (v < 0.0f)); }

// acc[i][q*4+e] += sum_k A_s[row(i)][k] * Bg[k][col(q,e)] for k < kdim, col < ncol
// (zero outside).  A_s has row stride lda (a multiple of 4) and must hold
// zeros in columns [kdim, 16*ceil(kdim/16)).  Bg is row-major with leading
// dimension ldb.  Starts with a __syncthreads (so A_s written just before is
// visible) and ends with one (so A_s and B_s may be rewritten right after).
template <class TL>
__device__ __forceinline__ void gemm_acc(float (&acc)[TL::RM][TL::RN], const float *A_s, int lda,
                                         const float *__restrict__ Bg, int kdim, int ncol, int ldb,
                                         float *B_s)
{
    const int NSTAGE = (kdim + TL::KC - 1) / TL::KC;
    constexpr int PER_T = TL::KC * TL::MP / NT;
    const Idx<TL> ix;
    const int tid = threadIdx.x;
    float stage[PER_T];

    auto load = [&](int s) {
#pragma unroll
        for (int j = 0; j < PER_T; ++j) {
            int e = tid + j * NT;
            int r = e / TL::MP, c = e % TL::MP;
            int k = s * TL::KC + r;
            stage[j] = (k < kdim && c < ncol) ? __ldg(Bg + (size_t)k * ldb + c) : 0.0f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int j = 0; j < PER_T; ++j) B_s[buf * TL::KC * TL::MP + tid + j * NT] = stage[j];
    };

    load(0);
    store(0);
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < NSTAGE; ++s) {
        if (s + 1 < NSTAGE) load(s + 1);
        const float *Bs = B_s + (s & 1) * TL::KC * TL::MP;
#pragma unroll
        for (int kk = 0; kk < TL::KC; kk += 4) {
            float4 a4[TL::RM];
#pragma unroll
            for (int i = 0; i < TL::RM; ++i)
                a4[i] = *reinterpret_cast<const float4 *>(A_s + ix.row(i) * lda + s * TL::KC + kk);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float4 b4[TL::GPT];
#pragma unroll
                for (int q = 0; q < TL::GPT; ++q)
                    b4[q] = *reinterpret_cast<const float4 *>(Bs + (kk + u) * TL::MP + q * 4 * TL::TXN + 4 * ix.tx);
#pragma unroll
                for (int i = 0; i < TL::RM; ++i) {
                    float a = u == 0 ? a4[i].x : u == 1 ? a4[i].y : u == 2 ? a4[i].z : a4[i].w;
#pragma unroll
                    for (int q = 0; q < TL::GPT; ++q) {
                        acc[i][q * 4 + 0] = fmaf(a, b4[q].x, acc[i][q * 4 + 0]);
                        acc[i][q * 4 + 1] = fmaf(a, b4[q].y, acc[i][q * 4 + 1]);
                        acc[i][q * 4 + 2] = fmaf(a, b4[q].z, acc[i][q * 4 + 2]);
                        acc[i][q * 4 + 3] = fmaf(a, b4[q].w, acc[i][q * 4 + 3]);
                    }
                }
            }
        }
        if (s + 1 < NSTAGE) store((s + 1) & 1);
        __syncthreads();
    }
}

// Stores the thread's tile values v into A_s (float4 per column group).
template <class TL>
__device__ __forceinline__ void store_tile(float *A_s, const float (&v)[TL::RM][TL::RN])
{
    const Idx<TL> ix;
#pragma unroll
    for (int i = 0; i < TL::RM; ++i)
#pragma unroll
        for (int q = 0; q < TL::GPT; ++q)
            *reinterpret_cast<float4 *>(A_s + ix.row(i) * TL::LDA + q * 4 * TL::TXN + 4 * ix.tx) =
                make_float4(v[i][q * 4 + 0], v[i][q * 4 + 1], v[i][q * 4 + 2], v[i][q * 4 + 3]);
}

// Loads rows [row0, row0+NB) x cols [0, MP) of a row-major N x m global matrix
// (leading dimension ld) into v; zero outside N x m.
template <class TL>
__device__ __forceinline__ void load_rows(float (&v)[TL::RM][TL::RN], const float *__restrict__ G,
                                          int row0, int N, int m, size_t ld)
{
    const Idx<TL> ix;
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        int r = row0 + ix.row(i);
#pragma unroll
        for (int q = 0; q < TL::GPT; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int c = ix.col(q, e);
                v[i][q * 4 + e] = (r < N && c < m) ? __ldg(G + (size_t)r * ld + c) : 0.0f;
            }
    }
}

// Stores v to rows [row0, row0+NB) of a row-major N x m global matrix.
template <class TL>
__device__ __forceinline__ void store_rows(float *__restrict__ G, const float (&v)[TL::RM][TL::RN],
                                           int row0, int N, int m, size_t ld)
{
    const Idx<TL> ix;
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        int r = row0 + ix.row(i);
        if (r >= N) continue;
#pragma unroll
        for (int q = 0; q < TL::GPT; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int c = ix.col(q, e);
                if (c < m) G[(size_t)r * ld + c] = v[i][q * 4 + e];
            }
    }
}

// Packs the non-zero pattern of v into 32-bit support words (bit j%32 of word
// j/32) and writes them to out[row * W + word] for rows < N.  Eight
// consecutive lanes own one word; all lanes of the warp must call this.
template <class TL>
__device__ __forceinline__ void store_support_words(uint32_t *__restrict__ out,
                                                    const float (&v)[TL::RM][TL::RN],
                                                    int row0, int N, int W)
{
    const Idx<TL> ix;
#pragma unroll
    for (int i = 0; i < TL::RM; ++i) {
        int r = row0 + ix.row(i);
#pragma unroll
        for (int q = 0; q < TL::GPT; ++q) {
            uint32_t nib = (uint32_t)(v[i][q * 4 + 0] != 0.0f) | ((uint32_t)(v[i][q * 4 + 1] != 0.0f) << 1) |
                           ((uint32_t)(v[i][q * 4 + 2] != 0.0f) << 2) | ((uint32_t)(v[i][q * 4 + 3] != 0.0f) << 3);
            uint32_t w = nib << ((ix.tx & 7) * 4);
            w |= __shfl_xor_sync(0xffffffffu, w, 1);
            w |= __shfl_xor_sync(0xffffffffu, w, 2);
            w |= __shfl_xor_sync(0xffffffffu, w, 4);
            int word = (q * 4 * TL::TXN + (ix.tx >> 3) * 32) >> 5;
            if ((ix.tx & 7) == 0 && r < N && word < W) out[(size_t)r * W + word] = w;
        }
    }
}

}  // namespace simt
}  // namespace slista
