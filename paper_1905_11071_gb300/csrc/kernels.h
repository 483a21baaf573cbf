// Internal launcher interface between the C ABI (abi.cu) and the kernel
// translation units.  Arguments have been validated by the caller.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace slista {

struct PgdArgs {
    const float *B, *C;
    int m, N;
    float lam;
    const float *alpha;  // T steps, or nullptr for ISTA (step 1/L)
    const double *L;     // used when alpha == nullptr
    int T;
    float *Z;
    uint32_t *masks;     // nullable
    float *ckpt;         // nullable
    int ckpt_every;
};

struct BwdArgs {
    const float *B, *C;
    int m, N;
    float lam;
    const float *alpha;
    int T;
    const uint32_t *masks;
    const float *ckpt;
    int ckpt_every;
    const float *gZ;     // nullable
    float *dalpha;
};

struct ObjArgs {
    const float *B, *C;
    const double *xsq;
    const float *Z;
    int m, N;
    float lam;
    double *F, *gap;
};

struct OistaArgs {
    const float *B, *C;
    const float *D;      // nullable: n x m dictionary, for supports larger than 64
    int n, m, N;
    float lam;
    const double *L;
    int T;
    float *Z;
    double *LS;          // nullable
    int *accepted;       // nullable
    int prec;            // SLISTA_PREC_FP32 (SIMT layers) or BF16 / BF16X3 (tensor-core layers)
};

struct ConvArgs {
    const float *F;      // K x Lf filters
    int K, Lf;
    const float *X;      // N x n
    int N, n;
    float lam;
    const float *alpha;  // T steps, or nullptr: 1 / L
    const double *L;
    int T;
    float *Z;            // N x K (n - Lf + 1)
};

struct Conv2dArgs {
    const float *F;      // K x Lh x Lw filters
    int K, Lh, Lw;
    const float *X;      // N x H x W images
    int N, H, W;
    float lam;
    const float *alpha;  // T steps, or nullptr: 1 / L
    const double *L;
    int T;
    float *Z;            // N x K x (H - Lh + 1) x (W - Lw + 1)
};

struct ListaArgs {
    const float *D;      // n x m
    int n, m;
    const float *X;      // N x n
    int N;
    const float *W;      // T x n x m, one matrix per layer
    const float *alpha, *beta;  // T each (device)
    float lam;
    int T;
    float *Z;            // N x m
};

struct SupportLsArgs {
    const float *B;
    const float *D;      // nullable: n x m dictionary, for supports larger than 64
    int n, m, N;
    const uint32_t *S;   // N x ceil(m/32) support words
    const double *L;     // L_empty
    double *LS;          // N
};

namespace simt {
int padded_mp(int m);  // 32/64/128/256, or 0 if m > 256
int launch_forward(const PgdArgs &a, cudaStream_t st);
int launch_backward(const BwdArgs &a, void *ws, cudaStream_t st);
size_t backward_ws_bytes(int m, int N, int T, int K);
int launch_objective(const ObjArgs &a, cudaStream_t st);
int launch_oista(const OistaArgs &a, void *ws, cudaStream_t st);
size_t oista_ws_bytes(int m, int N, int T, int prec);
int launch_support_lipschitz(const SupportLsArgs &a, void *ws, cudaStream_t st);
size_t support_ls_ws_bytes(int m, int N);
}  // namespace simt

namespace gram {
int launch_lipschitz_from_D(const float *D, int n, int m, double *L, cudaStream_t st);
int launch_lipschitz_from_B(const float *B, int m, double *L, cudaStream_t st);
}  // namespace gram

namespace tcg {
// tcgen05 products with the FP32-class six-product BF16 split: B = D^T D,
// C = X D and ||x||^2 (n >= 1, m <= 1024); the objective and gap (m <= 256).
int launch_gram(const float *D, int n, int m, const float *X, int N, float *B, float *C, double *xsq,
                cudaStream_t st);
bool objective_supported(int m);
int read_and_clear_flag(cudaStream_t st);
int launch_objective(const ObjArgs &a, cudaStream_t st);
// coupled LISTA layers (Eq. lista_layer): two products per layer
size_t lista_ws_bytes(int n, int N);
int launch_lista(const ListaArgs &a, void *ws, cudaStream_t st);
}  // namespace tcg

namespace tc {
// tcgen05 forward (SLISTA_PREC_BF16 / SLISTA_PREC_BF16X3).
bool supported(int m);
size_t forward_ws_bytes(int m);
int launch_forward(const PgdArgs &a, int prec, void *ws, cudaStream_t st);
// tcgen05 adjoint (recompute of each segment + reverse sweep); K <= 256.
size_t backward_ws_bytes(int m, int N, int T, int K);
int launch_backward(const BwdArgs &a, int prec, void *ws, cudaStream_t st);
int launch_forward_noalloc(const PgdArgs &a, int prec, cudaStream_t st);
int noalloc_max_m();
// rows per tile of the layer kernels (0: spread the batch evenly over the SMs)
int set_tile_rows(int rows);
int tile_rows();
// One-pass backward: the forward writes the adjoint's inputs (the
// trajectory, traj_floats() floats; 1 <= T <= 256), the backward is one
// reverse sweep (gZ, if given, replaces dF/dz^(T)).
size_t traj_floats(int m, int N, int T);
size_t backward_traj_ws_bytes(int m, int N, int T);
int launch_forward_traj(const PgdArgs &a, int prec, float *traj, void *ws, cudaStream_t st);
int launch_backward_traj(const BwdArgs &a, int prec, const float *traj, void *ws, cudaStream_t st);
// B -> B_hi, B_lo (BF16, zero-padded to MP, the engine's swizzled layout): 4 MP^2 bytes
int split_operands(const float *B, int m, int MP, uint8_t *out, cudaStream_t st);
}  // namespace tc

namespace tco {
// Oracle-ISTA as one cooperative kernel (split BF16, 128 < m <= 256, at most
// 128 samples per SM): the layers, condition (star) and the L_S solves of
// the whole grid between grid-wide barriers.
bool supported(int m, int N, int prec);
size_t ws_bytes(int m, int N, int T);
int launch(const OistaArgs &a, void *ws, cudaStream_t st);
int read_and_clear_flag(cudaStream_t st);
}  // namespace tco

namespace tcw {
// tcgen05 layers for 256 < m <= 1024 and for batches of problems: one launch
// per layer, state in HBM.
struct Problem {
    const float *B, *C;
    int m, N;
    float lam;
    const float *alpha;  // T steps, or nullptr: 1 / L
    const double *L;
    float *Z;
    uint32_t *masks;
    float *ckpt;
    const float *gZ;
    float *dalpha;
};
bool supported(int m);
size_t forward_batch_ws_bytes(const Problem *P, int count);
size_t backward_batch_ws_bytes(const Problem *P, int count, int T, int K);
int forward_batch(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st);
int backward_batch(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st);
// the same through the persistent batch kernels (one launch per 64 problems)
size_t persist_forward_ws_bytes(const Problem *P, int count);
size_t persist_backward_ws_bytes(const Problem *P, int count, int T, int K);
int forward_batch_persist(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st);
int backward_batch_persist(const Problem *P, int count, int T, int K, int prec, void *ws, cudaStream_t st);
size_t forward_ws_bytes(int m, int N);
int launch_forward(const PgdArgs &a, int prec, void *ws, cudaStream_t st);
size_t backward_ws_bytes(int m, int N, int T, int K);
int launch_backward(const BwdArgs &a, int prec, void *ws, cudaStream_t st);
int read_and_clear_flag(cudaStream_t st);

// Oracle-ISTA layer on the tensor cores (m <= 256, state in place).
struct OistaStep {
    const uint8_t *tiles;      // split B (oista_split)
    const float *C;
    float *Zs, *Gs, *Zfinal;
    const double *L, *LSv;
    int *flag;
    uint32_t *Scur;
    const uint32_t *Sprev;
    const int *valid;
    int *list, *counter;       // next layer's lists (3 classes, stride listN) and lengths
    int listN;
    int *accepted;
    double *LS_out;
    int m, N, t, T, want_ls;
    float lam;
};
size_t oista_tiles_bytes(int m);
int oista_split(const float *B, int m, uint8_t *tiles, cudaStream_t st);
int launch_oista_step(const OistaStep &o, int prec, cudaStream_t st);
}  // namespace tcw

// Device-side error flag (set by bounded waits that expire).
int read_and_clear_device_flag(cudaStream_t st);
namespace tc {
int launch_wait_probe(long long limit_cycles, cudaStream_t st);
}

namespace conv {
// layers on a 1-D convolutional dictionary (FP32, CUDA cores)
bool supported(int K, int Lf, int n);
int launch_forward(const ConvArgs &a, cudaStream_t st);
// trajectory forward and its adjoint (filters of at most 32 taps)
bool traj_supported(int K, int Lf, int n, int T);
size_t traj_floats(int K, int Lf, int n, int N, int T);
size_t backward_ws_bytes(int K, int Lf, int n, int N, int T);
int launch_forward_traj(const ConvArgs &a, float *traj, cudaStream_t st);
int launch_backward(const ConvArgs &a, const float *traj, float *dalpha, void *ws, cudaStream_t st);
// layers on a 2-D convolutional dictionary (FP32, CUDA cores)
bool supported2d(int K, int Lh, int Lw, int H, int W);
int launch_forward2d(const Conv2dArgs &a, cudaStream_t st);
}

}  // namespace slista
