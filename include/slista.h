/*
 * slista.h - C ABI of the GB300 (sm_103a) library for batched unfolded ISTA,
 * Step-LISTA (SLISTA) and Oracle-ISTA (OISTA) on the Lasso
 *
 *     F_x(z) = 1/2 ||x - D z||^2 + lam ||z||_1          (arXiv 1905.11071, Eq. lasso)
 *
 * solved for N samples at once by T unfolded proximal-gradient layers
 *
 *     z^(t+1) = ST(z^(t) - alpha_t (B z^(t) - c), alpha_t lam),  z^(0) = 0
 *
 * with B = D^T D and c = D^T x (Eq. pgd / Eq. steprec; ISTA is alpha_t = 1/L,
 * Eq. ista).
 *
 * Data layout (all row-major, sample-major):
 *   D     n x m   float32   dictionary (unit-norm columns in the paper's setups)
 *   X     N x n   float32   samples
 *   B     m x m   float32   Gram matrix D^T D (symmetric)
 *   C     N x m   float32   correlations, row i = (D^T x_i)^T
 *   xsq   N       float64   ||x_i||^2
 *   Z     N x m   float32   codes z_i^(T)
 *   alpha T       float32   per-layer step sizes (device memory)
 *   L     1       float64   Lipschitz constant, largest eigenvalue of B (device memory)
 *   masks T x N x W uint32  W = ceil(m/32); bit (j % 32) of word j/32 of row i of
 *                           layer t is 1 iff z_ij^(t+1) != 0 (the support after layer t)
 *   ckpt            float32  checkpoints every K = ckpt_every layers: checkpoint s
 *                           (s = 1 .. ceil(T/K)-1, layer t = sK) holds z^(t) (N x m)
 *                           followed by g^(t) = c - B z^(t) (N x m)
 *
 * Conventions for every entry point:
 *   - Every pointer is a DEVICE pointer owned by the caller unless stated
 *     otherwise; the library allocates no memory.  Scratch space is passed as
 *     (ws, ws_bytes); size it with slista_workspace_bytes().  ws must start on
 *     a 256-byte boundary (cudaMalloc and PyTorch allocations do), else
 *     SLISTA_ERR_WORKSPACE.
 *   - Calls are asynchronous on the CUDA stream passed as `stream`
 *     (a cudaStream_t cast to void*; NULL = legacy default stream).
 *   - Return value: SLISTA_OK (0) or a negative SLISTA_ERR_* code; the message
 *     of the last failure on the calling host thread is slista_last_error().
 *     Arguments are validated before anything is launched; on error no kernel
 *     runs and outputs are untouched.
 *   - Calls on distinct streams with distinct output and workspace buffers may
 *     run concurrently.
 *   - Buffers whose length is not fixed by the shape arguments alone - the
 *     support masks (T x N x ceil(m/32) words), the checkpoints (a function
 *     of ckpt_every) and the trajectory (a device-dependent tile layout) -
 *     are passed with their length in elements (mask_words, ckpt_floats,
 *     traj_floats).  A length below what the call needs
 *     (slista_mask_words, slista_ckpt_floats, slista_traj_floats) returns
 *     SLISTA_ERR_WORKSPACE before any launch.
 */
#ifndef SLISTA_H
#define SLISTA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SLISTA_API __attribute__((visibility("default")))
#else
#define SLISTA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SLISTA_OK               0
#define SLISTA_ERR_ARG         -1  /* null pointer, non-positive size, alpha <= 0, lam < 0 ... */
#define SLISTA_ERR_UNSUPPORTED -2  /* shape or precision not built */
#define SLISTA_ERR_WORKSPACE   -3  /* ws_bytes smaller than slista_workspace_bytes(), ws not 256-byte aligned,
                                    * or a caller buffer (masks, ckpt, traj) shorter than its stated length needs */
#define SLISTA_ERR_CUDA        -4  /* a CUDA runtime call failed */
#define SLISTA_ERR_TIMEOUT     -5  /* a kernel's bounded wait expired (see slista_device_status) */

/* ---- precision of the B z contraction ---------------------------------- */
#define SLISTA_PREC_FP32    0  /* FP32 on the CUDA cores (SIMT); any m */
#define SLISTA_PREC_TF32    1  /* reserved, returns SLISTA_ERR_UNSUPPORTED */
#define SLISTA_PREC_BF16    2  /* tcgen05 tensor cores, BF16 operands, FP32 accumulation */
#define SLISTA_PREC_BF16X3  3  /* tcgen05, split BF16: hi*hi + hi*lo + lo*hi, FP32 accumulation */

/* ---- function ids for slista_workspace_bytes --------------------------- */
#define SLISTA_FN_GRAM       0
#define SLISTA_FN_ISTA       1
#define SLISTA_FN_SLISTA_FWD 2
#define SLISTA_FN_SLISTA_BWD 3
#define SLISTA_FN_OISTA      4
#define SLISTA_FN_OBJECTIVE  5
#define SLISTA_FN_SLISTA_BWD_TRAJ 6
#define SLISTA_FN_SUPPORT_LIPSCHITZ 7

/* Message describing the last failed call on this host thread ("" if none). */
SLISTA_API const char *slista_last_error(void);

/* Synchronises `stream`, then reads and clears the library's device-side
 * error flag, which a kernel sets when one of its bounded waits expires.
 * Returns SLISTA_OK, SLISTA_ERR_TIMEOUT or SLISTA_ERR_CUDA. */
SLISTA_API int slista_device_status(void *stream);

/* Failure-detection check (the paper has no counterpart): launches, on
 * `stream`, one kernel that waits with the library's bounded wait on an
 * mbarrier that nothing arrives at, with the limit lowered to limit_cycles
 * (1 .. 1e8 SM cycles, else SLISTA_ERR_ARG), so that the wait expires and
 * raises the device flag as an expired wait of a layer kernel would.  The
 * next slista_device_status() on that stream then returns
 * SLISTA_ERR_TIMEOUT and clears the flag.  Nothing else is touched. */
SLISTA_API int slista_wait_probe(long long limit_cycles, void *stream);

/* Tuning of the tensor-core layer kernels for m <= 256 (the paper has no
 * counterpart): rows of the batch per tile of the persistent forward /
 * adjoint kernels.  0 (the default) spreads the batch evenly over the SMs
 * (ceil(N / (rounds x SMs)) rows, at most 128); 32 <= rows <= 128 fixes it.
 * The tile layout decides the sizes of slista_traj_floats and of the
 * backward workspaces, so a setting applies to buffers sized after it and
 * must stay unchanged between a forward and the backward that reads its
 * trajectory or checkpoints.  Process-wide; results do not depend on it
 * (samples are independent).  slista_get_tile_rows returns the setting. */
SLISTA_API int slista_set_tile_rows(int rows);
SLISTA_API int slista_get_tile_rows(void);

/* Bytes of scratch the call `fn` needs for these sizes (0 if none). */
SLISTA_API size_t slista_workspace_bytes(int fn, int m, int N, int T, int prec, int ckpt_every);

/* Number of float32 values in the checkpoint buffer of slista_forward /
 * slista_backward: 2 * N * m * (ceil(T / ckpt_every) - 1). */
SLISTA_API size_t slista_ckpt_floats(int m, int N, int T, int ckpt_every);

/* Number of uint32 words in the per-layer support masks: T * N * ceil(m/32). */
SLISTA_API size_t slista_mask_words(int m, int N, int T);

/* Gram quantities of the Lasso: B = D^T D (the matrix behind W_z = Id - D^T D / L,
 * Section 4), C = X D (the D^T x term of the gradient D^T(Dz - x), Eq. ista),
 * xsq_i = ||x_i||^2, and optionally L = largest eigenvalue of D^T D (Section 1,
 * after Eq. ista).  L is taken from the smaller of D^T D and D D^T when that
 * side is <= 128 (Lanczos with full reorthogonalisation on FP32 products,
 * then bisection on the tridiagonal matrix; relative accuracy about 1e-6),
 * else by power iteration on B; a diagonal B gives its largest entry exactly.
 * D: n x m, X: N x n (inputs).  B: m x m, C: N x m, xsq: N, L: 1 (outputs;
 * L may be NULL to skip it).  n, m >= 1, N >= 0. */
SLISTA_API int lasso_gram(const float *D, int n, int m, const float *X, int N,
               float *B, float *C, double *xsq, double *L, void *stream);

/* L = largest eigenvalue of the symmetric PSD matrix B (m x m) (Section 1:
 * L is the largest eigenvalue of D^T D), by the method of lasso_gram applied
 * to B itself. */
SLISTA_API int lasso_lipschitz(const float *B, int m, double *L, void *stream);

/* ISTA, Eq. ista: T layers with the constant step 1/L from z^(0) = 0.
 * L is a device pointer to one double (for example the output of lasso_gram).
 * Z (N x m) receives z^(T).  prec: SLISTA_PREC_*. */
SLISTA_API int ista_forward(const float *B, const float *C, int m, int N, float lam, const double *L,
                 int T, int prec, float *Z, void *ws, size_t ws_bytes, void *stream);

/* Step-LISTA forward, Eq. steprec (Section 4): T layers with the learned
 * steps alpha[0..T-1] (device, all > 0 - checked on the device side is not
 * possible, so positivity is the caller's contract; the host-side wrapper
 * checks it).  Z (N x m) receives z^(T).
 * masks (nullable): per-layer support bits, layout above.
 * mask_words: length of masks (>= slista_mask_words(m, N, T) when masks is
 * given).
 * ckpt (nullable, needs masks): checkpoints every ckpt_every layers, layout above;
 * ckpt_every >= 1 (ignored when ckpt is NULL); ckpt_floats: its length
 * (>= slista_ckpt_floats(m, N, T, ckpt_every) when ckpt is given).  masks
 * and ckpt are what slista_backward consumes. */
SLISTA_API int slista_forward(const float *B, const float *C, int m, int N, float lam,
                   const float *alpha, int T, int prec, float *Z,
                   uint32_t *masks, size_t mask_words, float *ckpt, size_t ckpt_floats, int ckpt_every,
                   void *ws, size_t ws_bytes, void *stream);

/* Step-LISTA forward on the tensor cores (SLISTA_PREC_BF16 or
 * SLISTA_PREC_BF16X3) that allocates nothing and takes no workspace.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory when they call - code whose device memory is owned
 * by another allocator or reserved in full at start-up (a framework's
 * caching pool, a fixed arena, a per-process quota), and loops that cannot
 * afford the device-wide synchronisation cudaMalloc / cudaFree imply.
 * Arguments, results and arithmetic are those of slista_forward with
 * ckpt = NULL (the same kernel runs); masks (nullable) holds mask_words
 * words, at least slista_mask_words(m, N, T) when given.  Its only scratch, the split copy of B
 * (256 KiB), lives in a static device array of the library, which every GPU
 * that loads the library holds until the process exits; m is limited to
 * m <= 256 by its size (larger m: SLISTA_ERR_UNSUPPORTED).
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it; make that first call before any stream
 * capture.  The cached address belongs to the device's current context: it
 * is not looked up again after cudaDeviceReset (or any other teardown of the
 * primary context), so do not call this entry point on a device after
 * resetting it in the same process.  All calls share the array and each call rewrites it completely
 * before use: calls whose work may overlap on the GPU (different streams
 * without ordering between them) race on it and must be serialised by the
 * caller. */
SLISTA_API int slista_forward_noalloc(const float *B, const float *C, int m, int N, float lam,
                                      const float *alpha, int T, int prec, float *Z, uint32_t *masks,
                                      size_t mask_words, void *stream);

/* Step-LISTA backward: the sub-gradient of sum_i F_{x_i}(z_i^(T)) (the
 * empirical form of Eq. unsupervised) with respect to alpha, obtained by the
 * chain rule on Eq. steprec, with derivative 0 at the kinks of ST and of |z|
 * (sign(0) = 0).  The paper takes it by automatic differentiation
 * (Appendix E); here it is the hand-written adjoint
 *     G = dF/dz^(T) = B z^(T) - c + lam sign(z^(T))   (or gZ if not NULL)
 *     for t = T-1 .. 0:  h = G * mask_t;
 *                        dalpha_t = sum_i <h_i, g_i^(t) - lam sign(z_i^(t+1))>;
 *                        G = h - alpha_t B h
 * where g^(t) = c - B z^(t).  Iterates between checkpoints are recomputed
 * from `ckpt`, so masks, ckpt and ckpt_every must come from a slista_forward
 * call with the same B, C, lam, alpha and T; mask_words and ckpt_floats are
 * their lengths (at least slista_mask_words(m, N, T) and, when ckpt_every <
 * T, slista_ckpt_floats(m, N, T, ckpt_every)).
 * prec selects the arithmetic of the recompute and of B h:
 *   SLISTA_PREC_FP32: CUDA cores, FP32.  After a tensor-core forward the
 *     recomputed segments follow the FP32 trajectory from each checkpoint.
 *   SLISTA_PREC_BF16 / SLISTA_PREC_BF16X3: tcgen05 tensor cores with the
 *     products of slista_forward at that precision; with masks and ckpt from
 *     a forward at the same precision the recompute reproduces the forward's
 *     iterates bit for bit.  At most 256 layers between checkpoints
 *     (min(ckpt_every, T) <= 256, else SLISTA_ERR_UNSUPPORTED).
 * gZ (nullable, N x m): upstream gradient dLoss/dz^(T).  dalpha (T, float32)
 * receives the sub-gradient; the per-layer sums are reduced in FP64 in a
 * fixed order, so repeated calls give identical results.
 * ws: at least slista_workspace_bytes(SLISTA_FN_SLISTA_BWD, m, N, T, prec,
 * ckpt_every) bytes (else SLISTA_ERR_WORKSPACE). */
SLISTA_API int slista_backward(const float *B, const float *C, int m, int N, float lam,
                    const float *alpha, int T, int prec,
                    const uint32_t *masks, size_t mask_words, const float *ckpt, size_t ckpt_floats,
                    int ckpt_every,
                    const float *gZ, float *dalpha,
                    void *ws, size_t ws_bytes, void *stream);

/* ---- one-pass backward (tensor cores, m <= 256, 1 <= T <= 256) -----------
 *
 * The same sub-gradient as slista_backward without the recompute: the
 * forward also writes the adjoint's inputs, the trajectory: for every layer
 * t = 0 .. T-1 either
 *     q_t = g^(t) - lam sign(z^(t+1))      (layers that rebuild g from C)
 * or the step z^(t) - z^(t+1), which is -alpha_t q_t on the support of
 * z^(t+1), the only codes the adjoint reads (Eq. steprec); then dF/dz^(T).
 * The backward is a single reverse sweep over them.  Memory for speed: the trajectory holds
 * (T + 1) x N x m floats (plus tile padding) against the checkpoints'
 * ceil(T/K) - 1 pairs of N x m.
 *
 * slista_traj_floats: length of the trajectory buffer (float32) for the
 * current device (its layout follows the tiling of the batch over the
 * device's SMs and is internal: only slista_forward_traj writes it and only
 * slista_backward_traj on the same device reads it); 0 if (m, T) is outside
 * the path's range.
 * slista_forward_traj: slista_forward at SLISTA_PREC_BF16 / BF16X3 writing
 * Z, masks (required: the backward reads them; mask_words >=
 * slista_mask_words(m, N, T)) and traj (traj_floats >=
 * slista_traj_floats(m, N, T)); ws as for slista_forward
 * (SLISTA_FN_SLISTA_FWD).
 * slista_backward_traj: dalpha (T) from masks and traj of a
 * slista_forward_traj call with the same B, lam, alpha, T, prec and N (with
 * the same lengths mask_words and traj_floats as there); gZ
 * (nullable, N x m) replaces dF/dz^(T) as in slista_backward.  ws:
 * slista_workspace_bytes(SLISTA_FN_SLISTA_BWD_TRAJ, m, N, T, prec, 1). */
SLISTA_API size_t slista_traj_floats(int m, int N, int T);
SLISTA_API int slista_forward_traj(const float *B, const float *C, int m, int N, float lam,
                                   const float *alpha, int T, int prec, float *Z, uint32_t *masks,
                                   size_t mask_words, float *traj, size_t traj_floats, void *ws,
                                   size_t ws_bytes, void *stream);
SLISTA_API int slista_backward_traj(const float *B, int m, int N, float lam, const float *alpha, int T,
                                    int prec, const uint32_t *masks, size_t mask_words, const float *traj,
                                    size_t traj_floats, const float *gZ, float *dalpha, void *ws,
                                    size_t ws_bytes, void *stream);

/* ---- ragged batches (many independent problems in one launch per layer) ----
 *
 * Each problem has its own dictionary width m, batch size N, lam, step sizes
 * and buffers; T, ckpt_every and the precision are shared.  The layers of
 * all problems run as one launch per layer (up to 64 problems per launch),
 * on the tensor-core layer kernel for wide dictionaries (any 1 <= m <= 1024):
 * the state (z, g) of every problem lives in the workspace between layers
 * and each launch computes, for every 128-sample x 256-code block of every
 * problem, the block of (z - z') B and the block's z', g' (Eq. steprec).
 * `problems` is a HOST array of `count` descriptors holding device pointers;
 * it is read during the call only.  prec: SLISTA_PREC_BF16 or
 * SLISTA_PREC_BF16X3 (else SLISTA_ERR_UNSUPPORTED).  The paper has no
 * batched entry point: it trains one problem at a time. */
typedef struct slista_problem {
    const float *B;      /* m x m, B = D^T D */
    const float *C;      /* N x m, row i = (D^T x_i)^T */
    int m;               /* 1 <= m <= 1024 */
    int N;               /* >= 0 */
    float lam;           /* >= 0 */
    const float *alpha;  /* T step sizes (> 0) */
    float *Z;            /* forward: N x m codes z^(T) (out) */
    uint32_t *masks;     /* T x N x ceil(m/32) support words: written by the forward
                          * (nullable there), read by the backward */
    size_t mask_words;   /* length of masks (>= slista_mask_words(m, N, T) when given) */
    float *ckpt;         /* slista_ckpt_floats(m, N, T, ckpt_every) floats: written by
                          * the forward, read by the backward; may be NULL when
                          * ckpt_every >= T */
    size_t ckpt_floats;  /* length of ckpt */
    const float *gZ;     /* backward: upstream gradient dLoss/dz^(T) (N x m), nullable */
    float *dalpha;       /* backward: T floats (out) */
} slista_problem_t;

/* Workspace of slista_forward_batched (fn = SLISTA_FN_SLISTA_FWD) or
 * slista_backward_batched (fn = SLISTA_FN_SLISTA_BWD) for these problems. */
SLISTA_API size_t slista_batched_workspace_bytes(int fn, const slista_problem_t *problems, int count, int T,
                                                 int prec, int ckpt_every);

/* Step-LISTA forward (Eq. steprec) of every problem: Z, and masks / ckpt where
 * given (checkpoint layout of slista_forward, every ckpt_every layers). */
SLISTA_API int slista_forward_batched(const slista_problem_t *problems, int count, int T, int prec,
                                      int ckpt_every, void *ws, size_t ws_bytes, void *stream);

/* Step-size sub-gradient of every problem (the adjoint of slista_backward),
 * from the masks and checkpoints of a slista_forward_batched call with the
 * same problems, T, prec and ckpt_every; dalpha per problem. */
SLISTA_API int slista_backward_batched(const slista_problem_t *problems, int count, int T, int prec,
                                       int ckpt_every, void *ws, size_t ws_bytes, void *stream);

/* Oracle-ISTA, Algorithm 1 (Section 3): at every layer, S = supp(z^(t)),
 * L_S = largest eigenvalue of B_SS (Eq. spca; L_empty = L, recomputed only
 * when S changes), y = ST(z - (Bz - c)/L_S, lam/L_S); z^(t+1) = y when
 * supp(y) is inside S (condition (star)), else the ISTA step with 1/L.
 * Condition (star) is decided before L_S (off S it reads |(c - Bz)_j| <= lam,
 * independent of L_S), so L_S is computed only for accepted steps.  L_S comes
 * from Lanczos in FP32 on B_SS, or, for |S| > 64 when D (n x m, nullable) is
 * given, on D_S D_S^T (same non-zero spectrum, n <= 64); relative accuracy
 * about 1e-6.  Outputs: Z (N x m) = z^(T); LS (N, nullable) = the L_S of
 * supp(z^(T-1)), the support the last layer's candidate step used;
 * accepted (T ints, nullable) = number of samples whose step t met condition
 * (star) (zeroed by the call).  Workspace: the per-sample state of the layer
 * loop (slista_workspace_bytes(SLISTA_FN_OISTA, ...)).  prec: SLISTA_PREC_FP32
 * (layers on the CUDA cores) or SLISTA_PREC_BF16X3 / SLISTA_PREC_BF16 (layer
 * products on the tensor cores); TF32 is not built.  m <= 256.
 * With SLISTA_PREC_BF16X3, 128 < m <= 256 and N <= 128 x (the device's SM
 * count), the call is one cooperative kernel (every layer, condition (star)
 * and the L_S solves of the whole grid between grid-wide barriers, the
 * state on chip); otherwise two kernels per layer (the solves, then the
 * layer) with the state in the workspace.  The results agree up to the
 * rounding order of the products. */
SLISTA_API int oista_forward(const float *B, const float *C, const float *D, int n, int m, int N,
                             float lam, const double *L, int T, int prec, float *Z, double *LS,
                             int *accepted, void *ws, size_t ws_bytes, void *stream);

/* Selects the Oracle-ISTA implementation where both apply: 1 (default) the
 * cooperative kernel, 0 the two kernels per layer.  Process-wide; returns
 * SLISTA_ERR_ARG for other values.  slista_get_oista_fused reads it. */
SLISTA_API int slista_set_oista_fused(int enable);
SLISTA_API int slista_get_oista_fused(void);

/* L_S = largest eigenvalue of B_SS for N given supports S_i (Eq. spca,
 * Section 3; L_empty = L), by the eigen-solver of oista_forward's layers:
 * Lanczos in FP32 on B_SS, or on D_S D_S^T for |S| > 64 when D (n x m,
 * nullable; used when n <= 64) is given; |S| = 1 gives B_jj exactly; relative
 * accuracy about 1e-6.  S: N x ceil(m/32) uint32 words, bit j % 32 of word
 * j / 32 of row i set iff code j is in S_i (one layer of the support masks);
 * bits of codes >= m are ignored.  L: device pointer to L (1 double).  LS: N
 * doubles (out).  All device pointers, caller-owned.  m <= 256.  Workspace:
 * slista_workspace_bytes(SLISTA_FN_SUPPORT_LIPSCHITZ, m, N, 0, 0, 0). */
SLISTA_API int lasso_support_lipschitz(const float *B, const float *D, int n, int m, int N, const uint32_t *S,
                                       const double *L, double *LS, void *ws, size_t ws_bytes, void *stream);

/* Coupled LISTA (Eq. lista_layer, Section 4): T layers from z^(0) = 0,
 *     z^(t+1) = ST(z^(t) - alpha_t W_t^T (D z^(t) - x), beta_t lam),
 * with one n x m matrix W_t and two positive scalars per layer; W_t = D and
 * alpha_t = beta_t = 1/L is ISTA.  D: n x m, X: N x n, W: T x n x m (layer t
 * at W + t n m), alpha, beta: T floats, Z: N x m (out), all device memory.
 * Each layer is two tensor-core products with the FP32-class split of the
 * Gram products (R = Z D^T - X, then R W_t finished into the soft-threshold).
 * ws: lista_workspace_bytes(n, m, N) bytes (the residual R, N x n floats).
 * n, m <= 1024. */
SLISTA_API size_t lista_workspace_bytes(int n, int m, int N);
SLISTA_API int lista_forward(const float *D, int n, int m, const float *X, int N, const float *W,
                             const float *alpha, const float *beta, float lam, int T, float *Z, void *ws,
                             size_t ws_bytes, void *stream);

/* Step-LISTA / ISTA forward on a 1-D convolutional dictionary, the
 * structured dictionaries of Section 6 (future work there): K filters d_k of
 * length Lf (filters: K x Lf, row k = d_k), signals of length n, and codes of
 * K maps of P = n - Lf + 1 entries each (valid positions), so that
 *     (D z)[i] = sum_k sum_l d_k[l] z_k[i - l],  m = K P,
 * and column k P + j of the equivalent dense dictionary holds d_k at rows
 * j .. j + Lf - 1.  The layers are Eq. pgd with the product B z replaced by
 * the operator z -> D^T (D z) (2 K P Lf multiply-adds per sample and layer
 * instead of m^2); steps alpha[0..T-1] (device, > 0, Eq. steprec) or, with
 * alpha NULL, 1/L from the device double *L (ISTA, Eq. ista).  X: N x n,
 * Z: N x m (out), sample-major, device memory.  FP32 on the CUDA cores.
 * Limits: n <= 8192, K Lf <= 8192, the filters, two signals and one code
 * vector within 200 KiB of shared memory (SLISTA_ERR_UNSUPPORTED beyond). */
SLISTA_API int conv_slista_forward(const float *filters, int K, int Lf, const float *X, int N, int n,
                                   float lam, const float *alpha, const double *L, int T, float *Z,
                                   void *stream);

/* Step-LISTA / ISTA forward on a 2-D convolutional dictionary (Section 6's
 * structured dictionaries, on images): K filters of Lh x Lw taps (filters:
 * K x Lh x Lw, row-major), images of H x W pixels (X: N x H x W, row-major)
 * and codes of K maps of Ph x Pw = (H - Lh + 1) x (W - Lw + 1) valid
 * positions (Z: N x K x Ph x Pw, out), so that
 *     (D z)[i, j] = sum_k sum_{a,b} d_k[a, b] z_k[i - a, j - b],
 * and column (k Ph + p) Pw + q of the equivalent dense dictionary holds d_k
 * with its top-left tap at pixel (p, q).  The layers are Eq. pgd with B z
 * replaced by z -> D^T (D z); steps alpha[0..T-1] (device, > 0, Eq. steprec)
 * or, with alpha NULL, 1/L from the device double *L (Eq. ista).  Device
 * memory throughout; FP32 on the CUDA cores.  Limits: H W <= 16384,
 * K Lh Lw <= 8192, the filters, two images and one code vector within
 * 200 KiB of shared memory (SLISTA_ERR_UNSUPPORTED beyond). */
SLISTA_API int conv2d_slista_forward(const float *filters, int K, int Lh, int Lw, const float *X, int N, int H,
                                     int W, float lam, const float *alpha, const double *L, int T, float *Z,
                                     void *stream);

/* Step-size sub-gradient on a 1-D convolutional dictionary: the adjoint of
 * conv_slista_forward's Step-LISTA layers (Eq. steprec), the analogue of
 * slista_forward_traj / slista_backward_traj for the structured
 * dictionaries of Section 6.  Filters of at most 32 taps.
 *
 * traj: device, conv_slista_traj_floats(K, Lf, n, N, T) floats, 16-byte
 * aligned, written by conv_slista_forward_traj and read by
 * conv_slista_backward: z^(t+1) of every layer t, sample s, layer t, map k
 * at ((s T + t) K + k) PQ with PQ = P rounded up to a multiple of 4 (entries
 * P .. PQ-1 of a map are zero).  traj_floats is its length; a shorter buffer
 * returns SLISTA_ERR_WORKSPACE before any launch.
 *
 * conv_slista_forward_traj: conv_slista_forward with steps alpha (device,
 * T >= 1, > 0) that also writes traj; Z (N x m) = z^(T).
 *
 * conv_slista_backward: dalpha (device, T floats) = the sub-gradient with
 * respect to alpha of sum_i F_{x_i}(z_i^(T)) (Eq. lasso), from the traj of a
 * conv_slista_forward_traj call with the same filters, X, lam, alpha, T:
 * per sample G = D^T (D z^(T) - x) + lam sign(z^(T)), then for t = T-1..0
 * h = G on the support of z^(t+1), dalpha_t += <h, z^(t+1) - z^(t)> / alpha_t,
 * G = h - alpha_t D^T (D h).  ws: conv_slista_backward_workspace_bytes(K, Lf,
 * n, N, T) bytes of device memory (256-byte aligned; per-CTA partial sums,
 * reduced in FP64 in a fixed order, so the result is run-to-run identical);
 * 0 when the sizes are outside the limits.  Limits: Lf <= 32 and the padded
 * filters, signal, residual, per-pair partial sums and three code vectors
 * within 200 KiB of shared memory (SLISTA_ERR_UNSUPPORTED beyond). */
SLISTA_API size_t conv_slista_traj_floats(int K, int Lf, int n, int N, int T);
SLISTA_API size_t conv_slista_backward_workspace_bytes(int K, int Lf, int n, int N, int T);
SLISTA_API int conv_slista_forward_traj(const float *filters, int K, int Lf, const float *X, int N, int n,
                                        float lam, const float *alpha, int T, float *Z, float *traj,
                                        size_t traj_floats, void *stream);
SLISTA_API int conv_slista_backward(const float *filters, int K, int Lf, const float *X, int N, int n,
                                    float lam, const float *alpha, int T, const float *traj, size_t traj_floats,
                                    float *dalpha, void *ws, size_t ws_bytes, void *stream);

/* Per-sample Lasso objective (Eq. lasso) evaluated from the Gram quantities,
 *     F_i = 1/2 xsq_i - c_i^T z_i + 1/2 z_i^T B z_i + lam ||z_i||_1,
 * and (gap nullable) the duality gap of the standard Lasso dual (not in the
 * paper): with r = x - Dz, s = min(1, lam / ||c - Bz||_inf),
 *     gap_i = F_i - (s x^T r - s^2 ||r||^2 / 2),
 * x^T r = xsq - c^T z, ||r||^2 = xsq - 2 c^T z + z^T B z.
 * B z in FP32, every reduction in FP64.  F, gap: N doubles. */
SLISTA_API int lasso_objective(const float *B, const float *C, const double *xsq, const float *Z,
                    int m, int N, float lam, double *F, double *gap, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SLISTA_H */
