// C ABI of the library (include/slista.h): argument validation, status
// reporting and dispatch to the kernel translation units.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace slista {

static thread_local char g_msg[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}

void clear_error() { g_msg[0] = '\0'; }

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SLISTA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return SLISTA_OK;
}

namespace {
std::mutex g_smem_mu;
std::map<std::pair<const void *, int>, size_t> g_smem;  // (kernel, device) -> bytes opted in
}  // namespace

bool smem_known(const void *kernel, size_t bytes)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    const auto it = g_smem.find({kernel, dev});
    return it != g_smem.end() && it->second >= bytes;
}

void smem_record(const void *kernel, size_t bytes)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    size_t &v = g_smem[{kernel, dev}];
    if (bytes > v) v = bytes;
}

int num_sms()
{
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            cached = v;
        else
            cached = 1;
    }
    return cached;
}

}  // namespace slista

using namespace slista;

namespace {

// Oracle-ISTA with split BF16: the fused cooperative kernel where it applies
// (slista_set_oista_fused(0) selects the two-kernel path everywhere)
std::atomic<int> g_oista_fused{1};

bool valid_prec(int prec)
{
    return prec == SLISTA_PREC_FP32 || prec == SLISTA_PREC_TF32 || prec == SLISTA_PREC_BF16 ||
           prec == SLISTA_PREC_BF16X3;
}

int check_lam(float lam)
{
    if (!(lam >= 0.0f) || isinf(lam)) return fail(SLISTA_ERR_ARG, "lam must be finite and >= 0 (got %g)", (double)lam);
    return SLISTA_OK;
}

// The kernels move the workspace's operand tiles with 16-byte vector loads
// and bulk copies, which need aligned addresses.
bool ws_aligned(const void *ws) { return (reinterpret_cast<uintptr_t>(ws) & 255) == 0; }

// A caller buffer (masks, checkpoints, trajectory) whose stated length is
// below what the call writes or reads: refused before any launch.
int check_len(const void *buf, size_t have, size_t need, const char *fn, const char *what, const char *unit)
{
    if (buf && have < need)
        return fail(SLISTA_ERR_WORKSPACE, "%s: %s holds %zu %s, %zu needed", fn, what, have, unit, need);
    return SLISTA_OK;
}

int forward_common(const PgdArgs &a, int prec, void *ws, size_t ws_bytes, cudaStream_t st, const char *name)
{
    SLISTA_REQUIRE(valid_prec(prec), SLISTA_ERR_ARG, "%s: unknown precision %d", name, prec);
    if (prec == SLISTA_PREC_FP32) {
        SLISTA_REQUIRE(simt::padded_mp(a.m) != 0, SLISTA_ERR_UNSUPPORTED, "%s: FP32 path supports m <= 256", name);
        return simt::launch_forward(a, st);
    }
    if (prec == SLISTA_PREC_TF32) return fail(SLISTA_ERR_UNSUPPORTED, "%s: TF32 is not built", name);
    SLISTA_REQUIRE(tc::supported(a.m) || tcw::supported(a.m), SLISTA_ERR_UNSUPPORTED,
                   "%s: tensor-core path supports m <= 1024 (got %d)", name, a.m);
    if (!tc::supported(a.m)) {  // m > 256: one launch per layer
        const size_t need = tcw::forward_ws_bytes(a.m, a.N);
        SLISTA_REQUIRE(ws_bytes >= need && ws != nullptr && ws_aligned(ws), SLISTA_ERR_WORKSPACE,
                       "%s: workspace of %zu bytes (256-byte aligned) needed, %zu given", name, need, ws_bytes);
        return tcw::launch_forward(a, prec, ws, st);
    }
    const size_t need = tc::forward_ws_bytes(a.m);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws != nullptr && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "%s: workspace of %zu bytes (256-byte aligned) needed, %zu given", name, need, ws_bytes);
    return tc::launch_forward(a, prec, ws, st);
}

}  // namespace

extern "C" {

const char *slista_last_error(void) { return g_msg; }

int slista_device_status(void *stream)
{
    clear_error();
    cudaStream_t st = as_stream(stream);
    SLISTA_CUDA_TRY(cudaStreamSynchronize(st));
    return read_and_clear_device_flag(st);
}

int slista_set_tile_rows(int rows)
{
    clear_error();
    SLISTA_REQUIRE(rows == 0 || (rows >= 32 && rows <= 128), SLISTA_ERR_ARG,
                   "slista_set_tile_rows: 0 or 32 <= rows <= 128 (got %d)", rows);
    return tc::set_tile_rows(rows);
}

int slista_get_tile_rows(void) { return tc::tile_rows(); }

int slista_wait_probe(long long limit_cycles, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(limit_cycles >= 1 && limit_cycles <= 100000000LL, SLISTA_ERR_ARG,
                   "slista_wait_probe: 1 <= limit_cycles <= 1e8 (got %lld)", limit_cycles);
    return tc::launch_wait_probe(limit_cycles, as_stream(stream));
}

size_t slista_ckpt_floats(int m, int N, int T, int ckpt_every)
{
    if (m <= 0 || N <= 0 || T <= 0 || ckpt_every <= 0) return 0;
    const size_t nck = (size_t)((T + ckpt_every - 1) / ckpt_every) - 1;
    return 2 * (size_t)N * (size_t)m * nck;
}

size_t slista_mask_words(int m, int N, int T)
{
    if (m <= 0 || N <= 0 || T <= 0) return 0;
    return (size_t)T * (size_t)N * (size_t)((m + 31) / 32);
}

size_t slista_workspace_bytes(int fn, int m, int N, int T, int prec, int ckpt_every)
{
    if (m <= 0 || N < 0 || T < 0) return 0;
    switch (fn) {
        case SLISTA_FN_ISTA:
        case SLISTA_FN_SLISTA_FWD:
            if (prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3)
                return tc::supported(m) ? tc::forward_ws_bytes(m) : tcw::supported(m) ? tcw::forward_ws_bytes(m, N) : 0;
            return 0;
        case SLISTA_FN_SLISTA_BWD:
            if (ckpt_every <= 0 || T <= 0) return 0;
            if (prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3) {
                const int K = ckpt_every < T ? ckpt_every : T;
                return tc::supported(m) ? tc::backward_ws_bytes(m, N, T, K)
                                        : tcw::supported(m) ? tcw::backward_ws_bytes(m, N, T, K) : 0;
            }
            return simt::backward_ws_bytes(m, N, T, ckpt_every < T ? ckpt_every : T);
        case SLISTA_FN_OISTA: {
            if (!simt::padded_mp(m)) return 0;
            const size_t two = simt::oista_ws_bytes(m, N, T, prec);
            // the fused kernel's workspace whenever it may be chosen
            const size_t one = (prec == SLISTA_PREC_BF16X3 && m > 128) ? tco::ws_bytes(m, N, T) : 0;
            return two > one ? two : one;
        }
        case SLISTA_FN_SLISTA_BWD_TRAJ:
            if ((prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3) && tc::supported(m) && T >= 1)
                return tc::backward_traj_ws_bytes(m, N, T);
            return 0;
        case SLISTA_FN_SUPPORT_LIPSCHITZ: return simt::padded_mp(m) && N > 0 ? simt::support_ls_ws_bytes(m, N) : 0;
        default: return 0;
    }
}

int lasso_gram(const float *D, int n, int m, const float *X, int N, float *B, float *C, double *xsq, double *L,
               void *stream)
{
    clear_error();
    SLISTA_REQUIRE(n >= 1 && m >= 1 && N >= 0, SLISTA_ERR_ARG, "lasso_gram: bad sizes n=%d m=%d N=%d", n, m, N);
    SLISTA_REQUIRE(D && B, SLISTA_ERR_ARG, "lasso_gram: D and B must not be NULL");
    SLISTA_REQUIRE(N == 0 || (X && C && xsq), SLISTA_ERR_ARG, "lasso_gram: X, C, xsq must not be NULL");
    SLISTA_REQUIRE(m <= 1024, SLISTA_ERR_UNSUPPORTED, "lasso_gram: m <= 1024 supported (got %d)", m);
    cudaStream_t st = as_stream(stream);
    int rc = tcg::launch_gram(D, n, m, X, N, B, C, xsq, st);
    if (rc) return rc;
    if (L) {
        if ((n <= m ? n : m) <= 128) return gram::launch_lipschitz_from_D(D, n, m, L, st);
        return gram::launch_lipschitz_from_B(B, m, L, st);
    }
    return SLISTA_OK;
}

int lasso_lipschitz(const float *B, int m, double *L, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(B && L, SLISTA_ERR_ARG, "lasso_lipschitz: B and L must not be NULL");
    SLISTA_REQUIRE(m >= 1 && m <= 1024, SLISTA_ERR_ARG, "lasso_lipschitz: 1 <= m <= 1024 (got %d)", m);
    return gram::launch_lipschitz_from_B(B, m, L, as_stream(stream));
}

int ista_forward(const float *B, const float *C, int m, int N, float lam, const double *L, int T, int prec,
                 float *Z, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 0, SLISTA_ERR_ARG, "ista_forward: bad sizes m=%d N=%d T=%d", m, N, T);
    SLISTA_REQUIRE(B && L, SLISTA_ERR_ARG, "ista_forward: B and L must not be NULL");
    SLISTA_REQUIRE(N == 0 || (C && Z), SLISTA_ERR_ARG, "ista_forward: C and Z must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    PgdArgs a{B, C, m, N, lam, nullptr, L, T, Z, nullptr, nullptr, 1};
    return forward_common(a, prec, ws, ws_bytes, as_stream(stream), "ista_forward");
}

int slista_forward(const float *B, const float *C, int m, int N, float lam, const float *alpha, int T, int prec,
                   float *Z, uint32_t *masks, size_t mask_words, float *ckpt, size_t ckpt_floats, int ckpt_every,
                   void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 0, SLISTA_ERR_ARG, "slista_forward: bad sizes m=%d N=%d T=%d", m, N,
                   T);
    SLISTA_REQUIRE(B && (T == 0 || alpha), SLISTA_ERR_ARG, "slista_forward: B and alpha must not be NULL");
    SLISTA_REQUIRE(N == 0 || (C && Z), SLISTA_ERR_ARG, "slista_forward: C and Z must not be NULL");
    SLISTA_REQUIRE(!ckpt || ckpt_every >= 1, SLISTA_ERR_ARG, "slista_forward: ckpt_every must be >= 1");
    int rc = check_lam(lam);
    if (rc) return rc;
    rc = check_len(masks, mask_words, slista_mask_words(m, N, T), "slista_forward", "masks", "words");
    if (rc) return rc;
    if (ckpt && ckpt_every < T) {
        rc = check_len(ckpt, ckpt_floats, slista_ckpt_floats(m, N, T, ckpt_every), "slista_forward", "ckpt", "floats");
        if (rc) return rc;
    }
    PgdArgs a{B, C, m, N, lam, alpha, nullptr, T, Z, masks, ckpt, ckpt ? ckpt_every : 1};
    return forward_common(a, prec, ws, ws_bytes, as_stream(stream), "slista_forward");
}

int slista_forward_noalloc(const float *B, const float *C, int m, int N, float lam, const float *alpha, int T,
                           int prec, float *Z, uint32_t *masks, size_t mask_words, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 0, SLISTA_ERR_ARG, "slista_forward_noalloc: bad sizes m=%d N=%d T=%d", m,
                   N, T);
    SLISTA_REQUIRE(B && (T == 0 || alpha), SLISTA_ERR_ARG, "slista_forward_noalloc: B and alpha must not be NULL");
    SLISTA_REQUIRE(N == 0 || (C && Z), SLISTA_ERR_ARG, "slista_forward_noalloc: C and Z must not be NULL");
    SLISTA_REQUIRE(prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3, SLISTA_ERR_UNSUPPORTED,
                   "slista_forward_noalloc: precision must be SLISTA_PREC_BF16 or SLISTA_PREC_BF16X3 (got %d)", prec);
    SLISTA_REQUIRE(m <= tc::noalloc_max_m(), SLISTA_ERR_UNSUPPORTED,
                   "slista_forward_noalloc: m = %d exceeds the static scratch limit m <= %d", m, tc::noalloc_max_m());
    int rc = check_lam(lam);
    if (rc) return rc;
    rc = check_len(masks, mask_words, slista_mask_words(m, N, T), "slista_forward_noalloc", "masks", "words");
    if (rc) return rc;
    PgdArgs a{B, C, m, N, lam, alpha, nullptr, T, Z, masks, nullptr, 1};
    return tc::launch_forward_noalloc(a, prec, as_stream(stream));
}

int slista_backward(const float *B, const float *C, int m, int N, float lam, const float *alpha, int T, int prec,
                    const uint32_t *masks, size_t mask_words, const float *ckpt, size_t ckpt_floats, int ckpt_every,
                    const float *gZ, float *dalpha, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 1, SLISTA_ERR_ARG, "slista_backward: bad sizes m=%d N=%d T=%d", m, N,
                   T);
    const bool tcp = prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3;
    SLISTA_REQUIRE(prec == SLISTA_PREC_FP32 || tcp, prec == SLISTA_PREC_TF32 ? SLISTA_ERR_UNSUPPORTED : SLISTA_ERR_ARG,
                   "slista_backward: precision %d not supported", prec);
    SLISTA_REQUIRE(tcp ? (tc::supported(m) || tcw::supported(m)) : simt::padded_mp(m) != 0, SLISTA_ERR_UNSUPPORTED,
                   "slista_backward: m <= %d supported with this precision (got %d)", tcp ? 1024 : 256, m);
    SLISTA_REQUIRE(B && alpha && dalpha, SLISTA_ERR_ARG, "slista_backward: B, alpha, dalpha must not be NULL");
    SLISTA_REQUIRE(ckpt_every >= 1, SLISTA_ERR_ARG, "slista_backward: ckpt_every must be >= 1");
    const int K = ckpt_every < T ? ckpt_every : T;
    SLISTA_REQUIRE(!tcp || K <= 256, SLISTA_ERR_UNSUPPORTED,
                   "slista_backward: tensor-core adjoint needs at most 256 layers between checkpoints (got %d)", K);
    SLISTA_REQUIRE(N == 0 || (C && masks), SLISTA_ERR_ARG, "slista_backward: C and masks must not be NULL");
    SLISTA_REQUIRE(N == 0 || K >= T || ckpt, SLISTA_ERR_ARG, "slista_backward: ckpt must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    rc = check_len(masks, mask_words, slista_mask_words(m, N, T), "slista_backward", "masks", "words");
    if (rc) return rc;
    if (K < T) {
        rc = check_len(ckpt, ckpt_floats, slista_ckpt_floats(m, N, T, K), "slista_backward", "ckpt", "floats");
        if (rc) return rc;
    }
    const bool wide = tcp && !tc::supported(m);
    const size_t need = wide  ? tcw::backward_ws_bytes(m, N, T, K)
                        : tcp ? tc::backward_ws_bytes(m, N, T, K)
                              : simt::backward_ws_bytes(m, N, T, K);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "slista_backward: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    BwdArgs a{B, C, m, N, lam, alpha, T, masks, ckpt, K, gZ, dalpha};
    if (wide) return tcw::launch_backward(a, prec, ws, as_stream(stream));
    if (tcp) return tc::launch_backward(a, prec, ws, as_stream(stream));
    return simt::launch_backward(a, ws, as_stream(stream));
}

size_t slista_traj_floats(int m, int N, int T)
{
    if (m <= 0 || N < 0 || T < 1) return 0;
    return tc::traj_floats(m, N, T);
}

int slista_forward_traj(const float *B, const float *C, int m, int N, float lam, const float *alpha, int T, int prec,
                        float *Z, uint32_t *masks, size_t mask_words, float *traj, size_t traj_floats, void *ws,
                        size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 1, SLISTA_ERR_ARG, "slista_forward_traj: bad sizes m=%d N=%d T=%d", m, N,
                   T);
    SLISTA_REQUIRE(prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3,
                   valid_prec(prec) ? SLISTA_ERR_UNSUPPORTED : SLISTA_ERR_ARG,
                   "slista_forward_traj: precision %d not supported (BF16 or BF16X3)", prec);
    SLISTA_REQUIRE(tc::supported(m) && T <= 256, SLISTA_ERR_UNSUPPORTED,
                   "slista_forward_traj: m <= 256 and T <= 256 supported (got m=%d, T=%d)", m, T);
    SLISTA_REQUIRE(B && alpha, SLISTA_ERR_ARG, "slista_forward_traj: B and alpha must not be NULL");
    SLISTA_REQUIRE(N == 0 || (C && Z && masks && traj), SLISTA_ERR_ARG,
                   "slista_forward_traj: C, Z, masks and traj must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    rc = check_len(masks, mask_words, slista_mask_words(m, N, T), "slista_forward_traj", "masks", "words");
    if (rc) return rc;
    rc = check_len(traj, traj_floats, slista_traj_floats(m, N, T), "slista_forward_traj", "traj", "floats");
    if (rc) return rc;
    const size_t need = tc::forward_ws_bytes(m);
    SLISTA_REQUIRE(ws_bytes >= need && ws != nullptr && ws_aligned(ws), SLISTA_ERR_WORKSPACE,
                   "slista_forward_traj: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    PgdArgs a{B, C, m, N, lam, alpha, nullptr, T, Z, masks, nullptr, T};
    return tc::launch_forward_traj(a, prec, traj, ws, as_stream(stream));
}

int slista_backward_traj(const float *B, int m, int N, float lam, const float *alpha, int T, int prec,
                         const uint32_t *masks, size_t mask_words, const float *traj, size_t traj_floats,
                         const float *gZ, float *dalpha, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 1, SLISTA_ERR_ARG, "slista_backward_traj: bad sizes m=%d N=%d T=%d", m,
                   N, T);
    SLISTA_REQUIRE(prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3,
                   valid_prec(prec) ? SLISTA_ERR_UNSUPPORTED : SLISTA_ERR_ARG,
                   "slista_backward_traj: precision %d not supported (BF16 or BF16X3)", prec);
    SLISTA_REQUIRE(tc::supported(m) && T <= 256, SLISTA_ERR_UNSUPPORTED,
                   "slista_backward_traj: m <= 256 and T <= 256 supported (got m=%d, T=%d)", m, T);
    SLISTA_REQUIRE(B && alpha && dalpha, SLISTA_ERR_ARG, "slista_backward_traj: B, alpha, dalpha must not be NULL");
    SLISTA_REQUIRE(N == 0 || (masks && traj), SLISTA_ERR_ARG, "slista_backward_traj: masks and traj must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    rc = check_len(masks, mask_words, slista_mask_words(m, N, T), "slista_backward_traj", "masks", "words");
    if (rc) return rc;
    rc = check_len(traj, traj_floats, slista_traj_floats(m, N, T), "slista_backward_traj", "traj", "floats");
    if (rc) return rc;
    const size_t need = tc::backward_traj_ws_bytes(m, N, T);
    SLISTA_REQUIRE(ws_bytes >= need && ws != nullptr && ws_aligned(ws), SLISTA_ERR_WORKSPACE,
                   "slista_backward_traj: workspace of %zu bytes (256-byte aligned) needed, %zu given", need,
                   ws_bytes);
    BwdArgs a{B, nullptr, m, N, lam, alpha, T, masks, nullptr, T, gZ, dalpha};
    return tc::launch_backward_traj(a, prec, traj, ws, as_stream(stream));
}

int slista_set_oista_fused(int enable)
{
    clear_error();
    SLISTA_REQUIRE(enable == 0 || enable == 1, SLISTA_ERR_ARG, "slista_set_oista_fused: 0 or 1 (got %d)", enable);
    g_oista_fused.store(enable, std::memory_order_relaxed);
    return SLISTA_OK;
}

int slista_get_oista_fused(void) { return g_oista_fused.load(std::memory_order_relaxed); }

int oista_forward(const float *B, const float *C, const float *D, int n, int m, int N, float lam, const double *L,
                  int T, int prec, float *Z, double *LS, int *accepted, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0 && T >= 0, SLISTA_ERR_ARG, "oista_forward: bad sizes m=%d N=%d T=%d", m, N, T);
    SLISTA_REQUIRE(valid_prec(prec), SLISTA_ERR_ARG, "oista_forward: unknown precision %d", prec);
    SLISTA_REQUIRE(prec != SLISTA_PREC_TF32, SLISTA_ERR_UNSUPPORTED, "oista_forward: TF32 is not built");
    SLISTA_REQUIRE(simt::padded_mp(m) != 0, SLISTA_ERR_UNSUPPORTED, "oista_forward: m <= 256 supported");
    SLISTA_REQUIRE(B && L, SLISTA_ERR_ARG, "oista_forward: B and L must not be NULL");
    SLISTA_REQUIRE(!D || n >= 1, SLISTA_ERR_ARG, "oista_forward: n must be >= 1 when D is given");
    SLISTA_REQUIRE(N == 0 || (C && Z), SLISTA_ERR_ARG, "oista_forward: C and Z must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    OistaArgs a{B, C, D, D ? n : 0, m, N, lam, L, T, Z, LS, accepted, prec};
    if (g_oista_fused.load(std::memory_order_relaxed) && tco::supported(m, N, prec)) {
        const size_t need = tco::ws_bytes(m, N, T);
        SLISTA_REQUIRE(ws_bytes >= need && ws && ws_aligned(ws), SLISTA_ERR_WORKSPACE,
                       "oista_forward: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
        return tco::launch(a, ws, as_stream(stream));
    }
    const size_t need = simt::oista_ws_bytes(m, N, T, prec);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "oista_forward: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    return simt::launch_oista(a, ws, as_stream(stream));
}

int conv_slista_forward(const float *filters, int K, int Lf, const float *X, int N, int n, float lam,
                        const float *alpha, const double *L, int T, float *Z, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(K >= 1 && Lf >= 1 && n >= Lf && N >= 0 && T >= 0, SLISTA_ERR_ARG,
                   "conv_slista_forward: bad sizes K=%d Lf=%d n=%d N=%d T=%d (need n >= Lf >= 1)", K, Lf, n, N, T);
    SLISTA_REQUIRE(conv::supported(K, Lf, n), SLISTA_ERR_UNSUPPORTED,
                   "conv_slista_forward: n <= 8192, K Lf <= 8192 and K (n - Lf + 1) + K Lf + 2 n floats within 200 KiB "
                   "of shared memory (got K=%d Lf=%d n=%d)", K, Lf, n);
    SLISTA_REQUIRE(filters, SLISTA_ERR_ARG, "conv_slista_forward: filters must not be NULL");
    SLISTA_REQUIRE(alpha || L, SLISTA_ERR_ARG, "conv_slista_forward: alpha or L must be given");
    SLISTA_REQUIRE(N == 0 || (X && Z), SLISTA_ERR_ARG, "conv_slista_forward: X and Z must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    ConvArgs a{filters, K, Lf, X, N, n, lam, alpha, L, T, Z};
    return conv::launch_forward(a, as_stream(stream));
}

int conv2d_slista_forward(const float *filters, int K, int Lh, int Lw, const float *X, int N, int H, int W,
                          float lam, const float *alpha, const double *L, int T, float *Z, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(K >= 1 && Lh >= 1 && Lw >= 1 && H >= Lh && W >= Lw && N >= 0 && T >= 0, SLISTA_ERR_ARG,
                   "conv2d_slista_forward: bad sizes K=%d Lh=%d Lw=%d H=%d W=%d N=%d T=%d (need H >= Lh >= 1, "
                   "W >= Lw >= 1)", K, Lh, Lw, H, W, N, T);
    SLISTA_REQUIRE(conv::supported2d(K, Lh, Lw, H, W), SLISTA_ERR_UNSUPPORTED,
                   "conv2d_slista_forward: H W <= 16384, K Lh Lw <= 8192 and the filters, two images and one code "
                   "vector within 200 KiB of shared memory (got K=%d Lh=%d Lw=%d H=%d W=%d)", K, Lh, Lw, H, W);
    SLISTA_REQUIRE(filters, SLISTA_ERR_ARG, "conv2d_slista_forward: filters must not be NULL");
    SLISTA_REQUIRE(alpha || L, SLISTA_ERR_ARG, "conv2d_slista_forward: alpha or L must be given");
    SLISTA_REQUIRE(N == 0 || (X && Z), SLISTA_ERR_ARG, "conv2d_slista_forward: X and Z must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    Conv2dArgs a{filters, K, Lh, Lw, X, N, H, W, lam, alpha, L, T, Z};
    return conv::launch_forward2d(a, as_stream(stream));
}

static int conv_traj_check(const char *fn, const float *filters, int K, int Lf, const float *alpha, int N, int n,
                           int T, float lam)
{
    SLISTA_REQUIRE(K >= 1 && Lf >= 1 && n >= Lf && N >= 0 && T >= 1, SLISTA_ERR_ARG,
                   "%s: bad sizes K=%d Lf=%d n=%d N=%d T=%d (need n >= Lf >= 1, T >= 1)", fn, K, Lf, n, N, T);
    SLISTA_REQUIRE(conv::supported(K, Lf, n) && conv::traj_supported(K, Lf, n, T), SLISTA_ERR_UNSUPPORTED,
                   "%s: filters of at most 32 taps, n <= 8192, and the padded buffers within 200 KiB of shared "
                   "memory (got K=%d Lf=%d n=%d T=%d)", fn, K, Lf, n, T);
    SLISTA_REQUIRE(filters && alpha, SLISTA_ERR_ARG, "%s: filters and alpha must not be NULL", fn);
    return check_lam(lam);
}

size_t conv_slista_backward_workspace_bytes(int K, int Lf, int n, int N, int T)
{
    if (K < 1 || Lf < 1 || n < Lf || N < 0 || T < 1) return 0;
    if (!conv::supported(K, Lf, n) || !conv::traj_supported(K, Lf, n, T)) return 0;
    return conv::backward_ws_bytes(K, Lf, n, N, T);
}

size_t conv_slista_traj_floats(int K, int Lf, int n, int N, int T)
{
    if (K < 1 || Lf < 1 || n < Lf || N < 0 || T < 1) return 0;
    return conv::traj_floats(K, Lf, n, N, T);
}

static int conv_traj_buffer_check(const char *fn, const float *traj, size_t traj_floats, int K, int Lf, int n, int N,
                                  int T)
{
    const size_t need = conv::traj_floats(K, Lf, n, N, T);
    SLISTA_REQUIRE(traj_floats >= need, SLISTA_ERR_WORKSPACE,
                   "%s: traj of %zu floats (conv_slista_traj_floats) needed, %zu given", fn, need, traj_floats);
    SLISTA_REQUIRE(need == 0 || (reinterpret_cast<uintptr_t>(traj) & 15) == 0, SLISTA_ERR_ARG,
                   "%s: traj must be 16-byte aligned", fn);
    return SLISTA_OK;
}

int conv_slista_forward_traj(const float *filters, int K, int Lf, const float *X, int N, int n, float lam,
                             const float *alpha, int T, float *Z, float *traj, size_t traj_floats, void *stream)
{
    clear_error();
    int rc = conv_traj_check("conv_slista_forward_traj", filters, K, Lf, alpha, N, n, T, lam);
    if (rc) return rc;
    SLISTA_REQUIRE(N == 0 || (X && Z && traj), SLISTA_ERR_ARG,
                   "conv_slista_forward_traj: X, Z and traj must not be NULL");
    rc = conv_traj_buffer_check("conv_slista_forward_traj", traj, traj_floats, K, Lf, n, N, T);
    if (rc) return rc;
    ConvArgs a{filters, K, Lf, X, N, n, lam, alpha, nullptr, T, Z};
    return conv::launch_forward_traj(a, traj, as_stream(stream));
}

int conv_slista_backward(const float *filters, int K, int Lf, const float *X, int N, int n, float lam,
                         const float *alpha, int T, const float *traj, size_t traj_floats, float *dalpha, void *ws,
                         size_t ws_bytes, void *stream)
{
    clear_error();
    int rc = conv_traj_check("conv_slista_backward", filters, K, Lf, alpha, N, n, T, lam);
    if (rc) return rc;
    SLISTA_REQUIRE(dalpha && (N == 0 || (X && traj)), SLISTA_ERR_ARG,
                   "conv_slista_backward: dalpha, X and traj must not be NULL");
    rc = conv_traj_buffer_check("conv_slista_backward", traj, traj_floats, K, Lf, n, N, T);
    if (rc) return rc;
    const size_t need = N > 0 ? conv::backward_ws_bytes(K, Lf, n, N, T) : 0;
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "conv_slista_backward: workspace of %zu bytes (256-byte aligned) needed, %zu given", need,
                   ws_bytes);
    ConvArgs a{filters, K, Lf, X, N, n, lam, alpha, nullptr, T, nullptr};
    return conv::launch_backward(a, traj, dalpha, ws, as_stream(stream));
}

size_t lista_workspace_bytes(int n, int m, int N)
{
    if (n < 1 || m < 1 || N < 0) return 0;
    return tcg::lista_ws_bytes(n, N);
}

int lista_forward(const float *D, int n, int m, const float *X, int N, const float *W, const float *alpha,
                  const float *beta, float lam, int T, float *Z, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(n >= 1 && m >= 1 && N >= 0 && T >= 0, SLISTA_ERR_ARG, "lista_forward: bad sizes n=%d m=%d N=%d T=%d",
                   n, m, N, T);
    SLISTA_REQUIRE(m <= 1024 && n <= 1024, SLISTA_ERR_UNSUPPORTED, "lista_forward: n, m <= 1024 supported");
    SLISTA_REQUIRE(D && (T == 0 || (W && alpha && beta)), SLISTA_ERR_ARG,
                   "lista_forward: D, W, alpha and beta must not be NULL");
    SLISTA_REQUIRE(N == 0 || (X && Z), SLISTA_ERR_ARG, "lista_forward: X and Z must not be NULL");
    int rc = check_lam(lam);
    if (rc) return rc;
    const size_t need = tcg::lista_ws_bytes(n, N);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "lista_forward: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    ListaArgs a{D, n, m, X, N, W, alpha, beta, lam, T, Z};
    return tcg::launch_lista(a, ws, as_stream(stream));
}

int lasso_support_lipschitz(const float *B, const float *D, int n, int m, int N, const uint32_t *S, const double *L,
                            double *LS, void *ws, size_t ws_bytes, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0, SLISTA_ERR_ARG, "lasso_support_lipschitz: bad sizes m=%d N=%d", m, N);
    SLISTA_REQUIRE(simt::padded_mp(m) != 0, SLISTA_ERR_UNSUPPORTED, "lasso_support_lipschitz: m <= 256 supported");
    SLISTA_REQUIRE(!D || n >= 1, SLISTA_ERR_ARG, "lasso_support_lipschitz: n must be >= 1 when D is given");
    SLISTA_REQUIRE(N == 0 || (B && S && L && LS), SLISTA_ERR_ARG,
                   "lasso_support_lipschitz: B, S, L and LS must not be NULL");
    const size_t need = N > 0 ? simt::support_ls_ws_bytes(m, N) : 0;
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "lasso_support_lipschitz: workspace of %zu bytes (256-byte aligned) needed, %zu given", need,
                   ws_bytes);
    SupportLsArgs a{B, D, D ? n : 0, m, N, S, L, LS};
    return simt::launch_support_lipschitz(a, ws, as_stream(stream));
}

int lasso_objective(const float *B, const float *C, const double *xsq, const float *Z, int m, int N, float lam,
                    double *F, double *gap, void *stream)
{
    clear_error();
    SLISTA_REQUIRE(m >= 1 && N >= 0, SLISTA_ERR_ARG, "lasso_objective: bad sizes m=%d N=%d", m, N);
    SLISTA_REQUIRE(B, SLISTA_ERR_ARG, "lasso_objective: B must not be NULL");
    SLISTA_REQUIRE(N == 0 || (C && xsq && Z && F), SLISTA_ERR_ARG,
                   "lasso_objective: C, xsq, Z, F must not be NULL");
    SLISTA_REQUIRE(m <= 1024, SLISTA_ERR_UNSUPPORTED, "lasso_objective: m <= 1024 supported (got %d)", m);
    int rc = check_lam(lam);
    if (rc) return rc;
    ObjArgs a{B, C, xsq, Z, m, N, lam, F, gap};
    if (tcg::objective_supported(m)) return tcg::launch_objective(a, as_stream(stream));
    return simt::launch_objective(a, as_stream(stream));
}

static int batch_args(const slista_problem_t *problems, int count, int T, int prec, int ckpt_every, bool bwd,
                      std::vector<tcw::Problem> &out, const char *name)
{
    SLISTA_REQUIRE(count >= 0 && T >= 0 && (count == 0 || problems), SLISTA_ERR_ARG, "%s: bad batch (count=%d T=%d)",
                   name, count, T);
    SLISTA_REQUIRE(valid_prec(prec), SLISTA_ERR_ARG, "%s: unknown precision %d", name, prec);
    SLISTA_REQUIRE(prec == SLISTA_PREC_BF16 || prec == SLISTA_PREC_BF16X3, SLISTA_ERR_UNSUPPORTED,
                   "%s: batches run on the tensor cores (SLISTA_PREC_BF16 or SLISTA_PREC_BF16X3)", name);
    SLISTA_REQUIRE(ckpt_every >= 1, SLISTA_ERR_ARG, "%s: ckpt_every must be >= 1", name);
    SLISTA_REQUIRE(!bwd || T >= 1, SLISTA_ERR_ARG, "%s: T must be >= 1", name);
    out.resize(count);
    for (int i = 0; i < count; ++i) {
        const slista_problem_t &q = problems[i];
        SLISTA_REQUIRE(q.m >= 1 && q.N >= 0, SLISTA_ERR_ARG, "%s: problem %d: bad sizes m=%d N=%d", name, i, q.m, q.N);
        SLISTA_REQUIRE(tcw::supported(q.m), SLISTA_ERR_UNSUPPORTED, "%s: problem %d: m <= 1024 supported (got %d)",
                       name, i, q.m);
        SLISTA_REQUIRE(q.B && (T == 0 || q.alpha), SLISTA_ERR_ARG, "%s: problem %d: B and alpha must not be NULL",
                       name, i);
        SLISTA_REQUIRE(q.N == 0 || q.C, SLISTA_ERR_ARG, "%s: problem %d: C must not be NULL", name, i);
        SLISTA_REQUIRE(!(q.lam < 0.0f) && !isnan(q.lam) && !isinf(q.lam), SLISTA_ERR_ARG,
                       "%s: problem %d: lam must be finite and >= 0", name, i);
        const bool needs_ck = ckpt_every < T;
        char what[64];
        snprintf(what, sizeof(what), "problem %d masks", i);
        int rl = check_len(q.masks, q.mask_words, slista_mask_words(q.m, q.N, T), name, what, "words");
        if (rl) return rl;
        if (needs_ck) {
            snprintf(what, sizeof(what), "problem %d ckpt", i);
            rl = check_len(q.ckpt, q.ckpt_floats, slista_ckpt_floats(q.m, q.N, T, ckpt_every), name, what, "floats");
            if (rl) return rl;
        }
        if (bwd) {
            SLISTA_REQUIRE(q.dalpha, SLISTA_ERR_ARG, "%s: problem %d: dalpha must not be NULL", name, i);
            SLISTA_REQUIRE(q.N == 0 || (q.masks && (!needs_ck || q.ckpt)), SLISTA_ERR_ARG,
                           "%s: problem %d: masks and ckpt must not be NULL", name, i);
        } else {
            SLISTA_REQUIRE(q.N == 0 || q.Z, SLISTA_ERR_ARG, "%s: problem %d: Z must not be NULL", name, i);
        }
        tcw::Problem &p = out[i];
        p = tcw::Problem{};
        p.B = q.B;
        p.C = q.C;
        p.m = q.m;
        p.N = q.N;
        p.lam = q.lam;
        p.alpha = q.alpha;
        p.Z = q.Z;
        p.masks = q.masks;
        p.ckpt = q.ckpt;
        p.gZ = q.gZ;
        p.dalpha = q.dalpha;
    }
    return SLISTA_OK;
}

size_t slista_batched_workspace_bytes(int fn, const slista_problem_t *problems, int count, int T, int prec,
                                      int ckpt_every)
{
    if (count <= 0 || !problems || T < 0 || ckpt_every < 1) return 0;
    (void)prec;
    std::vector<tcw::Problem> v(count);
    for (int i = 0; i < count; ++i) {
        v[i] = tcw::Problem{};
        v[i].m = problems[i].m;
        v[i].N = problems[i].N;
        if (!tcw::supported(v[i].m) || v[i].N < 0) return 0;
    }
    if (fn == SLISTA_FN_SLISTA_FWD) return tcw::persist_forward_ws_bytes(v.data(), count);
    if (fn == SLISTA_FN_SLISTA_BWD && T >= 1) return tcw::persist_backward_ws_bytes(v.data(), count, T, ckpt_every);
    return 0;
}

int slista_forward_batched(const slista_problem_t *problems, int count, int T, int prec, int ckpt_every, void *ws,
                           size_t ws_bytes, void *stream)
{
    clear_error();
    std::vector<tcw::Problem> v;
    int rc = batch_args(problems, count, T, prec, ckpt_every, false, v, "slista_forward_batched");
    if (rc) return rc;
    const size_t need = tcw::persist_forward_ws_bytes(v.data(), count);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "slista_forward_batched: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    return tcw::forward_batch_persist(v.data(), count, T, ckpt_every, prec, ws, as_stream(stream));
}

int slista_backward_batched(const slista_problem_t *problems, int count, int T, int prec, int ckpt_every, void *ws,
                            size_t ws_bytes, void *stream)
{
    clear_error();
    std::vector<tcw::Problem> v;
    int rc = batch_args(problems, count, T, prec, ckpt_every, true, v, "slista_backward_batched");
    if (rc) return rc;
    const size_t need = tcw::persist_backward_ws_bytes(v.data(), count, T, ckpt_every);
    SLISTA_REQUIRE(ws_bytes >= need && (need == 0 || (ws && ws_aligned(ws))), SLISTA_ERR_WORKSPACE,
                   "slista_backward_batched: workspace of %zu bytes (256-byte aligned) needed, %zu given", need, ws_bytes);
    return tcw::backward_batch_persist(v.data(), count, T, ckpt_every, prec, ws, as_stream(stream));
}

}  // extern "C"
