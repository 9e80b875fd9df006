// mra_noalloc.cu -- an entry point that performs no device allocation.
//
// mra_dense_loglik_noalloc evaluates the single-region case of the library
// (M = 1: the root is the only leaf, so the likelihood is the exact Gaussian
// log-density log N(z; 0, C(S,S) + tau2 I)) for up to MRA_NOALLOC_MAX_N
// observations, in FP64.  It is the large-leaf posterior kernel of libmra
// reduced to one leaf with no coarser basis, and it keeps its working memory
// (the covariance and its factor, the solved vector, the reciprocal pivots)
// in a fixed array compiled into the library instead of memory from
// cudaMalloc.  The array lives on every device that loads the library until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mra.h"
#include "mra_kernels.cuh"

#define MRA_NOALLOC_MAX_N 1024
#define MRA_NOALLOC_SLOTS ((size_t)MRA_NOALLOC_MAX_N * MRA_NOALLOC_MAX_N + 2 * (size_t)MRA_NOALLOC_MAX_N)
#define MRA_NOALLOC_MAX_DEVICES 64

// Fixed working memory: V (n x n), then y (n), then 1/L_jj (n), in doubles.
static __device__ __align__(256) double g_noalloc_scratch[MRA_NOALLOC_SLOTS];

namespace mra {
void set_thread_error(const std::string &msg); // mra_api.cu: text of mra_last_error(NULL)
}

namespace {

// Device address of the array per device ordinal, and the context it was
// looked up in: a reset device (cudaDeviceReset) gets a new primary context in
// which the module, and with it the array, may sit elsewhere.
struct NoallocSlot {
    double *ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool ctx_known = false;
};
std::mutex g_noalloc_mu;
NoallocSlot g_noalloc_slot[MRA_NOALLOC_MAX_DEVICES];

// Unique id of the context current on this thread (cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime's driver entry points so that the
// library does not link the driver directly).  False when no context is
// current yet or the entry points are missing.
bool current_context_id(unsigned long long *id)
{
    typedef int (*get_current_fn)(void **);
    typedef int (*get_id_fn)(void *, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = (get_current_fn)f;
            get_id = (get_id_fn)g;
        }
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// One CTA: V = C(S,S) + tau2 I (lower triangle), V = L L' in place, y = L^{-1} z,
// loglik = -(log|V| + y'y + n log 2 pi) / 2.  Every scratch element read is
// written earlier in the same launch, so nothing has to start at zero.
__global__ void __launch_bounds__(mra::NT) k_dense_noalloc(const double *x, const double *y, const double *z, int n,
                                                          const double *theta, double *loglik, int *status,
                                                          double *scratch)
{
    using namespace mra;
    __shared__ double red[32];
    __shared__ double sc[2];
    __shared__ double sr;
    __shared__ int flag[4];
    const int tid = threadIdx.x;
    if (!theta_ok(theta)) {
        if (tid == 0) {
            *loglik = qnan();
            if (status) *status = ST_EINVAL;
        }
        return;
    }
    const double s2 = theta[0], ib = 1.0 / theta[1], tau2 = theta[2];
    double *V = scratch;
    double *yb = V + (size_t)n * n;
    double *rs = yb + n;
    const double ox = x[0], oy = y[0];
    if (tid == 0) flag[0] = 0;
    for (int a = tid; a < n; a += NT) yb[a] = z[a];
    for (int64_t e = tid; e < (int64_t)n * n; e += NT) {
        const int a = (int)(e / n), q = (int)(e % n);
        if (q <= a)
            V[(size_t)a * n + q] = cov64(s2, ib, (x[a] - ox) - (x[q] - ox), (y[a] - oy) - (y[q] - oy)) +
                                   (a == q ? tau2 : 0.0);
    }
    __syncthreads();
    chol_global(V, n, n, rs, flag, sc, &sr);
    fwd_solve_vec_big(V, n, rs, n, yb);
    double uv = 0.0;
    for (int a = tid; a < n; a += NT) uv += yb[a] * yb[a];
    uv = block_sum(uv, red);
    const double dv = logdet_small(V, n, n, red);
    if (tid == 0) {
        const bool ok = flag[0] == 0;
        *loglik = ok ? -0.5 * (dv + uv + (double)n * 1.8378770664093454836) : qnan();
        if (status) *status = ok ? ST_OK : ST_ENOTPD;
    }
}

} // namespace

extern "C" mra_status mra_dense_loglik_noalloc(const double *x_dev, const double *y_dev, const double *z_dev,
                                               int64_t n, const double *theta_dev, double *loglik_dev,
                                               int *status_dev, void *stream)
{
    if (n < 1 || n > MRA_NOALLOC_MAX_N) {
        mra::set_thread_error("mra_dense_loglik_noalloc: n must lie in [1, " + std::to_string(MRA_NOALLOC_MAX_N) +
                              "], got " + std::to_string((long long)n));
        return MRA_EINVAL;
    }
    if (!x_dev || !y_dev || !z_dev || !theta_dev || !loglik_dev) {
        mra::set_thread_error("mra_dense_loglik_noalloc: null pointer");
        return MRA_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MRA_NOALLOC_MAX_DEVICES) {
        mra::set_thread_error(std::string("mra_dense_loglik_noalloc: no usable current device: ") +
                              cudaGetErrorString(e));
        return MRA_ECUDA;
    }
    double *scratch;
    {
        // Once per device (and again if the device's context has changed since),
        // with that device current: the host-side name of the array is not a
        // device address, so ask the runtime for it.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoallocSlot &slot = g_noalloc_slot[dev];
        unsigned long long id = 0;
        bool have_id = current_context_id(&id);
        if (!slot.ptr || !have_id || !slot.ctx_known || slot.ctx_id != id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                mra::set_thread_error(std::string("mra_dense_loglik_noalloc: cudaGetSymbolAddress failed: ") +
                                      cudaGetErrorString(e));
                return MRA_ECUDA;
            }
            if (!have_id) have_id = current_context_id(&id); // the lookup made the primary context current
            slot.ptr = (double *)p;
            slot.ctx_id = id;
            slot.ctx_known = have_id;
        }
        scratch = slot.ptr;
    }
    k_dense_noalloc<<<1, mra::NT, 0, (cudaStream_t)stream>>>(x_dev, y_dev, z_dev, (int)n, theta_dev, loglik_dev,
                                                            status_dev, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        mra::set_thread_error(std::string("mra_dense_loglik_noalloc: launch failed: ") + cudaGetErrorString(e));
        return MRA_ECUDA;
    }
    return MRA_OK;
}
