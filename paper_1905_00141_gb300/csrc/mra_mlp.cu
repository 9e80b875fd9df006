// mra_mlp.cu -- the learned surrogate of loglik(theta)/n (include/mra_mlp.h):
// forward, backward and Adam kernels of a 3 -> 64 -> 64 -> 1 SiLU network with
// BF16 parameters and FP32 accumulation, and its C ABI.
//
// One CTA of 256 threads takes 64 samples.  Layer 2 (64 x 64) is the only
// real contraction; per sample it is 4096 multiply-adds, so the whole batch is
// a few tens of MFLOP and the kernels run on the FP32 pipe with the weights
// and the activations of the CTA's samples in shared memory.  Gradients are
// reduced deterministically: every CTA writes its partial sums to its own row
// of a [CTAs][NPARAM] array, and the Adam kernel adds the rows in a fixed
// order.  One training step is the pair (gradient kernel, Adam kernel); a
// CUDA graph of a run of steps is replayed to keep launch cost off the loop.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/mra_mlp.h"

namespace mra {
void set_thread_error(const std::string &msg); // mra_api.cu: text of mra_last_error(NULL)
}

namespace {

constexpr int H = MRA_MLP_HIDDEN;
constexpr int NPAR = MRA_MLP_NPARAM;
constexpr int O_W1 = 0, O_B1 = 3 * H, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H, O_B3 = O_W3 + H;
static_assert(O_B3 + 1 == NPAR, "parameter layout");
constexpr int S = 64;     // samples per CTA
constexpr int NTM = 256;  // threads per CTA
constexpr int LD = H + 1; // padded row of the activation tiles
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

struct Scale {
    double llo[3], inv_span[3]; // log lo, 1 / (log hi - log lo)
    double t_off, t_scale;
};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
// d/dz z s(z) = s(z) (1 + z (1 - s(z))), s the logistic function
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// Network inputs of theta: scaled logs in [-1, 1] over the box.
__device__ __forceinline__ void features(const Scale &sc, const double *th, float *x)
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const double v = th[i];
        x[i] = v > 0.0 ? (float)(2.0 * (log(v) - sc.llo[i]) * sc.inv_span[i] - 1.0) : __int_as_float(0x7fc00000);
    }
}

// Shared-memory weights (BF16 values widened to FP32).
struct SW {
    float w1[H * 3], b1[H], w2[H * LD], b2[H], w3[H], b3;
};

__device__ void load_weights(SW &w, const __nv_bfloat16 *p)
{
    for (int e = threadIdx.x; e < H * H; e += NTM) w.w2[(e / H) * LD + e % H] = __bfloat162float(p[O_W2 + e]);
    for (int e = threadIdx.x; e < 3 * H; e += NTM) w.w1[e] = __bfloat162float(p[O_W1 + e]);
    for (int e = threadIdx.x; e < H; e += NTM) {
        w.b1[e] = __bfloat162float(p[O_B1 + e]);
        w.b2[e] = __bfloat162float(p[O_B2 + e]);
        w.w3[e] = __bfloat162float(p[O_W3 + e]);
    }
    if (threadIdx.x == 0) w.b3 = __bfloat162float(p[O_B3]);
}

// h1 = SiLU(W1 x + b1) for the CTA's samples (Z1 optional: pre-activations).
__device__ void layer1(const SW &w, const float *X, float *Z1, float *A1)
{
    for (int e = threadIdx.x; e < S * H; e += NTM) {
        const int s = e / H, k = e % H;
        const float z = w.b1[k] + w.w1[3 * k] * X[3 * s] + w.w1[3 * k + 1] * X[3 * s + 1] + w.w1[3 * k + 2] * X[3 * s + 2];
        if (Z1) Z1[s * LD + k] = z;
        A1[s * LD + k] = silu(z);
    }
}

// ------------------------------------------------------------- forward --
__global__ void __launch_bounds__(NTM) k_mlp_predict(const __nv_bfloat16 *wp, Scale sc, const double *theta, int B,
                                                     double *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SW &w = *reinterpret_cast<SW *>(smem);
    float *X = reinterpret_cast<float *>(smem + sizeof(SW)); // S x 3
    float *A1 = X + 3 * S;                                  // S x LD
    const int s0 = blockIdx.x * S;
    load_weights(w, wp);
    for (int s = threadIdx.x; s < S; s += NTM) {
        if (s0 + s < B)
            features(sc, theta + 3 * (size_t)(s0 + s), X + 3 * s);
        else
            X[3 * s] = X[3 * s + 1] = X[3 * s + 2] = 0.f;
    }
    __syncthreads();
    layer1(w, X, nullptr, A1);
    __syncthreads();
    // thread (s, jg): units j = jg * 16 .. jg * 16 + 15 of sample s
    const int s = threadIdx.x >> 2, jg = threadIdx.x & 3;
    float y = 0.f;
    for (int jj = 0; jj < H / 4; jj++) {
        const int j = jg * (H / 4) + jj;
        float z = w.b2[j];
#pragma unroll 8
        for (int k = 0; k < H; k++) z = fmaf(w.w2[j * LD + k], A1[s * LD + k], z);
        y = fmaf(w.w3[j], silu(z), y);
    }
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    if (jg == 0 && s0 + s < B) out[s0 + s] = sc.t_off + sc.t_scale * (double)(y + w.b3);
}

// ------------------------------------------------------------ backward --
// Partial gradient of L = (1/2B) sum (yhat - t)^2 over this CTA's samples ->
// part[blockIdx.x][NPAR]; the partial loss -> lossp[blockIdx.x].  With
// `step` non-null, block 0 advances the Adam step counter.
__global__ void __launch_bounds__(NTM) k_mlp_grad(const __nv_bfloat16 *wp, Scale sc, const double *theta,
                                                  const double *target, int B, float *part, float *lossp, int *step)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SW &w = *reinterpret_cast<SW *>(smem);
    float *X = reinterpret_cast<float *>(smem + sizeof(SW)); // S x 3
    float *E = X + 3 * S;                                   // S: dL/dyhat
    float *Z1 = E + S;                                      // S x LD: z1, then dL/dz1
    float *A1 = Z1 + S * LD;                                // S x LD
    float *D2 = A1 + S * LD;                                // S x LD: dL/dz2
    float *A2 = D2 + S * LD;                                // S x LD
    __shared__ float red[NTM / 32];
    const int tid = threadIdx.x, s0 = blockIdx.x * S;
    if (step && blockIdx.x == 0 && tid == 0) *step += 1;
    load_weights(w, wp);
    __shared__ float T[S];
    for (int s = tid; s < S; s += NTM) {
        if (s0 + s < B) {
            features(sc, theta + 3 * (size_t)(s0 + s), X + 3 * s);
            T[s] = (float)((target[s0 + s] - sc.t_off) / sc.t_scale);
        } else {
            X[3 * s] = X[3 * s + 1] = X[3 * s + 2] = 0.f;
            T[s] = 0.f;
        }
    }
    __syncthreads();
    layer1(w, X, Z1, A1);
    __syncthreads();
    // layer 2 and the output, thread (s, jg) with 16 units of sample s
    const float invB = 1.0f / (float)B;
    float lsum = 0.f;
    {
        const int s = tid >> 2, jg = tid & 3;
        float z2[H / 4];
        float y = 0.f;
#pragma unroll
        for (int jj = 0; jj < H / 4; jj++) {
            const int j = jg * (H / 4) + jj;
            float z = w.b2[j];
#pragma unroll 8
            for (int k = 0; k < H; k++) z = fmaf(w.w2[j * LD + k], A1[s * LD + k], z);
            z2[jj] = z;
            const float a = silu(z);
            A2[s * LD + j] = a;
            y = fmaf(w.w3[j], a, y);
        }
        y += __shfl_xor_sync(0xffffffffu, y, 1);
        y += __shfl_xor_sync(0xffffffffu, y, 2);
        const bool valid = s0 + s < B;
        const float r = valid ? (y + w.b3 - T[s]) : 0.f;
        const float e = r * invB;
        if (jg == 0) {
            E[s] = e;
            lsum = 0.5f * r * r * invB;
        }
#pragma unroll
        for (int jj = 0; jj < H / 4; jj++) {
            const int j = jg * (H / 4) + jj;
            D2[s * LD + j] = e * w.w3[j] * dsilu(z2[jj]);
        }
    }
    __syncthreads();
    float *g = part + (size_t)blockIdx.x * NPAR;
    // dW2[j][k] = sum_s D2[s][j] A1[s][k]; thread (j, kg) with 16 k
    {
        const int j = tid >> 2, kg = tid & 3;
        float acc[H / 4];
#pragma unroll
        for (int kk = 0; kk < H / 4; kk++) acc[kk] = 0.f;
        float gb = 0.f, gw3 = 0.f;
        for (int s = 0; s < S; s++) {
            const float d = D2[s * LD + j];
#pragma unroll
            for (int kk = 0; kk < H / 4; kk++) acc[kk] = fmaf(d, A1[s * LD + kg * (H / 4) + kk], acc[kk]);
            if (kg == 0) gb += d;
            if (kg == 1) gw3 = fmaf(E[s], A2[s * LD + j], gw3);
        }
#pragma unroll
        for (int kk = 0; kk < H / 4; kk++) g[O_W2 + j * H + kg * (H / 4) + kk] = acc[kk];
        if (kg == 0) g[O_B2 + j] = gb;
        if (kg == 1) g[O_W3 + j] = gw3;
        if (kg == 2 && j == 0) {
            float gb3 = 0.f;
            for (int s = 0; s < S; s++) gb3 += E[s];
            g[O_B3] = gb3;
        }
    }
    // dz1[s][k] = (sum_j D2[s][j] W2[j][k]) SiLU'(z1[s][k]), in place of z1
    {
        const int s = tid >> 2, kg = tid & 3;
#pragma unroll 4
        for (int kk = 0; kk < H / 4; kk++) {
            const int k = kg * (H / 4) + kk;
            float a = 0.f;
#pragma unroll 8
            for (int j = 0; j < H; j++) a = fmaf(D2[s * LD + j], w.w2[j * LD + k], a);
            Z1[s * LD + k] = a * dsilu(Z1[s * LD + k]);
        }
    }
    __syncthreads();
    // dW1[k][i] = sum_s dz1[s][k] x[s][i] (192 threads), db1[k] (64 threads)
    if (tid < 3 * H) {
        const int k = tid / 3, i = tid % 3;
        float a = 0.f;
        for (int s = 0; s < S; s++) a = fmaf(Z1[s * LD + k], X[3 * s + i], a);
        g[O_W1 + tid] = a;
    } else {
        const int k = tid - 3 * H;
        float a = 0.f;
        for (int s = 0; s < S; s++) a += Z1[s * LD + k];
        g[O_B1 + k] = a;
    }
    // partial loss
    for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int i = 0; i < NTM / 32; i++) l += red[i];
        lossp[blockIdx.x] = l;
    }
}

// -------------------------------------------------------------- update --
// Sum the partial gradients of nblk CTAs in order; optionally store the sum
// (grad) and the loss (loss_out[0]); with lr > 0 apply one Adam step with the
// bias correction of the device step counter and refresh the BF16 copy; with
// hist, store the loss at hist[*step - 1 - base].
__global__ void __launch_bounds__(NTM) k_mlp_adam(const float *part, const float *lossp, int nblk, float *master,
                                                  float *m1, float *m2, __nv_bfloat16 *wbf, const int *step, float lr,
                                                  float *grad, float *loss_out, float *hist, int base)
{
    const int p = blockIdx.x * NTM + threadIdx.x;
    if (p == 0 && (loss_out || hist)) {
        float l = 0.f;
        for (int b = 0; b < nblk; b++) l += lossp[b];
        if (loss_out) loss_out[0] = l;
        if (hist) hist[*step - 1 - base] = l;
    }
    if (p >= NPAR) return;
    float gs = 0.f;
    for (int b = 0; b < nblk; b++) gs += part[(size_t)b * NPAR + p];
    if (grad) grad[p] = gs;
    if (lr > 0.f) {
        const int t = *step;
        const float a = kBeta1 * m1[p] + (1.f - kBeta1) * gs;
        const float v = kBeta2 * m2[p] + (1.f - kBeta2) * gs * gs;
        m1[p] = a;
        m2[p] = v;
        const float c1 = (float)(1.0 - pow((double)kBeta1, (double)t));
        const float c2 = (float)(1.0 - pow((double)kBeta2, (double)t));
        const float w = master[p] - lr * (a / c1) / (sqrtf(v / c2) + kEps);
        master[p] = w;
        wbf[p] = __float2bfloat16_rn(w);
    }
}

__global__ void k_mlp_cast(const float *master, __nv_bfloat16 *wbf)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPAR) wbf[p] = __float2bfloat16_rn(master[p]);
}

constexpr size_t smem_predict() { return sizeof(SW) + (3 * S + S * LD) * sizeof(float); }
constexpr size_t smem_grad() { return sizeof(SW) + (3 * S + S + 4 * S * LD) * sizeof(float); }

} // namespace

struct mra_mlp {
    int device = 0;
    Scale sc{};
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    int *d_step = nullptr;
    int step = 0;               // host mirror of *d_step
    float *part = nullptr;      // [maxblk][NPAR]
    float *lossp = nullptr;     // [maxblk]
    int maxblk = 0;
    cudaStream_t stream = nullptr;
};

namespace {

mra_status fail(mra_status st, const std::string &msg)
{
    mra::set_thread_error(msg);
    return st;
}

mra_status cuda_fail(const char *what, cudaError_t e)
{
    return fail(MRA_ECUDA, std::string("mra_mlp: ") + what + ": " + cudaGetErrorString(e));
}

bool smem_ready(int device)
{
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return false;
    if (done[device]) return true;
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_grad()) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_mlp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_predict()) !=
            cudaSuccess)
        return false;
    done[device] = true;
    return true;
}

mra_status ensure_blocks(mra_mlp *m, int nblk)
{
    if (nblk <= m->maxblk) return MRA_OK;
    cudaFree(m->part);
    cudaFree(m->lossp);
    m->part = nullptr;
    m->lossp = nullptr;
    m->maxblk = 0;
    cudaError_t e = cudaMalloc(&m->part, (size_t)nblk * NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->lossp, (size_t)nblk * sizeof(float));
    if (e != cudaSuccess) return fail(MRA_ENOMEM, "mra_mlp: cannot allocate the gradient partials");
    m->maxblk = nblk;
    return MRA_OK;
}

mra_status upload_params(mra_mlp *m, const float *params)
{
    cudaError_t e = cudaMemcpy(m->master, params, NPAR * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d_step, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail("parameter upload", e);
    k_mlp_cast<<<(NPAR + 255) / 256, 256, 0, m->stream>>>(m->master, m->wbf);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail("parameter cast", e);
    m->step = 0;
    return MRA_OK;
}

bool scaling_ok(const mra_mlp_scaling *s)
{
    if (!s) return false;
    for (int i = 0; i < 3; i++)
        if (!(s->lo[i] > 0.0) || !(s->hi[i] > s->lo[i]) || !std::isfinite(s->hi[i])) return false;
    return std::isfinite(s->t_off) && s->t_scale > 0.0 && std::isfinite(s->t_scale);
}

} // namespace

extern "C" {

mra_status mra_mlp_create(int device, const mra_mlp_scaling *scaling, const float *params, mra_mlp **out)
{
    if (!out) return fail(MRA_EINVAL, "mra_mlp_create: null output pointer");
    *out = nullptr;
    if (!params || !scaling_ok(scaling)) return fail(MRA_EINVAL, "mra_mlp_create: bad scaling or null parameters");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail("cudaSetDevice", e);
    if (!smem_ready(device)) return fail(MRA_ECUDA, "mra_mlp_create: cannot raise the shared-memory limit");
    mra_mlp *m = new mra_mlp;
    m->device = device;
    for (int i = 0; i < 3; i++) {
        m->sc.llo[i] = std::log(scaling->lo[i]);
        m->sc.inv_span[i] = 1.0 / (std::log(scaling->hi[i]) - std::log(scaling->lo[i]));
    }
    m->sc.t_off = scaling->t_off;
    m->sc.t_scale = scaling->t_scale;
    e = cudaMalloc(&m->master, NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->m1, NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->m2, NPAR * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->wbf, NPAR * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_step, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        mra_mlp_free(m);
        return fail(MRA_ENOMEM, std::string("mra_mlp_create: ") + cudaGetErrorString(e));
    }
    mra_status st = upload_params(m, params);
    if (st != MRA_OK) {
        mra_mlp_free(m);
        return st;
    }
    *out = m;
    return MRA_OK;
}

mra_status mra_mlp_set_params(mra_mlp *m, const float *params)
{
    if (!m || !params) return fail(MRA_EINVAL, "mra_mlp_set_params: null pointer");
    cudaSetDevice(m->device);
    return upload_params(m, params);
}

mra_status mra_mlp_get_params(const mra_mlp *m, float *params)
{
    if (!m || !params) return fail(MRA_EINVAL, "mra_mlp_get_params: null pointer");
    cudaSetDevice(m->device);
    cudaError_t e = cudaMemcpy(params, m->master, NPAR * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail("parameter download", e);
    return MRA_OK;
}

mra_status mra_mlp_set_target_scaling(mra_mlp *m, double t_off, double t_scale)
{
    if (!m || !std::isfinite(t_off) || !(t_scale > 0.0) || !std::isfinite(t_scale))
        return fail(MRA_EINVAL, "mra_mlp_set_target_scaling: bad scaling");
    m->sc.t_off = t_off;
    m->sc.t_scale = t_scale;
    return MRA_OK;
}

mra_status mra_mlp_predict(mra_mlp *m, const double *theta_dev, int batch, double *out_dev, void *stream)
{
    if (!m || batch < 0 || (batch > 0 && (!theta_dev || !out_dev)))
        return fail(MRA_EINVAL, "mra_mlp_predict: bad arguments");
    if (batch == 0) return MRA_OK;
    cudaSetDevice(m->device);
    const int nblk = (batch + S - 1) / S;
    k_mlp_predict<<<nblk, NTM, smem_predict(), (cudaStream_t)stream>>>(m->wbf, m->sc, theta_dev, batch, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("predict launch", e);
    return MRA_OK;
}

mra_status mra_mlp_grad(mra_mlp *m, const double *theta_dev, const double *target_dev, int batch, float *grad_dev,
                        float *loss_dev, void *stream)
{
    if (!m || batch < 1 || batch > MRA_MLP_MAX_BATCH || !theta_dev || !target_dev || !grad_dev || !loss_dev)
        return fail(MRA_EINVAL, "mra_mlp_grad: bad arguments");
    cudaSetDevice(m->device);
    const int nblk = (batch + S - 1) / S;
    if (mra_status st = ensure_blocks(m, nblk)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_grad<<<nblk, NTM, smem_grad(), s>>>(m->wbf, m->sc, theta_dev, target_dev, batch, m->part, m->lossp,
                                              nullptr);
    k_mlp_adam<<<(NPAR + NTM - 1) / NTM, NTM, 0, s>>>(m->part, m->lossp, nblk, m->master, m->m1, m->m2, m->wbf,
                                                      m->d_step, 0.f, grad_dev, loss_dev, nullptr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("grad launch", e);
    return MRA_OK;
}

mra_status mra_mlp_train(mra_mlp *m, const double *theta_dev, const double *target_dev, int batch, int steps,
                         float lr, float *loss_hist_dev)
{
    if (!m || batch < 1 || batch > MRA_MLP_MAX_BATCH || steps < 0 || !theta_dev || !target_dev || !(lr > 0.f))
        return fail(MRA_EINVAL, "mra_mlp_train: bad arguments");
    if (steps == 0) return MRA_OK;
    cudaSetDevice(m->device);
    const int nblk = (batch + S - 1) / S;
    if (mra_status st = ensure_blocks(m, nblk)) return st;
    const int base = m->step;
    auto one_step = [&](cudaStream_t s) {
        k_mlp_grad<<<nblk, NTM, smem_grad(), s>>>(m->wbf, m->sc, theta_dev, target_dev, batch, m->part, m->lossp,
                                                  m->d_step);
        k_mlp_adam<<<(NPAR + NTM - 1) / NTM, NTM, 0, s>>>(m->part, m->lossp, nblk, m->master, m->m1, m->m2, m->wbf,
                                                          m->d_step, lr, nullptr, nullptr, loss_hist_dev, base);
    };
    // a graph of G steps, replayed; the remainder launched directly
    const int G = steps < 64 ? steps : 64;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail("begin capture", e);
    for (int i = 0; i < G; i++) one_step(m->stream);
    e = cudaStreamEndCapture(m->stream, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail("graph capture", e);
    }
    for (int r = 0; r < steps / G && e == cudaSuccess; r++) e = cudaGraphLaunch(exec, m->stream);
    for (int i = 0; i < steps % G && e == cudaSuccess; i++) {
        one_step(m->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail("training steps", e);
    m->step += steps;
    return MRA_OK;
}

void mra_mlp_free(mra_mlp *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    void *ptrs[] = {m->master, m->m1, m->m2, m->wbf, m->d_step, m->part, m->lossp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

} // extern "C"
