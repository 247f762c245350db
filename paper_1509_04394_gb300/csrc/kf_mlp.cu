// kf_mlp.cu -- the learned cost model: a 3-layer MLP (width 64, ReLU, FP32) that predicts
// the log-runtime of a fused group from its features, trained on the GPU by this file's
// own kernels on runtimes the executor measured (kf_dag_time_groups). It stands in for
// the execution-time estimate C_i of the partition model (Sec. VI, Fig. 5), whose
// source (ref. [6]) the paper only cites.
//
// Parameters (one flat vector): W1 (64 x F, row = output unit), b1 (64), W2 (64 x 64),
// b2 (64), w3 (64), b3. Inputs are log1p(features) standardised by the training set's
// mean and deviation; the target is log(ms) standardised likewise. Loss: mean squared
// error. Training is full-batch Adam; gradients are summed per block over per-sample
// vectors kept in shared memory and then over blocks in a fixed order, so a training
// run is deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kf_ctx.h"
#include "kf_device.h"

namespace kf {

constexpr int F = KF_NFEAT;
constexpr int HID = 64;
constexpr int NP = HID * F + HID + HID * HID + HID + HID + 1;
constexpr int OFF_W1 = 0, OFF_B1 = HID * F, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID,
              OFF_B3 = OFF_W3 + HID;
constexpr int SPB = 64;  // samples per block in the gradient kernel
static_assert(NP == KF_MLP_NPARAMS, "parameter count");

struct CostModel {
    std::vector<float> p = std::vector<float>(NP, 0.0f);
    float fmean[F] = {}, fstd[F] = {}, ymean = 0, ystd = 1;
    bool trained = false;
};

void costmodel_free(kf_ctx *ctx)
{
    delete ctx->cm;
    ctx->cm = nullptr;
}

namespace {

// Per block: SPB samples; thread s < SPB runs sample s forward and backward into shared
// vectors, then all threads form the block's gradient sums. Writes part[block][NP] and
// part_loss[block].
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float *__restrict__ p, const float *__restrict__ x,
                                                      const float *__restrict__ y, int n, float inv_n, float *part,
                                                      float *part_loss)
{
    extern __shared__ float sh[];
    float *w = sh;                     // NP parameters
    float *xs = w + NP;                // SPB x F
    float *h1 = xs + SPB * F;          // SPB x HID
    float *h2 = h1 + SPB * HID;        // SPB x HID
    float *dz1 = h2 + SPB * HID;       // SPB x HID
    float *dz2 = dz1 + SPB * HID;      // SPB x HID
    float *dy = dz2 + SPB * HID;       // SPB
    float *lossb = dy + SPB;           // SPB
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * SPB;
    for (int i = tid; i < NP; i += blockDim.x) w[i] = p[i];
    for (int i = tid; i < SPB * F; i += blockDim.x) {
        const int s = s0 + i / F;
        xs[i] = s < n ? x[(int64_t)s * F + i % F] : 0.0f;
    }
    __syncthreads();
    if (tid < SPB) {
        const int s = s0 + tid;
        const bool live = s < n;
        const float *xi = xs + tid * F;
        float *a1 = h1 + tid * HID, *a2 = h2 + tid * HID, *d1 = dz1 + tid * HID, *d2 = dz2 + tid * HID;
        for (int j = 0; j < HID; ++j) {
            float z = w[OFF_B1 + j];
            for (int k = 0; k < F; ++k) z = fmaf(w[OFF_W1 + j * F + k], xi[k], z);
            a1[j] = fmaxf(z, 0.0f);
        }
        float out = w[OFF_B3];
        for (int j = 0; j < HID; ++j) {
            float z = w[OFF_B2 + j];
            for (int k = 0; k < HID; ++k) z = fmaf(w[OFF_W2 + j * HID + k], a1[k], z);
            a2[j] = fmaxf(z, 0.0f);
            out = fmaf(w[OFF_W3 + j], a2[j], out);
        }
        const float e = live ? out - y[s] : 0.0f;
        const float g = 2.0f * e * inv_n;
        dy[tid] = g;
        lossb[tid] = e * e * inv_n;
        for (int j = 0; j < HID; ++j) d2[j] = a2[j] > 0.0f ? g * w[OFF_W3 + j] : 0.0f;
        for (int k = 0; k < HID; ++k) {
            float t = 0.0f;
            for (int j = 0; j < HID; ++j) t = fmaf(w[OFF_W2 + j * HID + k], d2[j], t);
            d1[k] = a1[k] > 0.0f ? t : 0.0f;
        }
    }
    __syncthreads();
    float *out = part + (int64_t)blockIdx.x * NP;
    for (int i = tid; i < NP; i += blockDim.x) {
        float acc = 0.0f;
        if (i < OFF_B1) {  // W1[j][k] = sum_s dz1[s][j] x[s][k]
            const int j = i / F, k = i % F;
            for (int s = 0; s < SPB; ++s) acc = fmaf(dz1[s * HID + j], xs[s * F + k], acc);
        } else if (i < OFF_W2) {
            const int j = i - OFF_B1;
            for (int s = 0; s < SPB; ++s) acc += dz1[s * HID + j];
        } else if (i < OFF_B2) {  // W2[j][k] = sum_s dz2[s][j] h1[s][k]
            const int j = (i - OFF_W2) / HID, k = (i - OFF_W2) % HID;
            for (int s = 0; s < SPB; ++s) acc = fmaf(dz2[s * HID + j], h1[s * HID + k], acc);
        } else if (i < OFF_W3) {
            const int j = i - OFF_B2;
            for (int s = 0; s < SPB; ++s) acc += dz2[s * HID + j];
        } else if (i < OFF_B3) {  // w3[j] = sum_s dy[s] h2[s][j]
            const int j = i - OFF_W3;
            for (int s = 0; s < SPB; ++s) acc = fmaf(dy[s], h2[s * HID + j], acc);
        } else {
            for (int s = 0; s < SPB; ++s) acc += dy[s];
        }
        out[i] = acc;
    }
    if (tid == 0) {
        float l = 0.0f;
        for (int s = 0; s < SPB; ++s) l += lossb[s];
        part_loss[blockIdx.x] = l;
    }
}

// grad[i] = sum over blocks of part[b][i], in block order (deterministic)
__global__ void reduce_kernel(const float *part, const float *part_loss, int nb, float *grad, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) {
        float acc = 0.0f;
        for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * NP + i];
        grad[i] = acc;
    }
    if (i == 0) {
        float l = 0.0f;
        for (int b = 0; b < nb; ++b) l += part_loss[b];
        *loss = l;
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps, int t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float mi = b1 * m[i] + (1.0f - b1) * g[i];
    const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)t)), vh = vi / (1.0f - powf(b2, (float)t));
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

constexpr size_t GRAD_SMEM = sizeof(float) * (NP + SPB * F + 4 * SPB * HID + 2 * SPB);

// Input and output scaling of the inference kernel (standardise = 1): features go in as
// log1p(max(f, 0)) standardised by (fmean, fstd), and the raw output y comes out as
// exp(y ystd + ymean) milliseconds.
struct Norm {
    float fmean[F], fstd[F], ymean, ystd;
};

constexpr int FWD_THREADS = 128;  // samples per block of the inference kernel

// Inference: the forward pass for n samples, one thread per sample, the parameters
// staged in shared memory (all threads of a warp read the same weight at the same time:
// a broadcast, no bank conflicts). The first hidden layer stays in registers; the second
// is consumed unit by unit into the output, so it is never stored. Same operation order
// as the training kernel's forward pass.
__global__ void __launch_bounds__(FWD_THREADS) mlp_forward_kernel(const float *__restrict__ p, const float *__restrict__ x,
                                                                 int n, int standardise, Norm norm, float *__restrict__ y)
{
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = p[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xi[F], a1[HID];
#pragma unroll
    for (int k = 0; k < F; ++k) {
        const float v = x[(int64_t)s * F + k];
        xi[k] = standardise ? (log1pf(fmaxf(v, 0.0f)) - norm.fmean[k]) / norm.fstd[k] : v;
    }
#pragma unroll
    for (int j = 0; j < HID; ++j) {
        float z = w[OFF_B1 + j];
#pragma unroll
        for (int k = 0; k < F; ++k) z = fmaf(w[OFF_W1 + j * F + k], xi[k], z);
        a1[j] = fmaxf(z, 0.0f);
    }
    float out = w[OFF_B3];
#pragma unroll 4
    for (int j = 0; j < HID; ++j) {
        float z = w[OFF_B2 + j];
#pragma unroll
        for (int k = 0; k < HID; ++k) z = fmaf(w[OFF_W2 + j * HID + k], a1[k], z);
        out = fmaf(w[OFF_W3 + j], fmaxf(z, 0.0f), out);
    }
    y[s] = standardise ? expf(fmaf(out, norm.ystd, norm.ymean)) : out;
}

// n rows of x (host) through the network with parameters p (host) on the current device:
// raw outputs (standardise = 0) or predicted milliseconds (standardise = 1). Allocates
// device memory for the call's duration only.
cudaError_t forward_on_device(const float *p, const float *x, int n, int standardise, const Norm &norm, float *y)
{
    struct Bufs {
        float *p = nullptr, *x = nullptr, *y = nullptr;
        ~Bufs()
        {
            for (float *q : {p, x, y})
                if (q) cudaFree(q);
        }
    } d;
    cudaError_t e = cudaMalloc(&d.p, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.x, sizeof(float) * (size_t)n * F);
    if (e == cudaSuccess) e = cudaMalloc(&d.y, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(d.p, p, sizeof(float) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.x, x, sizeof(float) * (size_t)n * F, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    mlp_forward_kernel<<<(n + FWD_THREADS - 1) / FWD_THREADS, FWD_THREADS>>>(d.p, d.x, n, standardise, norm, d.y);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(y, d.y, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost);
    return e;
}

struct DevBufs {
    float *p = nullptr, *x = nullptr, *y = nullptr, *part = nullptr, *pl = nullptr, *g = nullptr, *m = nullptr,
          *v = nullptr, *loss = nullptr;
    ~DevBufs()
    {
        for (float *q : {p, x, y, part, pl, g, m, v, loss})
            if (q) cudaFree(q);
    }
};

cudaError_t alloc_bufs(DevBufs &d, int n)
{
    const int nb = (n + SPB - 1) / SPB;
    cudaError_t e = cudaMalloc(&d.p, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.x, sizeof(float) * (size_t)n * F);
    if (e == cudaSuccess) e = cudaMalloc(&d.y, sizeof(float) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d.part, sizeof(float) * (size_t)nb * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.pl, sizeof(float) * (size_t)nb);
    if (e == cudaSuccess) e = cudaMalloc(&d.g, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.m, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.v, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc(&d.loss, sizeof(float));
    return e;
}

cudaError_t grad_step(const DevBufs &d, int n)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nb = (n + SPB - 1) / SPB;
    mlp_grad_kernel<<<nb, 256, GRAD_SMEM>>>(d.p, d.x, d.y, n, 1.0f / (float)n, d.part, d.pl);
    reduce_kernel<<<(NP + 255) / 256, 256>>>(d.part, d.pl, nb, d.g, d.loss);
    return cudaGetLastError();
}

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double gauss(uint64_t &s)
{
    const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

float feature_in(float f) { return std::log1p(std::fmax(f, 0.0f)); }

CostModel *model_of(kf_ctx *ctx)
{
    if (!ctx->cm) ctx->cm = new (std::nothrow) CostModel;
    return ctx->cm;
}

}  // namespace
kf_status predict_on_host(const CostModel &c, const float *features, int n, float *ms);
}  // namespace kf

using namespace kf;

extern "C" {

kf_status kf_costmodel_grad(kf_ctx *ctx, const float *params, const float *x, const float *y, int n, float *grad,
                            float *loss)
{
    if (!ctx || !params || !x || !y || !grad || n < 1) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    kf::DeviceScope dev_scope(ctx->device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    DevBufs d;
    cudaError_t e = alloc_bufs(d, n);
    if (e == cudaSuccess) e = cudaMemcpy(d.p, params, sizeof(float) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.x, x, sizeof(float) * (size_t)n * F, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = grad_step(d, n);
    if (e == cudaSuccess) e = cudaMemcpy(grad, d.g, sizeof(float) * NP, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, d.loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        return KF_ECUDA;
    }
    return KF_OK;
}

kf_status kf_costmodel_train(kf_ctx *ctx, const float *features, const float *ms, int n, int steps, float lr,
                             unsigned seed, float *final_loss)
{
    if (!ctx || !features || !ms || n < 2 || steps < 1 || !(lr > 0)) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    for (int i = 0; i < n; ++i)
        if (!(ms[i] > 0) || !std::isfinite(ms[i])) return KF_EINVAL;
    CostModel *cm = model_of(ctx);
    if (!cm) return KF_ENOMEM;
    // standardisation of log1p(features) and of log(ms) over the training set
    std::vector<float> xs((size_t)n * F), ys((size_t)n);
    for (int k = 0; k < F; ++k) {
        double s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) {
            const double v = feature_in(features[(size_t)i * F + k]);
            s += v;
            s2 += v * v;
        }
        const double mu = s / n, var = std::fmax(s2 / n - mu * mu, 0.0);
        cm->fmean[k] = (float)mu;
        cm->fstd[k] = (float)std::fmax(std::sqrt(var), 1e-6);
    }
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
        const double v = std::log((double)ms[i]);
        s += v;
        s2 += v * v;
    }
    cm->ymean = (float)(s / n);
    cm->ystd = (float)std::fmax(std::sqrt(std::fmax(s2 / n - (s / n) * (s / n), 0.0)), 1e-6);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < F; ++k)
            xs[(size_t)i * F + k] = (feature_in(features[(size_t)i * F + k]) - cm->fmean[k]) / cm->fstd[k];
        ys[(size_t)i] = (float)((std::log((double)ms[i]) - cm->ymean) / cm->ystd);
    }
    // He initialisation
    uint64_t st = 0x5EEDull ^ ((uint64_t)seed << 17);
    std::vector<float> p(NP, 0.0f);
    for (int i = 0; i < HID * F; ++i) p[OFF_W1 + i] = (float)(gauss(st) * std::sqrt(2.0 / F));
    for (int i = 0; i < HID * HID; ++i) p[OFF_W2 + i] = (float)(gauss(st) * std::sqrt(2.0 / HID));
    for (int i = 0; i < HID; ++i) p[OFF_W3 + i] = (float)(gauss(st) * std::sqrt(1.0 / HID));
    kf::DeviceScope dev_scope(ctx->device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    DevBufs d;
    cudaError_t e = alloc_bufs(d, n);
    if (e == cudaSuccess) e = cudaMemcpy(d.p, p.data(), sizeof(float) * NP, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.x, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.y, ys.data(), sizeof(float) * ys.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d.m, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(d.v, 0, sizeof(float) * NP);
    for (int t = 1; t <= steps && e == cudaSuccess; ++t) {
        e = grad_step(d, n);
        if (e == cudaSuccess) {
            adam_kernel<<<(NP + 255) / 256, 256>>>(d.p, d.g, d.m, d.v, lr, 0.9f, 0.999f, 1e-8f, t);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = grad_step(d, n);  // loss at the final parameters
    float L = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&L, d.loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(cm->p.data(), d.p, sizeof(float) * NP, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        return KF_ECUDA;
    }
    cm->trained = true;
    if (final_loss) *final_loss = L;
    return KF_OK;
}

kf_status kf_costmodel_forward(kf_ctx *ctx, const float *params, const float *x, int n, float *y)
{
    if (!ctx || !params || !x || !y || n < 0) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    if (n == 0) return KF_OK;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e == cudaSuccess) e = forward_on_device(params, x, n, 0, Norm{}, y);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        return KF_ECUDA;
    }
    return KF_OK;
}

kf_status kf_costmodel_predict(kf_ctx *ctx, const float *features, int n, float *ms)
{
    if (!ctx || !features || !ms || n < 0) return KF_EINVAL;
    if (!ctx->cm || !ctx->cm->trained) return KF_ESTATE;
    if (n == 0) return KF_OK;
    if (ctx->device >= 0) {  // a context with a GPU: the inference kernel
        const CostModel &c = *ctx->cm;
        Norm norm;
        for (int k = 0; k < F; ++k) {
            norm.fmean[k] = c.fmean[k];
            norm.fstd[k] = c.fstd[k];
        }
        norm.ymean = c.ymean;
        norm.ystd = c.ystd;
        kf::DeviceScope dev_scope(ctx->device);
        cudaError_t e = dev_scope.status();
        if (e == cudaSuccess) e = forward_on_device(c.p.data(), features, n, 1, norm, ms);
        if (e != cudaSuccess) {
            ctx->last_cuda = (int)e;
            return KF_ECUDA;
        }
        return KF_OK;
    }
    return kf::predict_on_host(*ctx->cm, features, n, ms);
}

}  // extern "C"

namespace kf {
// The network evaluated on the host: for planning contexts without a GPU, and for the
// recompute planner's own queries, which it issues one group at a time from inside its
// dynamic program (a kernel launch and two copies per query would dominate planning).
kf_status predict_on_host(const CostModel &c, const float *features, int n, float *ms)
{
    const float *w = c.p.data();
    for (int i = 0; i < n; ++i) {
        float x[F], h1[HID];
        for (int k = 0; k < F; ++k) x[k] = (feature_in(features[(size_t)i * F + k]) - c.fmean[k]) / c.fstd[k];
        for (int j = 0; j < HID; ++j) {
            float z = w[OFF_B1 + j];
            for (int k = 0; k < F; ++k) z = std::fma(w[OFF_W1 + j * F + k], x[k], z);
            h1[j] = std::fmax(z, 0.0f);
        }
        float out = w[OFF_B3];
        for (int j = 0; j < HID; ++j) {
            float z = w[OFF_B2 + j];
            for (int k = 0; k < HID; ++k) z = std::fma(w[OFF_W2 + j * HID + k], h1[k], z);
            out = std::fma(w[OFF_W3 + j], std::fmax(z, 0.0f), out);
        }
        ms[i] = (float)std::exp((double)out * c.ystd + c.ymean);
    }
    return KF_OK;
}

kf_status predict_group_ms(kf_ctx *model, const float *features, float *ms)
{
    if (!model || !model->cm || !model->cm->trained) return KF_ESTATE;
    return predict_on_host(*model->cm, features, 1, ms);
}
}  // namespace kf

extern "C" {

kf_status kf_costmodel_get(kf_ctx *ctx, float *params, float *norm)
{
    if (!ctx || !params || !norm) return KF_EINVAL;
    if (!ctx->cm || !ctx->cm->trained) return KF_ESTATE;
    std::memcpy(params, ctx->cm->p.data(), sizeof(float) * NP);
    for (int k = 0; k < F; ++k) {
        norm[k] = ctx->cm->fmean[k];
        norm[F + k] = ctx->cm->fstd[k];
    }
    norm[2 * F] = ctx->cm->ymean;
    norm[2 * F + 1] = ctx->cm->ystd;
    return KF_OK;
}

kf_status kf_costmodel_set(kf_ctx *ctx, const float *params, const float *norm)
{
    if (!ctx || !params || !norm) return KF_EINVAL;
    for (int k = 0; k < F; ++k)
        if (!(norm[F + k] > 0)) return KF_EINVAL;
    if (!(norm[2 * F + 1] > 0)) return KF_EINVAL;
    CostModel *cm = model_of(ctx);
    if (!cm) return KF_ENOMEM;
    std::memcpy(cm->p.data(), params, sizeof(float) * NP);
    for (int k = 0; k < F; ++k) {
        cm->fmean[k] = norm[k];
        cm->fstd[k] = norm[F + k];
    }
    cm->ymean = norm[2 * F];
    cm->ystd = norm[2 * F + 1];
    cm->trained = true;
    return KF_OK;
}

}  // extern "C"
