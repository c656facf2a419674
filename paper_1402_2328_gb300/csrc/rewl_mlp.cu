// rewl_mlp.cu -- the warm-start network: a 3 -> 64 -> 64 -> 1 MLP (tanh, float32) that maps
// (e = E/N in the Potts convention, q, 1/L) to ln g(E)/N, trained on converged REWL results of
// small lattices and evaluated for a larger one.  Forward, backward (mean squared error),
// a fixed-order gradient reduction (results do not depend on scheduling) and Adam.
//
// Parameter vector (4481 floats): W1[64][3], b1[64], W2[64][64] (W2[i][j]: hidden-1 unit j ->
// hidden-2 unit i), b2[64], W3[64], b3.
//
// Sizes are tiny (a 64x64 layer over ~10^4 samples), so CUDA cores are used: a tensor-core
// GEMM would not change the cost of the warm start, which is dominated by the REWL runs.
#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "rewl.h"
#include "rewl_device.cuh"

namespace {

constexpr int HID = 64;
constexpr int OFF_W1 = 0, OFF_B1 = HID * 3, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == REWL_MLP_NPARAM, "parameter count");
constexpr int TILE = 128; // samples per CTA in the gradient kernel

thread_local std::string g_mlp_err;

__device__ __forceinline__ void load_params(const float *__restrict__ P, float *sP)
{
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sP[i] = P[i];
    __syncthreads();
}

// forward of one sample; h1, h2 receive the hidden activations
__device__ __forceinline__ float mlp_fwd1(const float *sP, float x0, float x1, float x2,
                                          float *h1, float *h2)
{
#pragma unroll 8
    for (int j = 0; j < HID; ++j) {
        const float z = sP[OFF_B1 + j] + sP[OFF_W1 + 3 * j] * x0 + sP[OFF_W1 + 3 * j + 1] * x1 +
                        sP[OFF_W1 + 3 * j + 2] * x2;
        h1[j] = tanhf(z);
    }
    float y = sP[OFF_B3];
    for (int i = 0; i < HID; ++i) {
        float z = sP[OFF_B2 + i];
        const float *w = sP + OFF_W2 + HID * i;
#pragma unroll 16
        for (int j = 0; j < HID; ++j) z += w[j] * h1[j];
        const float a = tanhf(z);
        h2[i] = a;
        y += sP[OFF_W3 + i] * a;
    }
    return y;
}

__global__ void k_mlp_forward(const float *__restrict__ P, const float *__restrict__ X,
                              float *__restrict__ Y, int n)
{
    extern __shared__ float sP[];
    load_params(P, sP);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h1[HID], h2[HID];
    Y[s] = mlp_fwd1(sP, X[3 * s], X[3 * s + 1], X[3 * s + 2], h1, h2);
}

// Gradient of the mean squared error over one tile of TILE samples, written to partial[tile].
// Sums over samples run in sample order, so the result is the same on every run.
__global__ void __launch_bounds__(TILE) k_mlp_grad_tile(const float *__restrict__ P,
                                                        const float *__restrict__ X,
                                                        const float *__restrict__ T, int n,
                                                        float *__restrict__ partial,
                                                        float *__restrict__ loss_partial)
{
    extern __shared__ float sm[];
    float *sP = sm;                         // NPARAM
    float *sH1 = sP + ((NPARAM + 3) & ~3);  // [TILE][HID+1]
    float *sZ2 = sH1 + TILE * (HID + 1);    // [TILE][HID+1]: h2, then dz2
    float *sX = sZ2 + TILE * (HID + 1);     // [TILE][3]
    float *sDy = sX + TILE * 3;             // [TILE]
    load_params(P, sP);
    const int t = threadIdx.x;
    const int s = blockIdx.x * TILE + t;
    const bool live = s < n;
    float h1[HID], h2[HID];
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, dy = 0.f;
    if (live) {
        x0 = X[3 * s];
        x1 = X[3 * s + 1];
        x2 = X[3 * s + 2];
        const float y = mlp_fwd1(sP, x0, x1, x2, h1, h2);
        const float r = y - T[s];
        dy = 2.0f * r / (float)n;
        sDy[t] = r * r;
    } else {
#pragma unroll
        for (int j = 0; j < HID; ++j) h1[j] = h2[j] = 0.f;
        sDy[t] = 0.f;
    }
    sX[3 * t] = x0;
    sX[3 * t + 1] = x1;
    sX[3 * t + 2] = x2;
    for (int j = 0; j < HID; ++j) {
        sH1[t * (HID + 1) + j] = h1[j];
        sZ2[t * (HID + 1) + j] = h2[j];
    }
    __syncthreads();
    // loss of the tile (fixed order) and dW3, db3 need h2 before it is overwritten
    if (t == 0) {
        float l = 0.f;
        for (int i = 0; i < TILE; ++i) l += sDy[i];
        loss_partial[blockIdx.x] = l;
    }
    __syncthreads();
    sDy[t] = dy;
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * NPARAM;
    if (t < HID) {
        float g = 0.f;
        for (int i = 0; i < TILE; ++i) g += sDy[i] * sZ2[i * (HID + 1) + t];
        out[OFF_W3 + t] = g;
    }
    if (t == HID) {
        float g = 0.f;
        for (int i = 0; i < TILE; ++i) g += sDy[i];
        out[OFF_B3] = g;
    }
    __syncthreads();
    // dz2 = dy W3 (1 - h2^2), then dz1 = (W2^T dz2) (1 - h1^2) for this thread's sample
    for (int i = 0; i < HID; ++i) {
        const float a = sZ2[t * (HID + 1) + i];
        sZ2[t * (HID + 1) + i] = dy * sP[OFF_W3 + i] * (1.f - a * a);
    }
    __syncthreads();
    float dz1[HID];
    for (int j = 0; j < HID; ++j) dz1[j] = 0.f;
    for (int i = 0; i < HID; ++i) {
        const float d = sZ2[t * (HID + 1) + i];
        const float *w = sP + OFF_W2 + HID * i;
#pragma unroll 16
        for (int j = 0; j < HID; ++j) dz1[j] += d * w[j];
    }
    // dW2[i][j] = sum_s dz2[s][i] h1[s][j]; db2[i] = sum_s dz2[s][i]
    for (int e = t; e < HID * HID; e += TILE) {
        const int i = e / HID, j = e % HID;
        float g = 0.f;
        for (int q = 0; q < TILE; ++q) g += sZ2[q * (HID + 1) + i] * sH1[q * (HID + 1) + j];
        out[OFF_W2 + e] = g;
    }
    if (t < HID) {
        float g = 0.f;
        for (int q = 0; q < TILE; ++q) g += sZ2[q * (HID + 1) + t];
        out[OFF_B2 + t] = g;
    }
    __syncthreads();
    // reuse sZ2 for dz1 of every sample
    for (int j = 0; j < HID; ++j) {
        const float a = sH1[t * (HID + 1) + j];
        sZ2[t * (HID + 1) + j] = dz1[j] * (1.f - a * a);
    }
    __syncthreads();
    for (int e = t; e < HID * 4; e += TILE) { // W1[j][c] (c < 3) and b1[j] (c == 3)
        const int j = e / 4, cc = e % 4;
        float g = 0.f;
        for (int q = 0; q < TILE; ++q) {
            const float v = cc == 3 ? 1.f : sX[3 * q + cc];
            g += sZ2[q * (HID + 1) + j] * v;
        }
        if (cc == 3) out[OFF_B1 + j] = g;
        else out[OFF_W1 + 3 * j + cc] = g;
    }
}

// grad[p] = sum over tiles of partial[tile][p] (tile order); loss = sum of tile losses / n
__global__ void k_mlp_reduce(const float *__restrict__ partial, const float *__restrict__ lpart,
                             int ntiles, int n, float *__restrict__ grad, float *__restrict__ loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) {
        float g = 0.f;
        for (int k = 0; k < ntiles; ++k) g += partial[(size_t)k * NPARAM + p];
        grad[p] = g;
    }
    if (p == 0 && loss) {
        float l = 0.f;
        for (int k = 0; k < ntiles; ++k) l += lpart[k];
        *loss = l / (float)n;
    }
}

// Adam (Kingma & Ba 2015), bias-corrected, step t >= 1
__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, int t, float lr, float b1, float b2, float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float gp = g[p];
    const float mp = b1 * m[p] + (1.f - b1) * gp;
    const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.f - powf(b1, (float)t));
    const float vh = vp / (1.f - powf(b2, (float)t));
    P[p] -= lr * mh / (sqrtf(vh) + eps);
}

// Glorot-uniform weights from Philox (key = seed), zero biases.
__global__ void k_mlp_init(float *__restrict__ P, uint32_t k0, uint32_t k1)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const rewl::u32x4 r = rewl::philox((uint32_t)p, 0u, 0u, 0x4d4c5000u, k0, k1);
    const float u = ((float)(r.x >> 8) + 0.5f) * 0x1p-24f * 2.f - 1.f; // (-1, 1)
    float a = 0.f;
    if (p < OFF_B1) a = sqrtf(6.f / (3 + HID));
    else if (p >= OFF_W2 && p < OFF_B2) a = sqrtf(6.f / (HID + HID));
    else if (p >= OFF_W3 && p < OFF_B3) a = sqrtf(6.f / (HID + 1));
    P[p] = a * u;
}

// Features and targets of a converged ln g: one sample per reachable bin, in bin order (one
// CTA of 1024 threads, block-wide scans), so the training sums always see the same order.
__global__ void __launch_bounds__(1024) k_mlp_samples(const double *__restrict__ lng, int B, int model,
                                                      int q, int L, float *__restrict__ X,
                                                      float *__restrict__ T, int *__restrict__ count)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int N = L * L;
    int base = 0;
    for (int b0 = 0; b0 <= B; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const double v = b <= B ? lng[b] : -INFINITY;
        const int f = v > -INFINITY ? 1 : 0;
        int x = f; // inclusive warp scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w; // inclusive prefix over warps
        }
        __syncthreads();
        const int pos = base + (wid ? wsum[wid - 1] : 0) + x - f;
        if (f) {
            const double e = model == 0 ? -2.0 + 2.0 * (double)b / N : -2.0 + (double)b / N;
            X[3 * pos] = (float)e;
            X[3 * pos + 1] = (float)q;
            X[3 * pos + 2] = 1.0f / (float)L;
            T[pos] = (float)(v / N);
        }
        base += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// ln g(E) = N * net(e, q, 1/L) for every bin of the target lattice (float64 output).
__global__ void k_mlp_predict(const float *__restrict__ P, int B, int model, int q, int L,
                              double *__restrict__ out)
{
    extern __shared__ float sP[];
    load_params(P, sP);
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > B) return;
    const int N = L * L;
    const float e = model == 0 ? -2.0f + 2.0f * (float)b / N : -2.0f + (float)b / N;
    float h1[HID], h2[HID];
    out[b] = (double)N * (double)mlp_fwd1(sP, e, (float)q, 1.0f / (float)L, h1, h2);
}

size_t grad_smem() { return (size_t)(((NPARAM + 3) & ~3) + 2 * TILE * (HID + 1) + TILE * 4) * 4; }

int fail(cudaError_t e, const char *where)
{
    g_mlp_err = std::string(where) + ": " + cudaGetErrorString(e);
    return REWL_ERR_CUDA;
}

} // namespace

extern "C" {

int rewl_mlp_forward(const float *P, const float *X, float *Y, int n, void *stream)
{
    if (!P || !X || !Y || n < 0) return REWL_ERR_INVALID_ARG;
    if (n == 0) return REWL_OK;
    k_mlp_forward<<<(n + 127) / 128, 128, NPARAM * sizeof(float), (cudaStream_t)stream>>>(P, X, Y, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_forward");
}

int rewl_mlp_workspace_floats(int n) { return ((n + TILE - 1) / TILE) * (NPARAM + 1) + 1; }

int rewl_mlp_grad(const float *P, const float *X, const float *T, int n, float *grad, float *loss,
                  float *work, void *stream)
{
    if (!P || !X || !T || !grad || !work || n < 1) return REWL_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int ntiles = (n + TILE - 1) / TILE;
    float *partial = work, *lpart = work + (size_t)ntiles * NPARAM;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)grad_smem());
    if (e != cudaSuccess) return fail(e, "rewl_mlp_grad");
    k_mlp_grad_tile<<<ntiles, TILE, grad_smem(), st>>>(P, X, T, n, partial, lpart);
    k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(partial, lpart, ntiles, n, grad, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_grad");
}

int rewl_mlp_adam(float *P, const float *grad, float *m, float *v, int t, double lr, void *stream)
{
    if (!P || !grad || !m || !v || t < 1 || !(lr > 0)) return REWL_ERR_INVALID_ARG;
    k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, grad, m, v, t, (float)lr,
                                                                       0.9f, 0.999f, 1e-8f);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_adam");
}

int rewl_mlp_train(float *P, const float *X, const float *T, int n, int steps, double lr,
                   int t0, float *m, float *v, float *grad, float *work, float *loss_out,
                   void *stream)
{
    if (!P || !X || !T || !m || !v || !grad || !work || n < 1 || steps < 0 || t0 < 0)
        return REWL_ERR_INVALID_ARG;
    for (int s = 0; s < steps; ++s) {
        int rc = rewl_mlp_grad(P, X, T, n, grad, s + 1 == steps ? loss_out : nullptr, work, stream);
        if (rc == REWL_OK) rc = rewl_mlp_adam(P, grad, m, v, t0 + s + 1, lr, stream);
        if (rc != REWL_OK) return rc;
    }
    return REWL_OK;
}

int rewl_mlp_init(float *P, uint64_t seed, void *stream)
{
    if (!P) return REWL_ERR_INVALID_ARG;
    k_mlp_init<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, (uint32_t)seed,
                                                                       (uint32_t)(seed >> 32));
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_init");
}

int rewl_mlp_samples(const double *lng, int model, int L, float *X, float *T, int *count,
                     void *stream)
{
    if (!lng || !X || !T || !count || L < 2 || (model != 0 && model < 2)) return REWL_ERR_INVALID_ARG;
    const int N = L * L, B = model == 0 ? N : 2 * N, q = model == 0 ? 2 : model;
    k_mlp_samples<<<1, 1024, 0, (cudaStream_t)stream>>>(lng, B, model, q, L, X, T, count);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_samples");
}

int rewl_mlp_predict(const float *P, int model, int L, double *lng, void *stream)
{
    if (!P || !lng || L < 2 || (model != 0 && model < 2)) return REWL_ERR_INVALID_ARG;
    const int N = L * L, B = model == 0 ? N : 2 * N, q = model == 0 ? 2 : model;
    k_mlp_predict<<<(B + 128) / 128, 128, NPARAM * sizeof(float), (cudaStream_t)stream>>>(P, B, model,
                                                                                        q, L, lng);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? REWL_OK : fail(e, "rewl_mlp_predict");
}

const char *rewl_mlp_last_error(void) { return g_mlp_err.c_str(); }

} // extern "C"
