// The per-cluster degree selector: a 12 -> 64 -> 64 -> 6 perceptron with ReLU
// hidden layers, its softmax cross-entropy gradient and an Adam step, in FP32.
// The paper fixes one interpolation degree for all clusters; this network is
// the project's addition that picks a degree class per cluster from the
// cluster features of learn.cu.
//
// Parameter vector (floats): mu[12] sd[12] W1[64][12] b1[64] W2[64][64] b2[64]
// W3[6][64] b3[6]; the input is normalised as (x - mu) / sd and mu, sd are not
// trained.  Every reduction runs in a fixed order, so results do not depend on
// scheduling.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace {

constexpr int NF = KITC_NFEAT, NH = KITC_MLP_HIDDEN, NC = KITC_MLP_CLASSES;
constexpr int NP = KITC_MLP_NPARAM;
constexpr int O_MU = 0, O_SD = NF, O_W1 = 2 * NF, O_B1 = O_W1 + NH * NF, O_W2 = O_B1 + NH,
              O_B2 = O_W2 + NH * NH, O_W3 = O_B2 + NH, O_B3 = O_W3 + NC * NH;
static_assert(O_B3 + NC == NP, "parameter layout");
constexpr int ROWS = 64;  // samples per block of the gradient kernel
constexpr int GT = 256;   // threads per block of the gradient kernel

struct Classes {
    int deg[NC];
    int zero_unused;  // rows with features 2..4 all zero (no accepting target) get degree 0
};

// Warp per sample: logits (and the degree of the largest logit, first on ties).
__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ prm,
                                                     const float *__restrict__ X, int64_t m,
                                                     float *__restrict__ logits, Classes cls,
                                                     int32_t *__restrict__ deg)
{
    __shared__ float P[NP];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) P[k] = prm[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t i = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5); i < m;
         i += (int64_t)gridDim.x * nw) {
        float z = 0.f;
        if (lane < NF) z = (X[i * NF + lane] - P[O_MU + lane]) / P[O_SD + lane];
        float h1[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int u = lane + 32 * q;
            float a = P[O_B1 + u];
#pragma unroll
            for (int k = 0; k < NF; ++k) a = fmaf(P[O_W1 + u * NF + k], __shfl_sync(0xffffffffu, z, k), a);
            h1[q] = fmaxf(a, 0.f);
        }
        float h2[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int u = lane + 32 * q;
            float a = P[O_B2 + u];
#pragma unroll 8
            for (int j = 0; j < 32; ++j) a = fmaf(P[O_W2 + u * NH + j], __shfl_sync(0xffffffffu, h1[0], j), a);
#pragma unroll 8
            for (int j = 0; j < 32; ++j)
                a = fmaf(P[O_W2 + u * NH + 32 + j], __shfl_sync(0xffffffffu, h1[1], j), a);
            h2[q] = fmaxf(a, 0.f);
        }
        float lg[NC];
#pragma unroll
        for (int o = 0; o < NC; ++o) {
            float s = fmaf(P[O_W3 + o * NH + lane], h2[0], P[O_W3 + o * NH + lane + 32] * h2[1]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
            lg[o] = s + P[O_B3 + o];
        }
        if (lane == 0) {
            int best = 0;
            for (int o = 0; o < NC; ++o) {
                if (logits) logits[i * NC + o] = lg[o];
                if (lg[o] > lg[best]) best = o;
            }
            if (deg) {
                const bool unused = cls.zero_unused && X[i * NF + 2] == 0.f &&
                                    X[i * NF + 3] == 0.f && X[i * NF + 4] == 0.f;
                deg[i] = unused ? 0 : cls.deg[best];
            }
        }
    }
}

// Block of ROWS samples: forward pass, softmax cross-entropy, and the chain
// rule layer by layer; the block's gradient sum goes to part[blockIdx.x].
__global__ void __launch_bounds__(GT) k_mlp_grad(const float *__restrict__ prm,
                                                 const float *__restrict__ X,
                                                 const int32_t *__restrict__ labels, int64_t m,
                                                 float *__restrict__ part, float *__restrict__ lpart)
{
    extern __shared__ float sm[];
    float *P = sm;                  // NP
    float *Z = P + NP;              // [ROWS][NF]
    float *H1 = Z + ROWS * NF;      // [ROWS][NH]
    float *H2 = H1 + ROWS * NH;     // [ROWS][NH]
    float *G = H2 + ROWS * NH;      // [ROWS][NC]   dL/dlogits
    float *GA2 = G + ROWS * NC;     // [ROWS][NH]
    float *GA1 = GA2 + ROWS * NH;   // [ROWS][NH]
    float *LS = GA1 + ROWS * NH;    // [ROWS][2]    loss, rejected label
    const int64_t i0 = (int64_t)blockIdx.x * ROWS;
    const int rows = (int)min((int64_t)ROWS, m - i0);
    const float invm = 1.f / (float)m;
    for (int k = threadIdx.x; k < NP; k += GT) P[k] = prm[k];
    __syncthreads();
    for (int q = threadIdx.x; q < ROWS * NF; q += GT) {
        int i = q / NF, k = q % NF;
        Z[q] = i < rows ? (X[(i0 + i) * NF + k] - P[O_MU + k]) / P[O_SD + k] : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ROWS * NH; q += GT) {
        int i = q / NH, u = q % NH;
        float a = P[O_B1 + u];
        for (int k = 0; k < NF; ++k) a = fmaf(P[O_W1 + u * NF + k], Z[i * NF + k], a);
        H1[q] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < ROWS * NH; q += GT) {
        int i = q / NH, u = q % NH;
        float a = P[O_B2 + u];
        for (int j = 0; j < NH; ++j) a = fmaf(P[O_W2 + u * NH + j], H1[i * NH + j], a);
        H2[q] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (threadIdx.x < ROWS) {  // softmax and dL/dlogits of one row
        const int i = threadIdx.x;
        float lg[NC];
        for (int o = 0; o < NC; ++o) {
            float a = P[O_B3 + o];
            for (int j = 0; j < NH; ++j) a = fmaf(P[O_W3 + o * NH + j], H2[i * NH + j], a);
            lg[o] = a;
        }
        const int y = i < rows ? labels[i0 + i] : -1;
        const bool ok = y >= 0 && y < NC;
        float mx = lg[0];
        for (int o = 1; o < NC; ++o) mx = fmaxf(mx, lg[o]);
        float se = 0.f;
        for (int o = 0; o < NC; ++o) se += expf(lg[o] - mx);
        for (int o = 0; o < NC; ++o)
            G[i * NC + o] = ok ? (expf(lg[o] - mx) / se - (o == y ? 1.f : 0.f)) * invm : 0.f;
        LS[2 * i] = ok ? (logf(se) + mx - lg[y]) : 0.f;
        LS[2 * i + 1] = (i < rows && !ok) ? 1.f : 0.f;
    }
    __syncthreads();
    float *out = part + (size_t)blockIdx.x * NP;
    for (int q = threadIdx.x; q < NC * NH; q += GT) {  // dW3 = G^T H2
        int o = q / NH, j = q % NH;
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a = fmaf(G[i * NC + o], H2[i * NH + j], a);
        out[O_W3 + q] = a;
    }
    if (threadIdx.x < NC) {
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a += G[i * NC + threadIdx.x];
        out[O_B3 + threadIdx.x] = a;
    }
    for (int q = threadIdx.x; q < ROWS * NH; q += GT) {  // dA2 = (G W3) . [A2 > 0]
        int i = q / NH, j = q % NH;
        float a = 0.f;
        for (int o = 0; o < NC; ++o) a = fmaf(G[i * NC + o], P[O_W3 + o * NH + j], a);
        GA2[q] = H2[q] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NH * NH; q += GT) {  // dW2 = dA2^T H1
        int u = q / NH, j = q % NH;
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a = fmaf(GA2[i * NH + u], H1[i * NH + j], a);
        out[O_W2 + q] = a;
    }
    if (threadIdx.x < NH) {
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a += GA2[i * NH + threadIdx.x];
        out[O_B2 + threadIdx.x] = a;
    }
    for (int q = threadIdx.x; q < ROWS * NH; q += GT) {  // dA1 = (dA2 W2) . [A1 > 0]
        int i = q / NH, j = q % NH;
        float a = 0.f;
        for (int u = 0; u < NH; ++u) a = fmaf(GA2[i * NH + u], P[O_W2 + u * NH + j], a);
        GA1[q] = H1[q] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NH * NF; q += GT) {  // dW1 = dA1^T Z
        int u = q / NF, k = q % NF;
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a = fmaf(GA1[i * NH + u], Z[i * NF + k], a);
        out[O_W1 + q] = a;
    }
    if (threadIdx.x < NH) {
        float a = 0.f;
        for (int i = 0; i < ROWS; ++i) a += GA1[i * NH + threadIdx.x];
        out[O_B1 + threadIdx.x] = a;
    }
    if (threadIdx.x < 2 * NF) out[threadIdx.x] = 0.f;  // mu, sd are fixed
    if (threadIdx.x == 0) {
        float a = 0.f, r = 0.f;
        for (int i = 0; i < ROWS; ++i) a += LS[2 * i], r += LS[2 * i + 1];
        lpart[2 * blockIdx.x] = a;
        lpart[2 * blockIdx.x + 1] = r;
    }
}

// grad[k] = sum over blocks of part[b][k] in block order; loss = [mean loss,
// rejected labels].
__global__ void k_mlp_reduce(const float *__restrict__ part, const float *__restrict__ lpart,
                             int nblk, int64_t m, float *__restrict__ grad, float *__restrict__ loss)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NP) {
        float a = 0.f;
        for (int b = 0; b < nblk; ++b) a += part[(size_t)b * NP + k];
        grad[k] = a;
    } else if (k == NP) {
        float a = 0.f, r = 0.f;
        for (int b = 0; b < nblk; ++b) a += lpart[2 * b], r += lpart[2 * b + 1];
        loss[0] = a / (float)m;
        loss[1] = r;
    }
}

// One Adam step (bias-corrected; c1 = 1 - beta1^t, c2 = 1 - beta2^t); the
// normalisation entries mu, sd are left as they are.
__global__ void k_mlp_adam(float *__restrict__ prm, const float *__restrict__ g,
                           float *__restrict__ m1, float *__restrict__ m2, float lr, float b1,
                           float b2, float eps, float c1, float c2)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 2 * NF || k >= NP) return;
    float a = fmaf(b1, m1[k], (1.f - b1) * g[k]);
    float v = fmaf(b2, m2[k], (1.f - b2) * g[k] * g[k]);
    m1[k] = a;
    m2[k] = v;
    prm[k] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

size_t grad_smem() { return sizeof(float) * (NP + ROWS * NF + 4 * ROWS * NH + ROWS * NC + 2 * ROWS); }

}  // namespace

extern "C" {

size_t kitc_mlp_workspace_bytes(int64_t m)
{
    if (m < 1) return 0;
    int64_t nblk = (m + ROWS - 1) / ROWS;
    return (size_t)nblk * (NP + 2) * sizeof(float) + 256;
}

kitc_status kitc_mlp_forward(const float *params, const float *features, int64_t m, float *logits,
                             const int32_t *class_degree, int zero_unused, int32_t *degrees,
                             void *stream)
{
    if (!params || !features || m < 1 || m > (int64_t)INT32_MAX || (!logits && !degrees) ||
        (degrees && !class_degree))
        return KITC_ERR_INVALID_ARG;
    Classes cls{};
    cls.zero_unused = zero_unused != 0;
    for (int o = 0; o < NC; ++o) {
        cls.deg[o] = class_degree ? class_degree[o] : 0;
        if (degrees && (cls.deg[o] < 0 || cls.deg[o] > KITC_MAX_DEGREE)) return KITC_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    KITC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = std::min<int64_t>((m + 7) / 8, (int64_t)sms * 8);
    kitc_count_launch();
    k_mlp_forward<<<(unsigned)grid, 256, 0, s>>>(params, features, m, logits, cls, degrees);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status kitc_mlp_loss_grad(const float *params, const float *features, const int32_t *labels,
                               int64_t m, float *loss, float *grad, void *work, void *stream)
{
    if (!params || !features || !labels || !loss || !grad || !work || m < 1 ||
        m > (int64_t)INT32_MAX)
        return KITC_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(work) & 15u) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nblk = (int)((m + ROWS - 1) / ROWS);
    float *part = reinterpret_cast<float *>(work);
    float *lpart = part + (size_t)nblk * NP;
    static std::atomic<int> configured[64] = {};  // the attribute's value never changes
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev].load()) {
        KITC_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grad_smem()));
        if (dev >= 0 && dev < 64) configured[dev].store(1);
    }
    kitc_count_launch();
    k_mlp_grad<<<nblk, GT, grad_smem(), s>>>(params, features, labels, m, part, lpart);
    kitc_count_launch();
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, s>>>(part, lpart, nblk, m, grad, loss);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status kitc_mlp_adam_step(float *params, const float *grad, float *m1, float *m2, int step,
                               float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!params || !grad || !m1 || !m2 || step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float c1 = (float)(1.0 - pow((double)beta1, step));
    const float c2 = (float)(1.0 - pow((double)beta2, step));
    kitc_count_launch();
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, s>>>(params, grad, m1, m2, lr, beta1, beta2, eps, c1, c2);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

}  // extern "C"
