// Inputs of the per-cluster degree selector: features of every source cluster
// and, for training, the far-field error each cluster makes at its accepting
// targets, measured against the direct sum over the cluster's own sources.
//
// The paper interpolates every cluster at one degree n (Sec. 3).  The error of
// one cluster's far field at a target x, |sum_k k(x, s_k) fhat_k - sum_{y_j in
// C} k(x, y_j) f_j| (Eqs. pc_approximation_3D and pc_interaction_3D), is what
// the degree controls; these kernels measure it on sampled (target, cluster)
// pairs of the interaction lists so that a per-cluster degree can be chosen.
#include <float.h>

#include "common.cuh"
#include "kmath.cuh"

namespace {

// Targets of batch b: slots [s0, s1) of the target tree order.
__device__ __forceinline__ void batch_slots(const LearnArgs &a, int64_t b, int64_t &s0, int64_t &s1)
{
    s0 = a.bdesc ? (int64_t)a.bdesc[b] : b * a.batch;
    s1 = a.bdesc ? s0 + a.bdesc[a.nb + b] : min(a.nt, s0 + a.batch);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Weight statistics of a cluster, 8 doubles: sum_j f_j (w_in <= 6 components),
// sum_j |f_j|, max_j |f_j|.
constexpr int WS = 8;

// Block per leaf: the statistics over the leaf's sources.
__global__ void k_feat_leaf(const LearnArgs a, const double *__restrict__ w, double *__restrict__ acc)
{
    const int c = blockIdx.x;
    if (a.n_child[c] != 0) return;
    const int p0 = a.cbegin[c], p1 = a.cend[c];
    double v[WS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const double *f = w + (int64_t)a.perm[p] * a.win;
        double q = 0.0;
        for (int l = 0; l < a.win; ++l) {
            v[l] += f[l];
            q += f[l] * f[l];
        }
        q = sqrt(q);
        v[6] += q;
        v[7] = fmax(v[7], q);
    }
    __shared__ double red[4][WS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = warp_sum(v[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[7] = fmax(v[7], __shfl_xor_sync(0xffffffffu, v[7], o));
    if (lane == 0)
        for (int k = 0; k < WS; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x < WS) {
        const int k = threadIdx.x;
        double t = red[0][k];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = k == 7 ? fmax(t, red[q][k]) : t + red[q][k];
        acc[(size_t)c * WS + k] = t;
    }
}

// Thread per cluster of one level: the statistics of an internal cluster from
// its children's (in child order).
__global__ void k_feat_merge(const LearnArgs a, int lb, int le, double *__restrict__ acc)
{
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int nch = a.n_child[c];
    if (nch == 0) return;
    double v[WS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nch; ++i) {
        const double *u = acc + (size_t)(a.first_child[c] + i) * WS;
        for (int k = 0; k < 7; ++k) v[k] += u[k];
        v[7] = fmax(v[7], u[7]);
    }
    for (int k = 0; k < WS; ++k) acc[(size_t)c * WS + k] = v[k];
}

// Warp per target batch: for every far entry (batch, cluster) the accepting
// targets' ratios q = r / |x - y_c| go into the cluster's count, sum, min, max.
__global__ void k_feat_targets(const LearnArgs a, unsigned long long *__restrict__ cnt,
                               double *__restrict__ qsum, unsigned *__restrict__ qmin,
                               unsigned *__restrict__ qmax)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= a.nb) return;
    int64_t s0, s1;
    batch_slots(a, b, s0, s1);
    double x[2][3];
    for (int t = 0; t < 2; ++t) {
        int64_t sl = min(s0 + lane + 32 * t, s1 - 1);
        for (int l = 0; l < 3; ++l) x[t][l] = a.txs[l * a.nt + sl];
    }
    for (int64_t e = a.far_off[b]; e < a.far_off[b + 1]; ++e) {
        const int c = a.far_id[e];
        const uint64_t mk = a.far_mask[e];
        const dvec4 g = a.ctr[c];
        // FP32 ratios (the features are FP32): offsets formed in FP64 first
        const float r = (float)g.w;
        float qs = 0.f;
        float mn = FLT_MAX, mx = 0.f;
        for (int t = 0; t < 2; ++t) {
            if (!((mk >> (lane + 32 * t)) & 1ull)) continue;
            float dx = (float)(x[t][0] - g.x), dy = (float)(x[t][1] - g.y), dz = (float)(x[t][2] - g.z);
            float R2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float q = R2 > 0.f ? r * rsqrtf(R2) : 0.f;
            qs += q;
            mn = fminf(mn, q);
            mx = fmaxf(mx, q);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qs += __shfl_xor_sync(0xffffffffu, qs, o);
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0 && mk) {
            atomicAdd(cnt + c, (unsigned long long)__popcll(mk));
            atomicAdd(qsum + c, (double)qs);
            atomicMin(qmin + c, __float_as_uint(mn));  // q >= 0: bit order is value order
            atomicMax(qmax + c, __float_as_uint(mx));
        }
    }
}

__global__ void k_feat_init(int m, unsigned long long *cnt, double *qsum, unsigned *qmin, unsigned *qmax)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    cnt[c] = 0;
    qsum[c] = 0.0;
    qmin[c] = __float_as_uint(FLT_MAX);
    qmax[c] = 0u;
}

// The 12 features of each cluster (FP32, row c of feat).
__global__ void k_feat_final(const LearnArgs a, int m, const double *__restrict__ acc,
                             const unsigned long long *__restrict__ cnt,
                             const double *__restrict__ qsum, const unsigned *__restrict__ qmin,
                             const unsigned *__restrict__ qmax, float *__restrict__ feat)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const dvec4 g = a.ctr[c], lo = a.clo[c], hi = a.chi[c];
    const double r = g.w;
    const double nc = (double)(a.cend[c] - a.cbegin[c]);
    const unsigned long long k = cnt[c];
    double side[3] = {hi.x - lo.x, hi.y - lo.y, hi.z - lo.z};
    // sort the three sides: s0 >= s1 >= s2
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (side[j] < side[j + 1]) {
                double tmp = side[j];
                side[j] = side[j + 1];
                side[j + 1] = tmp;
            }
    float *o = feat + (size_t)c * KITC_NFEAT;
    o[0] = (float)log1p(nc);
    o[1] = (float)log(fmax(r, 1e-12));
    o[2] = k ? __uint_as_float(qmin[c]) : 0.f;
    o[3] = k ? (float)(qsum[c] / (double)k) : 0.f;
    o[4] = k ? __uint_as_float(qmax[c]) : 0.f;
    o[5] = (float)fmin(a.eps / fmax(r, 1e-300), 10.0);
    const double *u = acc + (size_t)c * WS;
    double n2 = 0.0;
    for (int l = 0; l < a.win; ++l) n2 += u[l] * u[l];
    o[6] = (float)log(1e-30 + sqrt(n2));
    o[7] = (float)log(1e-30 + u[6]);
    o[8] = (float)log(1e-30 + u[7]);
    o[9] = side[0] > 0.0 ? (float)(side[1] / side[0]) : 1.f;
    o[10] = side[0] > 0.0 ? (float)(side[2] / side[0]) : 1.f;
    o[11] = (float)a.level[c];
}

// A counter-based uniform number in [0, 1) of (seed, cluster, target slot)
// (the SplitMix64 finaliser).
__device__ __forceinline__ double unit_hash(unsigned long long seed, int c, int64_t slot)
{
    unsigned long long z = seed ^ ((unsigned long long)(unsigned)c << 32) ^ (unsigned long long)slot;
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Warp per target batch.  Of the targets that accept cluster c, a sample with
// probability min(1, S / cnt[c]) is taken; for each, lanes split the (n_c+1)^3
// grid points (far field with the cluster's FP64 modified weights) and then the
// cluster's sources (direct sum), and err2[c] += |far - direct|^2 (times the
// 1/(8 pi) of the kernels).
template <int K>
__global__ void k_far_errors(const LearnArgs a, const double *__restrict__ w, int S,
                             unsigned long long seed, const unsigned long long *__restrict__ cnt,
                             double *__restrict__ err2, int *__restrict__ nsamp)
{
    constexpr int WIN = KT<K>::WIN, WOUT = KT<K>::WOUT;
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= a.nb) return;
    int64_t s0, s1;
    batch_slots(a, b, s0, s1);
    double x[2][3];
    for (int t = 0; t < 2; ++t) {
        int64_t sl = min(s0 + lane + 32 * t, s1 - 1);
        for (int l = 0; l < 3; ++l) x[t][l] = a.txs[l * a.nt + sl];
    }
    const double e2 = a.eps * a.eps, e4 = e2 * e2;
    for (int64_t e = a.far_off[b]; e < a.far_off[b + 1]; ++e) {
        const int c = a.far_id[e];
        const uint64_t mk = a.far_mask[e];
        const double pc = fmin(1.0, (double)S / (double)max(cnt[c], 1ull));
        uint64_t sel = 0;
        for (int t = 0; t < 2; ++t) {
            int i = lane + 32 * t;
            bool take = ((mk >> i) & 1ull) && unit_hash(seed, c, s0 + i) < pc;
            unsigned bal = __ballot_sync(0xffffffffu, take);
            sel |= (uint64_t)bal << (32 * t);
        }
        if (!sel) continue;
        const int np = a.cdeg ? a.cdeg[c] + 1 : a.degree + 1;
        if (np < 2) {
            if (lane == 0) atomicExch(a.err, 1);
            continue;
        }
        const int P = np * np * np;
        const double *fh = a.fhat + (a.foff ? a.foff[c] : (int64_t)c * P * WIN);
        const double *ct = a.chebt + (size_t)(np - 1) * (KITC_MAX_DEGREE + 1);
        const dvec4 lo = a.clo[c], hi = a.chi[c];
        const double lx[3] = {lo.x, lo.y, lo.z}, hx[3] = {hi.x, hi.y, hi.z};
        const int p0 = a.cbegin[c], p1 = a.cend[c];
        while (sel) {
            const int i = __ffsll((long long)sel) - 1;
            sel &= sel - 1;
            const int t = i >> 5, src = i & 31;
            double xi[3];
            for (int l = 0; l < 3; ++l) xi[l] = __shfl_sync(0xffffffffu, x[t][l], src);
            double uf[WOUT], ud[WOUT];
            for (int q = 0; q < WOUT; ++q) uf[q] = ud[q] = 0.0;
            for (int k = lane; k < P; k += 32) {
                const int k1 = k / (np * np), k2 = (k / np) % np, k3 = k % np;
                const int kk[3] = {k1, k2, k3};
                double d[3];
                for (int l = 0; l < 3; ++l)
                    d[l] = xi[l] - 0.5 * ((lx[l] + hx[l]) + ct[kk[l]] * (hx[l] - lx[l]));
                double f[WIN];
                for (int q = 0; q < WIN; ++q) f[q] = fh[(size_t)k * WIN + q];
                pair<K, true, double>(d[0], d[1], d[2], f, e2, e4, uf,
                                      fma(d[0], d[0], fma(d[1], d[1], fma(d[2], d[2], e2))));
            }
            for (int p = p0 + lane; p < p1; p += 32) {
                double d[3];
                for (int l = 0; l < 3; ++l) d[l] = xi[l] - a.sxs[l * a.ns + p];
                const double *fp = w + (int64_t)a.perm[p] * WIN;
                double f[WIN];
                for (int q = 0; q < WIN; ++q) f[q] = fp[q];
                pair<K, true, double>(d[0], d[1], d[2], f, e2, e4, ud,
                                      fma(d[0], d[0], fma(d[1], d[1], fma(d[2], d[2], e2))));
            }
            double s = 0.0;
            for (int q = 0; q < WOUT; ++q) {
                double df = warp_sum(uf[q] - ud[q]) * 0.039788735772973836;  // 1/(8 pi)
                s += df * df;
            }
            if (lane == 0) {
                atomicAdd(err2 + c, s);
                atomicAdd(nsamp + c, 1);
            }
        }
    }
}

}  // namespace

kitc_status learn_features(const LearnArgs &a, const std::vector<int32_t> &level_start,
                           const double *w, float *feat, DevBuf &scratch, cudaStream_t s)
{
    const int m = a.nclus;
    size_t bytes = (size_t)m * (WS * sizeof(double) + sizeof(unsigned long long) + sizeof(double) +
                                2 * sizeof(unsigned));
    KITC_TRY(scratch.reserve(bytes + 64, s));
    double *acc = scratch.as<double>();
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(acc + WS * (size_t)m);
    double *qsum = reinterpret_cast<double *>(cnt + m);
    unsigned *qmin = reinterpret_cast<unsigned *>(qsum + m);
    unsigned *qmax = qmin + m;
    const unsigned g = (unsigned)((m + 255) / 256);
    kitc_count_launch();
    k_feat_init<<<g, 256, 0, s>>>(m, cnt, qsum, qmin, qmax);
    kitc_count_launch();
    k_feat_leaf<<<m, 128, 0, s>>>(a, w, acc);
    for (int L = (int)level_start.size() - 2; L >= 0; --L) {  // deepest level first
        const int lb = level_start[L], le = level_start[L + 1];
        if (le <= lb) continue;
        kitc_count_launch();
        k_feat_merge<<<(le - lb + 127) / 128, 128, 0, s>>>(a, lb, le, acc);
    }
    if (a.nb > 0) {
        kitc_count_launch();
        k_feat_targets<<<(unsigned)((a.nb + 7) / 8), 256, 0, s>>>(a, cnt, qsum, qmin, qmax);
    }
    kitc_count_launch();
    k_feat_final<<<g, 256, 0, s>>>(a, m, acc, cnt, qsum, qmin, qmax, feat);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status learn_far_errors(int kernel, const LearnArgs &a, const double *w, int S,
                             unsigned long long seed, double *err2, int *nsamp, DevBuf &scratch,
                             cudaStream_t s)
{
    const int m = a.nclus;
    KITC_TRY(scratch.reserve((size_t)m * (sizeof(unsigned long long) + sizeof(double) +
                                          2 * sizeof(unsigned)) + 64, s));
    unsigned long long *cnt = scratch.as<unsigned long long>();
    double *qsum = reinterpret_cast<double *>(cnt + m);
    unsigned *qmin = reinterpret_cast<unsigned *>(qsum + m);
    unsigned *qmax = qmin + m;
    const unsigned g = (unsigned)((m + 255) / 256);
    KITC_CUDA(cudaMemsetAsync(err2, 0, sizeof(double) * m, s));
    KITC_CUDA(cudaMemsetAsync(nsamp, 0, sizeof(int) * m, s));
    kitc_count_launch();
    k_feat_init<<<g, 256, 0, s>>>(m, cnt, qsum, qmin, qmax);
    if (a.nb == 0) return KITC_OK;
    const unsigned gb = (unsigned)((a.nb + 7) / 8);
    kitc_count_launch();
    k_feat_targets<<<gb, 256, 0, s>>>(a, cnt, qsum, qmin, qmax);
    kitc_count_launch();
    switch (kernel) {
    case KITC_STOKESLET: k_far_errors<KITC_STOKESLET><<<gb, 256, 0, s>>>(a, w, S, seed, cnt, err2, nsamp); break;
    case KITC_ROTLET: k_far_errors<KITC_ROTLET><<<gb, 256, 0, s>>>(a, w, S, seed, cnt, err2, nsamp); break;
    case KITC_STOKESLET_ROTLET:
        k_far_errors<KITC_STOKESLET_ROTLET><<<gb, 256, 0, s>>>(a, w, S, seed, cnt, err2, nsamp);
        break;
    default: return KITC_ERR_INVALID_ARG;
    }
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}
