// Modified weights of every cluster (Sec. 4-5, Eq. modified_weights,
// Algorithm 1) in FP64, and the packed records the evaluator streams.
//
//   fhat[c][k1][k2][k3][q] = sum_{y_j in c} L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) f_j[q]
//
// Each L is the barycentric form of Eq. Barycentric-1D with the simple
// weights of Eq. barycentric_weights at the Chebyshev points of Eq.
// Chebyshev_points mapped to the cluster's box (Sec. 3 interval map); a
// coordinate within DBL_MIN of a point s_m takes L_k = delta_km (Sec. 3,
// Algorithm 1).  The sum per axis is normalized before the product, which
// equals Algorithm 1's division by sum1*sum2*sum3 and cannot overflow.
//
// GPU form: the contraction over j is a batched outer-product sum.  For a
// chunk of particles a CTA stages h_j[k1,k2] = L_k1 L_k2 and g_j[k3,q] =
// L_k3 f_j[q] in shared memory and every thread accumulates its outputs with
// one FP64 FMA per particle.  Chunks of one cluster write partial sums that a
// second kernel adds in a fixed order, so the result is deterministic.
//
// Split-precision products (the mixed-precision form, k_weights_split): the
// FP64 basis values L and the weights f are held as FP32 pairs hi + lo (lo
// the rounded remainder); h = L1 L2 and g = L3 f and then each product h g are
// formed from pairs (the exact product of the high parts by FMA, TwoProduct,
// plus the cross terms); runs of up to 256 particles are summed in FP32 pairs
// with TwoSum, and each run's value is added to the FP64 sum.  Products carry
// about 2^-47 relative error; the barycentric basis and the accumulation
// across runs stay FP64.
#include <float.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "common.cuh"

namespace {

constexpr int WT = 256;       // threads of the weights kernels
constexpr int ACC_MAX = 16;   // outputs per thread per pass, at most
constexpr int CHUNK = 2048;   // particles per work item
constexpr size_t UP_SMEM_MAX = 200 * 1024;
constexpr size_t CHUNK_SMEM_MAX = 96 * 1024;  // dynamic shared memory of k_weights_chunk
kitc_status allow_up_smem();  // shared-memory attribute of the upward kernels

// Particles staged per round of k_weights_chunk (at most; fewer when the
// round's shared memory would exceed CHUNK_SMEM_MAX).
#ifndef KITC_WEIGHTS_SB
#define KITC_WEIGHTS_SB 64
#endif

struct Cheb {
    double t[KITC_MAX_DEGREE + 1];  // cos(k pi / n)
    double w[KITC_MAX_DEGREE + 1];  // (-1)^k delta_k
    int n;
};

Cheb make_cheb(int n)
{
    Cheb c;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k <= KITC_MAX_DEGREE; ++k) {
        c.t[k] = k <= n ? cos((double)k * pi / (double)n) : 0.0;
        double d = (k == 0 || k == n) ? 0.5 : 1.0;
        c.w[k] = k <= n ? ((k & 1) ? -d : d) : 0.0;
    }
    c.n = n;
    return c;
}

struct Item {
    int32_t c, p0, p1, pad;
};

// Barycentric basis of one coordinate on [a, b] (Eq. Barycentric-1D with the
// coincident-point rule), written to L[0..n].
__device__ void bary_basis(const Cheb &cb, double a, double b, double y, double *L)
{
    int n = cb.n;
    int flag = -1;
    double sum = 0.0;
    double ab = __dadd_rn(a, b), ba = __dsub_rn(b, a);
    for (int k = 0; k <= n; ++k) {
        double s = __dmul_rn(0.5, __dadd_rn(ab, __dmul_rn(cb.t[k], ba)));
        double diff = y - s;
        if (fabs(diff) <= DBL_MIN) {
            flag = k;
            L[k] = 0.0;
        } else {
            // w_k is +-1 or +-1/2, so w_k times the correctly rounded 1/diff is
            // exactly the correctly rounded w_k / diff (scaling by a power of 2)
            L[k] = cb.w[k] * __drcp_rn(diff);
            sum += L[k];
        }
    }
    if (flag >= 0) {
        for (int k = 0; k <= n; ++k) L[k] = (k == flag) ? 1.0 : 0.0;
    } else {
        double inv = __drcp_rn(sum);  // = 1.0 / sum, correctly rounded
        for (int k = 0; k <= n; ++k) L[k] *= inv;
    }
}

// An FP64 value as an FP32 pair hi + lo (lo = the rounded remainder).
__device__ __forceinline__ float2 split_f2(double v)
{
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

// (a.x + a.y)(b.x + b.y) as an FP32 pair: the exact product of the high parts
// (TwoProduct by FMA) plus the cross terms, renormalised (Fast2Sum).
__device__ __forceinline__ float2 mul_f2(float2 a, float2 b)
{
    const float p = a.x * b.x;
    const float e = __fmaf_rn(a.x, b.x, -p);
    const float c = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
    const float hi = p + c;
    return make_float2(hi, c - (hi - p));
}

template <int ACC>
__global__ void __launch_bounds__(WT) k_weights_chunk(
    Cheb cb, const Item *__restrict__ items, int64_t n, const double *__restrict__ xs,
    const int32_t *__restrict__ perm, const double *__restrict__ w, int win,
    const dvec4 *__restrict__ lo, const dvec4 *__restrict__ hi, int sb,
    double *__restrict__ partial, const int *__restrict__ nitems_dev)
{
    if (nitems_dev && (int)blockIdx.x >= *nitems_dev) return;  // device-planned items: past the end
    extern __shared__ double sm[];
    const int np = cb.n + 1;
    const int np2 = np * np, nw = np * win;
    const int pwin = np2 * np * win;
    double *Ls = sm;                        // [sb][3][np]
    double *hs = Ls + (size_t)sb * 3 * np;  // [sb][np2]
    double *gs = hs + (size_t)sb * np2;     // [sb][nw]
    Item it = items[blockIdx.x];
    int obase = blockIdx.y * ACC * WT;
    dvec4 blo = lo[it.c], bhi = hi[it.c];
    double acc[ACC];
#pragma unroll
    for (int i = 0; i < ACC; ++i) acc[i] = 0.0;
    int rowoff[ACC], coloff[ACC];
#pragma unroll
    for (int i = 0; i < ACC; ++i) {
        int o = obase + i * WT + threadIdx.x;
        rowoff[i] = o < pwin ? o / nw : 0;
        coloff[i] = o < pwin ? o % nw : 0;
    }
    for (int j0 = it.p0; j0 < it.p1; j0 += sb) {
        int cnt = min(sb, it.p1 - j0);
        for (int q = threadIdx.x; q < cnt * 3; q += WT) {
            int j = q / 3, l = q % 3;
            double a = l == 0 ? blo.x : (l == 1 ? blo.y : blo.z);
            double b = l == 0 ? bhi.x : (l == 1 ? bhi.y : bhi.z);
            bary_basis(cb, a, b, xs[l * n + j0 + j], Ls + (j * 3 + l) * np);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < cnt * np2; q += WT) {
            int j = q / np2, r = q % np2;
            hs[j * np2 + r] = Ls[(j * 3 + 0) * np + r / np] * Ls[(j * 3 + 1) * np + r % np];
        }
        for (int q = threadIdx.x; q < cnt * nw; q += WT) {
            int j = q / nw, r = q % nw;
            gs[j * nw + r] = Ls[(j * 3 + 2) * np + r / win] * w[(int64_t)perm[j0 + j] * win + r % win];
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const double *h = hs + j * np2, *g = gs + j * nw;
#pragma unroll
            for (int i = 0; i < ACC; ++i) acc[i] = fma(h[rowoff[i]], g[coloff[i]], acc[i]);
        }
        __syncthreads();
    }
    double *dst = partial + (size_t)blockIdx.x * pwin;
#pragma unroll
    for (int i = 0; i < ACC; ++i) {
        int o = obase + i * WT + threadIdx.x;
        if (o < pwin) dst[o] = acc[i];
    }
}

// Modified weights of a parent from those of its children.  For a child c the
// parent's Lagrange polynomials L^P_k, restricted to c's box, are polynomials
// of degree n in each variable, so interpolating them at c's Chebyshev points
// reproduces them exactly (Sec. 2).  Summing Eq. modified_weights over the
// children therefore gives
//   fhat_P[k1,k2,k3] = sum_c sum_k' L^P_k1(s^c_k1') L^P_k2(s^c_k2') L^P_k3(s^c_k3') fhat_c[k'],
// three 1D contractions per child instead of (n+1)^3 work per particle.
// One CTA per child (a level holds few parents but eight times as many
// children): child c writes its contribution, three 1D contractions, to
// contrib[c - cb0], and k_upward_sum adds each parent's children in child
// order.
__device__ void upward_child(const Cheb &cb, int c, const dvec4 *__restrict__ lo,
                             const dvec4 *__restrict__ hi, const int32_t *__restrict__ parent,
                             int win, const double *__restrict__ fhat, double *__restrict__ C,
                             double *sm)
{
    const int p = parent[c];
    const int np = cb.n + 1, np2 = np * np, pw = np2 * np * win;
    double *T1 = sm, *T2 = T1 + pw, *M = T2 + pw;  // M[l][k'][k] = L^P_k(s^c_k')
    const dvec4 plo = lo[p], phi = hi[p], clo = lo[c], chi = hi[c];
    for (int q = threadIdx.x; q < 3 * np; q += WT) {
        int l = q / np, kp = q % np;
        double ca = l == 0 ? clo.x : (l == 1 ? clo.y : clo.z);
        double cb_ = l == 0 ? chi.x : (l == 1 ? chi.y : chi.z);
        double pa = l == 0 ? plo.x : (l == 1 ? plo.y : plo.z);
        double pb = l == 0 ? phi.x : (l == 1 ? phi.y : phi.z);
        double y = __dmul_rn(0.5, __dadd_rn(__dadd_rn(ca, cb_), __dmul_rn(cb.t[kp], __dsub_rn(cb_, ca))));
        double L[KITC_MAX_DEGREE + 1];
        bary_basis(cb, pa, pb, y, L);
        for (int k = 0; k < np; ++k) M[(l * np + kp) * np + k] = L[k];
    }
    __syncthreads();
    const double *F = fhat + (size_t)c * pw;
    for (int o = threadIdx.x; o < pw; o += WT) {  // contract k3
        int q = o % win, k3 = (o / win) % np, r = o / (win * np);
        double v = 0.0;
        for (int kp = 0; kp < np; ++kp) v = fma(M[(2 * np + kp) * np + k3], F[(r * np + kp) * win + q], v);
        T1[o] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < pw; o += WT) {  // contract k2
        int q = o % win, k3 = (o / win) % np, k2 = (o / (win * np)) % np, k1 = o / (win * np2);
        double v = 0.0;
        for (int kp = 0; kp < np; ++kp)
            v = fma(M[(np + kp) * np + k2], T1[((k1 * np + kp) * np + k3) * win + q], v);
        T2[o] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < pw; o += WT) {  // contract k1
        int q = o % win, k3 = (o / win) % np, k2 = (o / (win * np)) % np, k1 = o / (win * np2);
        double v = 0.0;
        for (int kp = 0; kp < np; ++kp)
            v = fma(M[kp * np + k1], T2[((kp * np + k2) * np + k3) * win + q], v);
        C[o] = v;
    }
}

__global__ void __launch_bounds__(WT) k_upward_child(Cheb cb, int cb0, const dvec4 *__restrict__ lo,
                                                     const dvec4 *__restrict__ hi,
                                                     const int32_t *__restrict__ parent, int win,
                                                     const double *__restrict__ fhat,
                                                     double *__restrict__ contrib)
{
    extern __shared__ double sm[];
    const int pw = (cb.n + 1) * (cb.n + 1) * (cb.n + 1) * win;
    upward_child(cb, cb0 + blockIdx.x, lo, hi, parent, win, fhat, contrib + (size_t)blockIdx.x * pw, sm);
}

// Level bounds from a tree's state block: the clusters of level L are
// [*lb, *le); false when the tree has no level L.
__device__ __forceinline__ bool level_range(const BuildState *bs, int L, int *lb, int *le)
{
    const int D = bs->depth;
    if (L >= D) return false;
    *lb = bs->level_start[L];
    *le = L + 1 < D ? bs->level_start[L + 1] : bs->nclus;
    return true;
}

// k_upward_child for a tree known only on the device: the children at level
// L + 1, CTAs striding over them.
__global__ void __launch_bounds__(WT) k_upward_child_dev(Cheb cb, const BuildState *__restrict__ bs,
                                                         int L, const dvec4 *__restrict__ lo,
                                                         const dvec4 *__restrict__ hi,
                                                         const int32_t *__restrict__ parent, int win,
                                                         const double *__restrict__ fhat,
                                                         double *__restrict__ contrib)
{
    extern __shared__ double sm[];
    int cb0, ce;
    if (!level_range(bs, L + 1, &cb0, &ce)) return;
    const int pw = (cb.n + 1) * (cb.n + 1) * (cb.n + 1) * win;
    for (int c = cb0 + blockIdx.x; c < ce; c += gridDim.x) {
        upward_child(cb, c, lo, hi, parent, win, fhat, contrib + (size_t)(c - cb0) * pw, sm);
        __syncthreads();  // the shared tables are rewritten for the next child
    }
}

// fhat of every parent [lb, le) with children: the sum of its children's
// contributions (children are contiguous, contrib indexed from cb0).
__global__ void k_upward_sum(int lb, int le, int cb0, int pw, const int32_t *__restrict__ first_child,
                             const int32_t *__restrict__ n_child, const double *__restrict__ contrib,
                             double *__restrict__ fhat)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = lb + (int)(i / pw), o = (int)(i % pw);
    if (p >= le) return;
    const int nch = n_child[p];
    if (nch == 0) return;
    const int fc = first_child[p];
    double a = 0.0;
    for (int ci = 0; ci < nch; ++ci) a += contrib[(size_t)(fc + ci - cb0) * pw + o];
    fhat[(size_t)p * pw + o] = a;
}

// k_upward_sum for a tree known only on the device: the parents at level L.
__global__ void k_upward_sum_dev(const BuildState *__restrict__ bs, int L, int pw,
                                 const int32_t *__restrict__ first_child,
                                 const int32_t *__restrict__ n_child,
                                 const double *__restrict__ contrib, double *__restrict__ fhat)
{
    int lb, le, cb0, ce;
    if (!level_range(bs, L + 1, &cb0, &ce)) return;
    level_range(bs, L, &lb, &le);
    const int64_t tot = (int64_t)(le - lb) * pw;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p = lb + (int)(i / pw), o = (int)(i % pw);
        const int nch = n_child[p];
        if (nch == 0) continue;
        const int fc = first_child[p];
        double a = 0.0;
        for (int ci = 0; ci < nch; ++ci) a += contrib[(size_t)(fc + ci - cb0) * pw + o];
        fhat[(size_t)p * pw + o] = a;
    }
}

// fhat[c] = sum of the partials of c's work items, in item order.
__global__ void k_weights_reduce(const int32_t *__restrict__ first_item, int pwin,
                                 const double *__restrict__ partial, double *__restrict__ fhat)
{
    int c = blockIdx.x;
    int i0 = first_item[c], i1 = first_item[c + 1];
    if (i0 == i1) return;  // computed by the upward pass
    for (int o = threadIdx.x; o < pwin; o += blockDim.x) {
        double s = 0.0;
        for (int i = i0; i < i1; ++i) s += partial[(size_t)i * pwin + o];
        fhat[(size_t)c * pwin + o] = s;
    }
}

// nclus_dev given: the records of the first *nclus_dev clusters only (np3 each).
template <bool MIXED>
__global__ void k_pack_proxies(int64_t nrec, int win, const double *__restrict__ fhat,
                               void *__restrict__ out, const int *__restrict__ nclus_dev, int np3)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (nclus_dev) nrec = min(nrec, (int64_t)*nclus_dev * np3);
    if (r >= nrec) return;
    const double *f = fhat + r * win;
    if (MIXED) {
        float4 *o = reinterpret_cast<float4 *>(out);
        if (win == 3) {
            o[r] = make_float4((float)f[0], (float)f[1], (float)f[2], 0.f);
        } else {
            o[2 * r] = make_float4((float)f[0], (float)f[1], (float)f[2], 0.f);
            o[2 * r + 1] = make_float4((float)f[3], (float)f[4], (float)f[5], 0.f);
        }
    } else {
        double *o = reinterpret_cast<double *>(out);
        if (win == 3) {
            o[4 * r + 0] = f[0];
            o[4 * r + 1] = f[1];
            o[4 * r + 2] = f[2];
            o[4 * r + 3] = 0.0;
        } else {
            for (int q = 0; q < 6; ++q) o[6 * r + q] = f[q];
        }
    }
}

// Source records in slot order.  t == NULL: slots are the caller's order and
// coordinates come from xyz (n x 3).
template <bool MIXED>
__global__ void k_pack_sources(int64_t n, int win, const double *__restrict__ xs,
                               const int32_t *__restrict__ perm, const double *__restrict__ xyz,
                               const double *__restrict__ w, void *__restrict__ out)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t j = perm ? perm[p] : p;
    double x[3];
    for (int l = 0; l < 3; ++l) x[l] = perm ? xs[l * n + p] : xyz[3 * p + l];
    const double *f = w + j * win;
    if (MIXED) {
        float v[12];
        for (int l = 0; l < 3; ++l) {
            float h = __double2float_rn(x[l]);
            v[l] = h;
            v[3 + l] = __double2float_rn(x[l] - (double)h);
        }
        for (int q = 0; q < 6; ++q) v[6 + q] = q < win ? (float)f[q] : 0.f;
        float4 *o = reinterpret_cast<float4 *>(out) + 3 * p;
        o[0] = make_float4(v[0], v[1], v[2], v[3]);
        o[1] = make_float4(v[4], v[5], v[6], v[7]);
        o[2] = make_float4(v[8], v[9], v[10], v[11]);
    } else {
        int stride = win == 3 ? 6 : 10;
        double *o = reinterpret_cast<double *>(out) + p * stride;
        for (int l = 0; l < 3; ++l) o[l] = x[l];
        for (int q = 0; q < win; ++q) o[3 + q] = f[q];
        if (win == 6) o[9] = 0.0;
    }
}

// Paired records of a direct sum for the FP32x2 evaluator (Stokeslet forces or
// rotlet torques as the weights): two consecutive sources share a 80-byte
// record (negated hi/lo coordinates, so that the packed add forms x - y, then
// the weights):
//   [-yh_x0 -yh_x1 -yh_y0 -yh_y1][-yh_z0 -yh_z1 -yl_x0 -yl_x1]
//   [-yl_y0 -yl_y1 -yl_z0 -yl_z1][f_x0 f_x1 f_y0 f_y1][f_z0 f_z1 0 0]
// An odd source count is padded with a zero-weight point at 1e18, whose term
// is exactly zero.  put_pair_half writes half h (0 or 1) of record rec.
__device__ __forceinline__ void put_pair_half(float *__restrict__ rec, int h, const double *x,
                                              const double *f)
{
    for (int l = 0; l < 3; ++l) {
        float hi = __double2float_rn(x[l]);
        float lo = __double2float_rn(x[l] - (double)hi);
        rec[2 * l + h] = -hi;
        rec[6 + 2 * l + h] = -lo;
        rec[12 + 2 * l + h] = (float)f[l];
    }
    rec[18 + h] = 0.f;
}

// Paired records of a tree's leaves with leaf offsets (KITC_MIXED_LEAF): two
// consecutive sources of one leaf share a 48-byte record of their offsets
// from the centre c of the leaf's box (negated, so that the packed add forms
// x' - y' from the target's offset x'), then the weights:
//   [-y'_x0 -y'_x1 -y'_y0 -y'_y1][-y'_z0 -y'_z1 f_x0 f_x1][f_y0 f_y1 f_z0 f_z1]
// The offset of a point p is leaf_offset(ph, pl, ch, cl) of the FP32 hi/lo
// parts of p and c, the same arithmetic the evaluator applies to each target,
// so that a target on a source gives x' - y' = 0 exactly.  A leaf of odd size
// is padded with a zero-weight point at 1e18.
__device__ __forceinline__ void put_leaf_pair_half(float *__restrict__ rec, int h, const double *x,
                                                   const float *ch, const float *cl, const double *f)
{
    for (int l = 0; l < 3; ++l) {
        const float xh = __double2float_rn(x[l]);
        const float xl = __double2float_rn(x[l] - (double)xh);
        rec[2 * l + h] = -leaf_offset(xh, xl, ch[l], cl[l]);
        rec[6 + 2 * l + h] = (float)f[l];
    }
}

// Block r packs the slot range [rb[r], re[r]) of leaf rc[r] from pair pb[r],
// as hi/lo records (put_pair_half) or, LEAF, as leaf-offset records.
template <bool LEAF>
__global__ void k_pack_pairs(const int32_t *__restrict__ rb, const int32_t *__restrict__ re,
                             const int32_t *__restrict__ pb, const int32_t *__restrict__ rc,
                             int64_t n, const double *__restrict__ xs,
                             const int32_t *__restrict__ perm, const dvec4 *__restrict__ clo,
                             const dvec4 *__restrict__ chi, const double *__restrict__ w,
                             float *__restrict__ out)
{
    const int r = blockIdx.x;
    const int64_t b = rb[r], e = re[r];
    const int64_t cnt2 = ((e - b + 1) / 2) * 2;
    if (cnt2 == 0) return;
    float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
    if (LEAF) leaf_centre(clo[rc[r]], chi[rc[r]], ch, cl);
    for (int64_t i = threadIdx.x; i < cnt2; i += blockDim.x) {
        int64_t slot = b + i;
        double x[3], f[3];
        if (slot < e) {
            int64_t j = perm[slot];
            for (int l = 0; l < 3; ++l) {
                x[l] = xs[l * n + slot];
                f[l] = w[3 * j + l];
            }
        } else {
            for (int l = 0; l < 3; ++l) {
                x[l] = 1e18;
                f[l] = 0.0;
            }
        }
        if (LEAF) put_leaf_pair_half(out + ((int64_t)pb[r] + i / 2) * 12, (int)(i & 1), x, ch, cl, f);
        else put_pair_half(out + ((int64_t)pb[r] + i / 2) * 20, (int)(i & 1), x, f);
    }
}

// Paired records of n sources in the caller's order (a direct sum): one
// thread per slot of the padded range [0, 2 ceil(n/2)).
__global__ void k_pack_pairs_flat(int64_t n, const double *__restrict__ xyz,
                                  const double *__restrict__ w, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ((n + 1) / 2) * 2) return;
    double x[3], f[3];
    for (int l = 0; l < 3; ++l) {
        x[l] = i < n ? xyz[3 * i + l] : 1e18;
        f[l] = i < n ? w[3 * i + l] : 0.0;
    }
    put_pair_half(out + (i / 2) * 20, (int)(i & 1), x, f);
}

// Record q of a cluster's paired grid records (pair_records): fh is the
// cluster's FP64 weights [k1][k2][k3][3]; the record is
// [fx_a fx_b fy_a fy_b][fz_a fz_b 0 0] for its two points a, b (a missing b
// has zero weight).
__device__ __forceinline__ void pack_pair_record(const double *__restrict__ fh, int np, bool rowpairs,
                                                 int64_t q, float4 *__restrict__ o)
{
    const double *a, *b = nullptr;
    if (rowpairs && (np & 1)) {  // point k3 of rows 2P and 2P + 1
        const int64_t P = q / np, ra = 2 * P;
        const int k3 = (int)(q - P * np);
        a = fh + (ra * np + k3) * 3;
        if (ra + 1 < (int64_t)np * np) b = fh + ((ra + 1) * np + k3) * 3;
    } else {                     // points k, k + 1 of row r
        const int h = (np + 1) / 2;
        const int64_t r = q / h;
        const int k = (int)(q - r * h) * 2;
        a = fh + (r * np + k) * 3;
        if (k + 1 < np) b = a + 3;
    }
    double g[3] = {0.0, 0.0, 0.0};
    if (b)
        for (int l = 0; l < 3; ++l) g[l] = b[l];
    o[0] = make_float4((float)a[0], (float)g[0], (float)a[1], (float)g[1]);
    o[1] = make_float4((float)a[2], (float)g[2], 0.f, 0.f);
}

// Paired records of every cluster (of the first *nclus_dev when given).
__global__ void k_pack_proxy_pairs(int64_t nclus, int np, bool rowpairs, const double *__restrict__ fhat,
                                   float4 *__restrict__ out, const int *__restrict__ nclus_dev)
{
    const int64_t R = pair_records(np, rowpairs);
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (nclus_dev) nclus = min(nclus, (int64_t)*nclus_dev);
    if (q >= nclus * R) return;
    const int64_t c = q / R;
    pack_pair_record(fhat + c * np * np * np * 3, np, rowpairs, q - c * R, out + 2 * q);
}

}  // namespace

int proxy_record_bytes(int win, bool mixed)
{
    return mixed ? (win == 3 ? 16 : 32) : (win == 3 ? 32 : 48);
}

int source_record_bytes(int win, bool mixed)
{
    return mixed ? 48 : (win == 3 ? 48 : 80);
}

void WeightsDev::release(cudaStream_t s)
{
    for (DevBuf *b : {&fhat, &proxy, &src, &pbegin, &partial, &items}) b->release(s);
}

size_t WeightsDev::bytes() const
{
    return fhat.bytes + proxy.bytes + src.bytes + pbegin.bytes + partial.bytes + items.bytes;
}

template <int ACC>
kitc_status launch_chunks(dim3 grid, size_t smem, cudaStream_t s, const Cheb &cb, const Item *items,
                          const TreeDev &t, const double *w, int win, int sb, double *partial,
                          const int *nitems_dev)
{
    // every plan keeps a chunk's shared memory within CHUNK_SMEM_MAX, so one
    // attribute value per device serves all launches (no race between threads)
    static std::atomic<int> configured[64] = {};
    if (smem > CHUNK_SMEM_MAX) return KITC_ERR_INVALID_ARG;
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev].load()) {
        KITC_CUDA(cudaFuncSetAttribute(k_weights_chunk<ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CHUNK_SMEM_MAX));
        if (dev >= 0 && dev < 64) configured[dev].store(1);
    }
    kitc_count_launch();
    k_weights_chunk<ACC><<<grid, WT, smem, s>>>(cb, items, t.n, t.xs.as<double>(), t.perm.as<int32_t>(), w,
                                                win, t.lo.as<dvec4>(), t.hi.as<dvec4>(), sb, partial,
                                                nitems_dev);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

using ChunkLauncher = kitc_status (*)(dim3, size_t, cudaStream_t, const Cheb &, const Item *,
                                      const TreeDev &, const double *, int, int, double *,
                                      const int *);

// Launchers of k_weights_chunk<1..16>.
const ChunkLauncher *chunk_table()
{
    static constexpr ChunkLauncher t64[ACC_MAX] = {
        &launch_chunks<1>, &launch_chunks<2>, &launch_chunks<3>, &launch_chunks<4>,
        &launch_chunks<5>, &launch_chunks<6>, &launch_chunks<7>, &launch_chunks<8>,
        &launch_chunks<9>, &launch_chunks<10>, &launch_chunks<11>, &launch_chunks<12>,
        &launch_chunks<13>, &launch_chunks<14>, &launch_chunks<15>, &launch_chunks<16>};
    return t64;
}

// ---------------------------------------------------------------------------
// Split-precision Algorithm 1 with register tiles (the mixed form's weights).
// * The two FP32 lanes of a packed FP32x2 instruction carry two consecutive
//   particles: h = L1 L2 and g = L3 f are stored pair-interleaved,
//   [hi_j hi_j+1 lo_j lo_j+1] per row (column), so one 128-bit shared load
//   gives a row's (column's) values for both particles.
// * Each thread owns an R x C tile of outputs (rows (k1, k2), columns
//   (k3, q)) and loads R + C values per particle pair for R C products.
// * Per product the arithmetic is TwoProduct of the high parts (by FMA), the
//   cross terms, TwoSum into the running FP32 pair; each lane sums every other
//   particle of a run, and the two lanes are added (TwoSum) when the run is
//   folded into the FP64 sum.
// * The FP64 basis takes the grid points once per item and one reciprocal per
//   axis (bary_basis_split).
// ---------------------------------------------------------------------------
namespace {

struct SplitPlan {
    int R = 0, C = 0, TR = 0, TC = 0, np2pad = 0, nwpad = 0, sb = 0, npass = 0;
    size_t smem = 0;
};

// a - b on both lanes (PTX sub.rn.f32x2)
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<const unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<const unsigned long long *>(&b);
    unsigned long long rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<const float2 *>(&rd);
}

// (a.x + a.y) + (b.x + b.y) as an FP32 pair: TwoSum of the high parts, the
// low parts added to its error, renormalised (Fast2Sum).
__device__ __forceinline__ float2 add_f2(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    const float c = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s, c);
    return make_float2(hi, __fsub_rn(c, __fsub_rn(hi, s)));
}

// 1 / (a.x + a.y) as an FP32 pair: the correctly rounded reciprocal r of the
// high part, then one Newton step r + r (1 - a r), the residual formed with
// the exact product a.x r (TwoProduct by FMA); relative error about 2^-46.
__device__ __forceinline__ float2 rcp_f2(float2 a)
{
    const float r = __frcp_rn(a.x);
    const float p = __fmul_rn(a.x, r);
    const float e = __fmaf_rn(a.x, r, -p);                       // a.x r = p + e
    const float res = __fmaf_rn(-a.y, r, __fsub_rn(__fsub_rn(1.f, p), e));  // 1 - a r
    const float c = __fmul_rn(r, res);
    const float hi = __fadd_rn(r, c);
    return make_float2(hi, __fsub_rn(c, __fsub_rn(hi, r)));
}

// Barycentric basis of the coordinate y at the grid points s[0..n] of an
// interval of width 1/iw, written to Lj as FP32 hi/lo pairs: the second
// barycentric form (Eq. Barycentric-1D) with the same coincident-point rule
// as bary_basis,
//   L_k = (w_k / q_k) / sum_j (w_j / q_j),   q_j = (y - s_j) iw,
// with the differences and q_j in FP64 and the reciprocals, the sum and the
// quotients in FP32 pairs (about 2^-45 relative), which leaves the FP64 pipe
// one subtraction, one product and the conversion of q_j per point.  iw keeps
// every q_j in [-1, 1]; a point whose |q_j| is at most 2^-60 is taken as
// coinciding too (its L_j is 1 to within 2^-58, beyond the pairs' range of
// reciprocals).
__device__ __forceinline__ void bary_basis_split(const Cheb &cb, const double *__restrict__ s, double iw,
                                                 double y, float2 *Lj)
{
    const int np = cb.n + 1;
    int flag = -1;
    float2 S = make_float2(0.f, 0.f);
    for (int k = 0; k < np; ++k) {
        const double d = y - s[k];
        const double q = d * iw;
        // |d| <= DBL_MIN or |q| <= 2^-60, tested on the bits (d and q are finite)
        if ((__double_as_longlong(d) & 0x7fffffffffffffffll) <= 0x0010000000000000ll ||
            (__double_as_longlong(q) & 0x7fffffffffffffffll) <= 0x3c30000000000000ll)
            flag = k;
        // w_k = (-1)^k, halved at both ends (the weights of make_cheb): exact
        const float wk = ((k & 1) ? -1.f : 1.f) * ((k == 0 || k == cb.n) ? 0.5f : 1.f);
        float2 r = rcp_f2(split_f2(q));
        r.x *= wk;
        r.y *= wk;
        Lj[k] = r;
        S = add_f2(S, r);
    }
    if (flag >= 0) {
        for (int k = 0; k < np; ++k) Lj[k] = make_float2(k == flag ? 1.f : 0.f, 0.f);
        return;
    }
    const float2 rS = rcp_f2(S);
    for (int k = 0; k < np; ++k) Lj[k] = mul_f2(Lj[k], rS);
}

template <int R, int C>
__global__ void __launch_bounds__(WT, 2) k_weights_split(
    Cheb cb, const Item *__restrict__ items, int64_t n, const double *__restrict__ xs,
    const int32_t *__restrict__ perm, const double *__restrict__ w, int win,
    const dvec4 *__restrict__ lo, const dvec4 *__restrict__ hi, SplitPlan sp,
    double *__restrict__ partial, const int *__restrict__ nitems_dev)
{
    if (nitems_dev && (int)blockIdx.x >= *nitems_dev) return;  // device-planned items: past the end
    extern __shared__ float4 smf4[];
    const int np = cb.n + 1, np2 = np * np, nw = np * win, pwin = np2 * nw;
    const int sb = sp.sb, np2pad = sp.np2pad, nwpad = sp.nwpad;
    float4 *h4 = smf4;                                            // [sb/2][np2pad]
    float4 *g4 = h4 + (size_t)(sb / 2) * np2pad;                  // [sb/2][nwpad]
    float2 *Lf = reinterpret_cast<float2 *>(g4 + (size_t)(sb / 2) * nwpad);  // [sb][3][np]
    float2 *wsf = Lf + (size_t)sb * 3 * np;                       // [sb][win]
    double *sg = reinterpret_cast<double *>(wsf + (size_t)sb * win);  // [3][np] grid points
    double *siw = sg + 3 * np;                                    // [3] 1 / box width
    uint8_t *tk1 = reinterpret_cast<uint8_t *>(siw + 3);          // row r = (k1, k2)
    uint8_t *tk2 = tk1 + np2pad;
    uint8_t *tk3 = tk2 + np2pad;                                  // column c = (k3, q)
    uint8_t *tq = tk3 + nwpad;
    const Item it = items[blockIdx.x];
    const dvec4 blo = lo[it.c], bhi = hi[it.c];
    // the item's grid points (the expression of bary_basis) and index tables
    for (int t = threadIdx.x; t < 3 * np; t += WT) {
        const int l = t / np, k = t % np;
        const double a = l == 0 ? blo.x : (l == 1 ? blo.y : blo.z);
        const double b = l == 0 ? bhi.x : (l == 1 ? bhi.y : bhi.z);
        sg[t] = __dmul_rn(0.5, __dadd_rn(__dadd_rn(a, b), __dmul_rn(cb.t[k], __dsub_rn(b, a))));
    }
    if (threadIdx.x < 3) {
        const int l = threadIdx.x;
        const double a = l == 0 ? blo.x : (l == 1 ? blo.y : blo.z);
        const double b = l == 0 ? bhi.x : (l == 1 ? bhi.y : bhi.z);
        siw[l] = b > a ? __drcp_rn(__dsub_rn(b, a)) : 0.0;  // a flat axis: every point coincides
    }
    for (int t = threadIdx.x; t < np2pad; t += WT) {
        tk1[t] = (uint8_t)(t < np2 ? t / np : 0);
        tk2[t] = (uint8_t)(t < np2 ? t % np : 0);
    }
    for (int t = threadIdx.x; t < nwpad; t += WT) {
        tk3[t] = (uint8_t)(t < nw ? t / win : 0);
        tq[t] = (uint8_t)(t < nw ? t % win : 0);
    }
    // this thread's start and stride in the (particle, row), (particle, column)
    // and (particle, component) loops of a round: no division inside them
    const int jh0 = threadIdx.x / np2pad, rh0 = threadIdx.x % np2pad;
    const int djh = WT / np2pad, drh = WT % np2pad;
    const int jg0 = threadIdx.x / nwpad, cg0 = threadIdx.x % nwpad;
    const int djg = WT / nwpad, dcg = WT % nwpad;
    const int jw0 = threadIdx.x / win, qw0 = threadIdx.x % win;
    const int djw = WT / win, dqw = WT % win;
    const int q = blockIdx.y * WT + threadIdx.x;
    const bool active = q < sp.TR * sp.TC;
    const int r0 = active ? (q / sp.TC) * R : 0, c0 = active ? (q % sp.TC) * C : 0;
    // the FP64 sums live in this item's partial row (each output has one
    // owner thread), touched once per run; the FP32 pairs in registers
    double *dst = partial + (size_t)blockIdx.x * pwin;
    float2 SH[R][C], SL[R][C];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int k = 0; k < C; ++k) SH[i][k] = SL[i][k] = make_float2(0.f, 0.f);
    constexpr int FLUSH = 4;  // chunks per FP32 run
    int nrun = 0;
    bool first = true;
    __syncthreads();
    for (int j0 = it.p0; j0 < it.p1; j0 += sb) {
        const int cnt = min(sb, it.p1 - j0), cnt2 = (cnt + 1) & ~1;
        for (int t = threadIdx.x; t < cnt * 3; t += WT) {
            const int j = t / 3, l = t % 3;
            bary_basis_split(cb, sg + l * np, siw[l], xs[l * n + j0 + j], Lf + (j * 3 + l) * np);
        }
        for (int j = jw0, qq = qw0; j < cnt;) {
            wsf[j * win + qq] = split_f2(w[(int64_t)perm[j0 + j] * win + qq]);
            j += djw;
            qq += dqw;
            if (qq >= win) {
                qq -= win;
                ++j;
            }
        }
        __syncthreads();
        // h and g of the round, pair-interleaved; padding rows, columns and the
        // missing partner of an odd last particle are zero
        for (int j = jh0, r = rh0; j < cnt2;) {
            float2 v = make_float2(0.f, 0.f);
            if (j < cnt && r < np2) v = mul_f2(Lf[(j * 3 + 0) * np + tk1[r]], Lf[(j * 3 + 1) * np + tk2[r]]);
            float *d = reinterpret_cast<float *>(h4 + (size_t)(j >> 1) * np2pad + r);
            d[j & 1] = v.x;
            d[2 + (j & 1)] = v.y;
            j += djh;
            r += drh;
            if (r >= np2pad) {
                r -= np2pad;
                ++j;
            }
        }
        for (int j = jg0, c = cg0; j < cnt2;) {
            float2 v = make_float2(0.f, 0.f);
            if (j < cnt && c < nw) v = mul_f2(Lf[(j * 3 + 2) * np + tk3[c]], wsf[j * win + tq[c]]);
            float *d = reinterpret_cast<float *>(g4 + (size_t)(j >> 1) * nwpad + c);
            d[j & 1] = v.x;
            d[2 + (j & 1)] = v.y;
            j += djg;
            c += dcg;
            if (c >= nwpad) {
                c -= nwpad;
                ++j;
            }
        }
        __syncthreads();
        if (active) {
            const float4 *hp = h4 + r0, *gp = g4 + c0;
            for (int jp = 0; jp < cnt2 / 2; ++jp, hp += np2pad, gp += nwpad) {
                float4 B[C];
                float2 nbh[C];
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    B[k] = gp[k];
                    nbh[k] = sub2(make_float2(0.f, 0.f), make_float2(B[k].x, B[k].y));
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float4 A = hp[i];
                    const float2 ah = make_float2(A.x, A.y), al = make_float2(A.z, A.w);
#pragma unroll
                    for (int k = 0; k < C; ++k) {
                        const float2 bh = make_float2(B[k].x, B[k].y), bl = make_float2(B[k].z, B[k].w);
                        const float2 p = __fmul2_rn(ah, bh);
                        const float2 en = __ffma2_rn(ah, nbh[k], p);  // p - ah bh, exact (= -e)
                        const float2 c = sub2(__ffma2_rn(ah, bl, __fmul2_rn(al, bh)), en);
                        const float2 t = __fadd2_rn(SH[i][k], p);      // TwoSum(SH, p)
                        const float2 bb = sub2(t, SH[i][k]);
                        const float2 er = __fadd2_rn(sub2(SH[i][k], sub2(t, bb)), sub2(p, bb));
                        SH[i][k] = t;
                        SL[i][k] = __fadd2_rn(SL[i][k], __fadd2_rn(er, c));
                    }
                }
            }
        }
        // into the FP64 sums every FLUSH chunks and at the item's end: the two
        // lanes added by TwoSum first
        if (++nrun == FLUSH || j0 + sb >= it.p1) {
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const float a = SH[i][k].x, b = SH[i][k].y;
                    const float s = a + b, bb = s - a;
                    const float e = (a - (s - bb)) + (b - bb);
                    const double run = (double)s + (double)((SL[i][k].x + SL[i][k].y) + e);
                    if (active && r0 + i < np2 && c0 + k < nw) {
                        double *o = dst + (r0 + i) * nw + c0 + k;
                        *o = first ? run : *o + run;
                    }
                    SH[i][k] = SL[i][k] = make_float2(0.f, 0.f);
                }
            nrun = 0;
            first = false;
        }
        __syncthreads();
    }
}

// Tile shape of the split kernel for degree np - 1: among R, C in 2..4 with
// R C <= 12 (two CTAs of 256 threads per SM at <= 128 registers), the fewest
// passes over the particles (each pass stages the bases again), then the
// least work per thread, then the fewest tiles.
SplitPlan split_plan(int np, int win)
{
    const int np2 = np * np, nw = np * win;
    SplitPlan best;
    int64_t best_cost = -1;
    for (int R = 2; R <= 4; ++R)
        for (int C = 2; C <= 4; ++C) {
            if (R * C > 12) continue;
            const int TR = (np2 + R - 1) / R, TC = (nw + C - 1) / C, tiles = TR * TC;
            const int passes = (tiles + WT - 1) / WT;
            const int64_t cost = ((int64_t)passes * (R * C + 6)) * 1000000 + tiles;
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best.R = R;
                best.C = C;
                best.TR = TR;
                best.TC = TC;
                best.npass = passes;
            }
        }
    best.np2pad = best.TR * best.R;
    best.nwpad = best.TC * best.C;
    const size_t per = 8 * ((size_t)best.np2pad + best.nwpad + 3 * (size_t)np + win);  // bytes per particle
    // grid points, box widths and the index tables
    const size_t fixed = 8 * (3 * (size_t)np + 3) + 2 * ((size_t)best.np2pad + best.nwpad) + 16;
    int sb = KITC_WEIGHTS_SB;
    while (sb > 8 && per * sb + fixed > CHUNK_SMEM_MAX) sb /= 2;
    best.sb = sb;
    best.smem = per * sb + fixed;
    return best;
}

template <int R, int C>
kitc_status launch_split_rc(dim3 grid, const SplitPlan &sp, cudaStream_t s, const Cheb &cb,
                            const Item *items, const TreeDev &t, const double *w, int win,
                            double *partial, const int *nitems_dev)
{
    static std::atomic<int> configured[64] = {};  // one attribute value per device, never changed
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[dev].load()) {
        KITC_CUDA(cudaFuncSetAttribute(k_weights_split<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)CHUNK_SMEM_MAX));
        if (dev >= 0 && dev < 64) configured[dev].store(1);
    }
    kitc_count_launch();
    k_weights_split<R, C><<<grid, WT, sp.smem, s>>>(cb, items, t.n, t.xs.as<double>(), t.perm.as<int32_t>(),
                                                    w, win, t.lo.as<dvec4>(), t.hi.as<dvec4>(), sp, partial,
                                                    nitems_dev);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

// Algorithm 1 over nitems work items (grid.x; with nitems_dev, items past
// *nitems_dev exit): the tiled split kernel for the mixed form, else the FP64
// k_weights_chunk with the fewest accumulators per thread that cover the
// outputs in one pass.
kitc_status launch_items(bool split, int degree, int win, int64_t nitems, const Item *items,
                         const TreeDev &t, const double *w, double *partial, const int *nitems_dev,
                         cudaStream_t s)
{
    if (nitems <= 0) return KITC_OK;
    const int np = degree + 1, pwin = np * np * np * win;
    const Cheb cb = make_cheb(degree);
    if (split) {
        const SplitPlan sp = split_plan(np, win);
        if (sp.smem > CHUNK_SMEM_MAX) return KITC_ERR_INVALID_ARG;
        const dim3 grid((unsigned)nitems, (unsigned)sp.npass);
        switch (sp.R * 10 + sp.C) {
        case 22: return launch_split_rc<2, 2>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 23: return launch_split_rc<2, 3>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 24: return launch_split_rc<2, 4>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 32: return launch_split_rc<3, 2>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 33: return launch_split_rc<3, 3>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 34: return launch_split_rc<3, 4>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 42: return launch_split_rc<4, 2>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        case 43: return launch_split_rc<4, 3>(grid, sp, s, cb, items, t, w, win, partial, nitems_dev);
        default: return KITC_ERR_INVALID_ARG;
        }
    }
    const size_t per = sizeof(double) * (3 * np + np * np + np * win);
    int sb = KITC_WEIGHTS_SB;
    while (sb > 8 && per * sb > CHUNK_SMEM_MAX) sb /= 2;
    const int acc = std::min(ACC_MAX, (pwin + WT - 1) / WT);
    const int npass = (pwin + acc * WT - 1) / (acc * WT);
    return chunk_table()[acc - 1](dim3((unsigned)nitems, (unsigned)npass), per * sb, s, cb, items, t, w,
                                  win, sb, partial, nitems_dev);
}

}  // namespace

size_t upward_child_smem(int np, int win)
{
    size_t pw = (size_t)np * np * np * win;
    return sizeof(double) * (2 * pw + 3 * (size_t)np * np);
}


namespace {

// ---------------------------------------------------------------------------
// Plans made on the device: the work items of Algorithm 1 in cluster order
// (chunks of CHUNK slots) and the ranges of the paired source records (one
// per leaf, in cluster order), by single-block scans over the clusters.  The
// cluster count comes from a tree's device state block (bs), or from the host
// (m_fixed) for a tree built by tree_build.  Every buffer is sized from bounds
// that hold for any tree of at most cap clusters:
//   items <= cap + (levels counted per slot) * ceil(n / CHUNK)
//   pairs <= (n + cap) / 2 + 1   (each leaf adds at most half a pair)
// ---------------------------------------------------------------------------
// Exclusive prefix of one value per thread over a block of 1024 threads;
// *total receives the block's sum (every thread).
__device__ int64_t block_prefix(int64_t v, int64_t *total)
{
    __shared__ int64_t ws[32];
    __shared__ int64_t tot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        const int64_t t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        int64_t u = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        ws[lane] = u - t;
        if (lane == 31) tot = u;
    }
    __syncthreads();
    const int64_t r = ws[w] + x - v;
    *total = tot;
    __syncthreads();  // ws and tot are reused by the next call
    return r;
}

__device__ __forceinline__ int items_of(int c, int m, bool upward, const int32_t *begin,
                                        const int32_t *end, const int32_t *n_child)
{
    if (c >= m || (upward && n_child[c] > 0)) return 0;
    return (end[c] - begin[c] + CHUNK - 1) / CHUNK;
}

// first[c] (c <= cap): the first work item of cluster c, items in cluster
// order, chunks of CHUNK slots; clamped to itemcap.  One block of 1024.
__global__ void __launch_bounds__(1024) k_items_plan(const BuildState *__restrict__ bs, int m_fixed,
                                                     int cap, bool upward,
                                                     const int32_t *__restrict__ begin,
                                                     const int32_t *__restrict__ end,
                                                     const int32_t *__restrict__ n_child,
                                                     int32_t *__restrict__ first, int itemcap,
                                                     int *__restrict__ nitems, int *__restrict__ err)
{
    const int m = min(bs ? bs->nclus : m_fixed, cap);
    const int per = (cap + blockDim.x - 1) / blockDim.x;
    const int c0 = min(cap, (int)threadIdx.x * per), c1 = min(cap, c0 + per);
    int64_t loc = 0;
    for (int c = c0; c < c1; ++c) loc += items_of(c, m, upward, begin, end, n_child);
    int64_t total = 0;
    int64_t run = block_prefix(loc, &total);
    for (int c = c0; c < c1; ++c) {
        first[c] = (int32_t)min(run, (int64_t)itemcap);
        run += items_of(c, m, upward, begin, end, n_child);
    }
    if (threadIdx.x == 0) {
        first[cap] = (int32_t)min(total, (int64_t)itemcap);
        *nitems = (int)min(total, (int64_t)itemcap);
        if (total > itemcap) atomicOr(err, ASYNC_RECORD_OVERFLOW);
    }
}

__global__ void k_items_fill(const BuildState *__restrict__ bs, int m_fixed, int cap,
                             const int32_t *__restrict__ first, const int32_t *__restrict__ begin,
                             const int32_t *__restrict__ end, Item *__restrict__ items)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= min(bs ? bs->nclus : m_fixed, cap)) return;
    const int32_t b = begin[c], e = end[c];
    for (int i = first[c]; i < first[c + 1]; ++i) {
        const int32_t p = b + (i - first[c]) * CHUNK;
        items[i] = Item{c, p, min(e, p + CHUNK), 0};
    }
}

// Paired-record plan: pb_all = [first pair per cluster (cap, -1 off the
// leaves) | range begin (cap) | range end (cap) | first pair (cap) | leaf of
// the range (cap)], one range per leaf in cluster order, empty ranges after
// the last leaf.  One block.
__global__ void __launch_bounds__(1024) k_pairs_plan(const BuildState *__restrict__ bs, int m_fixed,
                                                     int cap, const int32_t *__restrict__ begin,
                                                     const int32_t *__restrict__ end,
                                                     const int32_t *__restrict__ n_child,
                                                     int32_t *__restrict__ pb_all, int64_t paircap,
                                                     int *__restrict__ err)
{
    const int m = min(bs ? bs->nclus : m_fixed, cap);
    int32_t *cpb = pb_all, *rb = pb_all + cap, *re = rb + cap, *pb = re + cap, *rc = pb + cap;
    const int per = (cap + blockDim.x - 1) / blockDim.x;
    const int c0 = min(cap, (int)threadIdx.x * per), c1 = min(cap, c0 + per);
    int64_t nl = 0, np = 0;
    for (int c = c0; c < c1; ++c)
        if (c < m && n_child[c] == 0) {
            nl++;
            np += (end[c] - begin[c] + 1) / 2;
        }
    int64_t nleaves = 0, npairs = 0;
    int64_t r = block_prefix(nl, &nleaves);
    int64_t q = block_prefix(np, &npairs);
    const bool over = npairs > paircap;  // cannot happen for a valid tree (bound above)
    for (int c = c0; c < c1; ++c) {
        if (c < m && n_child[c] == 0) {
            cpb[c] = over ? 0 : (int32_t)q;
            rb[r] = begin[c];
            re[r] = over ? begin[c] : end[c];
            pb[r] = over ? 0 : (int32_t)q;
            rc[r] = c;
            r++;
            q += (end[c] - begin[c] + 1) / 2;
        } else {
            cpb[c] = -1;
        }
    }
    for (int64_t k = nleaves + threadIdx.x; k < cap; k += blockDim.x) rb[k] = re[k] = pb[k] = rc[k] = 0;
    if (threadIdx.x == 0 && over) atomicOr(err, ASYNC_RECORD_OVERFLOW);
}

}  // namespace

// Plan of the weights pass for one tree: buffer sizes and launch shapes.  The
// work items themselves are planned on the device by each launch (k_items_plan,
// in cluster order), in room that bounds the items of a tree of these clusters
// and levels, so neither the plan nor the launch reads anything back and the
// launch can be captured in a CUDA graph.
kitc_status weights_plan(const TreeDev &t, int win, int degree, int mode, cudaStream_t s,
                         WeightsDev &wd)
{
    if (wd.planned && !wd.var && wd.degree == degree && wd.win == win && wd.mode == mode)
        return KITC_OK;
    wd.planned = false;
    const int np = degree + 1;
    const int pwin = np * np * np * win;
    const bool upward = mode == KITC_WEIGHTS_UPWARD && upward_child_smem(np, win) <= UP_SMEM_MAX;
    const int64_t itemcap = weights_async_itemcap(t.nclus, std::max(1, t.depth), t.n,
                                                  upward ? KITC_WEIGHTS_UPWARD : KITC_WEIGHTS_ALGORITHM1);
    if (itemcap > INT32_MAX / 2) return KITC_ERR_OOM;
    // items (itemcap) | first item of each cluster (nclus + 1) | item count | error word
    KITC_TRY(wd.items.reserve(sizeof(Item) * itemcap + sizeof(int32_t) * ((size_t)t.nclus + 3) + 64, s));
    size_t rows = (size_t)itemcap;  // item partials, then the upward contributions
    if (upward)
        for (size_t L = 1; L < t.level_start.size(); ++L) {
            const int e = L + 1 < t.level_start.size() ? t.level_start[L + 1] : t.nclus;
            rows = std::max<size_t>(rows, (size_t)(e - t.level_start[L]));
        }
    KITC_TRY(wd.partial.reserve(sizeof(double) * pwin * rows, s));
    KITC_TRY(wd.fhat.reserve(sizeof(double) * pwin * t.nclus, s));
    wd.nitems = (size_t)itemcap;
    wd.upward = upward;
    if (upward) KITC_TRY(allow_up_smem());
    wd.degree = degree;
    wd.win = win;
    wd.mode = mode;
    wd.var = false;
    wd.planned = true;
    return KITC_OK;
}

kitc_status weights_launch(const TreeDev &t, const double *w_user, WeightsDev &wd, cudaStream_t s)
{
    if (!wd.planned) return KITC_ERR_STATE;
    const int np = wd.degree + 1, win = wd.win;
    const int pwin = np * np * np * win;
    const int nclus = t.nclus, itemcap = (int)wd.nitems;
    Item *d_items = wd.items.as<Item>();
    int32_t *d_first = reinterpret_cast<int32_t *>(d_items + itemcap);
    int *d_nitems = d_first + nclus + 1;
    const Cheb cb = make_cheb(wd.degree);
    kitc_count_launch();
    k_items_plan<<<1, 1024, 0, s>>>(nullptr, nclus, nclus, wd.upward, t.begin.as<int32_t>(),
                                    t.end.as<int32_t>(), t.n_child.as<int32_t>(), d_first, itemcap,
                                    d_nitems, d_nitems + 1);
    kitc_count_launch();
    k_items_fill<<<(nclus + 255) / 256, 256, 0, s>>>(nullptr, nclus, nclus, d_first, t.begin.as<int32_t>(),
                                                     t.end.as<int32_t>(), d_items);
    KITC_CUDA(cudaGetLastError());
    KITC_TRY(launch_items(wd.split, wd.degree, win, itemcap, d_items, t, w_user,
                          wd.partial.as<double>(), d_nitems, s));
    kitc_count_launch();
    k_weights_reduce<<<nclus, 256, 0, s>>>(d_first, pwin, wd.partial.as<double>(),
                                           wd.fhat.as<double>());
    KITC_CUDA(cudaGetLastError());
    if (wd.upward) {
        const size_t us = upward_child_smem(np, win);
        const int nlev = (int)t.level_start.size();
        // deepest parents first: level L needs every child at level L + 1; the
        // children's contributions go to the (now free) item partials
        for (int L = nlev - 2; L >= 0; --L) {
            const int lb = t.level_start[L], le = t.level_start[L + 1];
            const int cb0 = t.level_start[L + 1], ce = L + 2 < nlev ? t.level_start[L + 2] : t.nclus;
            kitc_count_launch();
            k_upward_child<<<ce - cb0, WT, us, s>>>(cb, cb0, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                                    t.parent.as<int32_t>(), win, wd.fhat.as<double>(),
                                                    wd.partial.as<double>());
            kitc_count_launch();
            const int64_t tot = (int64_t)(le - lb) * pwin;
            k_upward_sum<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
                lb, le, cb0, pwin, t.first_child.as<int32_t>(), t.n_child.as<int32_t>(),
                wd.partial.as<double>(), wd.fhat.as<double>());
            KITC_CUDA(cudaGetLastError());
        }
    }
    return KITC_OK;
}

kitc_status weights_compute(const TreeDev &t, const double *w_user, int win, int degree, int mode,
                            cudaStream_t s, WeightsDev &wd)
{
    KITC_TRY(weights_plan(t, win, degree, mode, s, wd));
    return weights_launch(t, w_user, wd, s);
}

kitc_status pack_proxies(const TreeDev &t, WeightsDev &wd, bool mixed, cudaStream_t s)
{
    int np = wd.degree + 1;
    int64_t nrec = (int64_t)t.nclus * np * np * np;
    KITC_TRY(wd.proxy.reserve((size_t)proxy_record_bytes(wd.win, mixed) * nrec, s));
    unsigned g = (unsigned)((nrec + 255) / 256);
    kitc_count_launch();
    if (mixed)
        k_pack_proxies<true><<<g, 256, 0, s>>>(nrec, wd.win, wd.fhat.as<double>(), wd.proxy.ptr,
                                               nullptr, 0);
    else
        k_pack_proxies<false><<<g, 256, 0, s>>>(nrec, wd.win, wd.fhat.as<double>(), wd.proxy.ptr,
                                                nullptr, 0);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status pack_sources(const TreeDev *t, const double *xyz_user, const double *w_user,
                         int64_t n, int win, bool mixed, cudaStream_t s, DevBuf &out)
{
    KITC_TRY(out.reserve((size_t)source_record_bytes(win, mixed) * n, s));
    unsigned g = (unsigned)((n + 255) / 256);
    const double *xs = t ? t->xs.as<double>() : nullptr;
    const int32_t *perm = t ? t->perm.as<int32_t>() : nullptr;
    kitc_count_launch();
    if (mixed)
        k_pack_sources<true><<<g, 256, 0, s>>>(n, win, xs, perm, xyz_user, w_user, out.ptr);
    else
        k_pack_sources<false><<<g, 256, 0, s>>>(n, win, xs, perm, xyz_user, w_user, out.ptr);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

// Plan of the paired records, made on the device (k_pairs_plan): one range per
// leaf in cluster order, in room for any leaf sizes of this tree; pbegin
// receives [first pair of each cluster (nclus, -1 off the leaves) | range
// begin | range end | first pair | leaf (nclus each; empty ranges after the
// last leaf) | an error word].  Reads nothing back.
kitc_status pack_pairs_plan(const TreeDev *t, int64_t n, bool leaf, cudaStream_t s, DevBuf &out,
                            DevBuf &pbegin, int *nranges)
{
    if (!t) return KITC_ERR_INVALID_ARG;
    const int nclus = t->nclus;
    const int64_t paircap = (n + nclus) / 2 + 1;
    KITC_TRY(out.reserve(pair_record_bytes(leaf) * paircap + 16, s));
    KITC_TRY(pbegin.reserve(sizeof(int32_t) * (5 * (size_t)nclus + 1) + 16, s));
    int32_t *d = pbegin.as<int32_t>();
    kitc_count_launch();
    k_pairs_plan<<<1, 1024, 0, s>>>(nullptr, nclus, nclus, t->begin.as<int32_t>(), t->end.as<int32_t>(),
                                    t->n_child.as<int32_t>(), d, paircap,
                                    reinterpret_cast<int *>(d + 5 * (size_t)nclus));
    KITC_CUDA(cudaGetLastError());
    *nranges = nclus;
    return KITC_OK;
}

kitc_status pack_pairs_launch(const TreeDev *t, const double *w_user, int64_t n, int nranges,
                              bool leaf, cudaStream_t s, DevBuf &out, DevBuf &pbegin)
{
    if (!t) return KITC_ERR_INVALID_ARG;
    const int nclus = t->nclus;
    int32_t *d = pbegin.as<int32_t>();
    kitc_count_launch();
    (leaf ? k_pack_pairs<true> : k_pack_pairs<false>)<<<(unsigned)nranges, 256, 0, s>>>(d + nclus, d + nclus + nranges,
                                                   d + nclus + 2 * nranges, d + nclus + 3 * nranges, n,
                                                   t->xs.as<double>(), t->perm.as<int32_t>(),
                                                   t->lo.as<dvec4>(), t->hi.as<dvec4>(), w_user,
                                                   out.as<float>());
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status pack_proxy_pairs(const TreeDev &t, WeightsDev &wd, cudaStream_t s)
{
    const int np = wd.degree + 1;
    const int64_t nrec = (int64_t)t.nclus * pair_records(np, wd.rowpairs);
    KITC_TRY(wd.proxy.reserve((size_t)32 * nrec, s));
    unsigned g = (unsigned)((nrec + 255) / 256);
    kitc_count_launch();
    k_pack_proxy_pairs<<<g, 256, 0, s>>>(t.nclus, np, wd.rowpairs, wd.fhat.as<double>(),
                                         wd.proxy.as<float4>(), nullptr);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

size_t direct_record_bytes(int64_t n, int win, bool mixed, bool pairs)
{
    return pairs ? (size_t)80 * ((n + 1) / 2) : (size_t)source_record_bytes(win, mixed) * n;
}

kitc_status pack_direct_records(const double *xyz, const double *w, int64_t n, int win, bool mixed,
                                bool pairs, void *out, cudaStream_t s)
{
    if (pairs) {
        unsigned g = (unsigned)((((n + 1) / 2) * 2 + 255) / 256);
        kitc_count_launch();
        k_pack_pairs_flat<<<g, 256, 0, s>>>(n, xyz, w, reinterpret_cast<float *>(out));
    } else {
        unsigned g = (unsigned)((n + 255) / 256);
        kitc_count_launch();
        if (mixed)
            k_pack_sources<true><<<g, 256, 0, s>>>(n, win, nullptr, nullptr, xyz, w, out);
        else
            k_pack_sources<false><<<g, 256, 0, s>>>(n, win, nullptr, nullptr, xyz, w, out);
    }
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status pack_direct_preload(size_t *lmem)
{
    const void *kerns[] = {reinterpret_cast<const void *>(k_pack_pairs_flat),
                           reinterpret_cast<const void *>(k_pack_sources<true>),
                           reinterpret_cast<const void *>(k_pack_sources<false>)};
    for (const void *k : kerns) {
        cudaFuncAttributes at;
        KITC_CUDA(cudaFuncGetAttributes(&at, k));
        *lmem = std::max(*lmem, (size_t)at.localSizeBytes);
    }
    return KITC_OK;
}

// ---------------------------------------------------------------------------
// Degree per cluster (kitc_set_degrees).  Cluster c has degree deg[c] (0: no
// modified weights); its FP64 weights start at fhat + foff[c] and its grid
// records at proxy + roff[c] bytes.
//
// Upward form (used when its shared memory fits): let A_c be the largest degree
// on the path from the root to c.  Leaves get Algorithm 1 at degree A_c, every
// parent gets the weights at A_p from its children through the parent's
// barycentric basis at the children's points (exact: A_child >= A_p, so a
// child's degree-A_child interpolation reproduces the parent's degree-A_p
// Lagrange polynomials, Sec. 2), and a cluster with deg[c] < A_c is then taken
// down to deg[c] the same way with its own points as the source (exact for
// the same reason).  Otherwise every cluster runs Algorithm 1 at deg[c].
// Either way fhat equals Eq. modified_weights at each cluster's degree up to
// rounding.
// ---------------------------------------------------------------------------
namespace {

// Sums the work-item partials of cluster c (icount[c] > 0) into fhat + roff[c]
// at degree rdeg[c].
__global__ void k_weights_reduce_var(const int32_t *__restrict__ rdeg, int win,
                                     const int64_t *__restrict__ pstart,
                                     const int32_t *__restrict__ icount,
                                     const int64_t *__restrict__ roff,
                                     const double *__restrict__ partial, double *__restrict__ fhat)
{
    int c = blockIdx.x;
    int ni = icount[c];
    if (ni <= 0) return;
    int np = rdeg[c] + 1, pw = np * np * np * win;
    const double *src = partial + pstart[c];
    for (int o = threadIdx.x; o < pw; o += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < ni; ++i) s += src[(size_t)i * pw + o];
        fhat[roff[c] + o] = s;
    }
}

// Block per destination cluster p of [lb, lb + gridDim.x).  UP: p's weights at
// degree adeg[p] from its children's (degree adeg[child], at goff); otherwise
// p's own weights at adeg[p] taken down to deg[p] (written at foff[p]).
// Three 1D contractions per source (the grids are tensor products).
template <bool UP>
__global__ void __launch_bounds__(WT) k_transfer(
    int lb, const Cheb *__restrict__ chebs, const dvec4 *__restrict__ lo,
    const dvec4 *__restrict__ hi, const int32_t *__restrict__ first_child,
    const int32_t *__restrict__ n_child, const int32_t *__restrict__ adeg,
    const int32_t *__restrict__ deg, const int64_t *__restrict__ goff,
    const int64_t *__restrict__ foff, int win, int pmax, double *__restrict__ fhat)
{
    extern __shared__ double sm[];
    const int p = lb + blockIdx.x;
    int dd, nsrc, src0;
    double *dst;
    if (UP) {
        dd = adeg[p];
        nsrc = n_child[p];
        if (dd <= 0 || nsrc == 0) return;
        src0 = first_child[p];
        dst = fhat + goff[p];
    } else {
        dd = deg[p];
        if (dd <= 0 || dd == adeg[p]) return;
        nsrc = 1;
        src0 = p;
        dst = fhat + foff[p];
    }
    const Cheb &cd = chebs[dd];
    const int pd = dd + 1, pdw = pd * pd * pd * win;
    const size_t big = (size_t)pmax * pmax * pmax * win;
    double *T1 = sm, *T2 = T1 + big, *A = T2 + big, *M = A + big;  // M[l][k'][k] = L^dst_k(s^src_k')
    for (int i = threadIdx.x; i < pdw; i += WT) A[i] = 0.0;
    const dvec4 plo = lo[p], phi = hi[p];
    for (int ci = 0; ci < nsrc; ++ci) {
        const int c = src0 + ci;
        const int ds = adeg[c], ps = ds + 1;
        const Cheb &cs = chebs[ds];
        const dvec4 clo = lo[c], chi = hi[c];
        __syncthreads();
        for (int q = threadIdx.x; q < 3 * ps; q += WT) {
            int l = q / ps, kp = q % ps;
            double ca = l == 0 ? clo.x : (l == 1 ? clo.y : clo.z);
            double cb_ = l == 0 ? chi.x : (l == 1 ? chi.y : chi.z);
            double pa = l == 0 ? plo.x : (l == 1 ? plo.y : plo.z);
            double pb = l == 0 ? phi.x : (l == 1 ? phi.y : phi.z);
            double y = __dmul_rn(0.5, __dadd_rn(__dadd_rn(ca, cb_), __dmul_rn(cs.t[kp], __dsub_rn(cb_, ca))));
            double L[KITC_MAX_DEGREE + 1];
            bary_basis(cd, pa, pb, y, L);
            for (int k = 0; k < pd; ++k) M[(l * ps + kp) * pd + k] = L[k];
        }
        __syncthreads();
        const double *F = fhat + goff[c];  // [ks1][ks2][ks3][q]
        const int n1 = ps * ps * pd * win;
        for (int o = threadIdx.x; o < n1; o += WT) {  // T1[ks1][ks2][kd3][q]
            int q = o % win, k3 = (o / win) % pd, r = o / (win * pd);
            double v = 0.0;
            for (int kp = 0; kp < ps; ++kp) v = fma(M[(2 * ps + kp) * pd + k3], F[(r * ps + kp) * win + q], v);
            T1[o] = v;
        }
        __syncthreads();
        const int n2 = ps * pd * pd * win;
        for (int o = threadIdx.x; o < n2; o += WT) {  // T2[ks1][kd2][kd3][q]
            int q = o % win, k3 = (o / win) % pd, k2 = (o / (win * pd)) % pd, k1 = o / (win * pd * pd);
            double v = 0.0;
            for (int kp = 0; kp < ps; ++kp)
                v = fma(M[(ps + kp) * pd + k2], T1[((k1 * ps + kp) * pd + k3) * win + q], v);
            T2[o] = v;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < pdw; o += WT) {  // A[kd1][kd2][kd3][q] += ...
            int q = o % win, k3 = (o / win) % pd, k2 = (o / (win * pd)) % pd, k1 = o / (win * pd * pd);
            double v = 0.0;
            for (int kp = 0; kp < ps; ++kp)
                v = fma(M[kp * pd + k1], T2[((kp * pd + k2) * pd + k3) * win + q], v);
            A[o] += v;
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < pdw; o += WT) dst[o] = A[o];
}

// Block per cluster: grid records of the cluster, paired (FP32x2 evaluator)
// or one record per point (other forms), at proxy + roff[c].
template <int FORM>  // 0: pairs, 1: FP32 float4 per point, 2: FP64 per point
__global__ void k_pack_proxies_var(const int32_t *__restrict__ deg, int win,
                                   const int64_t *__restrict__ foff,
                                   const int64_t *__restrict__ roff, const double *__restrict__ fhat,
                                   unsigned char *__restrict__ proxy, bool rowpairs)
{
    int c = blockIdx.x;
    int d = deg[c];
    if (d <= 0) return;
    int np = d + 1;
    const double *fh = fhat + foff[c];
    unsigned char *out = proxy + roff[c];
    if (FORM == 0) {
        const int64_t R = pair_records(np, rowpairs);
        for (int64_t q = threadIdx.x; q < R; q += blockDim.x)
            pack_pair_record(fh, np, rowpairs, q, reinterpret_cast<float4 *>(out) + 2 * q);
    } else {
        int P = np * np * np;
        for (int r = threadIdx.x; r < P; r += blockDim.x) {
            const double *f = fh + (size_t)r * win;
            if (FORM == 1) {
                float4 *o = reinterpret_cast<float4 *>(out);
                o[(win == 3 ? 1 : 2) * r] = make_float4((float)f[0], (float)f[1], (float)f[2], 0.f);
                if (win == 6)
                    o[2 * r + 1] = make_float4((float)f[3], (float)f[4], (float)f[5], 0.f);
            } else {
                double *o = reinterpret_cast<double *>(out) + (size_t)r * (win == 3 ? 4 : 6);
                for (int q = 0; q < (win == 3 ? 4 : 6); ++q) o[q] = q < win ? f[q] : 0.0;
            }
        }
    }
}


size_t transfer_smem(int pmax, int win)
{
    size_t big = (size_t)pmax * pmax * pmax * win;
    return sizeof(double) * (3 * big + 3 * (size_t)pmax * pmax);
}

// The upward kernels run with at most UP_SMEM_MAX bytes of dynamic shared
// memory (their plans check it); the attribute is set to that bound once per
// device, so concurrent plans never lower it under each other's launches.
kitc_status allow_up_smem()
{
    static std::atomic<int> done[64] = {};
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev].load()) return KITC_OK;
    KITC_CUDA(cudaFuncSetAttribute(k_upward_child, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)UP_SMEM_MAX));
    KITC_CUDA(cudaFuncSetAttribute(k_upward_child_dev, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)UP_SMEM_MAX));
    KITC_CUDA(cudaFuncSetAttribute(k_transfer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)UP_SMEM_MAX));
    KITC_CUDA(cudaFuncSetAttribute(k_transfer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)UP_SMEM_MAX));
    if (dev >= 0 && dev < 64) done[dev].store(1);
    return KITC_OK;
}

}  // namespace

kitc_status weights_plan_var(const TreeDev &t, int win, const std::vector<int32_t> &hdeg,
                             cudaStream_t s, WeightsDev &wd)
{
    wd.planned = false;
    const int m = t.nclus;
    std::vector<int32_t> hb(m), he(m), hpar(m), hnc(m);
    KITC_CUDA(cudaMemcpyAsync(hb.data(), t.begin.ptr, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(he.data(), t.end.ptr, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(hpar.data(), t.parent.ptr, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(hnc.data(), t.n_child.ptr, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    // A_c: largest degree on the path root..c (parents precede children)
    std::vector<int32_t> adeg(m);
    int amax = 0;
    for (int c = 0; c < m; ++c) {
        int up = hpar[c] >= 0 && hpar[c] < c ? adeg[hpar[c]] : 0;
        adeg[c] = std::max(hdeg[c], up);
        amax = std::max(amax, adeg[c]);
    }
    const bool upward = amax > 0 && transfer_smem(amax + 1, win) <= UP_SMEM_MAX;
    // degree of the Algorithm 1 work of each cluster, and which clusters get it
    std::vector<int32_t> rdeg(m, 0);
    for (int c = 0; c < m; ++c)
        rdeg[c] = upward ? (hnc[c] == 0 ? adeg[c] : 0) : hdeg[c];
    std::vector<int64_t> goff(m, 0), foff(m, 0), pstart(m, 0);
    int64_t ofs = 0;
    auto P = [&](int d) { return (int64_t)(d + 1) * (d + 1) * (d + 1) * win; };
    if (upward) {
        for (int c = 0; c < m; ++c)
            if (adeg[c] > 0) goff[c] = ofs, ofs += P(adeg[c]);
        for (int c = 0; c < m; ++c) {
            if (hdeg[c] <= 0) continue;
            if (hdeg[c] == adeg[c]) foff[c] = goff[c];
            else foff[c] = ofs, ofs += P(hdeg[c]);
        }
    } else {
        for (int c = 0; c < m; ++c)
            if (hdeg[c] > 0) foff[c] = goff[c] = ofs, ofs += P(hdeg[c]);
    }
    // Algorithm 1 work items grouped by degree
    std::vector<Item> items;
    std::vector<int32_t> icount(m, 0);
    wd.groups.clear();
    int64_t pofs = 0;
    for (int d = 1; d <= KITC_MAX_DEGREE; ++d) {
        WeightsDev::Group g;
        g.degree = d;
        g.item0 = items.size();
        g.pofs = pofs;
        for (int c = 0; c < m; ++c) {
            if (rdeg[c] != d) continue;
            pstart[c] = pofs;
            for (int32_t p = hb[c]; p < he[c]; p += CHUNK) {
                items.push_back(Item{c, p, std::min(he[c], p + CHUNK), 0});
                pofs += P(d);
                icount[c]++;
            }
        }
        g.nitems = items.size() - g.item0;
        if (g.nitems) wd.groups.push_back(g);
    }
    size_t ni = items.size();
    size_t bytes = sizeof(Item) * ni + sizeof(int64_t) * 3 * m + sizeof(int32_t) * 4 * m +
                   sizeof(Cheb) * (KITC_MAX_DEGREE + 1) + 256;
    KITC_TRY(wd.items.reserve(bytes, s));
    Item *d_items = wd.items.as<Item>();
    int64_t *d_p = reinterpret_cast<int64_t *>(d_items + ni);
    int64_t *d_f = d_p + m, *d_g = d_f + m;
    int32_t *d_c = reinterpret_cast<int32_t *>(d_g + m);
    int32_t *d_r = d_c + m, *d_a = d_r + m, *d_d = d_a + m;
    Cheb *d_cheb = reinterpret_cast<Cheb *>(
        (reinterpret_cast<uintptr_t>(d_d + m) + 15) & ~static_cast<uintptr_t>(15));
    std::vector<Cheb> chebs(KITC_MAX_DEGREE + 1);
    for (int d = 1; d <= KITC_MAX_DEGREE; ++d) chebs[d] = make_cheb(d);
    chebs[0] = make_cheb(1);
    KITC_CUDA(cudaMemcpyAsync(d_items, items.data(), sizeof(Item) * ni, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_p, pstart.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_f, foff.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_g, goff.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_c, icount.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_r, rdeg.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_a, adeg.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_d, hdeg.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(d_cheb, chebs.data(), sizeof(Cheb) * chebs.size(), cudaMemcpyHostToDevice, s));
    KITC_TRY(wd.partial.reserve(sizeof(double) * std::max<int64_t>(pofs, 1), s));
    KITC_TRY(wd.fhat.reserve(sizeof(double) * std::max<int64_t>(ofs, 1), s));
    KITC_CUDA(cudaStreamSynchronize(s));  // the host vectors must outlive the copies
    if (upward) KITC_TRY(allow_up_smem());
    wd.nitems = ni;
    wd.fhat_len = ofs;
    wd.win = win;
    wd.degree = -1;
    wd.var_upward = upward;
    wd.var_pmax = amax + 1;
    wd.var = true;
    wd.planned = true;
    return KITC_OK;
}

kitc_status weights_launch_var(const TreeDev &t, const double *w_user, WeightsDev &wd,
                               cudaStream_t s)
{
    if (!wd.planned || !wd.var) return KITC_ERR_STATE;
    const int win = wd.win, m = t.nclus;
    Item *d_items = wd.items.as<Item>();
    int64_t *d_p = reinterpret_cast<int64_t *>(d_items + wd.nitems);
    int64_t *d_f = d_p + m, *d_g = d_f + m;
    int32_t *d_c = reinterpret_cast<int32_t *>(d_g + m);
    int32_t *d_r = d_c + m, *d_a = d_r + m, *d_d = d_a + m;
    const Cheb *d_cheb = reinterpret_cast<const Cheb *>(
        (reinterpret_cast<uintptr_t>(d_d + m) + 15) & ~static_cast<uintptr_t>(15));
    for (const auto &g : wd.groups)
        KITC_TRY(launch_items(wd.split, g.degree, win, (int64_t)g.nitems, d_items + g.item0, t, w_user,
                              wd.partial.as<double>() + g.pofs, nullptr, s));
    kitc_count_launch();
    k_weights_reduce_var<<<m, 256, 0, s>>>(d_r, win, d_p, d_c, wd.var_upward ? d_g : d_f,
                                           wd.partial.as<double>(), wd.fhat.as<double>());
    KITC_CUDA(cudaGetLastError());
    if (wd.var_upward) {
        const size_t sm = transfer_smem(wd.var_pmax, win);
        for (int L = (int)t.level_start.size() - 2; L >= 0; --L) {
            int lb = t.level_start[L], le = t.level_start[L + 1];
            if (le <= lb) continue;
            kitc_count_launch();
            k_transfer<true><<<le - lb, WT, sm, s>>>(lb, d_cheb, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                                     t.first_child.as<int32_t>(), t.n_child.as<int32_t>(),
                                                     d_a, d_d, d_g, d_f, win, wd.var_pmax,
                                                     wd.fhat.as<double>());
        }
        kitc_count_launch();
        k_transfer<false><<<m, WT, sm, s>>>(0, d_cheb, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                            t.first_child.as<int32_t>(), t.n_child.as<int32_t>(), d_a,
                                            d_d, d_g, d_f, win, wd.var_pmax, wd.fhat.as<double>());
        KITC_CUDA(cudaGetLastError());
    }
    return KITC_OK;
}

// Record offsets (bytes) of each cluster's grid records in the given form.
int64_t proxy_offsets_var(const std::vector<int32_t> &hdeg, int win, bool mixed, bool pairs,
                          bool rowpairs, std::vector<int64_t> &roff)
{
    roff.assign(hdeg.size(), 0);
    int64_t o = 0;
    for (size_t c = 0; c < hdeg.size(); ++c) {
        roff[c] = o;
        int d = hdeg[c];
        if (d <= 0) continue;
        int64_t np = d + 1;
        o += pairs ? pair_records((int)np, rowpairs) * 32 : np * np * np * proxy_record_bytes(win, mixed);
    }
    return o;
}

kitc_status pack_proxies_var(const TreeDev &t, WeightsDev &wd, const int32_t *d_deg,
                             const int64_t *d_roff, bool mixed, bool pairs, cudaStream_t s)
{
    Item *d_items = wd.items.as<Item>();
    const int64_t *d_f = reinterpret_cast<int64_t *>(d_items + wd.nitems) + t.nclus;
    kitc_count_launch();
    if (pairs)
        k_pack_proxies_var<0><<<t.nclus, 128, 0, s>>>(d_deg, wd.win, d_f, d_roff, wd.fhat.as<double>(),
                                                     wd.proxy.as<unsigned char>(), wd.rowpairs);
    else if (mixed)
        k_pack_proxies_var<1><<<t.nclus, 128, 0, s>>>(d_deg, wd.win, d_f, d_roff, wd.fhat.as<double>(),
                                                     wd.proxy.as<unsigned char>(), false);
    else
        k_pack_proxies_var<2><<<t.nclus, 128, 0, s>>>(d_deg, wd.win, d_f, d_roff, wd.fhat.as<double>(),
                                                     wd.proxy.as<unsigned char>(), false);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

const int64_t *weights_foff(const TreeDev &t, const WeightsDev &wd)
{
    if (!wd.planned || !wd.var) return nullptr;
    const Item *d_items = reinterpret_cast<const Item *>(wd.items.ptr);
    return reinterpret_cast<const int64_t *>(d_items + wd.nitems) + t.nclus;
}

// ---------------------------------------------------------------------------
// Weights pass for a tree known only on the device (the graph-capturable
// pipeline): the device plans above, the cluster count and the level starts
// read from the tree's state block, buffers sized once from the capacities.
// ---------------------------------------------------------------------------
int64_t weights_async_itemcap(int cap, int levels, int64_t n, int mode)
{
    const int64_t per = (n + CHUNK - 1) / CHUNK;
    return (int64_t)cap + (mode == KITC_WEIGHTS_UPWARD ? 1 : levels) * per + 1;
}

kitc_status weights_async_reserve(const TreeAsync &a, int win, int degree, int mode, bool split,
                                  bool mixed, bool pairs, bool rowpairs, bool leaf, cudaStream_t s,
                                  WeightsDev &wd)
{
    const TreeDev &t = a.t;
    const int cap = t.cap;
    wd.release(s);
    wd.planned = false;
    const int np = degree + 1, np3 = np * np * np;
    const int pwin = np3 * win;
    const bool upward = mode == KITC_WEIGHTS_UPWARD && upward_child_smem(np, win) <= UP_SMEM_MAX;
    const int64_t itemcap = weights_async_itemcap(cap, a.levels, t.n,
                                                  upward ? KITC_WEIGHTS_UPWARD : KITC_WEIGHTS_ALGORITHM1);
    if (itemcap > INT32_MAX / 2) return KITC_ERR_OOM;
    // items (itemcap) | first (cap + 1) | item count
    KITC_TRY(wd.items.reserve(sizeof(Item) * itemcap + sizeof(int32_t) * (cap + 2) + 64, s));
    const int64_t rows = std::max<int64_t>(itemcap, cap);  // item partials, then upward contributions
    KITC_TRY(wd.partial.reserve(sizeof(double) * pwin * rows, s));
    KITC_TRY(wd.fhat.reserve(sizeof(double) * pwin * cap, s));
    if (pairs) {
        const int64_t paircap = (t.n + cap) / 2 + 1;
        KITC_TRY(wd.proxy.reserve((size_t)32 * cap * pair_records(np, rowpairs), s));
        KITC_TRY(wd.src.reserve(pair_record_bytes(leaf) * paircap + 16, s));
        KITC_TRY(wd.pbegin.reserve(sizeof(int32_t) * 5 * (size_t)cap + 16, s));
        wd.paircap = paircap;
    } else {
        KITC_TRY(wd.proxy.reserve((size_t)proxy_record_bytes(win, mixed) * cap * np3, s));
        KITC_TRY(wd.src.reserve((size_t)source_record_bytes(win, mixed) * t.n, s));
        wd.paircap = 0;
    }
    wd.nitems = (size_t)itemcap;
    wd.upward = upward;
    if (upward) KITC_TRY(allow_up_smem());
    wd.split = split;
    wd.rowpairs = pairs && rowpairs;
    wd.leaf = pairs && leaf;
    wd.degree = degree;
    wd.win = win;
    wd.mode = mode;
    wd.var = false;
    wd.async = true;
    wd.planned = true;
    return KITC_OK;
}

kitc_status weights_async_launch(const TreeAsync &a, const double *w_user, WeightsDev &wd,
                                 bool mixed, bool pairs, int *err, cudaStream_t s)
{
    if (!wd.planned || !wd.async) return KITC_ERR_STATE;
    const TreeDev &t = a.t;
    const BuildState *bs = a.state();
    const int cap = t.cap, np = wd.degree + 1, win = wd.win;
    const int np3 = np * np * np, pwin = np3 * win;
    const int itemcap = (int)wd.nitems;
    Item *d_items = wd.items.as<Item>();
    int32_t *d_first = reinterpret_cast<int32_t *>(d_items + itemcap);
    int *d_nitems = d_first + cap + 1;
    const Cheb cb = make_cheb(wd.degree);
    kitc_count_launch();
    k_items_plan<<<1, 1024, 0, s>>>(bs, 0, cap, wd.upward, t.begin.as<int32_t>(), t.end.as<int32_t>(),
                                    t.n_child.as<int32_t>(), d_first, itemcap, d_nitems, err);
    kitc_count_launch();
    k_items_fill<<<(cap + 255) / 256, 256, 0, s>>>(bs, 0, cap, d_first, t.begin.as<int32_t>(),
                                                   t.end.as<int32_t>(), d_items);
    KITC_CUDA(cudaGetLastError());
    KITC_TRY(launch_items(wd.split, wd.degree, win, itemcap, d_items, t, w_user, wd.partial.as<double>(),
                          d_nitems, s));
    kitc_count_launch();
    k_weights_reduce<<<cap, 256, 0, s>>>(d_first, pwin, wd.partial.as<double>(), wd.fhat.as<double>());
    KITC_CUDA(cudaGetLastError());
    if (wd.upward) {
        const size_t us = upward_child_smem(np, win);
        const unsigned gch = (unsigned)std::min(cap, 4096);
        const unsigned gsum = (unsigned)std::min<int64_t>(((int64_t)cap * pwin + 255) / 256, 8192);
        for (int L = a.levels - 2; L >= 0; --L) {  // deepest parents first
            kitc_count_launch();
            k_upward_child_dev<<<gch, WT, us, s>>>(cb, bs, L, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                                   t.parent.as<int32_t>(), win, wd.fhat.as<double>(),
                                                   wd.partial.as<double>());
            kitc_count_launch();
            k_upward_sum_dev<<<gsum, 256, 0, s>>>(bs, L, pwin, t.first_child.as<int32_t>(),
                                                  t.n_child.as<int32_t>(), wd.partial.as<double>(),
                                                  wd.fhat.as<double>());
            KITC_CUDA(cudaGetLastError());
        }
    }
    const int *nclus_dev = &bs->nclus;
    if (pairs) {
        const int64_t nrec = (int64_t)cap * pair_records(np, wd.rowpairs);
        kitc_count_launch();
        k_pack_proxy_pairs<<<(unsigned)((nrec + 255) / 256), 256, 0, s>>>(
            cap, np, wd.rowpairs, wd.fhat.as<double>(), wd.proxy.as<float4>(), nclus_dev);
        int32_t *d = wd.pbegin.as<int32_t>();
        kitc_count_launch();
        k_pairs_plan<<<1, 1024, 0, s>>>(bs, 0, cap, t.begin.as<int32_t>(), t.end.as<int32_t>(),
                                        t.n_child.as<int32_t>(), d, wd.paircap, err);
        kitc_count_launch();
        (wd.leaf ? k_pack_pairs<true> : k_pack_pairs<false>)<<<(unsigned)cap, 256, 0, s>>>(d + cap, d + 2 * cap, d + 3 * cap, d + 4 * cap, t.n,
                                                   t.xs.as<double>(), t.perm.as<int32_t>(),
                                                   t.lo.as<dvec4>(), t.hi.as<dvec4>(), w_user,
                                                   wd.src.as<float>());
    } else {
        const int64_t nrec = (int64_t)cap * np3;
        const unsigned g = (unsigned)((nrec + 255) / 256);
        kitc_count_launch();
        if (mixed)
            k_pack_proxies<true><<<g, 256, 0, s>>>(nrec, win, wd.fhat.as<double>(), wd.proxy.ptr,
                                                   nclus_dev, np3);
        else
            k_pack_proxies<false><<<g, 256, 0, s>>>(nrec, win, wd.fhat.as<double>(), wd.proxy.ptr,
                                                    nclus_dev, np3);
        KITC_CUDA(cudaGetLastError());
        KITC_TRY(pack_sources(&t, nullptr, w_user, t.n, win, mixed, s, wd.src));
    }
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}
