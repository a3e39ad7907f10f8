// Interaction lists of target batches: the traversal of Algorithm 2.
//
// One warp walks the source tree for one batch of up to 64 targets (two per
// lane), depth first from the root, children in octant order.  Each stack
// entry carries the mask of the batch's targets still descending.  At a
// cluster C with mask M:
//   KITC_MAC_PARTICLE: A = {targets of M with r_C <= theta |x - y_C|} (Eq. MAC,
//     decided per target, so every target sees exactly Algorithm 2);
//   KITC_MAC_BATCH:    A = M if r_C <= theta dist(box_B, y_C), else empty.
//   KITC_MAC_ALL:      A = M if every target of M passes Eq. MAC, else empty.
// A non-empty A is a far entry (C, A); the rest R = M \ A becomes a near
// entry (C, R) if C is a leaf, else R descends into C's children.
// The MAC expressions round exactly as written (no contraction), so they
// agree bit for bit with any IEEE implementation of the same formulas.
// A first pass counts entries per batch, a scan sizes the arrays, a second
// pass writes them.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int LW = 8;                          // warps per block
constexpr int STK = 8 * KITC_MAX_LEVEL + 16;   // stack entries per warp

__device__ __forceinline__ double norm3_rn(double a, double b, double c)
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c)));
}

__device__ __forceinline__ double box_gap(double y, double lo, double hi)
{
    return y < lo ? __dsub_rn(lo, y) : (y > hi ? __dsub_rn(y, hi) : 0.0);
}

template <int PASS>
__global__ void __launch_bounds__(LW * 32) k_lists(
    int64_t nt, int batch, int64_t nb, const int32_t *__restrict__ bdesc, const double *__restrict__ txs,
    const dvec4 *__restrict__ ctr, const float4 *__restrict__ ctrf, const int32_t *__restrict__ cbegin,
    const int32_t *__restrict__ cend, const int32_t *__restrict__ first_child,
    const int32_t *__restrict__ n_child, double theta, int np3, const int32_t *__restrict__ cdeg, int mac,
    int64_t *__restrict__ counts, dvec4 *__restrict__ bctr, int64_t *__restrict__ totals,
    const int64_t *__restrict__ far_off, const int64_t *__restrict__ near_off,
    int32_t *__restrict__ far_id, uint64_t *__restrict__ far_mask, int32_t *__restrict__ near_id,
    uint64_t *__restrict__ near_mask, int *__restrict__ err, const int *__restrict__ skip)
{
    if (skip && *skip) return;  // lists over capacity: nothing is written
    __shared__ int32_t sid[LW][STK];
    __shared__ uint64_t smask[LW][STK];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t b = (int64_t)blockIdx.x * LW + w;
    if (b >= nb) return;
    // batch b: slots [s0, s1) of the target order; forests give each batch its
    // own slots and the root of its system's source tree
    int64_t s0 = bdesc ? (int64_t)bdesc[b] : b * batch;
    int64_t s1 = bdesc ? s0 + bdesc[nb + b] : min(nt, s0 + batch);
    const int root = bdesc ? bdesc[2 * nb + b] : 0;
    int64_t sa = s0 + lane, sb = s0 + 32 + lane;
    bool va = sa < s1, vb = sb < s1;
    double xa[3], xb[3], lo[3], hi[3];
    for (int l = 0; l < 3; ++l) {
        xa[l] = va ? txs[l * nt + sa] : txs[l * nt + s0];
        xb[l] = vb ? txs[l * nt + sb] : xa[l];
        lo[l] = fmin(xa[l], xb[l]);
        hi[l] = fmax(xa[l], xb[l]);
        for (int o = 16; o > 0; o >>= 1) {
            lo[l] = fmin(lo[l], __shfl_xor_sync(0xffffffffu, lo[l], o));
            hi[l] = fmax(hi[l], __shfl_xor_sync(0xffffffffu, hi[l], o));
        }
    }
    uint64_t m0 = (uint64_t)__ballot_sync(0xffffffffu, va) |
                  ((uint64_t)__ballot_sync(0xffffffffu, vb) << 32);
    double cb[3];
    for (int l = 0; l < 3; ++l) cb[l] = __dmul_rn(0.5, __dadd_rn(lo[l], hi[l]));
    if (PASS == 0 && lane == 0) bctr[b] = make_dvec4(cb[0], cb[1], cb[2], 0.0);
    // FP32 frame of the pre-test: offsets from the batch centre cb, which is
    // held as an FP32 hi/lo pair
    float cbh[3], cbl[3], xoa[3], xob[3], bl[3], bh[3];
    float sxa = 0.f, sxb = 0.f, sbx = 0.f;
    for (int l = 0; l < 3; ++l) {
        cbh[l] = __double2float_rn(cb[l]);
        cbl[l] = __double2float_rn(cb[l] - (double)cbh[l]);
        xoa[l] = __double2float_rn(xa[l] - cb[l]);
        xob[l] = __double2float_rn(xb[l] - cb[l]);
        bl[l] = __double2float_rn(lo[l] - cb[l]);
        bh[l] = __double2float_rn(hi[l] - cb[l]);
        sxa += fabsf(xoa[l]);
        sxb += fabsf(xob[l]);
        sbx += fmaxf(fabsf(bl[l]), fabsf(bh[l]));
    }
    const float thf = (float)theta;
    int64_t nfar = 0, nnear = 0, pairs = 0, points = 0, xpairs = 0, xpoints = 0;
    const int nvalid = __popcll(m0);
    int64_t fo = PASS ? far_off[b] : 0, no = PASS ? near_off[b] : 0;
    int sp = 0;
    if (lane == 0) {
        sid[w][0] = root;
        smask[w][0] = m0;
    }
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        --sp;
        int c = sid[w][sp];
        uint64_t M = smask[w][sp];
        __syncwarp();
        // MAC: an FP32 pre-test decides when the margin exceeds a bound on its
        // rounding error; otherwise the exact FP64 expression decides.  The
        // FP32 distance carries an absolute error <= 3u (|x - cb|_1 + |y_C - cb|_1)
        // (u = 2^-24) plus relative errors far below the 1e-5 margin.
        const float4 gh = ctrf[2 * c], gl = ctrf[2 * c + 1];
        float cc[3] = {(gh.x - cbh[0]) + (gl.x - cbl[0]), (gh.y - cbh[1]) + (gl.y - cbl[1]),
                       (gh.z - cbh[2]) + (gl.z - cbl[2])};
        const float scc = fabsf(cc[0]) + fabsf(cc[1]) + fabsf(cc[2]);
        const float rf = gh.w;
        auto pretest = [&](float dist, float err) -> int {  // 1 accept, 0 reject, 2 undecided
            if (rf < thf * (dist - err) * (1.f - 1e-5f)) return 1;
            if (rf > thf * (dist + err) * (1.f + 1e-5f)) return 0;
            return 2;
        };
        uint64_t A;
        if (mac != KITC_MAC_BATCH) {
            float da0 = xoa[0] - cc[0], da1 = xoa[1] - cc[1], da2 = xoa[2] - cc[2];
            float db0 = xob[0] - cc[0], db1 = xob[1] - cc[1], db2 = xob[2] - cc[2];
            int pa = pretest(sqrtf(fmaf(da0, da0, fmaf(da1, da1, da2 * da2))), 2e-7f * (sxa + scc));
            int pb = pretest(sqrtf(fmaf(db0, db0, fmaf(db1, db1, db2 * db2))), 2e-7f * (sxb + scc));
            if (pa == 2 || pb == 2) {
                const dvec4 g = ctr[c];  // centre, radius in w
                if (pa == 2) {
                    double Ra = norm3_rn(__dsub_rn(xa[0], g.x), __dsub_rn(xa[1], g.y), __dsub_rn(xa[2], g.z));
                    pa = g.w <= __dmul_rn(theta, Ra);
                }
                if (pb == 2) {
                    double Rb = norm3_rn(__dsub_rn(xb[0], g.x), __dsub_rn(xb[1], g.y), __dsub_rn(xb[2], g.z));
                    pb = g.w <= __dmul_rn(theta, Rb);
                }
            }
            A = ((uint64_t)__ballot_sync(0xffffffffu, pa == 1) |
                 ((uint64_t)__ballot_sync(0xffffffffu, pb == 1) << 32)) & M;
            if (mac == KITC_MAC_ALL && A != M) A = 0;  // one decision for the batch
        } else {
            float gap[3];
            for (int l = 0; l < 3; ++l)
                gap[l] = cc[l] < bl[l] ? bl[l] - cc[l] : (cc[l] > bh[l] ? cc[l] - bh[l] : 0.f);
            int p = pretest(sqrtf(fmaf(gap[0], gap[0], fmaf(gap[1], gap[1], gap[2] * gap[2]))),
                            2e-7f * (scc + sbx));
            if (p == 2) {
                const dvec4 g = ctr[c];
                double d = norm3_rn(box_gap(g.x, lo[0], hi[0]), box_gap(g.y, lo[1], hi[1]),
                                    box_gap(g.z, lo[2], hi[2]));
                p = g.w <= __dmul_rn(theta, d);
            }
            A = p == 1 ? M : 0;
        }
        uint64_t R = M & ~A;
        if (A) {
            if (PASS == 1 && lane == 0) {
                far_id[fo + nfar] = c;
                far_mask[fo + nfar] = A;
            }
            nfar++;
            int64_t g3 = np3;
            if (cdeg) {  // degree of cluster c; an accepted cluster must have weights
                int gn = cdeg[c] + 1;
                if (gn < 2 && lane == 0) atomicExch(err, 2);
                g3 = (int64_t)gn * gn * gn;
            }
            points += (int64_t)__popcll(A) * g3;
            xpoints += (int64_t)nvalid * g3;
        }
        if (R) {
            int nch = n_child[c];
            if (nch == 0) {
                if (PASS == 1 && lane == 0) {
                    near_id[no + nnear] = c;
                    near_mask[no + nnear] = R;
                }
                nnear++;
                pairs += (int64_t)__popcll(R) * (cend[c] - cbegin[c]);
                xpairs += (int64_t)nvalid * (cend[c] - cbegin[c]);
            } else {
                if (sp + nch > STK) {
                    if (lane == 0) atomicExch(err, 1);
                    break;
                }
                int fc = first_child[c];
                if (lane < nch) {  // pushed in reverse so that they pop in octant order
                    sid[w][sp + nch - 1 - lane] = fc + lane;
                    smask[w][sp + nch - 1 - lane] = R;
                }
                sp += nch;
                __syncwarp();
            }
        }
    }
    if (PASS == 0 && lane == 0) {
        counts[b] = nfar;
        counts[nb + b] = nnear;
        atomicAdd(reinterpret_cast<unsigned long long *>(&totals[0]), (unsigned long long)pairs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&totals[1]), (unsigned long long)points);
        atomicAdd(reinterpret_cast<unsigned long long *>(&totals[4]), (unsigned long long)xpairs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&totals[5]), (unsigned long long)xpoints);
    }
}

// Exclusive scan of in[0..m) into out[0..m] (out[m] = total); one block.
__global__ void k_scan64(const int64_t *__restrict__ in, int64_t m, int64_t *__restrict__ out,
                         int64_t *__restrict__ total)
{
    __shared__ int64_t sums[1024];
    int64_t per = (m + blockDim.x - 1) / blockDim.x;
    int64_t b = threadIdx.x * per, e = min(m, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    sums[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            int64_t v = sums[i];
            sums[i] = run;
            run += v;
        }
        out[m] = run;
        *total = run;
    }
    __syncthreads();
    int64_t run = sums[threadIdx.x];
    for (int64_t i = b; i < e; ++i) {
        out[i] = run;
        run += in[i];
    }
}

// Far-field grid points of existing lists under a degree map: warp per batch;
// totals[0] += points the batches' targets use, totals[1] += points evaluated,
// *err = 2 when an accepted cluster has degree 0.
__global__ void k_far_recount(int64_t nt, int batch, int64_t nb, const int32_t *__restrict__ bdesc,
                              const int64_t *__restrict__ far_off, const int32_t *__restrict__ far_id,
                              const uint64_t *__restrict__ far_mask, const int32_t *__restrict__ cdeg,
                              unsigned long long *__restrict__ totals, int *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= nb) return;
    const int64_t s0 = bdesc ? (int64_t)bdesc[b] : b * batch;
    const int64_t s1 = bdesc ? s0 + bdesc[nb + b] : min(nt, s0 + batch);
    const unsigned long long nvalid = (unsigned long long)(s1 - s0);
    unsigned long long pts = 0, xpts = 0;
    for (int64_t e = far_off[b] + lane; e < far_off[b + 1]; e += 32) {
        const int g = cdeg[far_id[e]] + 1;
        if (g < 2) atomicExch(err, 2);
        const unsigned long long g3 = (unsigned long long)g * g * g;
        pts += (unsigned long long)__popcll(far_mask[e]) * g3;
        xpts += nvalid * g3;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pts += __shfl_xor_sync(0xffffffffu, pts, o);
        xpts += __shfl_xor_sync(0xffffffffu, xpts, o);
    }
    if (lane == 0 && pts) {
        atomicAdd(totals, pts);
        atomicAdd(totals + 1, xpts);
    }
}

// After the scans of a capacity-sized build: if the lists exceed the room
// reserved for them, the writing pass is skipped (*skip) and every batch's
// offsets are zeroed, so that the evaluator finds empty lists; the error word
// records the overflow and a traversal stack overflow of the counting pass.
__global__ void k_lists_guard(int64_t nb, const int64_t *__restrict__ tot, int64_t cap_far,
                              int64_t cap_near, int64_t *__restrict__ far_off,
                              int64_t *__restrict__ near_off, int *__restrict__ skip,
                              int *__restrict__ err)
{
    const bool over = tot[2] > cap_far || tot[3] > cap_near;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *skip = over ? 1 : 0;
        if (over) atomicOr(err, ASYNC_LIST_OVERFLOW);
        if (reinterpret_cast<const int *>(tot + 6)[0] != 0) atomicOr(err, ASYNC_TRAVERSAL);
    }
    if (over && i <= nb) far_off[i] = near_off[i] = 0;
}

}  // namespace

kitc_status lists_recount(const int32_t *cdeg, cudaStream_t s, ListsDev &L)
{
    int64_t *tot = L.totals.as<int64_t>();
    KITC_CUDA(cudaMemsetAsync(tot + 6, 0, sizeof(int64_t) * 2, s));
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(tot + 6);
    int *err = reinterpret_cast<int *>(L.counts.as<int64_t>());  // the pass-0 counts are spent
    KITC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    if (L.nb > 0) {
        kitc_count_launch();
        k_far_recount<<<(unsigned)((L.nb + LW - 1) / LW), LW * 32, 0, s>>>(
            L.nt, L.batch, L.nb, L.forest ? L.bdesc.as<int32_t>() : nullptr, L.far_off.as<int64_t>(),
            L.far_id.as<int32_t>(), L.far_mask.as<uint64_t>(), cdeg, acc, err);
        KITC_CUDA(cudaGetLastError());
    }
    int64_t *h = nullptr;
    KITC_TRY(host_readback_buffer(reinterpret_cast<void **>(&h)));
    KITC_CUDA(cudaMemcpyAsync(h, tot + 6, sizeof(int64_t) * 2, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(h + 2, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    if (reinterpret_cast<int *>(h + 2)[0] != 0) return KITC_ERR_INVALID_ARG;
    L.far_points = h[0];
    L.far_exec = h[1];
    return KITC_OK;
}

void ListsDev::release(cudaStream_t s)
{
    for (DevBuf *b : {&bctr, &bdesc, &far_off, &near_off, &far_id, &near_id, &far_mask, &near_mask,
                      &counts, &totals})
        b->release(s);
    nb = nt = nfar = nnear = 0;
    async = false;
    cap_far = cap_near = 0;
}

size_t ListsDev::bytes() const
{
    size_t b = 0;
    for (const DevBuf *d : {&bctr, &bdesc, &far_off, &near_off, &far_id, &near_id, &far_mask,
                            &near_mask, &counts, &totals})
        b += d->bytes;
    return b;
}

// Per-system batches of a forest's target order: batch b covers slots
// [st[b], st[b] + sz[b]) of system rt[b]; never two systems in one batch.
static void forest_batches(const std::vector<int64_t> &off, int nsys, int batch, std::vector<int32_t> &all)
{
    std::vector<int32_t> st, sz, rt;
    for (int k = 0; k < nsys; ++k)
        for (int64_t p = off[k]; p < off[k + 1]; p += batch) {
            st.push_back((int32_t)p);
            sz.push_back((int32_t)std::min<int64_t>(batch, off[k + 1] - p));
            rt.push_back(k);
        }
    all = st;
    all.insert(all.end(), sz.begin(), sz.end());
    all.insert(all.end(), rt.begin(), rt.end());
}

kitc_status lists_build(const TreeDev &src, const TreeDev &tgt, int batch, double theta,
                        int degree, const int32_t *cdeg, int mac, cudaStream_t s, ListsDev &L)
{
    int64_t nt = tgt.n;
    int64_t nb = (nt + batch - 1) / batch;
    const int32_t *bdesc = nullptr;
    if (tgt.nsys > 1) {  // per-system batches: target system k meets source system k
        if (src.nsys != tgt.nsys) return KITC_ERR_INVALID_ARG;
        std::vector<int32_t> all;
        forest_batches(tgt.sys_off, tgt.nsys, batch, all);
        nb = (int64_t)all.size() / 3;
        KITC_TRY(L.bdesc.reserve(sizeof(int32_t) * 3 * nb, s));
        KITC_CUDA(cudaMemcpyAsync(L.bdesc.ptr, all.data(), sizeof(int32_t) * all.size(),
                                  cudaMemcpyHostToDevice, s));
        KITC_CUDA(cudaStreamSynchronize(s));  // the host vector must outlive the copy
        bdesc = L.bdesc.as<int32_t>();
    }
    L.forest = bdesc != nullptr;
    L.nt = nt;
    L.nb = nb;
    L.batch = batch;
    int np = degree + 1, np3 = np * np * np;
    KITC_TRY(L.bctr.reserve(sizeof(dvec4) * nb, s));
    KITC_TRY(L.counts.reserve(sizeof(int64_t) * 2 * nb, s));
    KITC_TRY(L.far_off.reserve(sizeof(int64_t) * (nb + 1), s));
    KITC_TRY(L.near_off.reserve(sizeof(int64_t) * (nb + 1), s));
    KITC_TRY(L.totals.reserve(sizeof(int64_t) * 8, s));
    int64_t *tot = L.totals.as<int64_t>();
    KITC_CUDA(cudaMemsetAsync(tot, 0, sizeof(int64_t) * 8, s));
    int *err = reinterpret_cast<int *>(tot + 6);
    unsigned grid = (unsigned)((nb + LW - 1) / LW);
    kitc_count_launch();
    k_lists<0><<<grid, LW * 32, 0, s>>>(nt, batch, nb, bdesc, tgt.xs.as<double>(), src.ctr.as<dvec4>(),
                                        src.ctrf.as<float4>(), src.begin.as<int32_t>(), src.end.as<int32_t>(),
                                        src.first_child.as<int32_t>(), src.n_child.as<int32_t>(),
                                        theta, np3, cdeg, mac, L.counts.as<int64_t>(),
                                        L.bctr.as<dvec4>(), tot, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, nullptr, err, nullptr);
    KITC_CUDA(cudaGetLastError());
    kitc_count_launch();
    k_scan64<<<1, 1024, 0, s>>>(L.counts.as<int64_t>(), nb, L.far_off.as<int64_t>(), tot + 2);
    kitc_count_launch();
    k_scan64<<<1, 1024, 0, s>>>(L.counts.as<int64_t>() + nb, nb, L.near_off.as<int64_t>(), tot + 3);
    KITC_CUDA(cudaGetLastError());
    int64_t *h = nullptr;
    KITC_TRY(host_readback_buffer(reinterpret_cast<void **>(&h)));
    KITC_CUDA(cudaMemcpyAsync(h, tot, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    if (reinterpret_cast<int *>(h + 6)[0] != 0) return KITC_ERR_INVALID_ARG;
    L.near_pairs = h[0];
    L.far_points = h[1];
    L.nfar = h[2];
    L.nnear = h[3];
    L.near_exec = h[4];
    L.far_exec = h[5];
    KITC_TRY(L.far_id.reserve(sizeof(int32_t) * (L.nfar + 1), s));
    KITC_TRY(L.far_mask.reserve(sizeof(uint64_t) * (L.nfar + 1), s));
    KITC_TRY(L.near_id.reserve(sizeof(int32_t) * (L.nnear + 1), s));
    KITC_TRY(L.near_mask.reserve(sizeof(uint64_t) * (L.nnear + 1), s));
    kitc_count_launch();
    k_lists<1><<<grid, LW * 32, 0, s>>>(nt, batch, nb, bdesc, tgt.xs.as<double>(), src.ctr.as<dvec4>(),
                                        src.ctrf.as<float4>(), src.begin.as<int32_t>(), src.end.as<int32_t>(),
                                        src.first_child.as<int32_t>(), src.n_child.as<int32_t>(),
                                        theta, np3, cdeg, mac, nullptr, nullptr, nullptr,
                                        L.far_off.as<int64_t>(), L.near_off.as<int64_t>(),
                                        L.far_id.as<int32_t>(), L.far_mask.as<uint64_t>(),
                                        L.near_id.as<int32_t>(), L.near_mask.as<uint64_t>(), err,
                                        nullptr);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status lists_async_reserve(const TreeAsync &src, const TreeAsync &tgt, int batch, int64_t cap_far,
                                int64_t cap_near, cudaStream_t s, ListsDev &L)
{
    L.release(s);
    const TreeDev &tt = tgt.t;
    int64_t nt = tt.n;
    int64_t nb = (nt + batch - 1) / batch;
    L.forest = tt.nsys > 1;
    if (L.forest) {
        if (src.t.nsys != tt.nsys) return KITC_ERR_INVALID_ARG;
        std::vector<int32_t> all;
        forest_batches(tt.sys_off, tt.nsys, batch, all);
        nb = (int64_t)all.size() / 3;
        KITC_TRY(L.bdesc.reserve(sizeof(int32_t) * all.size(), s));
        KITC_CUDA(cudaMemcpyAsync(L.bdesc.ptr, all.data(), sizeof(int32_t) * all.size(),
                                  cudaMemcpyHostToDevice, s));
        KITC_CUDA(cudaStreamSynchronize(s));  // the host vector must outlive the copy
    }
    L.nt = nt;
    L.nb = nb;
    L.batch = batch;
    KITC_TRY(L.bctr.reserve(sizeof(dvec4) * nb, s));
    KITC_TRY(L.counts.reserve(sizeof(int64_t) * 2 * nb, s));
    KITC_TRY(L.far_off.reserve(sizeof(int64_t) * (nb + 1), s));
    KITC_TRY(L.near_off.reserve(sizeof(int64_t) * (nb + 1), s));
    KITC_TRY(L.totals.reserve(sizeof(int64_t) * 10, s));  // 8 totals | skip flag
    KITC_TRY(L.far_id.reserve(sizeof(int32_t) * (cap_far + 1), s));
    KITC_TRY(L.far_mask.reserve(sizeof(uint64_t) * (cap_far + 1), s));
    KITC_TRY(L.near_id.reserve(sizeof(int32_t) * (cap_near + 1), s));
    KITC_TRY(L.near_mask.reserve(sizeof(uint64_t) * (cap_near + 1), s));
    L.cap_far = cap_far;
    L.cap_near = cap_near;
    L.nfar = L.nnear = -1;  // known on the device only
    L.async = true;
    return KITC_OK;
}

kitc_status lists_async_launch(const TreeAsync &srcA, const TreeAsync &tgtA, double theta, int degree,
                               int mac, int *perr, cudaStream_t s, ListsDev &L)
{
    if (!L.async) return KITC_ERR_STATE;
    const TreeDev &src = srcA.t, &tgt = tgtA.t;
    const int64_t nt = L.nt, nb = L.nb;
    const int batch = L.batch;
    const int32_t *bdesc = L.forest ? L.bdesc.as<int32_t>() : nullptr;
    const int np = degree + 1, np3 = np * np * np;
    int64_t *tot = L.totals.as<int64_t>();
    int *err = reinterpret_cast<int *>(tot + 6);
    int *skip = reinterpret_cast<int *>(tot + 8);
    KITC_CUDA(cudaMemsetAsync(tot, 0, sizeof(int64_t) * 8, s));
    const unsigned grid = (unsigned)((nb + LW - 1) / LW);
    kitc_count_launch();
    k_lists<0><<<grid, LW * 32, 0, s>>>(nt, batch, nb, bdesc, tgt.xs.as<double>(), src.ctr.as<dvec4>(),
                                        src.ctrf.as<float4>(), src.begin.as<int32_t>(), src.end.as<int32_t>(),
                                        src.first_child.as<int32_t>(), src.n_child.as<int32_t>(),
                                        theta, np3, nullptr, mac, L.counts.as<int64_t>(),
                                        L.bctr.as<dvec4>(), tot, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, nullptr, err, nullptr);
    KITC_CUDA(cudaGetLastError());
    kitc_count_launch();
    k_scan64<<<1, 1024, 0, s>>>(L.counts.as<int64_t>(), nb, L.far_off.as<int64_t>(), tot + 2);
    kitc_count_launch();
    k_scan64<<<1, 1024, 0, s>>>(L.counts.as<int64_t>() + nb, nb, L.near_off.as<int64_t>(), tot + 3);
    kitc_count_launch();
    k_lists_guard<<<(unsigned)((nb + 1 + 255) / 256), 256, 0, s>>>(
        nb, tot, L.cap_far, L.cap_near, L.far_off.as<int64_t>(), L.near_off.as<int64_t>(), skip, perr);
    kitc_count_launch();
    k_lists<1><<<grid, LW * 32, 0, s>>>(nt, batch, nb, bdesc, tgt.xs.as<double>(), src.ctr.as<dvec4>(),
                                        src.ctrf.as<float4>(), src.begin.as<int32_t>(), src.end.as<int32_t>(),
                                        src.first_child.as<int32_t>(), src.n_child.as<int32_t>(),
                                        theta, np3, nullptr, mac, nullptr, nullptr, nullptr,
                                        L.far_off.as<int64_t>(), L.near_off.as<int64_t>(),
                                        L.far_id.as<int32_t>(), L.far_mask.as<uint64_t>(),
                                        L.near_id.as<int32_t>(), L.near_mask.as<uint64_t>(), err, skip);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}
