// Sec. 6 tree of particle clusters, built level by level on the GPU.
//
// The root is the smallest box enclosing the particles.  A cluster holding
// more than N0 particles is bisected at the midpoint of every side longer than
// l_max / sqrt(2) (l_max = its longest side), into 8, 4 or 2 boxes; the
// non-empty ones become its children, ordered by octant code (bit 0 = upper x,
// bit 1 = upper y, bit 2 = upper z; a particle on the midpoint goes up).  Each
// split is a stable partition of the cluster's slot range, so the final order
// is unique and integer-exact.  Every floating-point decision (side, l_max /
// sqrt(2), midpoint, x >= mid) uses round-to-nearest operations with no
// contraction, so any IEEE implementation of the same expressions takes the
// same decisions.
//
// The level loop runs on the device: each level's kernels read the level's
// cluster range from a small state block that the previous level wrote, so the
// host queues several levels without waiting and reads the state back once
// (once per round of levels; one round covers the trees of the usual inputs).
// Cluster arrays are sized from a host bound; a tree that would exceed it sets
// an overflow flag, and the build is repeated with a larger bound.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace {

constexpr int BT = 1024;      // threads of the per-slot kernels
constexpr int RPB = 4;        // rounds of BT consecutive slots per block
constexpr int SPB = BT * RPB; // slots per block

struct SplitInfo {
    double mid[3];
    int mask;   // bit l set: axis l is bisected; 0: the cluster is a leaf
    int pad;
};

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

// Finite doubles as 64-bit integers of the same order (negative values have
// their magnitude bits flipped; -0 becomes +0), so that the root box's minima
// and maxima run on the integer ALU instead of the FP64 pipe.
__device__ __forceinline__ long long order_key(double v)
{
    long long k = __double_as_longlong(v);
    if (k == (long long)0x8000000000000000ull) return 0;
    return k < 0 ? k ^ 0x7fffffffffffffffll : k;
}
__device__ __forceinline__ double key_value(long long k)
{
    return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffll : k);
}

// Gathers the caller's n x 3 coordinates into SoA and sets the identity order.
__global__ void k_init(const double *__restrict__ xyz, int64_t n, double *__restrict__ xs,
                       int32_t *__restrict__ perm)
{
    int64_t base = (int64_t)blockIdx.x * SPB;
    for (int r = 0; r < RPB; ++r) {
        int64_t i = base + r * BT + threadIdx.x;
        if (i < n) {
            for (int l = 0; l < 3; ++l) xs[l * n + i] = xyz[3 * i + l];
            perm[i] = (int32_t)i;
        }
    }
}

// Bounding box of one chunk of one system's slots (chunk c covers
// [cb[c], ce[c]) of system cs[c]); also marks those slots as belonging to the
// system's root.
__global__ void __launch_bounds__(BT, 2) k_root_partial(const int32_t *__restrict__ cs,
                                                     const int64_t *__restrict__ cb,
                                                     const int64_t *__restrict__ ce, int64_t n,
                                                     const double *__restrict__ xs,
                                                     int32_t *__restrict__ node,
                                                     double *__restrict__ part)
{
    __shared__ long long red[6][BT / 32];
    const int c = blockIdx.x, sys = cs[c];
    long long l[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, h[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int64_t i = cb[c] + threadIdx.x; i < ce[c]; i += BT) {
        node[i] = sys;
        for (int a = 0; a < 3; ++a) {
            const long long v = order_key(xs[a * n + i]);
            l[a] = min(l[a], v);
            h[a] = max(h[a], v);
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            l[a] = min(l[a], __shfl_xor_sync(0xffffffffu, l[a], o));
            h[a] = max(h[a], __shfl_xor_sync(0xffffffffu, h[a], o));
        }
        if (lane == 0) {
            red[a][w] = l[a];
            red[3 + a][w] = h[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int q = threadIdx.x;
        long long v = red[q][0];
        for (int k = 1; k < BT / 32; ++k) v = q < 3 ? min(v, red[q][k]) : max(v, red[q][k]);
        part[6 * c + q] = key_value(v);
    }
}

// Root cluster of every system: the smallest box enclosing its particles,
// from the partial boxes of its chunks [c0[s], c0[s+1]).
__global__ void k_root_final(int nsys, const int32_t *__restrict__ c0, const int64_t *__restrict__ off,
                             const double *__restrict__ part, dvec4 *lo, dvec4 *hi, int32_t *begin,
                             int32_t *end, int32_t *first_child, int32_t *n_child, int32_t *level,
                             int32_t *parent)
{
    int sys = blockIdx.x * blockDim.x + threadIdx.x;
    if (sys >= nsys) return;
    double v[6];
    for (int q = 0; q < 6; ++q) v[q] = part[6 * c0[sys] + q];
    for (int c = c0[sys] + 1; c < c0[sys + 1]; ++c)
        for (int q = 0; q < 6; ++q) v[q] = q < 3 ? dmin(v[q], part[6 * c + q]) : dmax(v[q], part[6 * c + q]);
    lo[sys] = make_dvec4(v[0], v[1], v[2], 0.0);
    hi[sys] = make_dvec4(v[3], v[4], v[5], 0.0);
    begin[sys] = (int32_t)off[sys];
    end[sys] = (int32_t)off[sys + 1];
    first_child[sys] = -1;
    n_child[sys] = 0;
    level[sys] = 0;
    parent[sys] = -1;
}

// Split decision of each cluster of level lvl; clears the level's counts.
__global__ void k_split(BuildState *bs, int lvl, int leaf, const dvec4 *__restrict__ lo,
                        const dvec4 *__restrict__ hi, const int32_t *__restrict__ begin,
                        const int32_t *__restrict__ end, const int32_t *__restrict__ level,
                        SplitInfo *__restrict__ info, int32_t *__restrict__ ccount)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && bs->flip) {  // the previous level scattered
        bs->cur ^= 1;
        bs->flip = 0;
    }
    const LevelState L = bs->st[lvl & 1];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.nl) return;
    int c = L.lb + i;
    for (int k = 0; k < 8; ++k) ccount[i * 8 + k] = 0;
    SplitInfo s;
    s.mask = 0;
    s.pad = 0;
    double l[3] = {lo[c].x, lo[c].y, lo[c].z}, h[3] = {hi[c].x, hi[c].y, hi[c].z};
    double side[3], lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        side[a] = __dsub_rn(h[a], l[a]);
        if (side[a] > lmax) lmax = side[a];
        s.mid[a] = __dmul_rn(0.5, __dadd_rn(l[a], h[a]));
    }
    if (end[c] - begin[c] > leaf && level[c] < KITC_MAX_LEVEL && lmax > 0.0) {
        const double sqrt2 = 1.4142135623730951;  // correctly rounded sqrt(2)
        double thr = __ddiv_rn(lmax, sqrt2);
        for (int a = 0; a < 3; ++a)
            if (side[a] > thr) s.mask |= 1 << a;
    }
    info[i] = s;
}

__device__ __forceinline__ int slot_key(int64_t p, int64_t n, int lb, int nl,
                                        const double *__restrict__ xs,
                                        const int32_t *__restrict__ node,
                                        const SplitInfo *__restrict__ info, int *cl)
{
    int c = node[p] - lb;
    *cl = c;
    if (c < 0 || c >= nl) return 8;
    int m = info[c].mask;
    if (m == 0) return 8;
    int k = 0;
    for (int a = 0; a < 3; ++a)
        if (((m >> a) & 1) && xs[a * n + p] >= info[c].mid[a]) k |= 1 << a;
    return k;
}

// Per (cluster, code) counts and per (code, block) counts of the level.
__global__ void k_count(int64_t n, const BuildState *__restrict__ bs, int lvl,
                        const double *__restrict__ xsA, const double *__restrict__ xsB,
                        const int32_t *__restrict__ nodeA, const int32_t *__restrict__ nodeB,
                        const SplitInfo *__restrict__ info, int32_t *__restrict__ ccount,
                        int32_t *__restrict__ bcount, int nblk)
{
    const LevelState L = bs->st[lvl & 1];
    if (L.nl == 0) return;
    const int lb = L.lb, nl = L.nl;
    const bool cur = bs->cur != 0;
    const double *__restrict__ xs = cur ? xsB : xsA;
    const int32_t *__restrict__ node = cur ? nodeB : nodeA;
    __shared__ int sb[8];
    __shared__ int sc[8];
    __shared__ int c0s;
    if (threadIdx.x < 8) {
        sb[threadIdx.x] = 0;
        sc[threadIdx.x] = 0;
    }
    int64_t base = (int64_t)blockIdx.x * SPB;
    if (threadIdx.x == 0) c0s = (base < n) ? node[base] - lb : -1;
    __syncthreads();
    int c0 = c0s;
    for (int r = 0; r < RPB; ++r) {
        int64_t p = base + r * BT + threadIdx.x;
        int c = -1, k = 8;
        if (p < n) k = slot_key(p, n, lb, nl, xs, node, info, &c);
        unsigned key = 0xffffffffu;  // slots counted through global atomics
        if (k < 8) {
            atomicAdd(&sb[k], 1);
            if (c == c0) atomicAdd(&sc[k], 1);
            else key = (unsigned)c * 8u + (unsigned)k;
        }
        unsigned grp = __match_any_sync(0xffffffffu, key);
        if (key != 0xffffffffu && (threadIdx.x & 31) == __ffs(grp) - 1)
            atomicAdd(&ccount[key], __popc(grp));
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        bcount[threadIdx.x * nblk + blockIdx.x] = sb[threadIdx.x];
        if (c0 >= 0 && c0 < nl && sc[threadIdx.x] > 0)
            atomicAdd(&ccount[c0 * 8 + threadIdx.x], sc[threadIdx.x]);
    }
}

// In-place exclusive scan of a[0], a[stride], ... a[(m-1)*stride] by one block
// (each thread scans a contiguous segment; the segment sums are scanned with
// warp shuffles).
__device__ void block_scan_strided(int32_t *a, int m, int stride, int *tot_out)
{
    __shared__ int32_t wsum[BT / 32];
    int per = (m + blockDim.x - 1) / blockDim.x;
    int b = threadIdx.x * per, e = min(m, b + per);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += a[(int64_t)i * stride];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t v = lane < (int)(blockDim.x / 32) ? wsum[lane] : 0, x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane < (int)(blockDim.x / 32)) wsum[lane] = x - v;
        if (lane == 31 && tot_out) *tot_out = x;
    }
    __syncthreads();
    int32_t run = wsum[w] + incl - s;
    for (int i = b; i < e; ++i) {
        int32_t v = a[(int64_t)i * stride];
        a[(int64_t)i * stride] = run;
        run += v;
    }
    __syncthreads();
}

// Children of the level's clusters, in three kernels (a level can hold
// hundreds of thousands of clusters): a block-local pass over the clusters, one
// block that scans the block totals and advances the level state, and a wide
// pass that applies the block offsets and creates the children.
constexpr int CB = 256;  // clusters per block of the children kernels
constexpr int NT = 10;   // block totals: 8 code counts, children, splitting clusters

// Per cluster i of the level: the offset of each of its 8 codes inside it
// (childoff), and block-local exclusive prefixes over the clusters of the code
// counts (cprefix) and of the children counts (nchs); block totals to btot.
__global__ void __launch_bounds__(CB) k_children_local(
    const BuildState *__restrict__ bs, int lvl, const SplitInfo *__restrict__ info,
    const int32_t *__restrict__ ccount, int32_t *__restrict__ cprefix, int32_t *__restrict__ childoff,
    int32_t *__restrict__ nchs, int32_t *__restrict__ btot)
{
    const int nl = bs->st[lvl & 1].nl;
    if ((int64_t)blockIdx.x * CB >= nl) return;
    const int i = blockIdx.x * CB + threadIdx.x;
    int v[NT];
    if (i < nl) {
        const bool split = info[i].mask != 0;
        int off = 0, nch = 0;
        for (int k = 0; k < 8; ++k) {
            const int c = ccount[i * 8 + k];
            childoff[i * 8 + k] = off;
            off += c;
            v[k] = c;
            if (split && c > 0) nch++;
        }
        v[8] = nch;
        v[9] = nch > 0;
    } else {
        for (int k = 0; k < NT; ++k) v[k] = 0;
    }
    __shared__ int ws[CB / 32][NT];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl[NT];
    for (int k = 0; k < NT; ++k) {
        int x = v[k];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[k] = x;
        if (lane == 31) ws[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NT) {
        int run = 0;
        for (int q = 0; q < CB / 32; ++q) {
            const int t = ws[q][threadIdx.x];
            ws[q][threadIdx.x] = run;
            run += t;
        }
        btot[(int64_t)blockIdx.x * NT + threadIdx.x] = run;
    }
    __syncthreads();
    if (i < nl) {
        for (int k = 0; k < 8; ++k) cprefix[i * 8 + k] = ws[w][k] + incl[k] - v[k];
        nchs[i] = ws[w][8] + incl[8] - v[8];
    }
}

// Single block: exclusive scans of the per-block code counts of the slots
// (bcount) and of the cluster-block totals; then the capacity check and the
// next level's state (the new level holds the children, at most cap clusters
// in all).
__global__ void __launch_bounds__(BT) k_children_scan(BuildState *bs, int lvl, int cap,
                                                      int32_t *bcount, int nblk, int32_t *btot)
{
    const LevelState L = bs->st[lvl & 1];
    const int lb = L.lb, nl = L.nl, nclus = bs->nclus;
    if (nl == 0) {
        if (threadIdx.x == 0) bs->st[(lvl + 1) & 1] = LevelState{lb, 0};
        return;
    }
    for (int k = 0; k < 8; ++k) block_scan_strided(bcount + k * nblk, nblk, 1, nullptr);
    __shared__ int tot[NT];
    const int nb = (nl + CB - 1) / CB;
    for (int k = 0; k < NT; ++k) block_scan_strided(btot + k, nb, NT, &tot[k]);
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int total = tot[8], nsplit = tot[9];
    if ((int64_t)nclus + total > (int64_t)cap) {  // no room: stop the build, the host retries
        bs->overflow = 1;
        bs->st[(lvl + 1) & 1] = LevelState{nclus, 0};
        return;
    }
    bs->st[(lvl + 1) & 1] = LevelState{nclus, total};
    bs->nclus = nclus + total;
    bs->nleaves += nl - nsplit;
    bs->depth += 1;
    if (total > 0) bs->level_start[bs->depth] = nclus;
    bs->flip = total > 0;  // this level's scatter runs, then the next level flips cur
}

// Block offsets applied to the prefixes; children created: boxes (geometric
// halves of the parent), slot ranges, links.
__global__ void __launch_bounds__(CB) k_children_make(
    const BuildState *__restrict__ bs, int lvl, const SplitInfo *__restrict__ info,
    const int32_t *__restrict__ ccount, int32_t *__restrict__ cprefix,
    const int32_t *__restrict__ childoff, int32_t *__restrict__ childidx,
    const int32_t *__restrict__ nchs, const int32_t *__restrict__ btot, dvec4 *lo, dvec4 *hi,
    int32_t *begin, int32_t *end, int32_t *first_child, int32_t *n_child, int32_t *level,
    int32_t *parent)
{
    const LevelState L = bs->st[lvl & 1];
    const int lb = L.lb, nl = L.nl;
    if (nl == 0 || bs->overflow) return;
    const int i = blockIdx.x * CB + threadIdx.x;
    if (i >= nl) return;
    const int32_t *bt = btot + (int64_t)blockIdx.x * NT;  // exclusive over the blocks
    for (int k = 0; k < 8; ++k) cprefix[i * 8 + k] += bt[k];
    const int c = lb + i;
    const int m = info[i].mask;
    const int fc = bs->st[(lvl + 1) & 1].lb + bt[8] + nchs[i];
    int j = 0;
    for (int k = 0; k < 8; ++k) {
        const int v = ccount[i * 8 + k];
        childidx[i * 8 + k] = -1;
        if (m == 0 || v == 0) continue;
        const int id = fc + j++;
        childidx[i * 8 + k] = id;
        double l[3] = {lo[c].x, lo[c].y, lo[c].z}, h[3] = {hi[c].x, hi[c].y, hi[c].z};
        for (int a = 0; a < 3; ++a)
            if ((m >> a) & 1) {
                if ((k >> a) & 1) l[a] = info[i].mid[a];
                else h[a] = info[i].mid[a];
            }
        lo[id] = make_dvec4(l[0], l[1], l[2], 0.0);
        hi[id] = make_dvec4(h[0], h[1], h[2], 0.0);
        begin[id] = begin[c] + childoff[i * 8 + k];
        end[id] = begin[id] + v;
        first_child[id] = -1;
        n_child[id] = 0;
        level[id] = level[c] + 1;
        parent[id] = c;
    }
    first_child[c] = j > 0 ? fc : -1;
    n_child[c] = j;
}

// Stable scatter of the level's participating slots into their children,
// from the current buffers into the other ones.  Runs only when the level
// created children.
__global__ void __launch_bounds__(BT, 2) k_scatter(
    int64_t n, const BuildState *__restrict__ bs, int lvl, double *xsA, double *xsB, int32_t *permA,
    int32_t *permB, int32_t *nodeA, int32_t *nodeB, const SplitInfo *__restrict__ info,
    const int32_t *__restrict__ begin, const int32_t *__restrict__ cprefix,
    const int32_t *__restrict__ childoff, const int32_t *__restrict__ childidx,
    const int32_t *__restrict__ bprefix, int nblk)
{
    const LevelState L = bs->st[lvl & 1];
    if (L.nl == 0 || !bs->flip) return;
    const int lb = L.lb, nl = L.nl;
    const bool cur = bs->cur != 0;
    const double *__restrict__ xs = cur ? xsB : xsA;
    const int32_t *__restrict__ perm = cur ? permB : permA;
    const int32_t *__restrict__ node = cur ? nodeB : nodeA;
    double *__restrict__ xs2 = cur ? xsA : xsB;
    int32_t *__restrict__ perm2 = cur ? permA : permB;
    int32_t *__restrict__ node2 = cur ? nodeA : nodeB;
    // Each round of BT slots is staged in shared memory in the order of its
    // destinations (by code, then slot), so that consecutive threads write
    // consecutive addresses of the children's ranges.
    __shared__ int wcnt[BT / 32][9];
    __shared__ int run[8], rbase[10];
    __shared__ double sx[3][BT];
    __shared__ int32_t sperm[BT], snode[BT], sdst[BT];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < 8) run[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SPB;
    for (int r = 0; r < RPB; ++r) {
        int64_t p = base + r * BT + threadIdx.x;
        int c = -1, k = 8;
        if (p < n) k = slot_key(p, n, lb, nl, xs, node, info, &c);
        const int kk = p < n ? k : 9;  // 0..7 split codes, 8 slots that stay, 9 past the end
        unsigned grp = __match_any_sync(0xffffffffu, kk);
        int rank = __popc(grp & ((1u << lane) - 1u));
        if (lane < 9) wcnt[w][lane] = 0;
        __syncwarp();
        if (kk < 9 && rank == 0) wcnt[w][kk] = __popc(grp);
        __syncthreads();
        if (threadIdx.x < 9) {  // exclusive prefix over warps, per code (and per "stays")
            int t = 0;
            for (int q = 0; q < BT / 32; ++q) {
                int v = wcnt[q][threadIdx.x];
                wcnt[q][threadIdx.x] = t;
                t += v;
            }
            rbase[threadIdx.x] = t;  // round totals, turned into offsets below
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // offsets of the codes in the round's staged order
            int t = 0;
            for (int q = 0; q < 9; ++q) {
                int v = rbase[q];
                rbase[q] = t;
                t += v;
            }
            rbase[9] = t;  // staged slots of the round
        }
        __syncthreads();
        if (kk < 9) {
            int64_t dst;
            if (k < 8) {
                int g = bprefix[k * nblk + blockIdx.x] + run[k] + wcnt[w][k] + rank;
                dst = (int64_t)begin[lb + c] + childoff[c * 8 + k] + g - cprefix[c * 8 + k];
            } else {
                dst = p;
            }
            const int pos = rbase[kk] + wcnt[w][kk] + rank;
            for (int a = 0; a < 3; ++a) sx[a][pos] = xs[a * n + p];
            sperm[pos] = perm[p];
            snode[pos] = k < 8 ? childidx[c * 8 + k] : node[p];
            sdst[pos] = (int32_t)dst;
        }
        __syncthreads();
        if (threadIdx.x < rbase[9]) {
            const int64_t d = sdst[threadIdx.x];
            for (int a = 0; a < 3; ++a) xs2[a * n + d] = sx[a][threadIdx.x];
            perm2[d] = sperm[threadIdx.x];
            node2[d] = snode[threadIdx.x];
        }
        if (threadIdx.x < 8) run[threadIdx.x] += rbase[threadIdx.x + 1] - rbase[threadIdx.x];
        __syncthreads();
    }
}

// Cluster centre (box midpoint) and radius (half the diagonal), Fig. 1.
// Also writes the centre as FP32 hi/lo pairs and the radius in FP32
// (ctrf[2c] = hi xyz + radius, ctrf[2c+1] = lo xyz) for the list builder's
// FP32 pre-test of the MAC.
// With bs given, the clusters are bs->nclus (<= m).
__global__ void k_geometry(int m, const BuildState *__restrict__ bs, const dvec4 *__restrict__ lo,
                           const dvec4 *__restrict__ hi, dvec4 *__restrict__ ctr,
                           float4 *__restrict__ ctrf)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (bs) m = min(m, bs->nclus);
    if (c >= m) return;
    dvec4 a = lo[c], b = hi[c];
    double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y), dz = __dsub_rn(b.z, a.z);
    double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    dvec4 g = make_dvec4(__dmul_rn(0.5, __dadd_rn(a.x, b.x)), __dmul_rn(0.5, __dadd_rn(a.y, b.y)),
                         __dmul_rn(0.5, __dadd_rn(a.z, b.z)), __dmul_rn(0.5, __dsqrt_rn(s)));
    ctr[c] = g;
    float hx = __double2float_rn(g.x), hy = __double2float_rn(g.y), hz = __double2float_rn(g.z);
    ctrf[2 * c] = make_float4(hx, hy, hz, __double2float_rn(g.w));
    ctrf[2 * c + 1] = make_float4(__double2float_rn(g.x - (double)hx), __double2float_rn(g.y - (double)hy),
                                  __double2float_rn(g.z - (double)hz), 0.f);
}

// Initial state: one root per system, nothing split yet.
__global__ void k_state_init(BuildState *bs, int nsys)
{
    int *w = reinterpret_cast<int *>(bs);
    for (int i = threadIdx.x; i < (int)(sizeof(BuildState) / sizeof(int)); i += blockDim.x) w[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        bs->st[0] = LevelState{0, nsys};
        bs->nclus = nsys;
    }
}

// End of a build whose state the host never reads: brings the final slot
// order into the first buffers (when the last scattering level left it in the
// second ones) and flags a tree that ran out of clusters or of levels.
__global__ void k_tree_finish(int64_t n, const BuildState *__restrict__ bs, int levels,
                              double *__restrict__ xsA, const double *__restrict__ xsB,
                              int32_t *__restrict__ permA, const int32_t *__restrict__ permB,
                              int *__restrict__ err)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && (bs->overflow || bs->st[levels & 1].nl != 0))
        atomicOr(err, ASYNC_TREE_OVERFLOW);
    if ((bs->cur ^ bs->flip) == 0) return;
    int64_t base = (int64_t)blockIdx.x * SPB;
    for (int r = 0; r < RPB; ++r) {
        int64_t i = base + r * BT + threadIdx.x;
        if (i < n) {
            for (int l = 0; l < 3; ++l) xsA[l * n + i] = xsB[l * n + i];
            permA[i] = permB[i];
        }
    }
}

// Cluster arrays for cap clusters (contents not kept).
kitc_status alloc_clusters(TreeDev &t, int cap, cudaStream_t s)
{
    for (DevBuf *d : {&t.lo, &t.hi})
        KITC_TRY(d->reserve(sizeof(dvec4) * cap, s));
    for (DevBuf *d : {&t.begin, &t.end, &t.first_child, &t.n_child, &t.level, &t.parent})
        KITC_TRY(d->reserve(sizeof(int32_t) * cap, s));
    t.cap = cap;
    return KITC_OK;
}

// Pointers into the level scratch: the state block, then per cluster of the
// largest level: split info | ccount | cprefix | childoff | childidx (8 each)
// | children prefix | block totals of the children kernels.
struct LevelPtrs {
    BuildState *bs;
    SplitInfo *info;
    int32_t *ccount, *cprefix, *childoff, *childidx, *nchs, *btot;
};

size_t level_scratch_bytes(int64_t max_nl)
{
    const size_t per = (size_t)max_nl * 8;
    const size_t nbt = (size_t)((max_nl + CB - 1) / CB) * NT;
    return ((sizeof(BuildState) + 255) / 256) * 256 + sizeof(SplitInfo) * max_nl +
           sizeof(int32_t) * (4 * per + max_nl + nbt + 2) + 256;
}

LevelPtrs level_ptrs(const TreeScratch &sc)
{
    LevelPtrs q;
    char *b = sc.lvl.as<char>();
    const size_t per = (size_t)sc.max_nl * 8;
    q.bs = reinterpret_cast<BuildState *>(b);
    q.info = reinterpret_cast<SplitInfo *>(b + ((sizeof(BuildState) + 255) / 256) * 256);
    q.ccount = reinterpret_cast<int32_t *>(q.info + sc.max_nl);
    q.cprefix = q.ccount + per;
    q.childoff = q.cprefix + per;
    q.childidx = q.childoff + per;
    q.nchs = q.childidx + per;
    q.btot = q.nchs + sc.max_nl;
    return q;
}

// Root-box chunks of at most 64K slots, packed in offs as
// [off (nsys+1) | cb (nc) | ce (nc)] int64, then [c0 (nsys+1) | cs (nc)] int32,
// then the chunks' partial boxes (6 doubles each, 16-byte aligned).
struct RootPtrs {
    int64_t *d64;
    int32_t *d32;
    double *part;
};

RootPtrs root_ptrs(const TreeScratch &sc)
{
    RootPtrs r;
    r.d64 = sc.offs.as<int64_t>();
    r.d32 = reinterpret_cast<int32_t *>(r.d64 + sc.n64);
    r.part = reinterpret_cast<double *>(
        sc.offs.as<char>() + ((sizeof(int64_t) * sc.n64 + sizeof(int32_t) * sc.n32 + 15) / 16) * 16);
    return r;
}

// Slot arrays, cluster arrays for cap clusters and the scratch of one build of
// the n points (a forest of nsys systems when counts is given); uploads the
// root chunks.  The host copies of the chunks stay in hchunks until the
// scratch is released, so they outlive the upload.
kitc_status build_reserve(TreeDev &t, TreeScratch &sc, std::vector<int64_t> &h64,
                          std::vector<int32_t> &h32, int64_t n, int leaf, const int64_t *counts,
                          int nsys, int cap, cudaStream_t s)
{
    t.release(s);
    sc.release(s);
    t.n = n;
    t.leaf = leaf;
    sc.nsys = nsys;
    sc.cap = cap;
    sc.nblk = (int)((n + SPB - 1) / SPB);
    KITC_TRY(t.perm.reserve(sizeof(int32_t) * n, s));
    KITC_TRY(sc.perm2.reserve(sizeof(int32_t) * n, s));
    KITC_TRY(t.xs.reserve(sizeof(double) * 3 * n, s));
    KITC_TRY(sc.xs2.reserve(sizeof(double) * 3 * n, s));
    KITC_TRY(sc.node.reserve(sizeof(int32_t) * n, s));
    KITC_TRY(sc.node2.reserve(sizeof(int32_t) * n, s));
    sc.hoff.assign(nsys + 1, 0);
    for (int k = 0; k < nsys; ++k) sc.hoff[k + 1] = sc.hoff[k] + (counts ? counts[k] : n);
    if (sc.hoff[nsys] != n) return KITC_ERR_INVALID_ARG;
    const int64_t CH = 65536;
    std::vector<int64_t> cbv, cev;
    std::vector<int32_t> c0v(nsys + 1, 0), csv;
    for (int k = 0; k < nsys; ++k) {
        c0v[k] = (int32_t)cbv.size();
        for (int64_t p = sc.hoff[k]; p < sc.hoff[k + 1]; p += CH) {
            cbv.push_back(p);
            cev.push_back(std::min(sc.hoff[k + 1], p + CH));
            csv.push_back(k);
        }
    }
    sc.nc = (int)cbv.size();
    c0v[nsys] = sc.nc;
    h64 = sc.hoff;
    h64.insert(h64.end(), cbv.begin(), cbv.end());
    h64.insert(h64.end(), cev.begin(), cev.end());
    h32 = c0v;
    h32.insert(h32.end(), csv.begin(), csv.end());
    sc.n64 = h64.size();
    sc.n32 = h32.size();
    KITC_TRY(sc.offs.reserve(sizeof(int64_t) * sc.n64 + sizeof(int32_t) * sc.n32 +
                             sizeof(double) * 6 * sc.nc + 64, s));
    KITC_TRY(sc.bcount.reserve(sizeof(int32_t) * 8 * sc.nblk, s));
    KITC_TRY(alloc_clusters(t, cap, s));
    sc.max_nl = std::min<int64_t>(cap, n + nsys);  // the largest level
    KITC_TRY(sc.lvl.reserve(level_scratch_bytes(sc.max_nl), s));
    // every buffer the kernels write must exist before any launch
    for (const DevBuf *b : {&t.perm, &sc.perm2, &t.xs, &sc.xs2, &sc.node, &sc.node2, &sc.offs,
                            &sc.bcount, &sc.lvl, &t.lo, &t.hi, &t.begin, &t.end, &t.first_child,
                            &t.n_child, &t.level, &t.parent})
        if (!b->ptr) return KITC_ERR_OOM;
    const RootPtrs r = root_ptrs(sc);
    KITC_CUDA(cudaMemcpyAsync(r.d64, h64.data(), sizeof(int64_t) * h64.size(), cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(r.d32, h32.data(), sizeof(int32_t) * h32.size(), cudaMemcpyHostToDevice, s));
    return KITC_OK;
}

// State, slot order and root boxes.
kitc_status queue_root(TreeDev &t, const TreeScratch &sc, const double *xyz, cudaStream_t s)
{
    const LevelPtrs q = level_ptrs(sc);
    const RootPtrs r = root_ptrs(sc);
    const int nsys = sc.nsys, nc = sc.nc;
    kitc_count_launch();
    k_state_init<<<1, 128, 0, s>>>(q.bs, nsys);
    kitc_count_launch();
    k_init<<<sc.nblk, BT, 0, s>>>(xyz, t.n, t.xs.as<double>(), t.perm.as<int32_t>());
    KITC_CUDA(cudaGetLastError());
    kitc_count_launch();
    k_root_partial<<<nc, BT, 0, s>>>(r.d32 + nsys + 1, r.d64 + nsys + 1, r.d64 + nsys + 1 + nc, t.n,
                                     t.xs.as<double>(), sc.node.as<int32_t>(), r.part);
    KITC_CUDA(cudaGetLastError());
    kitc_count_launch();
    k_root_final<<<(nsys + 127) / 128, 128, 0, s>>>(nsys, r.d32, r.d64, r.part, t.lo.as<dvec4>(),
                                                    t.hi.as<dvec4>(), t.begin.as<int32_t>(),
                                                    t.end.as<int32_t>(), t.first_child.as<int32_t>(),
                                                    t.n_child.as<int32_t>(), t.level.as<int32_t>(),
                                                    t.parent.as<int32_t>());
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

// Levels [lv0, lv1).  Grids are sized from a host bound of each level's size
// (nsys 8^lv, at most the largest level); kernels of a level with no clusters
// exit at once.
kitc_status queue_levels(TreeDev &t, TreeScratch &sc, int leaf, int lv0, int lv1, cudaStream_t s)
{
    const LevelPtrs q = level_ptrs(sc);
    const int64_t n = t.n;
    const int nblk = sc.nblk;
    for (int lv = lv0; lv < lv1; ++lv) {
        int64_t cap_l = std::min<int64_t>(sc.max_nl, sc.nsys);
        for (int k = 0; k < lv && cap_l < sc.max_nl; ++k) cap_l = std::min<int64_t>(sc.max_nl, 8 * cap_l);
        kitc_count_launch();
        k_split<<<(unsigned)((cap_l + 255) / 256), 256, 0, s>>>(
            q.bs, lv, leaf, t.lo.as<dvec4>(), t.hi.as<dvec4>(), t.begin.as<int32_t>(),
            t.end.as<int32_t>(), t.level.as<int32_t>(), q.info, q.ccount);
        kitc_count_launch();
        k_count<<<nblk, BT, 0, s>>>(n, q.bs, lv, t.xs.as<double>(), sc.xs2.as<double>(),
                                    sc.node.as<int32_t>(), sc.node2.as<int32_t>(), q.info, q.ccount,
                                    sc.bcount.as<int32_t>(), nblk);
        const unsigned gc = (unsigned)((cap_l + CB - 1) / CB);
        kitc_count_launch();
        k_children_local<<<gc, CB, 0, s>>>(q.bs, lv, q.info, q.ccount, q.cprefix, q.childoff, q.nchs,
                                           q.btot);
        kitc_count_launch();
        k_children_scan<<<1, BT, 0, s>>>(q.bs, lv, sc.cap, sc.bcount.as<int32_t>(), nblk, q.btot);
        kitc_count_launch();
        k_children_make<<<gc, CB, 0, s>>>(q.bs, lv, q.info, q.ccount, q.cprefix, q.childoff,
                                          q.childidx, q.nchs, q.btot, t.lo.as<dvec4>(),
                                          t.hi.as<dvec4>(), t.begin.as<int32_t>(),
                                          t.end.as<int32_t>(), t.first_child.as<int32_t>(),
                                          t.n_child.as<int32_t>(), t.level.as<int32_t>(),
                                          t.parent.as<int32_t>());
        kitc_count_launch();
        k_scatter<<<nblk, BT, 0, s>>>(n, q.bs, lv, t.xs.as<double>(), sc.xs2.as<double>(),
                                      t.perm.as<int32_t>(), sc.perm2.as<int32_t>(),
                                      sc.node.as<int32_t>(), sc.node2.as<int32_t>(), q.info,
                                      t.begin.as<int32_t>(), q.cprefix, q.childoff, q.childidx,
                                      sc.bcount.as<int32_t>(), nblk);
        KITC_CUDA(cudaGetLastError());
    }
    return KITC_OK;
}

// Levels queued per round: the depth of a roughly uniform tree plus a few
// levels of slack.
int round_levels(int64_t n, int leaf, int nsys)
{
    int round = 4;
    for (int64_t m = std::max<int64_t>(1, n / std::max(1, nsys)); m > leaf; m = (m + 7) / 8) ++round;
    return round;
}

}  // namespace

BuildState *TreeScratch::state() const { return level_ptrs(*this).bs; }

void TreeScratch::release(cudaStream_t s)
{
    for (DevBuf *b : {&perm2, &xs2, &node, &node2, &offs, &bcount, &lvl}) b->release(s);
    nblk = nc = cap = 0;
    nsys = 1;
    max_nl = 0;
    n64 = n32 = 0;
    hoff.clear();
}

void TreeDev::release(cudaStream_t s)
{
    for (DevBuf *b : {&perm, &xs, &lo, &hi, &ctr, &ctrf, &begin, &end, &first_child, &n_child,
                      &level, &parent})
        b->release(s);
    nclus = cap = depth = nleaves = 0;
    nsys = 1;
    level_start.clear();
    sys_off.clear();
}

size_t TreeDev::bytes() const
{
    size_t b = 0;
    for (const DevBuf *d : {&perm, &xs, &lo, &hi, &ctr, &ctrf, &begin, &end, &first_child,
                            &n_child, &level, &parent})
        b += d->bytes;
    return b;
}

// One attempt at the build with room for cap clusters; *needed > cap on
// return means the tree did not fit (nothing else of t is valid then).
static kitc_status tree_build_cap(const double *xyz, int64_t n, int leaf, cudaStream_t s, TreeDev &t,
                                  const int64_t *counts, int nsys, int cap, int64_t *needed)
{
    *needed = 0;
    TreeScratch sc;
    std::vector<int64_t> h64;
    std::vector<int32_t> h32;
    auto fail = [&](kitc_status st) {
        sc.release(s);
        return st;
    };
    kitc_status st = build_reserve(t, sc, h64, h32, n, leaf, counts, nsys, cap, s);
    if (st == KITC_OK) st = queue_root(t, sc, xyz, s);
    if (st != KITC_OK) return fail(st);
    // Levels are queued in rounds, then the state is read back once; a deeper
    // tree takes further rounds.  Levels after the last one exit at once.
    const int round = round_levels(n, leaf, nsys);
    const BuildState *bs = sc.state();
    BuildState hs{};
    int lv = 0;
    for (;;) {
        const int lv_end = std::min(KITC_MAX_LEVEL + 1, lv + round);
        st = queue_levels(t, sc, leaf, lv, lv_end, s);
        if (st != KITC_OK) return fail(st);
        lv = lv_end;
        // the one read-back of the round (it also ends the life of the host
        // arrays uploaded by build_reserve)
        st = kitc_from_cuda(cudaMemcpyAsync(&hs, bs, sizeof(hs), cudaMemcpyDeviceToHost, s));
        if (st == KITC_OK) st = kitc_from_cuda(cudaStreamSynchronize(s));
        if (st != KITC_OK) return fail(st);
        if (hs.overflow || hs.st[lv & 1].nl == 0 || lv > KITC_MAX_LEVEL) break;
    }
    if (hs.overflow) {
        *needed = 2 * (int64_t)cap;
        return fail(KITC_OK);
    }
    if (hs.st[lv & 1].nl != 0) return fail(KITC_ERR_CUDA);  // cannot happen: a level past KITC_MAX_LEVEL splits nothing
    if ((hs.cur ^ hs.flip) != 0) {  // the final order is in the second buffers
        std::swap(t.xs, sc.xs2);
        std::swap(t.perm, sc.perm2);
    }
    sc.release(s);
    t.nclus = hs.nclus;
    t.depth = hs.depth;
    t.nleaves = hs.nleaves;
    t.nsys = nsys;
    t.sys_off.assign(h64.begin(), h64.begin() + nsys + 1);
    t.level_start.assign(hs.level_start, hs.level_start + hs.depth);
    KITC_TRY(t.ctr.reserve(sizeof(dvec4) * t.cap, s));
    KITC_TRY(t.ctrf.reserve(2 * sizeof(float4) * t.cap, s));
    kitc_count_launch();
    k_geometry<<<(t.nclus + 255) / 256, 256, 0, s>>>(t.nclus, nullptr, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                                   t.ctr.as<dvec4>(), t.ctrf.as<float4>());
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status tree_build(const double *xyz, int64_t n, int leaf, cudaStream_t s, TreeDev &t,
                       const int64_t *counts, int nsys)
{
    if (!counts) nsys = 1;
    // room for the clusters of a tree whose levels each split at most
    // n / (N0 + 1) clusters into 8, over 16 levels' worth; a tree that does not
    // fit is built again with twice the room
    int64_t cap = (int64_t)nsys + 16 * ((n + leaf) / (leaf + 1)) + 64;
    for (;;) {
        if (cap > (int64_t)INT32_MAX / 2) return KITC_ERR_OOM;
        int64_t needed = 0;
        KITC_TRY(tree_build_cap(xyz, n, leaf, s, t, counts, nsys, (int)cap, &needed));
        if (needed == 0) return KITC_OK;
        cap = needed;
    }
}

void TreeAsync::release(cudaStream_t s)
{
    t.release(s);
    sc.release(s);
    levels = 0;
}

size_t TreeAsync::bytes() const
{
    size_t b = t.bytes();
    for (const DevBuf *d : {&sc.perm2, &sc.xs2, &sc.node, &sc.node2, &sc.offs, &sc.bcount, &sc.lvl})
        b += d->bytes;
    return b;
}

kitc_status tree_async_reserve(TreeAsync &a, int64_t n, int leaf, const int64_t *counts, int nsys,
                               int cap, int levels, cudaStream_t s)
{
    if (!counts) nsys = 1;
    if (levels < 1 || levels > KITC_MAX_LEVEL + 1 || cap < nsys) return KITC_ERR_INVALID_ARG;
    std::vector<int64_t> h64;
    std::vector<int32_t> h32;
    kitc_status st = build_reserve(a.t, a.sc, h64, h32, n, leaf, counts, nsys, cap, s);
    if (st == KITC_OK) st = a.t.ctr.reserve(sizeof(dvec4) * cap, s);
    if (st == KITC_OK) st = a.t.ctrf.reserve(2 * sizeof(float4) * cap, s);
    if (st == KITC_OK) st = kitc_from_cuda(cudaStreamSynchronize(s));  // h64, h32 end here
    if (st != KITC_OK) {
        a.release(s);
        return st;
    }
    a.t.nsys = nsys;
    a.t.sys_off.assign(h64.begin(), h64.begin() + nsys + 1);
    a.t.nclus = -1;  // known on the device only
    a.levels = levels;
    return KITC_OK;
}

kitc_status tree_async_launch(TreeAsync &a, const double *xyz, int *err, cudaStream_t s)
{
    TreeDev &t = a.t;
    if (a.levels < 1 || !t.ctr.ptr || !t.ctrf.ptr) return KITC_ERR_STATE;
    KITC_TRY(queue_root(t, a.sc, xyz, s));
    KITC_TRY(queue_levels(t, a.sc, t.leaf, 0, a.levels, s));
    const BuildState *bs = a.state();
    kitc_count_launch();
    k_tree_finish<<<a.sc.nblk, BT, 0, s>>>(t.n, bs, a.levels, t.xs.as<double>(), a.sc.xs2.as<double>(),
                                           t.perm.as<int32_t>(), a.sc.perm2.as<int32_t>(), err);
    kitc_count_launch();
    k_geometry<<<(t.cap + 255) / 256, 256, 0, s>>>(t.cap, bs, t.lo.as<dvec4>(), t.hi.as<dvec4>(),
                                                 t.ctr.as<dvec4>(), t.ctrf.as<float4>());
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}
