// Fused near/far evaluator of Algorithm 2 (and of the direct sum), for the
// regularized Stokes kernels of Sec. 7 (Eqs. MRS_kernels, Velocity_1, MRS_2).
//
// Design (GB300, sm_103a):
//  * Persistent CTAs take target batches from an atomic work counter.
//  * A producer warp streams the batch's interaction list as tiles -- source
//    records of a near leaf (Eq. pc_interaction_3D) or modified-weight records
//    of a far cluster (Eq. pc_approximation_3D) -- global -> shared memory with
//    TMA bulk copies (cp.async.bulk) into a ring of stages guarded by
//    mbarriers (full: bytes landed; empty: all consumer warps done).
//  * Eight consumer warps hold the batch's <= 64 targets (two per lane) and
//    split every tile between them: near tiles by blocks of 8 sources, far
//    tiles by grid rows (k1, k2) of (n+1) points.  The (n+1)^3 grid of a
//    cluster is a tensor product, so only 3 (n+1) coordinates per cluster are
//    formed; the per-point work is one rsqrt and a few FMAs.
//  * KITC_MIXED: coordinate differences of near pairs come from hi/lo FP32
//    pairs (d = (xh - yh) + (xl - yl), relative error ~1e-7 at any distance);
//    KITC_MIXED_LEAF (FP32x2 path): d = (x - c) - (y - c) from offsets to the
//    leaf's box centre c, both formed by the same FP32 arithmetic on hi/lo
//    parts (leaf_offset), one packed add per coordinate instead of three.
//    Far-field points are taken relative to the batch centre in FP64 and then
//    rounded.  Kernel values are FP32, summed in FP32 over runs of at most 8
//    terms, those runs summed over at most 8, and so on one more level; the
//    per-leaf / per-cluster sums are accumulated in FP64.
//  * The mixed Stokeslet and rotlet run on packed FP32x2 arithmetic over pairs
//    of sources or grid points (paired records); the other forms take one
//    point at a time.
//  * Every barrier wait is bounded (globaltimer); a wait that runs out sets an
//    error flag, the CTA drains its own copies in flight and returns.
#include <type_traits>
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kmath.cuh"

namespace {

#ifndef KITC_NCW
#define KITC_NCW 8
#endif
constexpr int NCW = KITC_NCW;          // consumer warps
constexpr int NTH = (NCW + 1) * 32;    // plus one producer warp
#ifndef KITC_STAGES
#define KITC_STAGES 3
#endif
#ifndef KITC_TILE
#define KITC_TILE 24576
#endif
constexpr int STAGES = KITC_STAGES;    // ring of shared-memory stages
constexpr int TILE = KITC_TILE;        // bytes per stage
// Batches of <= 32 targets run the mixed Stokeslet with one target per lane
// instead of two (KITC_TPL1=0: two, the second idle).
#ifndef KITC_TPL1
#define KITC_TPL1 1
#endif
constexpr double INV8PI = 0.039788735772973836;

enum { K_FAR = 0, K_NEAR = 1, K_EXIT = 2 };
enum { F_FIRST_BATCH = 1, F_LAST_BATCH = 2, F_FIRST_ENTRY = 4, F_LAST_ENTRY = 8 };

struct TileMeta {
    int kind, flags, batch, id;
    int a, b;        // far: k1 planes [a, b); near: source slots [a, b)
    int seq;         // position of the tile within its batch (fixes the work split)
    int np;          // far: grid points per dimension of the cluster (n_c + 1)
    uint64_t mask;   // targets of the batch that use this entry
    dvec4 lo, hi;    // far: the cluster's box (read ahead by the producer)
    // FP32x2 path, far: cluster centre minus batch centre and half widths of
    // the box, formed in FP64 by the producer and rounded once; near with
    // leaf offsets: the leaf's box centre as FP32 hi (goff) and lo (ghw) parts
    float goff[3], ghw[3];
};

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            bar),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `parity` to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long limit_ns)
{
    if (mbar_try(bar, parity)) return true;
    unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Packed FP32x2 arithmetic of sm_100+ (one instruction, two FP32 lanes).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// The test kernel prod_l (1 + x_l y_l / 2)^3 f (FP64 only).
__device__ __forceinline__ void pair_poly(const double *x, double y0, double y1, double y2,
                                          const double *f, double *u)
{
    double q0 = 1.0 + 0.5 * x[0] * y0, q1 = 1.0 + 0.5 * x[1] * y1, q2 = 1.0 + 0.5 * x[2] * y2;
    double p = (q0 * q0 * q0) * (q1 * q1 * q1) * (q2 * q2 * q2);
    u[0] = fma(p, f[0], u[0]);
    u[1] = fma(p, f[1], u[1]);
    u[2] = fma(p, f[2], u[2]);
}

}  // namespace

namespace {

template <bool MIXED, int WIN> struct Rec {
    static constexpr int SRC = MIXED ? 48 : (WIN == 3 ? 48 : 80);
    static constexpr int PROXY = MIXED ? (WIN == 3 ? 16 : 32) : (WIN == 3 ? 32 : 48);
};

// Keep the per-target FP64 sums and the third FP32 sum level of the mixed
// path in shared memory instead of registers (they change every 8 / 64 runs).
#ifndef KITC_SMEM_ACC
#define KITC_SMEM_ACC 0
#endif

// FP32x2 path: keep a run's packed sums (even / odd points or sources)
// as float2 through the second summation level instead of adding the halves
// at every run.
#ifndef KITC_PACKED_RUNS
#define KITC_PACKED_RUNS 1
#endif

// FP32x2 path: grid rows per run of the Stokeslet far field (a warp's rows r,
// r + NCW, ...; the rotlet takes one) and source pairs per run of the near
// field.
#ifndef KITC_RPR
#define KITC_RPR 2
#endif
#ifndef KITC_NPB
#define KITC_NPB 8   // rotlet
#endif
#ifndef KITC_NPB_S
#define KITC_NPB_S 16  // Stokeslet
#endif
constexpr int RPR = KITC_RPR, NPB = KITC_NPB;

// FP32x2 path: the producer forms each far cluster's offset from the batch
// centre and its half widths (FP64, rounded to FP32) once per entry, and the
// consumers map the FP32 Chebyshev table with one FMA per grid coordinate
// (KITC_FAR_PROD=0: every consumer warp maps the points in FP64).
#ifndef KITC_FAR_PROD
#define KITC_FAR_PROD 1
#endif

// FP32x2 rotlet: FP64 sums and third FP32 level in shared memory (they change
// every 8 / 64 runs), which leaves the registers to the six-component run sums.
#ifndef KITC_ROT_SACC
#define KITC_ROT_SACC 1
#endif

template <int K> struct Smem {
    static constexpr int WOUT = KT<K>::WOUT;
    static constexpr size_t RED = (size_t)NCW * KITC_MAX_BATCH * WOUT * sizeof(double);
    static constexpr size_t META = STAGES * sizeof(TileMeta);
    static constexpr size_t BARS = (2 * STAGES + 2) * sizeof(uint64_t);
    static constexpr size_t GRID = (size_t)NCW * 3 * (KITC_MAX_DEGREE + 1) * sizeof(double);
    // KITC_SMEM_ACC: the FP64 sums and the third FP32 level of the mixed path
    static constexpr bool SA = KITC_SMEM_ACC || (KITC_ROT_SACC && K == KITC_ROTLET);
    static constexpr size_t ACCS = SA ? (size_t)NCW * KITC_MAX_BATCH * WOUT * 12 : 0;
    // FP32 Chebyshev table cos(k pi / n) [n][k] of the FP32x2 far field
    static constexpr size_t CHEBF = (size_t)(KITC_MAX_DEGREE + 1) * (KITC_MAX_DEGREE + 1) * sizeof(float);
    static constexpr size_t TOTAL = (size_t)STAGES * TILE + RED + META + BARS + GRID + ACCS + CHEBF;
};

// Weight components of a record as R values.
template <bool MIXED, int WIN, typename R>
__device__ __forceinline__ void load_proxy(const unsigned char *p, R *f)
{
    if constexpr (MIXED) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        f[0] = v.x; f[1] = v.y; f[2] = v.z;
        if constexpr (WIN == 6) {
            float4 u = *reinterpret_cast<const float4 *>(p + 16);
            f[3] = u.x; f[4] = u.y; f[5] = u.z;
        }
    } else {
        const double *d = reinterpret_cast<const double *>(p);
#pragma unroll
        for (int q = 0; q < WIN; ++q) f[q] = d[q];
    }
}

template <bool MIXED, int WIN, typename R>
__device__ __forceinline__ void load_source(const unsigned char *rec, R *yh, R *yl, R *f)
{
    if constexpr (MIXED) {
        float4 r0 = *reinterpret_cast<const float4 *>(rec);
        float4 r1 = *reinterpret_cast<const float4 *>(rec + 16);
        float4 r2 = *reinterpret_cast<const float4 *>(rec + 32);
        yh[0] = r0.x; yh[1] = r0.y; yh[2] = r0.z;
        yl[0] = r0.w; yl[1] = r1.x; yl[2] = r1.y;
        f[0] = r1.z; f[1] = r1.w; f[2] = r2.x;
        if constexpr (WIN == 6) { f[3] = r2.y; f[4] = r2.z; f[5] = r2.w; }
    } else {
        const double *d = reinterpret_cast<const double *>(rec);
        yh[0] = d[0]; yh[1] = d[1]; yh[2] = d[2];
        yl[0] = yl[1] = yl[2] = 0.0;
#pragma unroll
        for (int q = 0; q < WIN; ++q) f[q] = d[3 + q];
    }
}

// CTAs per SM the register budget targets: two for the FP32 Stokeslet (96
// registers a thread: a 9-warp CTA puts up to five warps of two CTAs on one
// scheduler), one for the wider FP64 and rotlet variants (168).
#ifndef KITC_PAIR_MINB
#define KITC_PAIR_MINB 2
#endif
template <int K, bool MIXED> struct MinBlocks {
    static constexpr int value = (MIXED && K == KITC_STOKESLET) ? KITC_PAIR_MINB : 1;
};

// LEAF: the FP32x2 near field reads leaf-offset records (KITC_MIXED_LEAF);
// otherwise double-float records (KITC_MIXED, and every direct sum).
template <int K, bool MIXED, bool EPS0, int TPL, bool LEAF>
__device__ __forceinline__ void eval_body(const EvalArgs &a)
{
    static_assert(TPL == 1 || TPL == 2, "one or two targets per lane");
    using SM = Smem<K>;
    constexpr int WIN = KT<K>::WIN, WOUT = KT<K>::WOUT;
    constexpr int SREC = Rec<MIXED, WIN>::SRC, PREC = Rec<MIXED, WIN>::PROXY;
    // FP32x2 path (Stokeslet, rotlet): paired source records and paired grid
    // points (see pack_pairs)
    constexpr bool PAIR = MIXED && (K == KITC_STOKESLET || K == KITC_ROTLET);
    constexpr bool ROT = K == KITC_ROTLET;
    constexpr bool OFF = PAIR && LEAF;  // near records: offsets from the leaf centre
    constexpr int PAIR_REC = OFF ? LEAF_PAIR_BYTES : 80;
    using R = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *tiles = smem;
    double *red = reinterpret_cast<double *>(smem + (size_t)STAGES * TILE);
    TileMeta *meta = reinterpret_cast<TileMeta *>(smem + (size_t)STAGES * TILE + SM::RED);
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(meta) +
                                                  SM::META);
    double *gridc = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(bars) +
                                               SM::BARS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool SACC = MIXED && SM::SA;
    double *accs = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(gridc) + SM::GRID) +
                   (size_t)warp * KITC_MAX_BATCH * WOUT;  // [64 targets][WOUT]
    float *a3s = reinterpret_cast<float *>(reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(gridc) +
                                                                      SM::GRID) +
                                           (size_t)NCW * KITC_MAX_BATCH * WOUT) +
                 (size_t)warp * KITC_MAX_BATCH * WOUT;
    float *chebf = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(gridc) + SM::GRID +
                                             SM::ACCS);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
    const uint32_t rbw = smem_u32(bars + 2 * STAGES), rbr = smem_u32(bars + 2 * STAGES + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, NCW);
        }
        mbar_init(rbw, NCW);
        mbar_init(rbr, NCW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (PAIR && KITC_FAR_PROD) {
        constexpr int NC = KITC_MAX_DEGREE + 1;
        for (int q = threadIdx.x; q < NC * NC; q += blockDim.x) {
            const int n = q / NC, k = q % NC;  // row n: degree n (cos(k pi / n), k <= n)
            double v = 0.0;
            if (a.chebt) v = a.chebt[q];
            else if (n == a.degree) v = a.cheb[k];
            chebf[q] = (float)v;
        }
    }
    __syncthreads();
    const int np0 = a.degree + 1;                                 // uniform degree
    const int near_unit = PAIR ? PAIR_REC : SREC;                 // one near item
    const int near_max = PAIR ? (TILE / PAIR_REC) / 4 * 4 : (TILE / SREC) / 8 * 8;
    const unsigned long long wait_ns = a.wait_ns;

    // ---------------------------------------------------------------- producer
    if (warp == NCW) {
        if (lane != 0) return;
        uint32_t it = 0;
        bool ok = true;
        auto emit = [&](const TileMeta &m, const unsigned char *src, uint32_t bytes) -> bool {
            int s = it % STAGES;
            uint32_t ph = (it / STAGES) & 1u;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, wait_ns)) return false;
            meta[s] = m;
            if (bytes) {
                mbar_arrive_tx(full0 + 8 * s, bytes);
                bulk_g2s(smem_u32(tiles + (size_t)s * TILE), src, bytes, full0 + 8 * s);
            } else {
                mbar_arrive(full0 + 8 * s);
            }
            ++it;
            return true;
        };
        const unsigned char *srcb = reinterpret_cast<const unsigned char *>(a.src);
        const unsigned char *pxb = reinterpret_cast<const unsigned char *>(a.proxy);
        const dvec4 zero4 = make_dvec4(0, 0, 0, 0);
        for (;;) {
            int b = atomicAdd(a.queue, 1);
            if (b >= a.nb) break;
            dvec4 pcB = zero4;
            if (PAIR && KITC_FAR_PROD && a.bctr && a.near_off) pcB = a.bctr[b];
            bool have = false, first = true;
            TileMeta pend{};
            const unsigned char *psrc = nullptr;
            uint32_t pbytes = 0;
            int tseq = 0;
            auto push = [&](const TileMeta &m0, const unsigned char *src, uint32_t bytes) -> bool {
                TileMeta m = m0;
                m.seq = tseq++;
                if (have) {
                    if (first) pend.flags |= F_FIRST_BATCH;
                    first = false;
                    if (!emit(pend, psrc, pbytes)) return false;
                }
                pend = m;
                psrc = src;
                pbytes = bytes;
                have = true;
                return true;
            };
            if (a.near_off) {
                int64_t f0 = a.far_off[b], f1 = a.far_off[b + 1];
                for (int64_t e = f0; e < f1 && ok; ++e) {
                    int c = a.far_id[e];
                    uint64_t mk = a.far_mask[e];
                    dvec4 lo = a.clo[c], hi = a.chi[c];
                    // grid of cluster c: (n_c+1)^3 records from its offset
                    const int np = a.cdeg ? a.cdeg[c] + 1 : np0;
                    if (np < 2 || np > KITC_MAX_DEGREE + 1) { ok = false; break; }
                    // a tile holds whole units: planes k1 of np grid rows, or
                    // (paired rotlet records, odd np) pairs of consecutive grid rows
                    const bool rowpairs = PAIR && ROT && (np & 1);
                    const int unit_bytes = rowpairs ? np * 32 : np * (PAIR ? (np + 1) / 2 * 32 : np * PREC);
                    const int nunits = rowpairs ? (np * np + 1) / 2 : np;
                    const int units_max = TILE / unit_bytes;
                    const unsigned char *cb = pxb + (a.roff ? (size_t)a.roff[c]
                                                            : (size_t)c * nunits * unit_bytes);
                    for (int k1 = 0; k1 < nunits && ok; k1 += units_max) {
                        int k2 = min(nunits, k1 + units_max);
                        TileMeta m{K_FAR, (k1 == 0 ? F_FIRST_ENTRY : 0) | (k2 == nunits ? F_LAST_ENTRY : 0),
                                   b, c, k1, k2, 0, np, mk, lo, hi};
                        if (PAIR && KITC_FAR_PROD && k1 == 0) {
                            m.goff[0] = (float)(0.5 * (lo.x + hi.x) - pcB.x);
                            m.goff[1] = (float)(0.5 * (lo.y + hi.y) - pcB.y);
                            m.goff[2] = (float)(0.5 * (lo.z + hi.z) - pcB.z);
                            m.ghw[0] = (float)(0.5 * (hi.x - lo.x));
                            m.ghw[1] = (float)(0.5 * (hi.y - lo.y));
                            m.ghw[2] = (float)(0.5 * (hi.z - lo.z));
                        }
                        ok = push(m, cb + (size_t)k1 * unit_bytes, (uint32_t)((k2 - k1) * unit_bytes));
                    }
                }
                int64_t n0 = a.near_off[b], n1 = a.near_off[b + 1];
                for (int64_t e = n0; e < n1 && ok; ++e) {
                    int c = a.near_id[e];
                    uint64_t mk = a.near_mask[e];
                    int p0 = a.cbegin[c], p1 = a.cend[c];
                    if (PAIR) {  // items are source pairs
                        int pc = (p1 - p0 + 1) / 2;
                        p0 = a.pbegin[c];
                        p1 = p0 + pc;
                    }
                    float lch[3] = {0.f, 0.f, 0.f}, lcl[3] = {0.f, 0.f, 0.f};  // OFF: leaf centre
                    if (OFF) leaf_centre(a.clo[c], a.chi[c], lch, lcl);
                    for (int q = p0; q < p1 && ok; q += near_max) {
                        int q1 = min(p1, q + near_max);
                        TileMeta m{K_NEAR, (q == p0 ? F_FIRST_ENTRY : 0) | (q1 == p1 ? F_LAST_ENTRY : 0),
                                   b, c, q, q1, 0, 0, mk, zero4, zero4};
                        for (int l = 0; l < 3; ++l) {
                            m.goff[l] = lch[l];
                            m.ghw[l] = lcl[l];
                        }
                        ok = push(m, srcb + (size_t)q * near_unit, (uint32_t)((q1 - q) * near_unit));
                    }
                }
            } else {
                int64_t p1 = PAIR ? (a.direct_ns + 1) / 2 : a.direct_ns;
                for (int64_t q = 0; q < p1 && ok; q += near_max) {
                    int64_t q1 = min(p1, q + (int64_t)near_max);
                    TileMeta m{K_NEAR, (q == 0 ? F_FIRST_ENTRY : 0) | (q1 == p1 ? F_LAST_ENTRY : 0),
                               b, -1, (int)q, (int)q1, 0, 0, ~0ull, zero4, zero4};
                    ok = push(m, srcb + (size_t)q * near_unit, (uint32_t)((q1 - q) * near_unit));
                }
            }
            if (!ok) break;
            if (!have) {  // no entries: one empty tile closes the batch
                pend = TileMeta{K_NEAR, F_FIRST_ENTRY | F_LAST_ENTRY, b, -1, 0, 0, 0, 0, 0ull, zero4, zero4};
                psrc = nullptr;
                pbytes = 0;
            }
            pend.flags |= F_LAST_BATCH | (first ? F_FIRST_BATCH : 0);
            if (!(ok = emit(pend, psrc, pbytes))) break;
        }
        if (ok) ok = emit(TileMeta{K_EXIT, 0, -1, -1, 0, 0, 0, 0, 0ull, zero4, zero4}, nullptr, 0);
        if (!ok) atomicExch(a.err, 1);
        // drain: the last phase of every stage this thread armed must complete
        uint32_t last = it;
        for (uint32_t j = (last > STAGES ? last - STAGES : 0); j < last; ++j)
            if (!mbar_wait(full0 + 8 * (j % STAGES), (j / STAGES) & 1u, wait_ns)) atomicExch(a.err, 1);
        return;
    }

    // --------------------------------------------------------------- consumers
    // Per target: a1 sums one run (a grid row of n+1 points or a block of <= 8
    // sources) and is added to a2 only if the target uses the entry; a2 holds
    // <= 8 runs, a3 <= 8 a2's, and every 64 runs a3 goes into the FP64 sum.
    // eps-derived constants come precomputed in the kernel parameters: rebuilt
    // from eps inside the loops they would cost FP64 multiplies and conversions
    const R e2 = MIXED ? (R)a.ecf[0] : (R)a.e2d, e4 = MIXED ? (R)a.ecf[1] : (R)a.e4d;
    R X[TPL][3], XL[TPL][3], XO[TPL][3];
    double acc[TPL][WOUT];
    R a1[TPL][WOUT], a2[TPL][WOUT], a3[TPL][WOUT];
    constexpr bool PRUN = PAIR && (KITC_PACKED_RUNS || ROT);  // the rotlet path always packs
    float2 a2p[TPL][WOUT];  // PRUN: second level of packed run sums
    int c2 = 0, c3 = 0;
    dvec4 cB = make_dvec4(0, 0, 0, 0);
    double xd[TPL][3];
    R *gs = reinterpret_cast<R *>(gridc + (size_t)warp * 3 * (KITC_MAX_DEGREE + 1));
    float *gsf = reinterpret_cast<float *>(gridc + (size_t)warp * 3 * (KITC_MAX_DEGREE + 1));
    float2 Xh2[TPL][3], Xl2[TPL][3];
    const float2 e22 = bc2(a.ecf[0]);
    // rotlet (times 8 pi): Q/2 = ri3 + 1.5 eps^2 ri5, D2/4 = ri5 (1.5 + 3.75 eps^2 ri2),
    // D1/4 = ri3 (-0.5 + ri2 (-0.75 eps^2 + 3.75 eps^4 ri2))
    const float2 cq = bc2(a.ecf[2]), cd2a = bc2(a.ecf[3]);
    const float2 cd1a = bc2(a.ecf[4]);
    const float2 cd1b = bc2(a.ecf[5]);
    const float2 c15 = bc2(1.5f), cm05 = bc2(-0.5f), m1 = bc2(-1.f);
    uint32_t it = 0, nbd = 0;
    int64_t bslot = 0;
    int bsize = 0;
#pragma unroll
    for (int t = 0; t < TPL; ++t)
#pragma unroll
        for (int c = 0; c < WOUT; ++c) acc[t][c] = 0.0, a1[t][c] = a2[t][c] = a3[t][c] = R(0);
#pragma unroll
    for (int t = 0; t < TPL; ++t)
#pragma unroll
        for (int c = 0; c < WOUT; ++c) a2p[t][c] = make_float2(0.f, 0.f);

    auto to_fp64 = [&]() {
#pragma unroll
        for (int t = 0; t < TPL; ++t)
#pragma unroll
            for (int c = 0; c < WOUT; ++c) {
                R p = R(0);
                if constexpr (PRUN) {
                    p = (R)(a2p[t][c].x + a2p[t][c].y);
                    a2p[t][c] = make_float2(0.f, 0.f);
                }
                if constexpr (SACC) {
                    const int i = (lane + 32 * t) * WOUT + c;
                    accs[i] += (double)(a3s[i] + (float)(a2[t][c] + p));
                    a3s[i] = 0.f;
                } else {
                    acc[t][c] += (double)(a3[t][c] + (a2[t][c] + p));
                }
                a2[t][c] = a3[t][c] = R(0);
            }
        c2 = c3 = 0;
    };
    auto step = [&](bool u0, bool u1) {
        if constexpr (MIXED) {
#pragma unroll
            for (int c = 0; c < WOUT; ++c) {
                a2[0][c] += u0 ? a1[0][c] : R(0);
                a1[0][c] = R(0);
                if constexpr (TPL > 1) {
                    a2[TPL - 1][c] += u1 ? a1[TPL - 1][c] : R(0);
                    a1[TPL - 1][c] = R(0);
                }
            }
            if (++c2 == 8) {
                c2 = 0;
#pragma unroll
                for (int t = 0; t < TPL; ++t)
#pragma unroll
                    for (int c = 0; c < WOUT; ++c) {
                        if constexpr (SACC) a3s[(lane + 32 * t) * WOUT + c] += (float)a2[t][c];
                        else a3[t][c] += a2[t][c];
                        a2[t][c] = R(0);
                    }
                if (++c3 == 8) to_fp64();
            }
        } else {
#pragma unroll
            for (int c = 0; c < WOUT; ++c) {
                acc[0][c] += u0 ? a1[0][c] : 0.0;
                a1[0][c] = 0.0;
                if constexpr (TPL > 1) {
                    acc[TPL - 1][c] += u1 ? a1[TPL - 1][c] : 0.0;
                    a1[TPL - 1][c] = 0.0;
                }
            }
        }
    };

    // PRUN: one run given as packed sums v0 (target lane) and v1 (target lane + 32;
    // not read with one target per lane)
    auto step2 = [&](bool u0, bool u1, const float2 *v0, const float2 *v1) {
#pragma unroll
        for (int c = 0; c < WOUT; ++c) {
            a2p[0][c] = u0 ? add2(a2p[0][c], v0[c]) : a2p[0][c];
            if constexpr (TPL > 1) a2p[TPL - 1][c] = u1 ? add2(a2p[TPL - 1][c], v1[c]) : a2p[TPL - 1][c];
        }
        if (++c2 == 8) {
            c2 = 0;
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < WOUT; ++c) {
                    const float h = a2p[t][c].x + a2p[t][c].y;
                    if constexpr (SACC) a3s[(lane + 32 * t) * WOUT + c] += h;
                    else a3[t][c] += (R)h;
                    a2p[t][c] = make_float2(0.f, 0.f);
                }
            if (++c3 == 8) to_fp64();
        }
    };

    // rotlet factors of a pair of points from rho^2: hQ = Q/2, qD1 = D1/4, qD2 = D2/4
    auto rot_factors = [&](float2 r2, float2 &hQ, float2 &qD1, float2 &qD2) {
        const float2 ri = make_float2(rsq<EPS0>(r2.x), rsq<EPS0>(r2.y));
        const float2 ri2 = mul2(ri, ri), ri3 = mul2(ri2, ri), ri5 = mul2(ri3, ri2);
        hQ = fma2(cq, ri5, ri3);
        qD2 = mul2(ri5, fma2(cd2a, ri2, c15));
        qD1 = mul2(ri3, fma2(fma2(cd1a, ri2, cd1b), ri2, cm05));
    };

    for (;;) {
        const int s = it % STAGES;
        if (!mbar_wait(full0 + 8 * s, (it / STAGES) & 1u, wait_ns)) {
            atomicExch(a.err, 1);
            break;
        }
        const TileMeta &mr = meta[s];
        const int kind = mr.kind, flags = mr.flags, batch = mr.batch, ta = mr.a, tb = mr.b;
        const int rot = mr.seq % NCW;  // depends on the batch only: results are deterministic
        const uint64_t mask = mr.mask;
        if (kind == K_EXIT) break;
        // far tiles: grid size of the tile's cluster
        const int np = mr.np, npair = (np + 1) / 2;
        const int row_bytes = PAIR ? npair * 32 : np * PREC;
        const unsigned char *tile = tiles + (size_t)s * TILE;
        const bool u0 = (mask >> lane) & 1ull, u1 = TPL > 1 && ((mask >> (lane + 32)) & 1ull);
        if (flags & F_FIRST_BATCH) {
            bslot = a.bstart ? (int64_t)a.bstart[batch] : (int64_t)batch * a.batch;
            bsize = a.bcount ? a.bcount[batch] : (int)min((int64_t)a.batch, a.nt - bslot);
            if (MIXED && a.bctr) cB = a.bctr[batch];
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                int i = lane + 32 * t;
                int64_t slot = bslot + i;
                int64_t sl = i < bsize ? slot : bslot;
                xd[t][0] = a.tx[sl * a.tstride];
                xd[t][1] = a.ty[sl * a.tstride];
                xd[t][2] = a.tz[sl * a.tstride];
                const double cb[3] = {cB.x, cB.y, cB.z};
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    if constexpr (MIXED) {
                        float h = __double2float_rn(xd[t][l]);
                        X[t][l] = h;
                        XL[t][l] = __double2float_rn(xd[t][l] - (double)h);
                        XO[t][l] = __double2float_rn(xd[t][l] - cb[l]);
                    } else {
                        X[t][l] = xd[t][l];
                        XL[t][l] = 0.0;
                        XO[t][l] = xd[t][l];
                    }
                }
#pragma unroll
                for (int c = 0; c < WOUT; ++c) {
                    acc[t][c] = 0.0;
                    if constexpr (SACC) {
                        accs[(lane + 32 * t) * WOUT + c] = 0.0;
                        a3s[(lane + 32 * t) * WOUT + c] = 0.f;
                    }
                }
                if constexpr (PAIR && !OFF) {
#pragma unroll
                    for (int l = 0; l < 3; ++l) {
                        Xh2[t][l] = bc2(X[t][l]);
                        Xl2[t][l] = bc2(XL[t][l]);
                    }
                }
            }
        }
        if constexpr (PAIR) {
            if (kind == K_FAR) {
                if (flags & F_FIRST_ENTRY) {
                    // grid points relative to the batch centre: x at gsf[0..], y at
                    // gsf[18..], -z at gsf[36..] (a missing odd point lies far away)
                    if constexpr (KITC_FAR_PROD) {
                        const float *cr = chebf + (np - 1) * (KITC_MAX_DEGREE + 1);
                        for (int q = lane; q < 3 * np; q += 32) {
                            const int l = q / np, k = q % np;
                            const float v = fmaf(mr.ghw[l], cr[k], mr.goff[l]);
                            gsf[18 * l + k] = l == 2 ? -v : v;
                        }
                    } else
                    for (int q = lane; q < 3 * np; q += 32) {
                        int l = q / np, k = q % np;
                        double lo_l = l == 0 ? mr.lo.x : (l == 1 ? mr.lo.y : mr.lo.z);
                        double hi_l = l == 0 ? mr.hi.x : (l == 1 ? mr.hi.y : mr.hi.z);
                        const double ck = a.chebt ? a.chebt[(np - 1) * (KITC_MAX_DEGREE + 1) + k] : a.cheb[k];
                        double sk = 0.5 * ((lo_l + hi_l) + ck * (hi_l - lo_l));
                        double cb_l = l == 0 ? cB.x : (l == 1 ? cB.y : cB.z);
                        float v = (float)(sk - cb_l);
                        gsf[18 * l + k] = l == 2 ? -v : v;
                    }
                    if (lane == 0 && (np & 1)) gsf[36 + np] = -1e18f;
                    __syncwarp();
                    if (ROT && (np & 1)) {  // row pairs: -z of each point on both lanes
                        for (int k = lane; k < np; k += 32) gsf[54 + 2 * k] = gsf[55 + 2 * k] = gsf[36 + k];
                        __syncwarp();
                    }
                }
                const int rows = (tb - ta) * np;
                // rows of the tile, split over the warps; the loop over the point
                // pairs of a row is unrolled for each (n+1)/2 so that the pairs'
                // z coordinates stay in registers for the whole tile
                auto far_rows = [&](auto npc) {
                    constexpr int NPAIR = decltype(npc)::value;
                    float2 ngz[NPAIR];
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) ngz[q] = *reinterpret_cast<const float2 *>(gsf + 36 + 2 * q);
                    int r = (warp + rot) % NCW;
                    int k1 = ta + r / np, k2 = r % np;  // advanced incrementally below
                    // a run is RPR rows of this warp (r, r + NCW, ...): one fold
                    // into the hierarchical sums per run
                    for (; r < rows; r += RPR * NCW) {
                        float2 ux[TPL], uy[TPL], uz[TPL];
#pragma unroll
                        for (int t = 0; t < TPL; ++t) ux[t] = uy[t] = uz[t] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int j = 0; j < RPR; ++j) {
                        if (j > 0 && r + j * NCW >= rows) break;  // uniform over the warp
                        const unsigned char *row = tile + (size_t)(r + j * NCW) * row_bytes;
                        float2 dx2[TPL], dy2[TPL], rxy2[TPL], z2[TPL], S[TPL];
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            const float dx = XO[t][0] - gsf[k1], dy = XO[t][1] - gsf[18 + k2];
                            dx2[t] = bc2(dx);
                            dy2[t] = bc2(dy);
                            rxy2[t] = bc2(fmaf(dx, dx, fmaf(dy, dy, (float)e2)));
                            z2[t] = bc2(XO[t][2]);
                            S[t] = make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < NPAIR; ++q) {
                            const float4 A = *reinterpret_cast<const float4 *>(row + q * 32);
                            const float4 B = *reinterpret_cast<const float4 *>(row + q * 32 + 16);
                            const float2 fx = make_float2(A.x, A.y), fy = make_float2(A.z, A.w);
                            const float2 fz = make_float2(B.x, B.y);
#pragma unroll
                            for (int t = 0; t < TPL; ++t) {
                                float2 dz = add2(z2[t], ngz[q]);
                                float2 r2 = fma2(dz, dz, rxy2[t]);
                                float2 ri = make_float2(rsq<EPS0>(r2.x), rsq<EPS0>(r2.y));
                                float2 ri3 = mul2(mul2(ri, ri), ri);
                                float2 H1 = fma2(e22, ri3, ri);
                                float2 fd = fma2(fx, dx2[t], fma2(fy, dy2[t], mul2(fz, dz)));
                                float2 sv = mul2(fd, ri3);
                                ux[t] = fma2(fx, H1, ux[t]);
                                uy[t] = fma2(fy, H1, uy[t]);
                                uz[t] = fma2(fz, H1, fma2(dz, sv, uz[t]));
                                S[t] = add2(S[t], sv);
                            }
                        }
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {  // the x and y parts of d s, summed over the row
                            ux[t] = fma2(dx2[t], S[t], ux[t]);
                            uy[t] = fma2(dy2[t], S[t], uy[t]);
                        }
                        k2 += NCW;
                        while (k2 >= np) {
                            k2 -= np;
                            ++k1;
                        }
                        }
                        if constexpr (PRUN) {
                            float2 v[TPL][3];
#pragma unroll
                            for (int t = 0; t < TPL; ++t) v[t][0] = ux[t], v[t][1] = uy[t], v[t][2] = uz[t];
                            step2(u0, u1, v[0], v[TPL - 1]);
                        } else {
#pragma unroll
                            for (int t = 0; t < TPL; ++t) {
                                a1[t][0] += ux[t].x + ux[t].y;
                                a1[t][1] += uy[t].x + uy[t].y;
                                a1[t][2] += uz[t].x + uz[t].y;
                            }
                            step(u0, u1);
                        }
                    }
                };
                // rotlet: one row per run.  With d = (dx, dy, dz_k) on a row, the
                // row needs per point only the sums S = sum hQ n, B = sum hQ dz n
                // (x, y), W = sum qD1 n, T = sum t, Z = sum t dz (t = (n.d) qD2):
                //   u = (B_y - dy S_z, dx S_z - B_x, dy S_x - dx S_y),
                //   w = (W_x + dx T, W_y + dy T, W_z + Z).
                auto far_rows_rot = [&](auto npc) {
                    constexpr int NPAIR = decltype(npc)::value;
                    float2 ngz[NPAIR];
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) ngz[q] = *reinterpret_cast<const float2 *>(gsf + 36 + 2 * q);
                    int r = (warp + rot) % NCW;
                    int k1 = ta + r / np, k2 = r % np;
                    for (; r < rows; r += NCW) {
                        const unsigned char *row = tile + (size_t)r * row_bytes;
                        float2 v[TPL][WOUT];
                        float dxs[TPL], dys[TPL];
                        float2 dx2[TPL], dy2[TPL], rxy2[TPL], z2[TPL];
                        float2 S0[TPL], S1[TPL], S2[TPL], B0[TPL], B1[TPL], W0[TPL], W1[TPL], W2[TPL], T[TPL], Z[TPL];
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            dxs[t] = XO[t][0] - gsf[k1];
                            dys[t] = XO[t][1] - gsf[18 + k2];
                            dx2[t] = bc2(dxs[t]);
                            dy2[t] = bc2(dys[t]);
                            rxy2[t] = bc2(fmaf(dxs[t], dxs[t], fmaf(dys[t], dys[t], (float)e2)));
                            z2[t] = bc2(XO[t][2]);
                            S0[t] = S1[t] = S2[t] = B0[t] = B1[t] = make_float2(0.f, 0.f);
                            W0[t] = W1[t] = W2[t] = T[t] = Z[t] = make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < NPAIR; ++q) {
                            const float4 A = *reinterpret_cast<const float4 *>(row + q * 32);
                            const float4 B = *reinterpret_cast<const float4 *>(row + q * 32 + 16);
                            const float2 nx = make_float2(A.x, A.y), ny = make_float2(A.z, A.w);
                            const float2 nz = make_float2(B.x, B.y);
#pragma unroll
                            for (int t = 0; t < TPL; ++t) {
                                const float2 dz = add2(z2[t], ngz[q]);
                                float2 hQ, qD1, qD2;
                                rot_factors(fma2(dz, dz, rxy2[t]), hQ, qD1, qD2);
                                const float2 nd = fma2(nx, dx2[t], fma2(ny, dy2[t], mul2(nz, dz)));
                                const float2 tt = mul2(nd, qD2);
                                S0[t] = fma2(hQ, nx, S0[t]);
                                S1[t] = fma2(hQ, ny, S1[t]);
                                S2[t] = fma2(hQ, nz, S2[t]);
                                const float2 hz = mul2(hQ, dz);
                                B0[t] = fma2(hz, nx, B0[t]);
                                B1[t] = fma2(hz, ny, B1[t]);
                                W0[t] = fma2(nx, qD1, W0[t]);
                                W1[t] = fma2(ny, qD1, W1[t]);
                                W2[t] = fma2(nz, qD1, W2[t]);
                                T[t] = add2(T[t], tt);
                                Z[t] = fma2(dz, tt, Z[t]);
                            }
                        }
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            v[t][0] = fma2(bc2(-dys[t]), S2[t], B1[t]);
                            v[t][1] = fma2(dx2[t], S2[t], mul2(m1, B0[t]));
                            v[t][2] = fma2(dy2[t], S0[t], mul2(bc2(-dxs[t]), S1[t]));
                            if constexpr (WOUT == 6) {
                                v[t][3] = fma2(dx2[t], T[t], W0[t]);
                                v[t][4] = fma2(dy2[t], T[t], W1[t]);
                                v[t][5] = add2(W2[t], Z[t]);
                            }
                        }
                        step2(u0, u1, v[0], v[TPL - 1]);
                        k2 += NCW;
                        while (k2 >= np) {
                            k2 -= np;
                            ++k1;
                        }
                    }
                };
                // Rotlet, odd n + 1: a record holds one k3 point of two
                // consecutive grid rows (row index k1 np + k2) on the two lanes,
                // the last row of the odd count paired with a zero-weight row
                // placed far away, instead of a padding point in every row.
                // Along a unit dx and dy stay constant per lane, so the row sums
                // fold per lane as above.  Unit u of the tile is rows 2 (ta + u)
                // and 2 (ta + u) + 1; a warp's units advance by NCW, its rows by
                // 2 NCW.  (The Stokeslet keeps its padded rows: at its
                // 96-register budget the second loop made the whole kernel slower.)
                auto unit_rows = [&](int k1, int k2, int t, float2 &dx2, float2 &dy2) {
                    int k2b = k2 + 1, k1b = k1;
                    if (k2b == np) {
                        k2b = 0;
                        ++k1b;
                    }
                    const bool pad = k1b >= np;
                    dx2 = make_float2(XO[t][0] - gsf[k1], pad ? 1e18f : XO[t][0] - gsf[k1b]);
                    dy2 = make_float2(XO[t][1] - gsf[18 + k2], pad ? 0.f : XO[t][1] - gsf[18 + k2b]);
                };
                auto far_rowpairs_rot = [&](auto npc) {
                    constexpr int NP = decltype(npc)::value;
                    const int units = tb - ta;
                    int u = (warp + rot) % NCW;
                    int k1 = (2 * (ta + u)) / NP, k2 = 2 * (ta + u) - k1 * NP;
                    for (; u < units; u += NCW) {
                        const unsigned char *row = tile + (size_t)u * (NP * 32);
                        float2 v[TPL][WOUT];
                        float2 dx2[TPL], dy2[TPL], rxy2[TPL], z2[TPL];
                        float2 S0[TPL], S1[TPL], S2[TPL], B0[TPL], B1[TPL], W0[TPL], W1[TPL], W2[TPL], T[TPL], Z[TPL];
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            unit_rows(k1, k2, t, dx2[t], dy2[t]);
                            rxy2[t] = fma2(dx2[t], dx2[t], fma2(dy2[t], dy2[t], e22));
                            z2[t] = bc2(XO[t][2]);
                            S0[t] = S1[t] = S2[t] = B0[t] = B1[t] = make_float2(0.f, 0.f);
                            W0[t] = W1[t] = W2[t] = T[t] = Z[t] = make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const float4 A = *reinterpret_cast<const float4 *>(row + q * 32);
                            const float4 B = *reinterpret_cast<const float4 *>(row + q * 32 + 16);
                            const float2 nx = make_float2(A.x, A.y), ny = make_float2(A.z, A.w);
                            const float2 nz = make_float2(B.x, B.y);
                            const float2 ngzq = *reinterpret_cast<const float2 *>(gsf + 54 + 2 * q);
#pragma unroll
                            for (int t = 0; t < TPL; ++t) {
                                const float2 dz = add2(z2[t], ngzq);
                                float2 hQ, qD1, qD2;
                                rot_factors(fma2(dz, dz, rxy2[t]), hQ, qD1, qD2);
                                const float2 nd = fma2(nx, dx2[t], fma2(ny, dy2[t], mul2(nz, dz)));
                                const float2 tt = mul2(nd, qD2);
                                S0[t] = fma2(hQ, nx, S0[t]);
                                S1[t] = fma2(hQ, ny, S1[t]);
                                S2[t] = fma2(hQ, nz, S2[t]);
                                const float2 hz = mul2(hQ, dz);
                                B0[t] = fma2(hz, nx, B0[t]);
                                B1[t] = fma2(hz, ny, B1[t]);
                                W0[t] = fma2(nx, qD1, W0[t]);
                                W1[t] = fma2(ny, qD1, W1[t]);
                                W2[t] = fma2(nz, qD1, W2[t]);
                                T[t] = add2(T[t], tt);
                                Z[t] = fma2(dz, tt, Z[t]);
                            }
                        }
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            v[t][0] = fma2(mul2(m1, dy2[t]), S2[t], B1[t]);
                            v[t][1] = fma2(dx2[t], S2[t], mul2(m1, B0[t]));
                            v[t][2] = fma2(dy2[t], S0[t], mul2(mul2(m1, dx2[t]), S1[t]));
                            if constexpr (WOUT == 6) {
                                v[t][3] = fma2(dx2[t], T[t], W0[t]);
                                v[t][4] = fma2(dy2[t], T[t], W1[t]);
                                v[t][5] = add2(W2[t], Z[t]);
                            }
                        }
                        step2(u0, u1, v[0], v[TPL - 1]);
                        k2 += 2 * NCW;
                        while (k2 >= NP) {
                            k2 -= NP;
                            ++k1;
                        }
                    }
                };
                auto far_any = [&](auto npc) {
                    if constexpr (ROT) far_rows_rot(npc);
                    else far_rows(npc);
                };
                bool done = false;
                if constexpr (ROT) {
                    if (np & 1) {
                        switch (np) {
                        case 3: far_rowpairs_rot(std::integral_constant<int, 3>{}); break;
                        case 5: far_rowpairs_rot(std::integral_constant<int, 5>{}); break;
                        case 7: far_rowpairs_rot(std::integral_constant<int, 7>{}); break;
                        case 9: far_rowpairs_rot(std::integral_constant<int, 9>{}); break;
                        case 11: far_rowpairs_rot(std::integral_constant<int, 11>{}); break;
                        case 13: far_rowpairs_rot(std::integral_constant<int, 13>{}); break;
                        case 15: far_rowpairs_rot(std::integral_constant<int, 15>{}); break;
                        default: far_rowpairs_rot(std::integral_constant<int, 17>{}); break;
                        }
                        done = true;
                    }
                }
                if (!done)
                switch (npair) {
                case 1: far_any(std::integral_constant<int, 1>{}); break;
                case 2: far_any(std::integral_constant<int, 2>{}); break;
                case 3: far_any(std::integral_constant<int, 3>{}); break;
                case 4: far_any(std::integral_constant<int, 4>{}); break;
                case 5: far_any(std::integral_constant<int, 5>{}); break;
                case 6: far_any(std::integral_constant<int, 6>{}); break;
                case 7: far_any(std::integral_constant<int, 7>{}); break;
                case 8: far_any(std::integral_constant<int, 8>{}); break;
                default: far_any(std::integral_constant<int, 9>{}); break;
                }
            } else {
                const int cnt = tb - ta;  // source pairs
                constexpr int NPBK = ROT ? NPB : KITC_NPB_S;  // source pairs per run
                const int nb4 = (cnt + NPBK - 1) / NPBK, nfull = cnt / NPBK;
                float2 ux[TPL], uy[TPL], uz[TPL];
                // OFF: the targets' offsets from the leaf centre, formed as the
                // records' offsets are
                float2 Xc2[TPL][3];
                if constexpr (OFF) {
#pragma unroll
                    for (int t = 0; t < TPL; ++t)
#pragma unroll
                        for (int l = 0; l < 3; ++l)
                            Xc2[t][l] = bc2(leaf_offset(X[t][l], XL[t][l], mr.goff[l], mr.ghw[l]));
                }
                // a record's source pair: the negated coordinates as they enter
                // x - y (leaf offsets, or hi and lo parts), and the weights
                auto load_pair = [&](const unsigned char *rec, float2 (&ny)[2][3], float2 (&w)[3]) {
                    const float4 A = *reinterpret_cast<const float4 *>(rec);
                    const float4 B = *reinterpret_cast<const float4 *>(rec + 16);
                    const float4 C = *reinterpret_cast<const float4 *>(rec + 32);
                    ny[0][0] = make_float2(A.x, A.y);
                    ny[0][1] = make_float2(A.z, A.w);
                    ny[0][2] = make_float2(B.x, B.y);
                    if constexpr (OFF) {
                        w[0] = make_float2(B.z, B.w);
                        w[1] = make_float2(C.x, C.y);
                        w[2] = make_float2(C.z, C.w);
                    } else {
                        const float4 D = *reinterpret_cast<const float4 *>(rec + 48);
                        const float4 E = *reinterpret_cast<const float4 *>(rec + 64);
                        ny[1][0] = make_float2(B.z, B.w);
                        ny[1][1] = make_float2(C.x, C.y);
                        ny[1][2] = make_float2(C.z, C.w);
                        w[0] = make_float2(D.x, D.y);
                        w[1] = make_float2(D.z, D.w);
                        w[2] = make_float2(E.x, E.y);
                    }
                };
                auto diff = [&](int t, int l, const float2 (&ny)[2][3]) -> float2 {
                    if constexpr (OFF) return add2(Xc2[t][l], ny[0][l]);
                    else return add2(add2(Xh2[t][l], ny[0][l]), add2(Xl2[t][l], ny[1][l]));
                };
                auto body = [&](int idx) {
                    float2 ny[2][3], fw[3];
                    load_pair(tile + (size_t)idx * PAIR_REC, ny, fw);
                    const float2 fx = fw[0], fy = fw[1], fz = fw[2];
#pragma unroll
                    for (int t = 0; t < TPL; ++t) {
                        float2 dx = diff(t, 0, ny);
                        float2 dy = diff(t, 1, ny);
                        float2 dz = diff(t, 2, ny);
                        float2 r2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e22)));
                        float2 ri = make_float2(rsq<EPS0>(r2.x), rsq<EPS0>(r2.y));
                        float2 ri3 = mul2(mul2(ri, ri), ri);
                        float2 H1 = fma2(e22, ri3, ri);
                        float2 fd = fma2(fx, dx, fma2(fy, dy, mul2(fz, dz)));
                        float2 sv = mul2(fd, ri3);
                        ux[t] = fma2(fx, H1, fma2(dx, sv, ux[t]));
                        uy[t] = fma2(fy, H1, fma2(dy, sv, uy[t]));
                        uz[t] = fma2(fz, H1, fma2(dz, sv, uz[t]));
                    }
                };
                // rotlet: u = hQ n x d as the positive (P) and negative (M)
                // products of the cross product, summed separately over a run
                float2 P[TPL][3], M[TPL][3], Wr[TPL][3];
                auto body_rot = [&](int idx) {
                    float2 nyc[2][3], nw[3];
                    load_pair(tile + (size_t)idx * PAIR_REC, nyc, nw);
                    const float2 nx = nw[0], ny = nw[1], nz = nw[2];
#pragma unroll
                    for (int t = 0; t < TPL; ++t) {
                        const float2 dx = diff(t, 0, nyc);
                        const float2 dy = diff(t, 1, nyc);
                        const float2 dz = diff(t, 2, nyc);
                        float2 hQ, qD1, qD2;
                        rot_factors(fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, e22))), hQ, qD1, qD2);
                        const float2 nd = fma2(nx, dx, fma2(ny, dy, mul2(nz, dz)));
                        const float2 tt = mul2(nd, qD2);
                        const float2 h0 = mul2(hQ, nx), h1 = mul2(hQ, ny), h2 = mul2(hQ, nz);
                        P[t][0] = fma2(h1, dz, P[t][0]);
                        M[t][0] = fma2(h2, dy, M[t][0]);
                        P[t][1] = fma2(h2, dx, P[t][1]);
                        M[t][1] = fma2(h0, dz, M[t][1]);
                        P[t][2] = fma2(h0, dy, P[t][2]);
                        M[t][2] = fma2(h1, dx, M[t][2]);
                        Wr[t][0] = fma2(nx, qD1, fma2(dx, tt, Wr[t][0]));
                        Wr[t][1] = fma2(ny, qD1, fma2(dy, tt, Wr[t][1]));
                        Wr[t][2] = fma2(nz, qD1, fma2(dz, tt, Wr[t][2]));
                    }
                };
                if constexpr (ROT) {
                    for (int blk = (warp + rot) % NCW; blk < nb4; blk += NCW) {
#pragma unroll
                        for (int t = 0; t < TPL; ++t)
#pragma unroll
                            for (int c = 0; c < 3; ++c) P[t][c] = M[t][c] = Wr[t][c] = make_float2(0.f, 0.f);
                        if (blk < nfull) {
#pragma unroll
                            for (int j = 0; j < NPB; ++j) body_rot(blk * NPB + j);
                        } else {
                            for (int idx = blk * NPB; idx < cnt; ++idx) body_rot(idx);
                        }
                        float2 v[TPL][WOUT];
#pragma unroll
                        for (int t = 0; t < TPL; ++t)
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                v[t][c] = fma2(m1, M[t][c], P[t][c]);
                                if constexpr (WOUT == 6) v[t][3 + c] = Wr[t][c];
                            }
                        step2(u0, u1, v[0], v[TPL - 1]);
                    }
                } else
                for (int blk = (warp + rot) % NCW; blk < nb4; blk += NCW) {
#pragma unroll
                    for (int t = 0; t < TPL; ++t) ux[t] = uy[t] = uz[t] = make_float2(0.f, 0.f);
                    if (blk < nfull) {
#pragma unroll
                        for (int j = 0; j < NPBK; ++j) body(blk * NPBK + j);
                    } else {
                        for (int idx = blk * NPBK; idx < cnt; ++idx) body(idx);
                    }
                    if constexpr (PRUN) {
                        float2 v[TPL][3];
#pragma unroll
                        for (int t = 0; t < TPL; ++t) v[t][0] = ux[t], v[t][1] = uy[t], v[t][2] = uz[t];
                        step2(u0, u1, v[0], v[TPL - 1]);
                    } else {
#pragma unroll
                        for (int t = 0; t < TPL; ++t) {
                            a1[t][0] += ux[t].x + ux[t].y;
                            a1[t][1] += uy[t].x + uy[t].y;
                            a1[t][2] += uz[t].x + uz[t].y;
                        }
                        step(u0, u1);
                    }
                }
            }
        } else if (kind == K_FAR) {
            if (flags & F_FIRST_ENTRY) {
                // mapped Chebyshev points of the cluster (Sec. 3 interval map);
                // FP32 runs take them relative to the batch centre
                for (int q = lane; q < 3 * np; q += 32) {
                    int l = q / np, k = q % np;
                    double lo_l = l == 0 ? mr.lo.x : (l == 1 ? mr.lo.y : mr.lo.z);
                    double hi_l = l == 0 ? mr.hi.x : (l == 1 ? mr.hi.y : mr.hi.z);
                    const double ck = a.chebt ? a.chebt[(np - 1) * (KITC_MAX_DEGREE + 1) + k] : a.cheb[k];
                        double sk = 0.5 * ((lo_l + hi_l) + ck * (hi_l - lo_l));
                    double cb_l = l == 0 ? cB.x : (l == 1 ? cB.y : cB.z);
                    gs[l * (KITC_MAX_DEGREE + 1) + k] = MIXED ? (R)(sk - cb_l) : (R)sk;
                }
                __syncwarp();
            }
            const R *gx = gs, *gy = gs + (KITC_MAX_DEGREE + 1), *gz = gs + 2 * (KITC_MAX_DEGREE + 1);
            const int rows = (tb - ta) * np;
            for (int r = (warp + rot) % NCW; r < rows; r += NCW) {
                const int k1 = ta + r / np, k2 = r % np;
                const unsigned char *row = tile + (size_t)r * np * PREC;
                R dx[TPL], dy[TPL], rxy[TPL];
#pragma unroll
                for (int t = 0; t < TPL; ++t) {
                    dx[t] = XO[t][0] - gx[k1];
                    dy[t] = XO[t][1] - gy[k2];
                    rxy[t] = fma(dx[t], dx[t], fma(dy[t], dy[t], e2));
                }
#pragma unroll 3
                for (int k3 = 0; k3 < np; ++k3) {
                    R f[WIN];
                    load_proxy<MIXED, WIN, R>(row + (size_t)k3 * PREC, f);
                    const R gzk = gz[k3];
#pragma unroll
                    for (int t = 0; t < TPL; ++t) {
                        if constexpr (K == KITC_TEST_POLY) {
                            pair_poly(xd[t], (double)gx[k1], (double)gy[k2], (double)gzk,
                                      reinterpret_cast<const double *>(f),
                                      reinterpret_cast<double *>(a1[t]));
                        } else {
                            R dz = XO[t][2] - gzk;
                            R r2 = fma(dz, dz, rxy[t]);
                            pair<K, EPS0, R>(dx[t], dy[t], dz, f, e2, e4, a1[t], r2);
                        }
                    }
                }
                step(u0, u1);
            }
        } else {
            const int cnt = tb - ta;
            const int nb8 = (cnt + 7) >> 3, nfull = cnt >> 3;
            auto body = [&](int idx) {
                R f[WIN], yh[3], yl[3];
                load_source<MIXED, WIN, R>(tile + (size_t)idx * SREC, yh, yl, f);
#pragma unroll
                for (int t = 0; t < TPL; ++t) {
                    if constexpr (K == KITC_TEST_POLY) {
                        pair_poly(xd[t], (double)yh[0], (double)yh[1], (double)yh[2],
                                  reinterpret_cast<const double *>(f),
                                  reinterpret_cast<double *>(a1[t]));
                    } else {
                        R dx, dy, dz;
                        if constexpr (MIXED) {
                            dx = (X[t][0] - yh[0]) + (XL[t][0] - yl[0]);
                            dy = (X[t][1] - yh[1]) + (XL[t][1] - yl[1]);
                            dz = (X[t][2] - yh[2]) + (XL[t][2] - yl[2]);
                        } else {
                            dx = X[t][0] - yh[0];
                            dy = X[t][1] - yh[1];
                            dz = X[t][2] - yh[2];
                        }
                        R r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e2)));
                        pair<K, EPS0, R>(dx, dy, dz, f, e2, e4, a1[t], r2);
                    }
                }
            };
            for (int blk = (warp + rot) % NCW; blk < nb8; blk += NCW) {
                if (blk < nfull) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) body(blk * 8 + j);
                } else {
                    for (int idx = blk * 8; idx < cnt; ++idx) body(idx);
                }
                step(u0, u1);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * s);
        ++it;
        if (flags & F_LAST_BATCH) {
            if constexpr (MIXED) to_fp64();
            // cross-warp sum: write partials, wait for all warps, add, write out
            if (!mbar_wait(rbr, (nbd & 1u) ^ 1u, wait_ns)) { atomicExch(a.err, 1); break; }
#pragma unroll
            for (int t = 0; t < TPL; ++t)
#pragma unroll
                for (int c = 0; c < WOUT; ++c)
                    red[((size_t)warp * KITC_MAX_BATCH + lane + 32 * t) * WOUT + c] =
                        SACC ? accs[(lane + 32 * t) * WOUT + c] : acc[t][c];
            __syncwarp();
            if (lane == 0) mbar_arrive(rbw);
            if (!mbar_wait(rbw, nbd & 1u, wait_ns)) { atomicExch(a.err, 1); break; }
            const double scale = (K == KITC_TEST_POLY) ? 1.0 : INV8PI;
            const int ne = bsize * WOUT;
            for (int e = warp * 32 + lane; e < ne; e += NCW * 32) {
                int i = e / WOUT, c = e % WOUT;
                int64_t slot = bslot + i;
                double v = 0.0;
#pragma unroll
                for (int q = 0; q < NCW; ++q) v += red[((size_t)q * KITC_MAX_BATCH + i) * WOUT + c];
                int64_t j = a.tperm ? (int64_t)a.tperm[slot] : slot;
                a.out[j * WOUT + c] = v * scale;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(rbr);
            ++nbd;
        }
    }
}

template <int K, bool MIXED, bool EPS0, int TPL, bool LEAF>
__global__ void __launch_bounds__(NTH, (MinBlocks<K, MIXED>::value)) k_eval(const EvalArgs a)
{
    eval_body<K, MIXED, EPS0, TPL, LEAF>(a);
}


// One thread waits on a barrier that is never completed; the bounded wait
// gives up after limit_ns and records the time-out.
__global__ void k_watchdog(unsigned long long limit_ns, int *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(b, 0, limit_ns)) atomicExch(err, 1);
}

template <int K, bool MIXED, bool EPS0>
kitc_status launch_k(const EvalArgs &a, cudaStream_t s)
{
    constexpr int WIN = KT<K>::WIN;
    int np = a.cdeg ? KITC_MAX_DEGREE + 1 : a.degree + 1;  // the largest grid of the launch
    constexpr bool PAIR = MIXED && (K == KITC_STOKESLET || K == KITC_ROTLET);
    if (a.cdeg && (!a.roff || !a.chebt)) return KITC_ERR_INVALID_ARG;
    size_t plane = PAIR ? (size_t)np * ((np + 1) / 2) * 32 : (size_t)np * np * Rec<MIXED, WIN>::PROXY;
    // one target per lane for batches of <= 32 (mixed Stokeslet)
    constexpr bool ONE = KITC_TPL1 && MIXED && K == KITC_STOKESLET;
    const bool one = ONE && a.batch <= 32;
    if (plane > (size_t)TILE) return KITC_ERR_INVALID_ARG;
    if (PAIR && a.near_off && !a.pbegin) return KITC_ERR_INVALID_ARG;
    // bulk copies need 16-byte aligned sources; records are multiples of 16 bytes
    if ((reinterpret_cast<uintptr_t>(a.src) & 15u) || (reinterpret_cast<uintptr_t>(a.proxy) & 15u))
        return KITC_ERR_INVALID_ARG;
    if (!a.src || (a.near_off && !a.proxy) || !a.out || !a.queue || !a.err)
        return KITC_ERR_INVALID_ARG;
    const size_t smem = Smem<K>::TOTAL;
    // leaf-offset near records: a tree's near field under KITC_MIXED_LEAF
    const bool leaf = PAIR && a.near_off && a.leaf;
    void (*kern)(const EvalArgs) = k_eval<K, MIXED, EPS0, 2, false>;
    if constexpr (PAIR) {
        if (leaf) kern = k_eval<K, MIXED, EPS0, 2, true>;
    }
    if constexpr (ONE) {
        if (one) kern = leaf ? k_eval<K, MIXED, EPS0, 1, true> : k_eval<K, MIXED, EPS0, 1, false>;
    }
    const int form = (one ? 1 : 0) + (leaf ? 2 : 0);
    static std::atomic<int> configured[4][64] = {};  // the attribute's value never changes
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !configured[form][dev].load()) {
        KITC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (dev >= 0 && dev < 64) configured[form][dev].store(1);
    }
    int sms = 0, occ = 0;
    KITC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    KITC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTH, smem));
    if (occ < 1) return KITC_ERR_CUDA;
    int64_t grid = std::min<int64_t>(a.nb, (int64_t)sms * occ);
    if (grid < 1) return KITC_OK;
    kitc_count_launch();
    kern<<<(unsigned)grid, NTH, smem, s>>>(a);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

template <int K, bool MIXED, bool EPS0>
kitc_status preload_k(size_t *lmem)
{
    cudaFuncAttributes at;
    KITC_CUDA(cudaFuncGetAttributes(&at, k_eval<K, MIXED, EPS0, 2, false>));
    *lmem = std::max(*lmem, (size_t)at.localSizeBytes);
    if constexpr (KITC_TPL1 && MIXED && K == KITC_STOKESLET) {
        KITC_CUDA(cudaFuncGetAttributes(&at, k_eval<K, MIXED, EPS0, 1, false>));
        *lmem = std::max(*lmem, (size_t)at.localSizeBytes);
        KITC_CUDA(cudaFuncGetAttributes(&at, k_eval<K, MIXED, EPS0, 1, true>));
        *lmem = std::max(*lmem, (size_t)at.localSizeBytes);
    }
    if constexpr (MIXED && (K == KITC_STOKESLET || K == KITC_ROTLET)) {
        KITC_CUDA(cudaFuncGetAttributes(&at, k_eval<K, MIXED, EPS0, 2, true>));
        *lmem = std::max(*lmem, (size_t)at.localSizeBytes);
    }
    return KITC_OK;
}

template <int K>
kitc_status preload_kernel(size_t *lmem)
{
    KITC_TRY((preload_k<K, true, true>(lmem)));
    KITC_TRY((preload_k<K, true, false>(lmem)));
    KITC_TRY((preload_k<K, false, true>(lmem)));
    return preload_k<K, false, false>(lmem);
}

template <int K, bool MIXED>
kitc_status launch_eps(const EvalArgs &a, cudaStream_t s)
{
    return a.eps == 0.0 ? launch_k<K, MIXED, true>(a, s) : launch_k<K, MIXED, false>(a, s);
}

}  // namespace

kitc_status watchdog_launch(unsigned long long limit_ns, int *err, cudaStream_t s)
{
    kitc_count_launch();
    k_watchdog<<<1, 32, 0, s>>>(limit_ns, err);
    KITC_CUDA(cudaGetLastError());
    return KITC_OK;
}

kitc_status evaluate_preload(size_t *lmem)
{
    KITC_TRY(preload_kernel<KITC_STOKESLET>(lmem));
    KITC_TRY(preload_kernel<KITC_ROTLET>(lmem));
    KITC_TRY(preload_kernel<KITC_STOKESLET_ROTLET>(lmem));
    return preload_k<KITC_TEST_POLY, false, false>(lmem);
}

kitc_status evaluate_launch(int kernel, bool mixed, const EvalArgs &a0, cudaStream_t s)
{
    EvalArgs a = a0;
    const double e2 = a.eps * a.eps;
    a.e2d = e2;
    a.e4d = e2 * e2;
    a.ecf[0] = (float)e2;
    a.ecf[1] = (float)(e2 * e2);
    a.ecf[2] = (float)(1.5 * e2);
    a.ecf[3] = (float)(3.75 * e2);
    a.ecf[4] = (float)(3.75 * e2 * e2);
    a.ecf[5] = (float)(-0.75 * e2);
    switch (kernel) {
    case KITC_STOKESLET:
        return mixed ? launch_eps<KITC_STOKESLET, true>(a, s) : launch_eps<KITC_STOKESLET, false>(a, s);
    case KITC_ROTLET:
        return mixed ? launch_eps<KITC_ROTLET, true>(a, s) : launch_eps<KITC_ROTLET, false>(a, s);
    case KITC_STOKESLET_ROTLET:
        return mixed ? launch_eps<KITC_STOKESLET_ROTLET, true>(a, s)
                     : launch_eps<KITC_STOKESLET_ROTLET, false>(a, s);
    case KITC_TEST_POLY:
        if (mixed) return KITC_ERR_INVALID_ARG;
        return launch_k<KITC_TEST_POLY, false, false>(a, s);
    default:
        return KITC_ERR_INVALID_ARG;
    }
}
