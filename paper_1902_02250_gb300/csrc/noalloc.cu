// kitc_direct_noalloc: the direct sum of kitc_direct for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates): a
// latency-critical loop where an allocation may stall or fail, an embedding
// whose own allocator owns all of the device's memory, or error handling that
// runs when memory is already exhausted.  This entry point keeps its scratch --
// the work counter and error flag, a small range descriptor and the packed
// source records -- in one file-scope device array of fixed size instead, so it
// needs only the caller's inputs and outputs.
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace {

// 8 MiB, 256-byte aligned, held by every GPU that loads the library until the
// process exits.  Layout: [0, 16) work counter + error flag (zeroed by every
// call), [64, 76) range descriptor, [256, ...) source records.
constexpr size_t SCRATCH_BYTES = (size_t)8 << 20;
constexpr size_t RECORDS_AT = 256;
constexpr int64_t MAX_SOURCES = 100000;  // 100000 * 80 B (the widest record) + 256 <= 8 MiB

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once with that device current.
void *g_scratch_addr[64] = {nullptr};
std::mutex g_scratch_mu;

kitc_status scratch_address(void **out)
{
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return KITC_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return kitc_from_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return KITC_OK;
}

bool readable_by_device(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
           at.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" kitc_status kitc_direct_noalloc(const double *tgt_xyz, int64_t n_tgt,
                                           const double *src_xyz, const double *w, int64_t n_src,
                                           const kitc_params *p, double *out, void *stream)
{
    if (!p || kitc_kernel_win(p->kernel) < 0 || !(p->eps >= 0.0) || !isfinite(p->eps) ||
        (p->precision != KITC_FP64 && p->precision != KITC_MIXED) || p->target_batch < 0 ||
        p->target_batch > KITC_MAX_BATCH ||
        (p->kernel == KITC_TEST_POLY && p->precision == KITC_MIXED))
        return KITC_ERR_INVALID_ARG;
    if (n_tgt < 1 || n_tgt > (int64_t)INT32_MAX - 1024 || n_src < 1) return KITC_ERR_INVALID_ARG;
    if (n_src > MAX_SOURCES) return KITC_ERR_TOO_LARGE;
    if (!readable_by_device(tgt_xyz) || !readable_by_device(src_xyz) || !readable_by_device(w) ||
        !readable_by_device(out))
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool mixed = p->precision == KITC_MIXED;
    const bool pairs = uses_pair_records(p->kernel, mixed);
    const int win = kitc_kernel_win(p->kernel);
    if (RECORDS_AT + direct_record_bytes(n_src, win, mixed, pairs) > SCRATCH_BYTES)
        return KITC_ERR_TOO_LARGE;
    void *base = nullptr;
    KITC_TRY(scratch_address(&base));
    unsigned char *sc = static_cast<unsigned char *>(base);
    int *flags = reinterpret_cast<int *>(sc);
    int32_t *range3 = reinterpret_cast<int32_t *>(sc + 64);
    void *records = sc + RECORDS_AT;
    KITC_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    KITC_TRY(pack_direct_records(src_xyz, w, n_src, win, mixed, pairs, range3, records, s));
    const int B = p->target_batch == 0 ? KITC_MAX_BATCH : p->target_batch;
    EvalArgs a{};
    a.tx = tgt_xyz;
    a.ty = tgt_xyz + 1;
    a.tz = tgt_xyz + 2;
    a.tstride = 3;
    a.nt = n_tgt;
    a.batch = B;
    a.nb = (n_tgt + B - 1) / B;
    a.direct_ns = n_src;
    a.src = records;
    a.degree = 1;
    cheb_cos_table(1, a.cheb);
    a.eps = p->eps;
    a.out = out;
    a.queue = flags;
    a.err = flags + 1;
    a.wait_ns = (unsigned long long)g_wait_limit_ms * 1000000ull;
    KITC_TRY(evaluate_launch(p->kernel, mixed, a, s));
    int err = 0;
    KITC_CUDA(cudaMemcpyAsync(&err, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return err ? KITC_ERR_TIMEOUT : KITC_OK;
}
