// kitc_direct_noalloc: the direct sum of kitc_direct for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates): a
// latency-critical loop where an allocation may stall or fail, an embedding
// whose own allocator owns all of the device's memory, or error handling that
// runs when memory is already exhausted.  This entry point keeps its scratch --
// the work counter and error flag and the packed source records -- in one
// file-scope device array of fixed size instead, so it needs only the caller's
// inputs and outputs.
//
// Set-up.  With lazy module loading (the CUDA default) neither the array nor
// the kernels exist on a device until something touches them, and loading
// them allocates device memory.  The first call on a device therefore does the
// set-up, with that device current: it looks up the array's device address
// with cudaGetSymbolAddress and loads every kernel this entry point can launch
// (cudaFuncGetAttributes), so that no later call loads anything.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace {

// 8 MiB, 256-byte aligned; it exists on a device from the set-up of that
// device until the process exits.  Layout: [0, 16) work counter + error flag
// (zeroed by every call), [256, ...) source records.
constexpr size_t SCRATCH_BYTES = (size_t)8 << 20;
constexpr size_t RECORDS_AT = 256;
constexpr int64_t MAX_SOURCES = 100000;  // 100000 * 80 B (the widest record) + 256 <= 8 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device, set by the set-up of that device.
void *g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// The set-up of the current device (once per device and process); returns the
// device address of g_scratch.  In host code g_scratch names a host-side
// stand-in, never the device array, so only this address goes to the kernels.
kitc_status device_setup(void **out)
{
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return KITC_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return kitc_from_cuda(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        size_t lmem = 0;
        KITC_TRY(evaluate_preload(&lmem));
        KITC_TRY(pack_direct_preload(&lmem));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return KITC_OK;
}

}  // namespace

extern "C" kitc_status kitc_direct_noalloc(const double *tgt_xyz, int64_t n_tgt,
                                           const double *src_xyz, const double *w, int64_t n_src,
                                           const kitc_params *p, double *out, void *stream)
{
    if (!valid_direct_params(p) || !valid_count(n_tgt) || n_src < 1) return KITC_ERR_INVALID_ARG;
    if (n_src > MAX_SOURCES) return KITC_ERR_TOO_LARGE;
    if (!device_accessible(tgt_xyz) || !device_accessible(src_xyz) || !device_accessible(w) ||
        !device_accessible(out))
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool mixed = is_mixed(p->precision);
    const bool pairs = uses_pair_records(p->kernel, mixed);
    const int win = kitc_kernel_win(p->kernel);
    if (RECORDS_AT + direct_record_bytes(n_src, win, mixed, pairs) > SCRATCH_BYTES)
        return KITC_ERR_TOO_LARGE;
    void *base = nullptr;
    KITC_TRY(device_setup(&base));
    unsigned char *sc = static_cast<unsigned char *>(base);
    int *flags = reinterpret_cast<int *>(sc);
    void *records = sc + RECORDS_AT;
    KITC_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    KITC_TRY(pack_direct_records(src_xyz, w, n_src, win, mixed, pairs, records, s));
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
