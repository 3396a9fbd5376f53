// sfde_step_batch_noalloc: the batched fine step without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree from inside this library, e.g. an
// application whose device memory is owned by another allocator (a framework's caching allocator
// holds the pool, so an extra cudaMalloc can fail or force that allocator to release its cache),
// or a latency-critical loop in which cudaFree would synchronise the whole device and stall other
// streams.  sfde_step_batch allocates its padded staging buffers and step workspace on every call;
// this variant uses one fixed, file-scope device array instead.
//
// The array lives in every GPU that loads this library until the process exits.  Host code may not
// use the symbol itself as a device pointer (it names a host-side shadow), so the device address is
// looked up once per device with cudaGetSymbolAddress, on the first call made while that device is
// current, and cached.  That first call should therefore be made before any stream capture.  A call
// must be made with the context's own device current (checked), and a call that fails with a CUDA
// error drops the cached address (a device reset would move the array).
#include <mutex>

#include "sfde_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[SFDE_NOALLOC_SCRATCH_DOUBLES];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// The array's device address on device `dev`, looked up once (with that device current) and cached.
sfde_status scratch_on_device(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return SFDE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        SFDE_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return SFDE_OK;
}

// Forget a device's cached address (after a failed call: the next call looks it up again).
void forget_scratch(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    g_scratch_addr[dev] = nullptr;
}

sfde_status step_batch_noalloc_impl(sfde_ctx* c, int n0, int dn, int batch, const double* in, double* out) {
    if (!c || !in || !out || batch < 1) return SFDE_EINVAL;
    if (c->op_kind != SFDE_OP_TENSOR) return SFDE_EUNSUPPORTED;   // the P1 step's CG needs a workspace
    const long long last = (long long)n0 + (long long)(batch - 1) * dn;
    if (n0 < 1 || n0 > c->nt || last < 1 || last > c->nt) return SFDE_EINVAL;
    // the scratch address is per device: the context's device must be the current one, or the
    // kernels on the context's stream would be handed another GPU's array
    int dev = -1;
    SFDE_CUDA(cudaGetDevice(&dev));
    if (dev != c->device) return SFDE_EINVAL;
    if (!sfde_is_device_ptr(in) || !sfde_is_device_ptr(out)) return SFDE_EINVAL;
    const size_t P2 = c->P2();
    // padded input, three intermediate products, padded output
    if ((size_t)batch * P2 * 5 > (size_t)SFDE_NOALLOC_SCRATCH_DOUBLES) return SFDE_ESCRATCH;
    double* s = nullptr;
    SFDE_TRY(scratch_on_device(dev, &s));
    double* pin = s;
    double* T1 = pin + (size_t)batch * P2;
    double* T2 = T1 + (size_t)batch * P2;
    double* T3 = T2 + (size_t)batch * P2;
    double* pout = T3 + (size_t)batch * P2;
    // every scratch element read below is written first in this call (the padding included),
    // so nothing left from an earlier call leaks into the result
    sfde_launch_pad(in, pin, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
    StepBatch sb{};
    sb.batch = batch;
    sb.src = pin; sb.src_stride = (long long)P2;
    sb.dst = pout; sb.dst_stride = (long long)P2;
    sb.dt = c->dt0; sb.n0 = n0; sb.dn = dn; sb.scheme = SCHEME_CN; sb.level0 = true;
    sfde_status st = sfde_step_fp64_into(c, sb, T1, T2, T3);
    if (st == SFDE_OK) {
        sfde_launch_unpad(pout, out, c->y.n, c->x.n, c->y.P, c->x.P, batch, c->stream);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            sfde_set_last_cuda_error(e, "sfde_step_batch_noalloc", __FILE__, __LINE__);
            st = SFDE_ECUDA;
        }
    }
    if (st == SFDE_ECUDA) forget_scratch(dev);
    return st;
}

}  // namespace

extern "C" sfde_status sfde_step_batch_noalloc(sfde_ctx* c, int n0, int dn, int batch, const double* in,
                                               double* out) {
    return sfde_no_throw([&] { return step_batch_noalloc_impl(c, n0, dn, batch, in, out); });
}
