// Allocation-free reconstruction T = T~ + T^ at caller-provided device
// points.
//
// Who needs it: callers that must not call cudaMalloc or cudaFree while they
// run, for example a monitoring hook inside a time-critical control loop
// (an allocation can block on a device-wide synchronisation and makes the
// call's latency unpredictable), or code embedded in a framework whose
// caching allocator already owns the free device memory (a raw cudaMalloc
// there either fails or fragments the pool).  sa_eval_T may allocate on its
// first call and when the point count grows; this variant never does.
//
// Its per-call working memory (the FP64 temperature coefficients of the
// current step's sources and the element centres used for the Newton start)
// lives in one file-scope __device__ array of fixed size, shared by every
// call and every context in the process.  Each device that loads the library
// holds the array until the process exits.
//
// The evaluation runs in FP64 in every context (FP64 source coefficients,
// FP64 Newton inversion and sums).  In an FP64 context it equals sa_eval_T
// to rounding; in an SA_MIXED context, whose sa_eval_T sums the sources in
// FP32, the two agree within the mixed tolerance (1e-4 relative, 0.05 K).
#include <mutex>

#include "sa_internal.h"

namespace {

constexpr size_t kSrcBytes = (size_t)SA_NOALLOC_MAX_SOURCES * sizeof(double4);
constexpr size_t kElemBytes = (size_t)SA_NOALLOC_MAX_ELEMENTS * 3 * sizeof(double);
constexpr size_t kScratchBytes = kSrcBytes + kElemBytes;   // 5 MiB

// In host code this name is only a host-side stand-in; the device address is
// obtained with cudaGetSymbolAddress below and passed to the kernels.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array.
cudaError_t scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = (unsigned char*)g_addr[dev];
    return cudaSuccess;
}

struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t enter(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != dev) {
            e = cudaSetDevice(dev);
            if (e != cudaSuccess) return e;
            switched = true;
        }
        return cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" sa_status sa_eval_T_noalloc(sa_ctx* c, const double* d_pts, int n, double* d_T_out) {
    if (!c) return SA_ERR_ARG;
    if (c->poisoned) return sa_fail(c, SA_ERR_STATE, "context poisoned by an earlier CUDA error");
    if (n < 0 || (n > 0 && (!d_pts || !d_T_out))) return sa_fail(c, SA_ERR_ARG, "bad argument");
    if (!c->has_patch || !c->has_material || !c->state_init)
        return sa_fail(c, SA_ERR_STATE,
                       "sa_eval_T_noalloc needs a context that has stepped (or had its state set)");
    if (c->n_elem > SA_NOALLOC_MAX_ELEMENTS)
        return sa_fail(c, SA_ERR_ARG, "sa_eval_T_noalloc: %d elements exceed the limit of %d",
                       c->n_elem, SA_NOALLOC_MAX_ELEMENTS);
    if (c->n_src > SA_NOALLOC_MAX_SOURCES)
        return sa_fail(c, SA_ERR_ARG, "sa_eval_T_noalloc: %d sources exceed the limit of %d",
                       c->n_src, SA_NOALLOC_MAX_SOURCES);
    if (n == 0) return SA_OK;
    DeviceGuard guard;
    cudaError_t e = guard.enter(c->device);
    if (e != cudaSuccess) return sa_fail(c, SA_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    unsigned char* base = nullptr;
    e = scratch_address(c->device, &base);
    if (e != cudaSuccess)
        return sa_fail(c, SA_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    double4* evT = (double4*)base;                  // the flux table is not needed here
    double* ecent = (double*)(base + kSrcBytes);
    cudaStream_t s = c->stream;
    e = launch_elem_centers(c->dp, ecent, s);
    if (e != cudaSuccess) return sa_cuda_fail(c, e, "element centres (no-alloc)");
    int n_active = 0;
    if (c->has_scan && c->src_dt > 0.0 && c->n_step > 0 && c->n_src > 0) {
        const double alpha = c->k / (c->rho * c->cp);
        e = launch_prologue(nullptr, c->n_step, nullptr, c->n_src, c->src_pos.p, c->src_dt, alpha,
                            c->spot_radius * c->spot_radius / (8.0 * alpha),
                            c->opt.half_space_factor * c->E / (c->rho * c->cp), SA_FP64, evT,
                            nullptr, nullptr, nullptr, s);
        if (e != cudaSuccess) return sa_cuda_fail(c, e, "prologue (no-alloc)");
        n_active = (int)(c->n_step < c->n_src ? c->n_step : c->n_src);
    }
    e = launch_eval_points(c->dp, d_pts, n, ecent, c->dperm.p, c->That.p, evT, n_active, c->x_ref,
                           c->y_ref, c->z_top, c->length_scale, d_T_out, s);
    if (e != cudaSuccess) return sa_cuda_fail(c, e, "eval (no-alloc)");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sa_cuda_fail(c, e, "eval (no-alloc) synchronize");
    return SA_OK;
}
