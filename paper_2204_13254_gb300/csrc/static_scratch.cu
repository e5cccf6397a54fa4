// dd_schur_apply_static: the interface-operator application of dd_schur_apply,
// but with its temporary vectors in a fixed, file-scope device array instead of
// the caller-bound workspace, so that a call allocates no device memory at all.
//
// Who needs this: code that runs where device allocation is not allowed or not
// safe -- for instance a caller inside a custom memory pool that must not grow,
// a callback or plugin that only receives pre-existing buffers, or a real-time
// loop where a cudaMalloc would synchronise the device and stall other streams.
// Such callers still own the inputs (lam) and the outputs (out); only the
// scratch lives here.
//
// The array is kStaticScratchDoubles doubles (8 MiB) on every GPU that loads
// the library and stays resident until the process exits.  All calls on a
// device share it: two calls whose kernels overlap on the GPU (different
// streams, or different handles on concurrent streams) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dd_internal.h"

namespace {

constexpr size_t kStaticScratchDoubles = size_t(1) << 20;  // 8 MiB

__device__ __align__(256) double g_dd_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_dd_scratch on the current device, looked up once per
// device.  The host-side symbol is only a stand-in; kernels need this address.
// The cache is keyed by device ordinal, i.e. it assumes the CUDA runtime's
// primary context of that device (the one the runtime and torch use); a
// caller that makes another driver-API context current on the same device
// would receive an address that is not valid there.
cudaError_t scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&p, g_dd_scratch);
        if (rc != cudaSuccess) return rc;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

size_t round32(size_t n) { return (n + 31) / 32 * 32; }

}  // namespace

extern "C" int dd_schur_apply_static(dd_handle* h, const double* lam, double* out, void* stream) {
    if (!h || !lam || !out) return DD_ERR_ARG;
    if (h->members > 1)
        return h->fail(DD_ERR_STATE, "dd_schur_apply_static is not available for an ensemble (members > 1)");
    const size_t n_local = h->sub_ptr.empty() ? 0 : (size_t)h->sub_ptr.back();
    const size_t nc = h->corner_dof.size();
    const size_t need = round32(n_local) + 2 * round32(nc);
    if (need > kStaticScratchDoubles)
        return h->fail(DD_ERR_ARG, "dd_schur_apply_static: problem needs " + std::to_string(need) +
                                       " scratch doubles (local unknowns + 2 x corners, each rounded up to 32); the "
                                       "static limit is " + std::to_string(kStaticScratchDoubles));
    if (!h->factored) return h->fail(DD_ERR_STATE, "dd_schur_apply_static before dd_factor");
    if (h->factored_scheme != DD_SCHEME_DP1)
        return h->fail(DD_ERR_STATE, "dd_schur_apply_static needs the DP1 factorisation");
    if (h->mult_dof.empty()) return DD_OK;
    int dev = 0;
    cudaError_t rc = cudaGetDevice(&dev);
    if (rc != cudaSuccess) return h->fail(DD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(rc));
    if (dev < 0 || dev >= kMaxDevices)
        return h->fail(DD_ERR_CUDA, "dd_schur_apply_static: device ordinal " + std::to_string(dev) + " >= " +
                                        std::to_string(kMaxDevices) + " is not supported");
    double* base = nullptr;
    rc = scratch_address(dev, &base);
    if (rc != cudaSuccess) return h->fail(DD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(rc));
    double* w = base;                       // per-slot operator pieces
    double* uC = base + round32(n_local);   // assembled corner vector
    double* vC = uC + round32(nc);          // K~cc^-1 uC
    // Every slot that is read below is written first in the same call, so the
    // previous call's contents need no clearing.
    const bool has_c = nc > 0;
    XSrc xs{};
    GemvOut go{};
    int e = 0;
    if (has_c) {
        xs = XSrc{};
        xs.kind = X_LAMBDA;
        xs.v = lam;
        go = GemvOut{w, nullptr, nullptr, nullptr, 1.0};
        e = launch_gemv(h, GEMV_SCHUR_C, DD_FP64, xs, go, false, stream);
        if (!e) e = launch_corner_gather(h, w, nullptr, nullptr, uC, nullptr, false, stream);
        if (!e) {
            xs = XSrc{};
            xs.kind = X_FLAT;
            xs.v = uC;
            go = GemvOut{vC, nullptr, nullptr, nullptr, 1.0};
            e = launch_gemv(h, GEMV_COARSE, DD_FP64, xs, go, false, stream);
        }
    }
    if (!e) {
        xs = XSrc{};
        xs.kind = X_LAMBDA_CV;
        xs.v = lam;
        xs.v3 = vC;
        go = GemvOut{w, nullptr, nullptr, nullptr, 1.0};
        e = launch_gemv(h, GEMV_SCHUR_G, DD_FP64, xs, go, false, stream);
    }
    if (!e) e = launch_jump(h, w, nullptr, nullptr, 1.0, out, stream);
    if (e) return h->fail(DD_ERR_CUDA, std::string("dd_schur_apply_static: ") + cudaGetErrorString((cudaError_t)e));
    return DD_OK;
}
