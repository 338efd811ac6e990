// ptsne_gradient_static: the exact gradient of one chunk (the per-row pass of
// k_grad.cu followed by the reduction of Z) without any device allocation.
//
// Who needs it.  Every other entry point works on a context whose workspace
// ptsne_create obtains with cudaMalloc.  Some callers cannot do that: a host
// framework that owns the whole device memory pool and forbids allocations
// outside its own accounting, and callers that must not block, since
// cudaMalloc may synchronise the device.  Such a caller allocates its inputs
// and outputs itself and calls this function, which allocates nothing: its
// scratch (per-row partial sums) lives in a fixed array in the library's own
// device memory, loaded with the module.
//
// Scratch contract.
//  - g_static_scratch holds kStaticScratchBytes (1 MiB): per-row Z partials
//    (z doubles) followed by per-row accumulators A_i, R_i (z x 2 x out_dim
//    floats), enough for PTSNE_STATIC_MAX_ROWS rows at out_dim 3.
//  - Its device address is looked up with cudaGetSymbolAddress once per
//    device, on the first call made while that device is current (that first
//    lookup may load the module).  The address is cached together with the identity of the CUDA context it
//    was taken in; when the device's context has been destroyed and created
//    again (cudaDeviceReset), the module may load at another address, so the
//    next call sees the new context and looks the address up again.
//  - Every call on a device shares the one array.  Calls whose kernels can
//    overlap on the GPU (different streams, or several host threads without
//    ordering) race on it and give wrong results; calls in one stream are
//    ordered and safe.
//  - Every scratch word a call reads is written earlier by the same call, so
//    nothing has to be cleared between calls.
#include <cuda.h>   // CUcontext / CUresult types of the two driver calls fetched below

#include <mutex>

#include "ptsne_internal.cuh"

namespace {

constexpr int kStaticMaxRows = PTSNE_STATIC_MAX_ROWS;
constexpr size_t kZBytes = sizeof(double) * kStaticMaxRows;                   // 256 KiB
constexpr size_t kAccBytes = sizeof(float) * 2 * 3 * kStaticMaxRows;          // 768 KiB
constexpr size_t kStaticScratchBytes = kZBytes + kAccBytes;                   // 1 MiB
constexpr int kMaxDevices = 64;
constexpr int kRowWarps = 8;
constexpr int kFinalThreads = 1024;

// Per device: the scratch address, the context it belongs to and the SM count.
struct ScratchSlot {
    unsigned long long ctx_id;   // 0: not looked up yet
    void* ptr;
    int sms;
};
std::mutex g_scratch_mu;
ScratchSlot g_slot[kMaxDevices];

// Unique id of the calling thread's current CUDA context (the driver's
// cuCtxGetCurrent and cuCtxGetId, fetched through the runtime so that the
// library does not link the driver library itself).  0 if unavailable.
unsigned long long current_ctx_id() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    typedef CUresult (*GetId)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
        tried = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

using ptsne::hw_rcp;
using ptsne::warp_sum;

// Per-row pass of one chunk: for row i the warp accumulates
//   A_i = sum_j p_ij w_ij (y_i - y_j),  R_i = sum_j w_ij^2 (y_i - y_j),
//   Z_i = sum_{j != i} w_ij,            w_ij = (1 + ||y_i - y_j||^2)^-1
// (the same sums as grad_rows_kernel), reading P row i with stride ld.
template <int OD>
__global__ void __launch_bounds__(kRowWarps * 32)
grad_rows_static_kernel(const float* __restrict__ P, int64_t ld, const float* __restrict__ Y, int z,
                        float* __restrict__ acc, double* __restrict__ rowz) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = blockIdx.x * kRowWarps + warp; i < z; i += gridDim.x * kRowWarps) {
        const float* prow = P + (int64_t)i * ld;
        float yi[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) yi[k] = Y[(int64_t)i * OD + k];
        float a[OD], r[OD], zs = 0.f;
#pragma unroll
        for (int k = 0; k < OD; ++k) { a[k] = 0.f; r[k] = 0.f; }
        for (int j = lane; j < z; j += 32) {
            if (j == i) continue;
            float dx[OD];
            float q = 1.0f;
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                dx[k] = yi[k] - Y[(int64_t)j * OD + k];
                q = fmaf(dx[k], dx[k], q);
            }
            const float w = hw_rcp(q);
            zs += w;
            const float pw = prow[j] * w, w2 = w * w;
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                a[k] = fmaf(pw, dx[k], a[k]);
                r[k] = fmaf(w2, dx[k], r[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < OD; ++k) {
            a[k] = warp_sum(a[k]);
            r[k] = warp_sum(r[k]);
        }
        const double zr = warp_sum((double)zs);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                acc[(int64_t)i * 2 * OD + k] = a[k];
                acc[(int64_t)i * 2 * OD + OD + k] = r[k];
            }
            rowz[i] = zr;
        }
    }
}

// Z = sum_i Z_i in FP64 (fixed order), then dC/dy_i = 4 (A_i - R_i / Z) (Eq. 6).
template <int OD>
__global__ void __launch_bounds__(kFinalThreads)
grad_final_static_kernel(const float* __restrict__ acc, const double* __restrict__ rowz, int z,
                         float* __restrict__ grad, double* __restrict__ Z_out) {
    __shared__ double part[kFinalThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s = 0.0;
    for (int i = threadIdx.x; i < z; i += kFinalThreads) s += rowz[i];
    s = warp_sum(s);
    if (lane == 0) part[warp] = s;
    __syncthreads();
    double Z = 0.0;
#pragma unroll 1
    for (int w = 0; w < kFinalThreads / 32; ++w) Z += part[w];
    if (threadIdx.x == 0 && Z_out) *Z_out = Z;
    const float invZ = (float)(1.0 / Z);
    for (int i = threadIdx.x; i < z; i += kFinalThreads) {
#pragma unroll
        for (int k = 0; k < OD; ++k)
            grad[(int64_t)i * OD + k] =
                4.0f * (acc[(int64_t)i * 2 * OD + k] - acc[(int64_t)i * 2 * OD + OD + k] * invZ);
    }
}

// Device address of g_static_scratch on the current device, and its SM count
// (looked up once per device and context; the runtime has made the device's
// primary context current by the time cudaGetSymbolAddress returns).
int static_scratch(unsigned char** out, int* sms_out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ptsne::set_last_error(cudaGetErrorString(e));
        return PTSNE_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        ptsne::set_last_error("ptsne_gradient_static: device ordinal beyond the supported 64 devices");
        return PTSNE_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& sl = g_slot[dev];
    const unsigned long long id = current_ctx_id();
    if (!sl.ptr || id == 0 || sl.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            ptsne::set_last_error(e != cudaSuccess ? cudaGetErrorString(e)
                                                   : "ptsne_gradient_static: scratch address lookup returned NULL");
            return PTSNE_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms < 1) {
            ptsne::set_last_error(e != cudaSuccess ? cudaGetErrorString(e)
                                                   : "ptsne_gradient_static: device reports no multiprocessors");
            return PTSNE_ECUDA;
        }
        sl.ptr = p;
        sl.sms = sms;
        sl.ctx_id = current_ctx_id();   // the lookup made the primary context current
    }
    *out = static_cast<unsigned char*>(sl.ptr);
    *sms_out = sl.sms;
    return PTSNE_OK;
}

}  // namespace

extern "C" int ptsne_gradient_static(const float* P_dev, int64_t ld, const float* Y_dev, int32_t z,
                                     int32_t out_dim, float* grad_out_dev, double* Z_out_dev, void* stream) {
    char msg[256];
    if (!P_dev || !Y_dev || !grad_out_dev) {
        ptsne::set_last_error("ptsne_gradient_static: P, Y and grad_out must be device pointers");
        return PTSNE_EINVAL;
    }
    if (out_dim != 2 && out_dim != 3) {
        snprintf(msg, sizeof msg, "ptsne_gradient_static: out_dim must be 2 or 3 (got %d)", (int)out_dim);
        ptsne::set_last_error(msg);
        return PTSNE_EINVAL;
    }
    if (z < 2 || z > kStaticMaxRows) {
        snprintf(msg, sizeof msg,
                 "ptsne_gradient_static: z = %d is outside [2, %d], the rows its fixed %zu-byte scratch holds",
                 (int)z, kStaticMaxRows, kStaticScratchBytes);
        ptsne::set_last_error(msg);
        return PTSNE_EINVAL;
    }
    if (ld < z) {
        snprintf(msg, sizeof msg, "ptsne_gradient_static: ld = %lld is smaller than z = %d", (long long)ld, (int)z);
        ptsne::set_last_error(msg);
        return PTSNE_EINVAL;
    }
    unsigned char* base = nullptr;
    int sms = 0;
    const int rc = static_scratch(&base, &sms);
    if (rc != PTSNE_OK) return rc;
    double* rowz = reinterpret_cast<double*>(base);
    float* acc = reinterpret_cast<float*>(base + kZBytes);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int blocks = (z + kRowWarps - 1) / kRowWarps;
    if (blocks > sms * 8) blocks = sms * 8;   // 8 blocks of 256 threads fill an SM
    if (out_dim == 2) {
        grad_rows_static_kernel<2><<<blocks, kRowWarps * 32, 0, s>>>(P_dev, ld, Y_dev, z, acc, rowz);
        grad_final_static_kernel<2><<<1, kFinalThreads, 0, s>>>(acc, rowz, z, grad_out_dev, Z_out_dev);
    } else {
        grad_rows_static_kernel<3><<<blocks, kRowWarps * 32, 0, s>>>(P_dev, ld, Y_dev, z, acc, rowz);
        grad_final_static_kernel<3><<<1, kFinalThreads, 0, s>>>(acc, rowz, z, grad_out_dev, Z_out_dev);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ptsne::set_last_error(cudaGetErrorString(e));
        return PTSNE_ECUDA;
    }
    return PTSNE_OK;
}
