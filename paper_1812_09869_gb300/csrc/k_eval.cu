// k-nearest-neighbour preservation of a map: for each query point q, the k
// nearest neighbours of q among the n input points (squared Euclidean
// distances of X rows, q itself excluded) and among the n map points (rows
// of Y), and the size of the overlap of the two sets.  It judges how well a
// map keeps the local structure of the data (the learned mapper's placement
// against ptSNE's own map).
//
// One block per query.  Each thread scans a strided share of the points with
// direct FP32 differences and keeps its own k best (distance, index) pairs in
// registers (insertion into a sorted list with compile-time positions); the
// block then sorts the threads' candidates in shared memory (bitonic sort of
// 64-bit keys: distance bits above the index, so ties go to the smaller
// index) and keeps the first k.  Distances are non-negative, so their float
// bits order like the values.
#include <float.h>
#include <stdio.h>

#include "ptsne_internal.cuh"

namespace {

constexpr int kKnnThreads = 256;
constexpr int kKnnMaxK = 32;

template <int K>
struct TopK {
    float d[K];
    int i[K];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int t = 0; t < K; ++t) { d[t] = FLT_MAX; i[t] = INT_MAX; }
    }
    __device__ __forceinline__ static bool less(float da, int ia, float db, int ib) {
        return da < db || (da == db && ia < ib);
    }
    // insert (dn, jn) if it is among the K best seen
    __device__ __forceinline__ void push(float dn, int jn) {
        if (!less(dn, jn, d[K - 1], i[K - 1])) return;
#pragma unroll
        for (int t = K - 1; t >= 0; --t) {
            const bool above = t > 0 && less(dn, jn, d[t - 1], i[t - 1]);   // the new pair goes above slot t
            if (less(dn, jn, d[t], i[t])) {
                d[t] = above ? d[t - 1] : dn;
                i[t] = above ? i[t - 1] : jn;
            }
        }
    }
};

// Sorts keys[0 .. kKnnThreads * K) ascending (bitonic network); the count is
// a power of two times the block size.
template <int N>
__device__ void block_bitonic(unsigned long long* keys) {
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long knn_key(float d, int i) {
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned int)i;
}

// The block's k nearest of point q among the n rows of A (dim columns),
// written to out[0 .. K) (indices), sorted by distance then index.
template <int K, int KP>
__device__ void block_knn(const float* __restrict__ A, int64_t n, int dim, int64_t q, unsigned long long* keys,
                          int* out) {
    TopK<K> top;
    top.clear();
    const float* aq = A + q * dim;
    for (int64_t j = threadIdx.x; j < n; j += kKnnThreads) {
        if (j == q) continue;
        const float* aj = A + j * dim;
        float s = 0.f;
        for (int k = 0; k < dim; ++k) {
            const float t = aq[k] - aj[k];
            s = fmaf(t, t, s);
        }
        top.push(s, (int)j);
    }
#pragma unroll
    for (int t = 0; t < KP; ++t)
        keys[threadIdx.x * KP + t] = t < K ? knn_key(top.d[t], top.i[t]) : ~0ull;
    block_bitonic<kKnnThreads * KP>(keys);
    if (threadIdx.x < K) out[threadIdx.x] = (int)(keys[threadIdx.x] & 0xffffffffu);
    __syncthreads();
}

template <int K, int KP>
__global__ void __launch_bounds__(kKnnThreads)
knn_overlap_kernel(const float* __restrict__ X, const float* __restrict__ Y, int64_t n, int d, int od,
                   const int32_t* __restrict__ queries, int k, int32_t* __restrict__ overlap,
                   int32_t* __restrict__ nbr_x, int32_t* __restrict__ nbr_y) {
    extern __shared__ unsigned long long keys[];   // kKnnThreads * KP
    __shared__ int sx[K], sy[K];
    const int qi = blockIdx.x;
    const int64_t q = queries[qi];
    if (q < 0 || q >= n) {   // a query outside [0, n) is reported, never dereferenced
        if (threadIdx.x == 0) overlap[qi] = -1;
        return;
    }
    block_knn<K, KP>(X, n, d, q, keys, sx);
    block_knn<K, KP>(Y, n, od, q, keys, sy);
    if (threadIdx.x < k) {
        if (nbr_x) nbr_x[(int64_t)qi * k + threadIdx.x] = sx[threadIdx.x];
        if (nbr_y) nbr_y[(int64_t)qi * k + threadIdx.x] = sy[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        int c = 0;
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) c += sx[a] == sy[b];
        overlap[qi] = c;
    }
}

template <int K, int KP>
cudaError_t launch_knn(const float* X, const float* Y, int64_t n, int d, int od, const int32_t* queries, int nq, int k,
                       int32_t* overlap, int32_t* nx, int32_t* ny, cudaStream_t s) {
    const size_t smem = sizeof(unsigned long long) * kKnnThreads * KP;
    cudaError_t e = cudaFuncSetAttribute(knn_overlap_kernel<K, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    knn_overlap_kernel<K, KP><<<(unsigned)nq, kKnnThreads, smem, s>>>(X, Y, n, d, od, queries, k, overlap, nx, ny);
    return cudaGetLastError();
}

}  // namespace

extern "C" int ptsne_knn_preservation(const float* X_dev, const float* Y_dev, int64_t n, int32_t d, int32_t od,
                                      const int32_t* queries_dev, int32_t nq, int32_t k, int32_t* overlap_out_dev,
                                      int32_t* nbr_x_out_dev, int32_t* nbr_y_out_dev, void* stream) {
    char msg[256];
    if (!X_dev || !Y_dev || !queries_dev || !overlap_out_dev) {
        ptsne::set_last_error("ptsne_knn_preservation: X, Y, queries and overlap_out must be device pointers");
        return PTSNE_EINVAL;
    }
    if (k < 1 || k > kKnnMaxK || n < (int64_t)k + 1 || n > 2147483647LL || d < 1 || d > 4096 || od < 1 ||
        od > 4096 || nq < 0) {
        snprintf(msg, sizeof msg,
                 "ptsne_knn_preservation: need 1 <= k <= %d, k < n < 2^31, 1 <= d, od <= 4096, nq >= 0 "
                 "(k %d, n %lld, d %d, od %d, nq %d)",
                 kKnnMaxK, (int)k, (long long)n, (int)d, (int)od, (int)nq);
        ptsne::set_last_error(msg);
        return PTSNE_EINVAL;
    }
    if (nq == 0) return PTSNE_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    // the per-thread list holds K >= k entries (power of two for the sort)
    if (k <= 8) e = launch_knn<8, 8>(X_dev, Y_dev, n, d, od, queries_dev, nq, k, overlap_out_dev, nbr_x_out_dev, nbr_y_out_dev, s);
    else if (k <= 16) e = launch_knn<16, 16>(X_dev, Y_dev, n, d, od, queries_dev, nq, k, overlap_out_dev, nbr_x_out_dev, nbr_y_out_dev, s);
    else e = launch_knn<32, 32>(X_dev, Y_dev, n, d, od, queries_dev, nq, k, overlap_out_dev, nbr_x_out_dev, nbr_y_out_dev, s);
    if (e != cudaSuccess) {
        ptsne::set_last_error(cudaGetErrorString(e));
        return PTSNE_ECUDA;
    }
    return PTSNE_OK;
}
