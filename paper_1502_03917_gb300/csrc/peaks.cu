// peaks.cu -- the roofs the library's kernels are measured against, taken on
// the device at hand with the library's own microbenchmarks (mg_device_peaks):
// the FP32 and FP64 fused multiply-add rates, the bandwidth of data resident
// in L2, and the HBM copy bandwidth.  Not part of the method.
#include <cuda_runtime.h>

#include <string>

#include "aaomg.h"
#include "errors.h"

namespace {

using aaomg::set_error;

constexpr int kChains = 8;  // independent accumulator chains per thread

// FP32: kChains pairs per thread, each step one packed FMA (two FMAs) per pair
__global__ void k_peak_fma32(float2* out, int iters, float seed) {
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = make_float2(seed + threadIdx.x + k, seed - k);
    const float2 m = make_float2(0.99999994f, 1.00000012f), c = make_float2(1e-7f, -1e-7f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s = __fadd2_rn(s, a[k]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64: kChains accumulators per thread, one FMA per step each
__global__ void k_peak_fma64(double* out, int iters, double seed) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + threadIdx.x + k;
    const double m = 0.9999999999999998, c = 1e-15;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// `passes` reads of a buffer small enough to stay in L2 (16-byte loads,
// consecutive threads on consecutive words)
__global__ void k_peak_read(const float4* __restrict__ buf, size_t n4, int passes, float* out) {
    float acc = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void k_peak_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n4) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) b[i] = a[i];
}

struct Scratch {
    void* p[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        for (void* q : p) cudaFree(q);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace

extern "C" int mg_device_peaks(double* fp32_tflops, double* fp64_tflops, double* l2_gbs, double* hbm_gbs) {
    if (!fp32_tflops || !fp64_tflops || !l2_gbs || !hbm_gbs) return set_error(AAOMG_ERR_BAD_ARG, "null output");
    int dev = 0, nsm = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev)) {
        cudaGetLastError();
        return set_error(AAOMG_ERR_NO_DEVICE, "no CUDA device");
    }
    Scratch S;
    const int threads = 256, blocks = nsm * 8;
    const size_t l2_bytes = (size_t)l2 / 4;              // a quarter of L2: resident on either die
    const size_t hbm_bytes = (size_t)1 << 31;            // 2 GB per copy buffer, far beyond L2
    if (cudaMalloc(&S.p[0], (size_t)blocks * threads * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&S.p[1], l2_bytes) != cudaSuccess || cudaMalloc(&S.p[2], hbm_bytes) != cudaSuccess ||
        cudaMalloc(&S.p[3], hbm_bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(AAOMG_ERR_OOM, "peak measurement buffers");
    }
    cudaEventCreate(&S.e0);
    cudaEventCreate(&S.e1);
    cudaMemset(S.p[1], 0, l2_bytes);
    cudaMemset(S.p[2], 0, hbm_bytes);
    auto timed = [&](auto launch, int reps) {
        launch();  // warm-up
        cudaEventRecord(S.e0);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(S.e1);
        cudaEventSynchronize(S.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, S.e0, S.e1);
        return (double)ms / reps;
    };
    const int it32 = 1 << 14, it64 = 1 << 10;
    const double t32 = timed([&] { k_peak_fma32<<<blocks, threads>>>((float2*)S.p[0], it32, 1.f); }, 5);
    const double t64 = timed([&] { k_peak_fma64<<<blocks, threads>>>((double*)S.p[0], it64, 1.0); }, 5);
    const int passes = 64;
    const double tl2 = timed([&] {
        k_peak_read<<<blocks, threads>>>((const float4*)S.p[1], l2_bytes / 16, passes, (float*)S.p[0]);
    }, 5);
    const double thbm = timed([&] {
        k_peak_copy<<<blocks, threads>>>((const float4*)S.p[2], (float4*)S.p[3], hbm_bytes / 16);
    }, 5);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AAOMG_ERR_CUDA, std::string("peak measurement: ") + cudaGetErrorString(e));
    const double nthreads = (double)blocks * threads;
    *fp32_tflops = nthreads * it32 * kChains * 4.0 / (t32 * 1e-3) / 1e12;  // 2 FMAs per packed step, 2 flops each
    *fp64_tflops = nthreads * it64 * kChains * 2.0 / (t64 * 1e-3) / 1e12;
    *l2_gbs = (double)l2_bytes * passes / (tl2 * 1e-3) / 1e9;
    *hbm_gbs = 2.0 * (double)hbm_bytes / (thbm * 1e-3) / 1e9;
    return AAOMG_OK;
}
