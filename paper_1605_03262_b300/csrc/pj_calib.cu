// Measurement kernels used by bench.py to put roofline denominators on the same box and clocks as
// the benchmark: FP64 FMA throughput, store-only HBM bandwidth, and the throughput of FP64 exp, log
// and division relative to FMA. Not part of the pyjac_b300 C ABI (separate libpjcalib.so).
#include <cuda_runtime.h>

#include <cstdint>

#include "pj_fastmath.cuh"

namespace {

constexpr int kChains = 8;

__global__ void dfma_chains(double *out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <int OP>
__global__ void func_chains(double *out, int iters, double seed) {
    double x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = seed + 1e-6 * (threadIdx.x + 32 * c);
    double acc = 0.0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v;
            if (OP == 0) v = exp(x[c]);
            else if (OP == 1) v = log(x[c]);
            else v = 1.0 / x[c];
            acc += v;
            x[c] = x[c] + 1e-9;
        }
    }
    if (acc == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void store_only(double2 *p, size_t n2) {
    size_t stride = size_t(gridDim.x) * blockDim.x;
    double2 z;
    z.x = 0.0;
    z.y = 0.0;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n2; i += stride) __stcs(p + i, z);
}

__global__ void fastmath_check(const double *x, int n, const pj::MathTables *tb, double *e_fast, double *e_lib,
                               double *l_fast, double *l_lib) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = x[i];
        e_fast[i] = pj::fast_exp(v, tb);
        e_lib[i] = exp(v);
        l_fast[i] = pj::fast_log(v, tb);
        l_lib[i] = log(v);
    }
}

int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

template <class F>
float time_ms(F &&launch, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();   // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / reps;
}

}  // namespace

extern "C" {

// FP64 FMA throughput in TFLOP/s (2 flops per FMA). Returns 0 on success.
__attribute__((visibility("default"))) int pjc_fp64_fma_tflops(int iters, double *tflops) {
    const int threads = 256, blocks = sms() * 8;
    double *out = nullptr;
    if (cudaMalloc(&out, size_t(threads) * blocks * sizeof(double)) != cudaSuccess) return -1;
    float ms = time_ms([&] { dfma_chains<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7); }, 3);
    cudaError_t e = cudaGetLastError();
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return -1;
    *tflops = 2.0 * kChains * double(iters) * threads * blocks / (ms * 1e-3) / 1e12;
    return 0;
}

// Throughput of FP64 exp (op 0), log (op 1) or reciprocal-division (op 2), in calls per second.
__attribute__((visibility("default"))) int pjc_fp64_func_rate(int op, int iters, double *calls_per_s) {
    const int threads = 256, blocks = sms() * 8;
    double *out = nullptr;
    if (op < 0 || op > 2) return -1;
    if (cudaMalloc(&out, size_t(threads) * blocks * sizeof(double)) != cudaSuccess) return -1;
    float ms = 0.f;
    if (op == 0) ms = time_ms([&] { func_chains<0><<<blocks, threads>>>(out, iters, 0.25); }, 3);
    if (op == 1) ms = time_ms([&] { func_chains<1><<<blocks, threads>>>(out, iters, 1.75); }, 3);
    if (op == 2) ms = time_ms([&] { func_chains<2><<<blocks, threads>>>(out, iters, 1.75); }, 3);
    cudaError_t e = cudaGetLastError();
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.f) return -1;
    *calls_per_s = 4.0 * double(iters) * threads * blocks / (ms * 1e-3);
    return 0;
}

// The table-driven exp/log of the Jacobian kernels next to CUDA's exp/log on device array x[n]
// (all pointers device pointers), for the accuracy test.
__attribute__((visibility("default"))) int pjc_fastmath_check(const double *x, int n, double *e_fast, double *e_lib,
                                                              double *l_fast, double *l_lib) {
    pj::MathTables h;
    pj::build_math_tables(h);
    pj::MathTables *d = nullptr;
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return -1;
    cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice);
    fastmath_check<<<sms() * 4, 256>>>(x, n, d, e_fast, e_lib, l_fast, l_lib);
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(d);
    return e == cudaSuccess ? 0 : -1;
}

// Store-only bandwidth (GB/s, bytes written) over a buffer of the given size.
__attribute__((visibility("default"))) int pjc_store_gbs(size_t bytes, double *gbs) {
    double2 *p = nullptr;
    bytes &= ~size_t(15);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return -1;
    const size_t n2 = bytes / 16;
    const int blocks = sms() * 8;
    float ms = time_ms([&] { store_only<<<blocks, 512>>>(p, n2); }, 5);
    cudaError_t e = cudaGetLastError();
    cudaFree(p);
    if (e != cudaSuccess || ms <= 0.f) return -1;
    *gbs = double(bytes) / (ms * 1e-3) / 1e9;
    return 0;
}

}  // extern "C"
