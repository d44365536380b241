// Arithmetic peaks and dependent-operation latencies of the GPU, measured by
// small kernels (no library calls).  They set the compute roofline of the
// wide-band path and the critical-path model of single long chains, whose
// per-row recurrence is a chain of dependent FMAs, a square root and a
// reciprocal.
//
// Throughput kernels: every thread runs 8 independent FMA chains (FP32 /
// FP64), or every warp issues independent mma.sync tiles (DMMA m8n8k4 FP64,
// TF32 m16n8k8), on a grid of 8 blocks per SM; the kernel time comes from
// CUDA events.  Latency kernels: one thread runs a chain of N dependent
// operations and reads clock64() around it.
//
// Output: one JSON object on stdout.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            std::fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            std::exit(1);                                                              \
        }                                                                              \
    } while (0)

constexpr int kChains = 8;

template <typename T>
__global__ void fma_throughput(T *out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// DMMA: D(8x8) = A(8x4) B(4x8) + C, FP64; each warp keeps 4 independent accumulators.
__global__ void dmma_throughput(double *out, int iters) {
    double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
    double d[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) { d[c][0] = 0.0; d[c][1] = 0.0; }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// TF32: D(16x8) = A(16x8) B(8x8) + C with FP32 accumulation.
__global__ void tf32_throughput(float *out, int iters) {
    unsigned a0 = 0x3f800000u, a1 = 0x3f800000u, a2 = 0x3f800000u, a3 = 0x3f800000u;
    unsigned b0 = 0x3f000000u, b1 = 0x3f000000u;
    float d[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[c][e] = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};\n"
                : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) s += d[c][e];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Dependent chains: op 0 FMA, 1 sqrt, 2 reciprocal square root, 3 division, 4 reciprocal.
template <typename T, int OP>
__global__ void latency(T *out, long long *cycles, int iters, T seed) {
    T x = seed;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (OP == 0) x = fma(x, T(0.999999), T(1e-7));
            if (OP == 1) x = sqrt(x) + T(0.5);
            if (OP == 2) x = rsqrt(x) + T(0.5);
            if (OP == 3) x = T(1.5) / x + T(0.25);
            if (OP == 4) x = T(1) / (x + T(0.25));
        }
    }
    const long long t1 = clock64();
    out[0] = x;
    cycles[0] = t1 - t0;
}

template <>
__global__ void latency<float, 2>(float *out, long long *cycles, int iters, float seed) {
    float x = seed;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) x = rsqrtf(x) + 0.5f;
    }
    const long long t1 = clock64();
    out[0] = x;
    cycles[0] = t1 - t0;
}

template <typename K>
static float time_kernel(K launch, int reps) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch();
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(a));
    for (int r = 0; r < reps; ++r) launch();
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    CK(cudaEventDestroy(a));
    CK(cudaEventDestroy(b));
    CK(cudaGetLastError());
    return ms / reps;
}

template <typename T, int OP>
static double cycles_per_op(T seed) {
    T *out;
    long long *cyc;
    CK(cudaMalloc(&out, sizeof(T)));
    CK(cudaMalloc(&cyc, sizeof(long long)));
    const int iters = 4096;
    latency<T, OP><<<1, 1>>>(out, cyc, 16, seed);          // warm-up
    latency<T, OP><<<1, 1>>>(out, cyc, iters, seed);
    CK(cudaGetLastError());
    long long c = 0;
    CK(cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost));
    CK(cudaFree(out));
    CK(cudaFree(cyc));
    return (double)c / (16.0 * iters);
}

int main() {
    int dev = 0, sms = 0, clk_khz = 0;
    CK(cudaSetDevice(dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    const int threads = 256, blocks = sms * 8;
    void *buf;
    CK(cudaMalloc(&buf, sizeof(double) * threads * blocks));

    const int it = 1 << 14;
    const float ms32 = time_kernel([&] { fma_throughput<float><<<blocks, threads>>>((float *)buf, it, 0.999f, 1e-3f); }, 5);
    const float ms64 = time_kernel([&] { fma_throughput<double><<<blocks, threads>>>((double *)buf, it / 8, 0.999, 1e-3); }, 3);
    const double fl32 = 2.0 * kChains * (double)it * threads * blocks / (ms32 * 1e-3);
    const double fl64 = 2.0 * kChains * (double)(it / 8) * threads * blocks / (ms64 * 1e-3);

    const int itd = 1 << 10;
    const float msd = time_kernel([&] { dmma_throughput<<<blocks, threads>>>((double *)buf, itd); }, 3);
    const double warps = (double)blocks * threads / 32.0;
    const double fld = warps * itd * 4 * (2.0 * 8 * 8 * 4) / (msd * 1e-3);
    const int itt = 1 << 12;
    const float mst = time_kernel([&] { tf32_throughput<<<blocks, threads>>>((float *)buf, itt); }, 3);
    const double flt = warps * itt * 4 * (2.0 * 16 * 8 * 8) / (mst * 1e-3);
    CK(cudaFree(buf));

    std::printf("{\"sms\": %d, \"sm_clock_mhz_attr\": %.0f, ", sms, clk_khz / 1e3);
    std::printf("\"fp32_fma_tflops\": %.3f, \"fp64_fma_tflops\": %.4f, ", fl32 / 1e12, fl64 / 1e12);
    std::printf("\"dmma_f64_tflops\": %.4f, \"mma_tf32_tflops\": %.2f, ", fld / 1e12, flt / 1e12);
    std::printf("\"latency_cycles\": {");
    std::printf("\"f32_fma\": %.2f, \"f32_sqrt\": %.2f, \"f32_rsqrt\": %.2f, \"f32_div\": %.2f, \"f32_rcp\": %.2f, ",
                cycles_per_op<float, 0>(1.0f), cycles_per_op<float, 1>(2.0f), cycles_per_op<float, 2>(2.0f),
                cycles_per_op<float, 3>(2.0f), cycles_per_op<float, 4>(2.0f));
    std::printf("\"f64_fma\": %.2f, \"f64_sqrt\": %.2f, \"f64_rsqrt\": %.2f, \"f64_div\": %.2f, \"f64_rcp\": %.2f}}\n",
                cycles_per_op<double, 0>(1.0), cycles_per_op<double, 1>(2.0), cycles_per_op<double, 2>(2.0),
                cycles_per_op<double, 3>(2.0), cycles_per_op<double, 4>(2.0));
    return 0;
}
