// FP64 throughput probe of one GPU: the denominator of the FP64 roofline
// fractions that bench.py reports.  Two instruction loops, each thread
// writing one result (every access in bounds):
//   dfma : 8 independent FP64 fused multiply-add chains per thread
//   dmma : 4 independent mma.sync m8n8k4 FP64 accumulations per warp
// over grids of 1..8 CTAs per SM and 128..512 threads, timed with CUDA
// events after a warm-up launch.  Prints one JSON line per configuration
// and a final line with the best of each.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_peak bench_fp64_peak.cu
#include <cstdio>
#include <cuda_runtime.h>

#define CHECK(x)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) {                                                      \
            std::printf("{\"error\": \"%s at line %d\"}\n", cudaGetErrorString(e_), __LINE__); \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

__global__ void k_dfma(double* out, int iters) {
    double a[8];
    const double b = 1.0000001, c = 1e-9;
    for (int j = 0; j < 8; j++) a[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0;
    for (int j = 0; j < 8; j++) s += a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dmma(double* out, int iters) {
    const double a = 1e-3 * threadIdx.x, b = 1.0 / (1 + threadIdx.x);
    double c[4][2];
    for (int j = 0; j < 4; j++) {
        c[j][0] = j;
        c[j][1] = j + 1;
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0;
    for (int j = 0; j < 4; j++) s += c[j][0] + c[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// half of the warps of every CTA run the DFMA loop, half the DMMA loop: the
// sum of both rates shows whether the two share the FP64 units
__global__ void k_mixed(double* out, int iters) {
    const int warp = threadIdx.x >> 5;
    if (warp & 1) {
        const double a = 1e-3 * threadIdx.x, b = 1.0 / (1 + threadIdx.x);
        double c[4][2];
        for (int j = 0; j < 4; j++) {
            c[j][0] = j;
            c[j][1] = j + 1;
        }
        for (int i = 0; i < iters; i++) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                             : "+d"(c[j][0]), "+d"(c[j][1])
                             : "d"(a), "d"(b));
        }
        double s = 0;
        for (int j = 0; j < 4; j++) s += c[j][0] + c[j][1];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else {
        double a[8];
        const double b = 1.0000001, c = 1e-9;
        for (int j = 0; j < 8; j++) a[j] = threadIdx.x * 1e-3 + j;
        for (int i = 0; i < 4 * iters; i++) {  // as many FMAs as the DMMA warp
#pragma unroll
            for (int j = 0; j < 8; j++) a[j] = fma(a[j], b, c);
        }
        double s = 0;
        for (int j = 0; j < 8; j++) s += a[j];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

template <typename K>
static float time_ms(K kern, double* out, int grid, int block, int iters) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kern<<<grid, block>>>(out, iters / 10);
    cudaDeviceSynchronize();
    cudaEventRecord(e0);
    kern<<<grid, block>>>(out, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int main() {
    cudaDeviceProp p;
    CHECK(cudaGetDeviceProperties(&p, 0));
    const int sms = p.multiProcessorCount;
    const size_t maxthreads = static_cast<size_t>(sms) * 8 * 512;
    double* out = nullptr;
    CHECK(cudaMalloc(&out, maxthreads * sizeof(double)));
    double best_fma = 0, best_mma = 0;
    const int it = 20000;
    for (int bpsm : {1, 2, 4, 8})
        for (int threads : {128, 256, 512}) {
            const int grid = sms * bpsm;
            if (static_cast<size_t>(grid) * threads > maxthreads) continue;
            float ms = time_ms(k_dfma, out, grid, threads, it);
            double tf = 2.0 * 8 * it * static_cast<double>(grid) * threads / (ms * 1e-3) / 1e12;
            if (tf > best_fma) best_fma = tf;
            std::printf("{\"kernel\": \"dfma\", \"ctas_per_sm\": %d, \"threads\": %d, \"ms\": %.3f, \"tflops\": %.4f}\n",
                        bpsm, threads, ms, tf);
            ms = time_ms(k_dmma, out, grid, threads, it);
            tf = 2.0 * 4 * it * static_cast<double>(grid * threads / 32) * 8 * 8 * 4 / (ms * 1e-3) / 1e12;
            if (tf > best_mma) best_mma = tf;
            std::printf("{\"kernel\": \"dmma_m8n8k4\", \"ctas_per_sm\": %d, \"threads\": %d, \"ms\": %.3f, \"tflops\": %.4f}\n",
                        bpsm, threads, ms, tf);
        }
    // mixed: per warp pair, one DMMA loop (4 x 256 FMA per iteration) and one
    // DFMA loop with as many FMAs (4 iterations of 8 x 32 each)
    for (int bpsm : {2, 4}) {
        const int threads = 256, grid = sms * bpsm;
        const float ms = time_ms(k_mixed, out, grid, threads, it);
        const double warps = static_cast<double>(grid) * threads / 32;
        const double fl = 2.0 * it * (warps / 2) * (4.0 * 256 + 4.0 * 8 * 32);
        std::printf("{\"kernel\": \"mixed_dfma_dmma\", \"ctas_per_sm\": %d, \"threads\": %d, \"ms\": %.3f, "
                    "\"tflops\": %.4f}\n", bpsm, threads, ms, fl / (ms * 1e-3) / 1e12);
    }
    CHECK(cudaGetLastError());
    std::printf("{\"gpu\": \"%s\", \"sms\": %d, \"best_dfma_tflops\": %.4f, \"best_dmma_tflops\": %.4f}\n", p.name, sms,
                best_fma, best_mma);
    cudaFree(out);
    return 0;
}
