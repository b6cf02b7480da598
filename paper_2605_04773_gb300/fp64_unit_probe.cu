// Measures the FP64 FMA rate of one SM of the GPU it runs on: one CTA per
// SM, 1, 2, 4 or 8 warps each issuing 8 independent FMA chains, timed with
// clock64 on every SM.  Prints one JSON object: cycles per FP64 warp
// instruction seen by one warp, and FMA lanes per clock per SM with all warps
// busy.  The FP64 roofline of the PCG kernels divides by this rate (bench.py
// --fp64-probe builds and runs this file).  Every thread writes only its own
// output slots; nothing waits.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kIters = 4096;

__global__ void fma_rate(int warps, double seed, long long *cyc, double *sink)
{
    const int w = threadIdx.x >> 5;
    if (w >= warps) return;
    double a[8];
    for (int k = 0; k < 8; ++k) a[k] = seed + 1e-3 * threadIdx.x + k;
    const long long t0 = clock64();
    for (int i = 0; i < kIters / 8; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], 1.0000001, 1e-12);
    const long long t1 = clock64();
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += a[k];   // every chain stays live
    sink[blockIdx.x * 256 + threadIdx.x] = s;
    if ((threadIdx.x & 31) == 0) cyc[blockIdx.x * 8 + w] = t1 - t0;
}

int main()
{
    int sms = 0, clk_khz = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    long long *cyc = nullptr;
    double *sink = nullptr;
    if (cudaMalloc(&cyc, (size_t)sms * 8 * sizeof(long long)) != cudaSuccess) return 1;
    if (cudaMalloc(&sink, (size_t)sms * 256 * sizeof(double)) != cudaSuccess) return 1;
    long long *h = new long long[(size_t)sms * 8];
    printf("{\"sms\": %d, \"sm_clock_mhz\": %.0f, \"per_warps\": {", sms, clk_khz / 1e3);
    double lanes_per_clk_8 = 0.0;
    const int counts[] = {1, 2, 4, 8};
    for (int ci = 0; ci < 4; ++ci) {
        const int nw = counts[ci];
        for (int rep = 0; rep < 2; ++rep) fma_rate<<<sms, 32 * nw>>>(nw, 1.0, cyc, sink);
        if (cudaDeviceSynchronize() != cudaSuccess) return 1;
        cudaMemcpy(h, cyc, (size_t)sms * 8 * sizeof(long long), cudaMemcpyDeviceToHost);
        double mean = 0.0;
        for (int b = 0; b < sms; ++b)
            for (int w = 0; w < nw; ++w) mean += (double)h[b * 8 + w];
        mean /= (double)sms * nw;
        const double per_instr = mean / kIters;              // cycles per FP64 warp instruction, one warp
        const double lanes = nw * 32.0 / per_instr;          // FMA lanes per clock per SM
        if (nw == 8) lanes_per_clk_8 = lanes;
        printf("%s\"%d\": {\"cycles_per_warp_instr\": %.1f, \"fma_lanes_per_clk_per_sm\": %.3f}", ci ? ", " : "", nw,
               per_instr, lanes);
    }
    printf("}, \"fma_lanes_per_clk_per_sm\": %.3f}\n", lanes_per_clk_8);
    delete[] h;
    return 0;
}
