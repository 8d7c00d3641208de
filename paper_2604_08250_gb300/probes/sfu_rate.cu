// sfu_rate.cu -- throughput of the special-function instructions the MLP
// path uses (tanh.approx.f32 for SiLU; ex2.approx for comparison), in lanes
// per clock per SM: 8 CTAs of 256 threads per SM, 8 independent chains per
// thread, 4096 iterations.  Prints one JSON line.  Built and run by
// `python bench.py --probe-sfu`.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

template <int OP>
__global__ void k_sfu(float *out, int iters, float seed)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + 0.001f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == 0) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(a[i]));
            if (OP == 1) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main()
{
    int sms = 0, clk_khz = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0) != cudaSuccess) {
        printf("{\"error\": \"no device\"}\n");
        return 1;
    }
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double rate[2];
    for (int op = 0; op < 2; ++op) {
        float ms = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            if (op == 0)
                k_sfu<0><<<blocks, threads>>>(out, iters, 0.3f);
            else
                k_sfu<1><<<blocks, threads>>>(out, iters, 0.3f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        const double lanes = (double)blocks * threads * iters * 8;
        rate[op] = lanes / (ms * 1e-3) / sms / (clk_khz * 1e3);  // per clock at the nominal maximum
    }
    printf("{\"tanh_approx_f32_per_clk_per_sm\": %.2f, \"ex2_approx_f32_per_clk_per_sm\": %.2f, \"sms\": %d, "
           "\"clock_mhz\": %d, \"status\": \"%s\"}\n",
           rate[0], rate[1], sms, clk_khz / 1000, cudaGetErrorString(cudaGetLastError()));
    cudaFree(out);
    return 0;
}
