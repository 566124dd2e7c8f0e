// Standalone probe (not part of libsta): FP64 add / fma / mul / div and int32 throughput on
// every SM, and the cost of an FP64 add issued with 32, 16, 8 or 1 active lanes of a warp.
// Build and run:  nvcc -gencode arch=compute_103a,code=sm_103a -O3 fp64_rate.cu -o fp64_rate
// Every thread writes only out[its global index].
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("error %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int OP> __global__ void k_op(double *out, int iters, double s, int active) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    double a0 = gid * 1e-9 + 1, a1 = a0 + .1, a2 = a0 + .2, a3 = a0 + .3, a4 = a0 + .4, a5 = a0 + .5, a6 = a0 + .6, a7 = a0 + .7;
    if (lane < active)
        for (int i = 0; i < iters; i++) {
            if (OP == 0) { a0 += s; a1 += s; a2 += s; a3 += s; a4 += s; a5 += s; a6 += s; a7 += s; }
            if (OP == 1) { a0 = fma(a0, s, 1e-9); a1 = fma(a1, s, 1e-9); a2 = fma(a2, s, 1e-9); a3 = fma(a3, s, 1e-9);
                           a4 = fma(a4, s, 1e-9); a5 = fma(a5, s, 1e-9); a6 = fma(a6, s, 1e-9); a7 = fma(a7, s, 1e-9); }
            if (OP == 2) { a0 *= s; a1 *= s; a2 *= s; a3 *= s; a4 *= s; a5 *= s; a6 *= s; a7 *= s; }
            if (OP == 3) { a0 /= s; a1 /= s; a2 /= s; a3 /= s; a4 /= s; a5 /= s; a6 /= s; a7 /= s; }
        }
    out[gid] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void k_int(unsigned *out, int iters, unsigned s) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned a0 = gid, a1 = a0 ^ 1, a2 = a0 ^ 2, a3 = a0 ^ 3, a4 = a0 ^ 4, a5 = a0 ^ 5, a6 = a0 ^ 6, a7 = a0 ^ 7;
    for (int i = 0; i < iters; i++) {
        a0 = (a0 + s) ^ a1; a1 = (a1 + s) ^ a2; a2 = (a2 + s) ^ a3; a3 = (a3 + s) ^ a4;
        a4 = (a4 + s) ^ a5; a5 = (a5 + s) ^ a6; a6 = (a6 + s) ^ a7; a7 = (a7 + s) ^ a0;
    }
    out[gid] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

int main() {
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    int clk = 0;
    CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
    const int blocks = p.multiProcessorCount * 8, thr = 256;
    const size_t n = (size_t)blocks * thr;
    double *out;
    CK(cudaMalloc(&out, n * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    printf("%s: %d SMs, max SM clock %.0f MHz\n", p.name, p.multiProcessorCount, clk / 1e3);
    const char *names[4] = {"add", "fma", "mul", "div"};
    for (int op = 0; op < 4; ++op) {
        const int iters = op == 3 ? 256 : 4096;
        float ms = 0;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            if (op == 0) k_op<0><<<blocks, thr>>>(out, iters, 1.0000001, 32);
            if (op == 1) k_op<1><<<blocks, thr>>>(out, iters, 1.0000001, 32);
            if (op == 2) k_op<2><<<blocks, thr>>>(out, iters, 1.0000001, 32);
            if (op == 3) k_op<3><<<blocks, thr>>>(out, iters, 1.0000001, 32);
            cudaEventRecord(e1);
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            cudaEventElapsedTime(&ms, e0, e1);
        }
        printf("fp64 %s: %.1f G lane-ops/s\n", names[op], (double)n * iters * 8 / ms / 1e6);
    }
    const int act[4] = {32, 16, 8, 1};
    for (int a = 0; a < 4; ++a) {
        float ms = 0;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0);
            k_op<0><<<blocks, thr>>>(out, 2048, 1.0000001, act[a]);
            cudaEventRecord(e1);
            CK(cudaEventSynchronize(e1));
            cudaEventElapsedTime(&ms, e0, e1);
        }
        printf("fp64 add, %2d active lanes per warp: %.3f ms\n", act[a], ms);
    }
    float ms = 0;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_int<<<blocks, thr>>>((unsigned *)out, 4096, 12345u);
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
    }
    printf("int32 add+xor: %.1f G lane-ops/s\n", (double)n * 4096 * 16 / ms / 1e6);
    CK(cudaFree(out));
    return 0;
}
