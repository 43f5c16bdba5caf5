// peak.cu -- integer-pipe throughput probe for the benchmark's ALU roofline
// (not part of the REI ABI; built into librei_peak.so).
//
// Every thread runs 8 independent chains of 3-input logic operations
// (lop3.b32, the instruction a bit-sliced AND-OR compiles to); the result is
// stored so nothing is optimised away.  Returns lane-operations per second.
#include <cuda_runtime.h>

#include <cstdint>

__global__ void k_lop3(uint32_t *out, uint32_t iters, uint32_t seed) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = seed * (threadIdx.x + 7u * i + 1u) ^ blockIdx.x;
    const uint32_t y = seed ^ 0x5A5A5A5Au, z = seed + 0x01234567u;
    for (uint32_t k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            // x = (x & y) | z   (truth table 0xEA), one instruction per chain step
            asm volatile("lop3.b32 %0, %0, %1, %2, 0xEA;" : "+r"(x[i]) : "r"(y), "r"(z));
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(z), "r"(y));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) acc ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

extern "C" double rei_peak_lop3(int device, double *ms_out) {
    if (cudaSetDevice(device) != cudaSuccess) return -1;
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, device);
    const int threads = 512, blocks = p.multiProcessorCount * 4;
    const uint32_t iters = 20000;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * threads * blocks) != cudaSuccess) return -1;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_lop3<<<blocks, threads>>>(out, iters / 10, 3);  // warm-up
    cudaEventRecord(a);
    k_lop3<<<blocks, threads>>>(out, iters, 3);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0) return -1;
    if (ms_out) *ms_out = ms;
    const double ops = (double)threads * blocks * iters * 8 * 2;
    return ops / (ms * 1e-3);
}

// L2 throughput for random 32-byte sectors: every thread runs 8 independent
// chains of 4-byte loads through L2 (ld.global.cg, as the search reads its
// bitmap of cached languages) at addresses drawn by a multiplicative
// congruential step over a buffer that fits the L2; each load moves one
// sector.  The next address depends on the loaded value, so no load can be
// skipped.
__global__ void k_l2_random(const uint32_t *buf, uint32_t mask, uint32_t iters, uint32_t *out) {
    uint32_t a[8], acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = (blockIdx.x * blockDim.x + threadIdx.x) * 8u + (uint32_t)i;
    for (uint32_t k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint32_t v = __ldcg(buf + ((a[i] * 8u) & mask));  // word index of a sector start
            a[i] = a[i] * 1664525u + 1013904223u + v;
            acc ^= v;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// bytes per second of random 32-byte sectors served by the L2 (buffer of
// `mib` MiB, at most a quarter of the L2 so that it stays resident)
extern "C" double rei_peak_l2_random(int device, int mib, double *ms_out) {
    if (cudaSetDevice(device) != cudaSuccess) return -1;
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, device);
    size_t bytes = (size_t)mib << 20;
    if (bytes > (size_t)p.l2CacheSize / 4) bytes = (size_t)p.l2CacheSize / 4;
    size_t words = 1;
    while (words * 2 * 4 <= bytes) words *= 2;  // a power of two
    const int threads = 512, blocks = p.multiProcessorCount * 4;
    const uint32_t iters = 400;
    uint32_t *buf = nullptr, *out = nullptr;
    if (cudaMalloc(&buf, words * 4) != cudaSuccess) return -1;
    if (cudaMalloc(&out, sizeof(uint32_t) * threads * blocks) != cudaSuccess) {
        cudaFree(buf);
        return -1;
    }
    cudaMemset(buf, 0, words * 4);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_l2_random<<<blocks, threads>>>(buf, (uint32_t)(words - 1), iters / 4, out);  // warm-up: the buffer into L2
    cudaEventRecord(a);
    k_l2_random<<<blocks, threads>>>(buf, (uint32_t)(words - 1), iters, out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0) return -1;
    if (ms_out) *ms_out = ms;
    const double sectors = (double)threads * blocks * iters * 8;
    return sectors * 32.0 / (ms * 1e-3);
}
