// Integer-ALU throughput probe: lane-operations per SM clock of the integer
// instructions the fill kernels are built from, measured on the device that runs
// this program. It is the basis of the integer roofline peak the benchmark
// reports (SMs x lane-ops per clock x SM clock).
//
// Each thread runs NCHAIN accumulators for ITERS iterations; every operation
// reads two or three different accumulators of the previous iteration (a ring),
// so the NCHAIN operations of an iteration are independent and no chain can be
// simplified algebraically. The grid fills every SM with resident warps; the
// reported rate is operations / (CUDA-event time x SMs x the maximum SM clock),
// i.e. lane-operations per SM per clock if the SM ran at its maximum clock
// (lower clocks lower every figure alike, so ratios between operations hold).
//
// Output, one line per operation: name, lane-ops per SM per clock, elapsed ms.
// "add" (add.s32), "max" (max.s32), "add3" (a + b + c), "max3" (three-input
// max, __vimax3_s32), "addmax" (max(a + b, c), __viaddmax_s32) and "relax"
// (two candidates of the line kernel, max(acc, w + y, z + c) with w <- w + y,
// counted as four operations: two adds and two maxes).
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

constexpr int NCHAIN = 8;
constexpr int ITERS = 4096;
constexpr int THREADS = 512;
constexpr int BLOCKS_PER_SM = 3;  // 3 x 512 threads: the 48 warps an SM holds, all resident at once

template <int OP>
__global__ void __launch_bounds__(THREADS) probe(int b, int c, int *out) {
    int a[NCHAIN], w[NCHAIN];
#pragma unroll
    for (int j = 0; j < NCHAIN; ++j) {
        a[j] = threadIdx.x + j;
        w[j] = threadIdx.x * 3 + j;
    }
#pragma unroll 4
    for (int i = 0; i < ITERS; ++i) {
        // every operation reads two or three different accumulators of the
        // previous iteration (a ring), so no chain can be simplified
        int n[NCHAIN], m[NCHAIN];
#pragma unroll
        for (int j = 0; j < NCHAIN; ++j) {
            const int x = a[j], y = a[(j + 1) % NCHAIN], z = a[(j + 2) % NCHAIN];
            if constexpr (OP == 0) {
                n[j] = x + y;
            } else if constexpr (OP == 1) {
                n[j] = max(x, y);
            } else if constexpr (OP == 2) {
                n[j] = x + y + z;
            } else if constexpr (OP == 3) {
                n[j] = __vimax3_s32(x, y, z);
            } else if constexpr (OP == 4) {
                n[j] = __viaddmax_s32(x, y, z);
            } else {
                // acc = max(acc, w + b, y + c), w <- w + b: two candidates of the line kernel
                m[j] = w[j] + y;
                n[j] = __vimax3_s32(x, m[j], z + c);
            }
        }
#pragma unroll
        for (int j = 0; j < NCHAIN; ++j) {
            a[j] = n[j];
            if constexpr (OP == 5) w[j] = m[j];
        }
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < NCHAIN; ++j) s += a[j] + w[j];
    out[blockIdx.x * THREADS + threadIdx.x] = s;
}

template <int OP>
static int run(const char *name, int ops_per_step, int sms, double clk_hz, int *d_out) {
    const int blocks = sms * BLOCKS_PER_SM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    probe<OP><<<blocks, THREADS>>>(3, -5, d_out);  // warm-up
    cudaEventRecord(e0);
    probe<OP><<<blocks, THREADS>>>(3, -5, d_out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = (double)blocks * THREADS * ITERS * NCHAIN * ops_per_step;
    printf("%s %.1f %.3f\n", name, ops / (ms * 1e-3) / sms / clk_hz, ms);
    return 0;
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    printf("sms %d max_clock_khz %d\n", sms, clk);
    int *d_out = nullptr;
    if (cudaMalloc(&d_out, sizeof(int) * sms * BLOCKS_PER_SM * THREADS) != cudaSuccess) return 2;
    const double hz = clk * 1e3;
    int rc = 0;
    rc |= run<0>("add", 1, sms, hz, d_out);
    rc |= run<1>("max", 1, sms, hz, d_out);
    rc |= run<2>("add3", 2, sms, hz, d_out);
    rc |= run<3>("max3", 2, sms, hz, d_out);
    rc |= run<4>("addmax", 2, sms, hz, d_out);
    rc |= run<5>("relax", 4, sms, hz, d_out);
    cudaFree(d_out);
    return rc;
}
