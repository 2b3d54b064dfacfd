// Issue-rate microbenchmark of the integer SIMD forms the fill could use on
// sm_103a: each thread runs 8 independent chains of one operation; the rate is
// reported in lane operations per clock per SM at the maximum SM clock.
#include <cstdio>
#include <cuda_runtime.h>

#define CHAINS 8

template <int OP>
__device__ __forceinline__ unsigned f(unsigned a, unsigned b, unsigned c) {
    if (OP == 0) return (unsigned)max((int)a + (int)b, (int)c);          // IADD + IMNMX
    if (OP == 1) return __viaddmax_s32(a, b, c);
    if (OP == 2) return __viaddmax_s32_relu(a, b, c);
    if (OP == 3) return __vimax3_s32(a, b, c);
    if (OP == 4) return __viaddmax_s16x2(a, b, c);
    if (OP == 5) return __viaddmax_s16x2_relu(a, b, c);
    if (OP == 6) return __vmaxs2(a, b);
    if (OP == 7) return __vimax3_s16x2_relu(a, b, c);
    if (OP == 8) return __vadd2(a, b);
    if (OP == 9) return __vsub2(a, b);
    if (OP == 10) return __vaddus4(a, b);
    if (OP == 11) return __vsubus4(a, b);
    if (OP == 12) return __vmaxu4(a, b);
    if (OP == 13) return __byte_perm(b, c, a);
    if (OP == 14) return (a ^ b) | (c & 0x8888u);  // LOP3
    if (OP == 15) return (unsigned)max((int)a, (int)b);
    if (OP == 16) return a + b;
    if (OP == 17) return __vimax_s16x2_relu(a, b);
    if (OP == 18) return __vmaxu2(a, b);
    if (OP == 19) return __viaddmax_u16x2(a, b, c);
    if (OP == 20) { bool p, q; unsigned r = __vibmax_s16x2(a, b, &p, &q); return r + (p ? 1u : 0u) + (q ? 0x10000u : 0u); }
    if (OP == 21) return __vmaxs4(a, b);
    return a;
}

template <int OP>
__global__ void kbench(unsigned *out, unsigned seed, int iters) {
    unsigned a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; k++) a[k] = seed * (k + 1) + threadIdx.x;
    unsigned b = seed * 3u + blockIdx.x, c = seed * 7u;
    for (int i = 0; i < iters; i++) {
        unsigned bi = b + (unsigned)i;
#pragma unroll
        for (int k = 0; k < CHAINS; k++) a[k] = f<OP>(a[k], bi, c);
    }
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; k++) r ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

template <int OP>
void run(const char *name, unsigned *d, int sms, int clk_khz) {
    int blocks = sms * 8, threads = 256, iters = 8192;
    kbench<OP><<<blocks, threads>>>(d, 12345u, 64);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    kbench<OP><<<blocks, threads>>>(d, 12345u, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = (double)blocks * threads * iters * CHAINS;
    double gops = ops / (ms * 1e-3) / 1e9;
    // per SM per clock at the reported max clock (lower bound on lanes/clk)
    double per_clk = ops / (ms * 1e-3) / sms / (clk_khz * 1e3);
    printf("%-26s %8.3f ms  %9.1f Gop/s  %6.1f thread-ops/clk/SM(@max)\n", name, ms, gops, per_clk);
}

int main() {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, 0);
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("%s sm_%d%d SMs=%d clock=%d kHz\n", p.name, p.major, p.minor, p.multiProcessorCount, clk);
    unsigned *d;
    cudaMalloc(&d, sizeof(unsigned) * p.multiProcessorCount * 8 * 256);
    int s = p.multiProcessorCount;
    for (int rep = 0; rep < 2; rep++) {
        run<16>("iadd", d, s, clk);
        run<15>("imax s32", d, s, clk);
        run<0>("iadd+imax", d, s, clk);
        run<1>("viaddmax_s32", d, s, clk);
        run<2>("viaddmax_s32_relu", d, s, clk);
        run<3>("vimax3_s32", d, s, clk);
        run<4>("viaddmax_s16x2", d, s, clk);
        run<5>("viaddmax_s16x2_relu", d, s, clk);
        run<6>("vmaxs2", d, s, clk);
        run<17>("vimax_s16x2_relu", d, s, clk);
        run<7>("vimax3_s16x2_relu", d, s, clk);
        run<18>("vmaxu2", d, s, clk);
        run<19>("viaddmax_u16x2", d, s, clk);
        run<20>("vibmax_s16x2", d, s, clk);
        run<8>("vadd2", d, s, clk);
        run<9>("vsub2", d, s, clk);
        run<10>("vaddus4", d, s, clk);
        run<11>("vsubus4", d, s, clk);
        run<12>("vmaxu4", d, s, clk);
        run<21>("vmaxs4", d, s, clk);
        run<13>("byte_perm", d, s, clk);
        run<14>("lop3", d, s, clk);
    }
    cudaError_t e = cudaGetLastError();
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
