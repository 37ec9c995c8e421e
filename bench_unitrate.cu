// bench_unitrate.cu -- a measurement helper of bench.py, not part of the sampler or of its
// C ABI (built into its own library, libbench_unitrate.so): the sustained rate of one
// instruction kind on this GPU, in lane-operations per second per SM.  The benchmark uses it
// as the measured peak of the pipe that bounds a kernel (the special-function unit for the
// tensor-core sweep's epilogue, the issue rate for the mixture sweep): one CTA of 32 warps per
// SM, each thread running 8 independent dependency chains of the instruction, timed with the
// global nanosecond timer (no assumption about the SM clock).  Chains whose instruction could
// be folded with itself (rcp of rcp) or would leave its domain (lg2 of lg2) carry one fp32 add
// per step, which runs on another pipe.
#include <cuda_runtime.h>
#include <vector>

// instruction kinds (unitrate_measure's unit argument)
enum { UNIT_EX2 = 0, UNIT_RCP = 1, UNIT_LG2 = 2, UNIT_FFMA = 3, UNIT_LOP3 = 4 };

namespace unitrate {

constexpr int kThreads = 1024;
constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(kThreads, 1)
rate_kernel(float* sink, long long* nanos, int iters)
{
    float a[kChains];
    unsigned u[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        a[k] = 1.0f + 0.001f * (threadIdx.x + k);
        u[k] = threadIdx.x * 2654435761u + k;
    }
    __syncthreads();
    long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (OP == UNIT_EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
            if (OP == UNIT_RCP)
                asm volatile("rcp.approx.ftz.f32 %0, %0;\n\tadd.f32 %0, %0, 0f3F800000;" : "+f"(a[k]));
            if (OP == UNIT_LG2)
                asm volatile("lg2.approx.ftz.f32 %0, %0;\n\tadd.f32 %0, %0, 0f40000000;" : "+f"(a[k]));
            if (OP == UNIT_FFMA) asm volatile("fma.rn.f32 %0, %0, %0, %0;" : "+f"(a[k]));
            if (OP == UNIT_LOP3) asm volatile("lop3.b32 %0, %0, %1, %0, 0x6a;" : "+r"(u[k]) : "r"(0x9E3779B9u));
        }
    }
    __syncthreads();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += a[k] + (float)(u[k] & 1u);
    sink[blockIdx.x * kThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0) nanos[blockIdx.x] = t1 - t0;
}

} // namespace unitrate

// Returns 0 and the rate in *lane_ops_per_s_per_sm, 1 for a bad argument, 2 when the scratch
// allocation fails, 3 for another CUDA error.  Allocates and frees a small scratch buffer and
// synchronises the device.
extern "C" int unitrate_measure(int unit, double* lane_ops_per_s_per_sm)
{
    using namespace unitrate;
    if (!lane_ops_per_s_per_sm || unit < UNIT_EX2 || unit > UNIT_LOP3) return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
    float* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)sms * kThreads) != cudaSuccess) return 2;
    if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) { cudaFree(sink); return 2; }
    const int iters = 8192;
    // 160 KB of (unused) dynamic shared memory keeps a second CTA off each SM
    const size_t smem = 160 * 1024;
    auto launch = [&](int reps) {
        for (int r = 0; r < reps; ++r) {
            switch (unit) {
#define UNITRATE_CASE(U)                                                                              \
            case U:                                                                                     \
                cudaFuncSetAttribute(rate_kernel<U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
                rate_kernel<U><<<sms, kThreads, smem>>>(sink, cyc, iters);                              \
                break;
            UNITRATE_CASE(UNIT_EX2)
            UNITRATE_CASE(UNIT_RCP)
            UNITRATE_CASE(UNIT_LG2)
            UNITRATE_CASE(UNIT_FFMA)
            UNITRATE_CASE(UNIT_LOP3)
#undef UNITRATE_CASE
            }
        }
    };
    launch(2);   // warm-up, then the timed launch
    launch(1);
    std::vector<long long> h(sms);
    int st = 0;
    if (cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost) != cudaSuccess) st = 3;
    cudaFree(sink);
    cudaFree(cyc);
    if (st != 0) return st;
    double rate = 0.0;
    for (int b = 0; b < sms; ++b) rate += (double)kThreads * iters * kChains / ((double)h[b] * 1e-9);
    *lane_ops_per_s_per_sm = rate / sms;
    return 0;
}
