// noalloc.cu -- oais_logsumexp_noalloc: the log-sum-exp reduction of oais_logsumexp for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden -- inside a
// CUDA-graph capture that must not allocate, in a process whose memory is owned by
// another allocator (a framework's caching pool, a real-time loop with a fixed
// memory budget), or in an embedding that only hands over its input and output
// buffers.  The ordinary entry point asks the caller for a scratch buffer; this one
// keeps its scratch in a fixed array of device memory that is part of the library
// image, so the caller passes only the input and the output.
//
// Scratch: g_noalloc_lse below, kNoAllocRecords records of 32 bytes (128 KiB).  Every GPU
// that loads the library holds this array until the process exits.  One record covers
// kNoAllocChunk = 4096 inputs, so n is limited to kNoAllocRecords * kNoAllocChunk =
// 16,777,216 elements; larger n is rejected with OAIS_EINVAL.
//
// Sharing: all calls on a device use the same array, and it keeps the last call's
// contents.  Each call writes every record it later reads, so nothing has to start at
// zero, but two calls whose kernels overlap on the GPU (different streams, or host
// threads without ordering between them) race on the array and may return wrong sums.
// Order such calls on one stream.
//
// Set-up: host code cannot use the array's name as a device address.  The first call on
// each device (with that device current) looks the address up with cudaGetSymbolAddress
// and caches it; make that first call before any stream capture on the device.  The cached
// address belongs to the device's current primary context: after cudaDeviceReset (or any
// other teardown of that context) the library's module is loaded again and the array may
// move, so a process that resets a device must not call this entry point on it afterwards.
//
// Errors go through the library's per-thread error text (oais_last_error(NULL)).  An error
// left pending by an earlier, unrelated CUDA call is cleared on entry, so a launch failure
// reported here is this call's own.
#include <cmath>
#include <mutex>

#include "internal.h"
#include "oais_device.cuh"
#include "../../include/oais.h"

namespace oais {
namespace noalloc {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kNoAllocChunk = kThreads * kItems;     // inputs per record
constexpr int kNoAllocRecords = 4096;
constexpr int64_t kMaxN = (int64_t)kNoAllocRecords * kNoAllocChunk;
constexpr int kMaxDevices = 64;

struct Record { double m1, s1, m2, s2; };

static __device__ __align__(256) Record g_noalloc_lse[kNoAllocRecords];

__device__ __forceinline__ void push(double& m, double& s, double v)
{
    if (v == -INFINITY) return;
    if (v > m) { s = s * exp(m - v) + 1.0; m = v; }
    else       { s += exp(v - m); }
}

__device__ void block_merge(double& m1, double& s1, double& m2, double& s2)
{
    __shared__ double sm1[kThreads], ss1[kThreads], sm2[kThreads], ss2[kThreads];
    const int tid = threadIdx.x;
    sm1[tid] = m1; ss1[tid] = s1; sm2[tid] = m2; ss2[tid] = s2;
    __syncthreads();
    for (int stride = kThreads / 2; stride > 0; stride >>= 1) {
        if (tid < stride) {
            double mm = sm1[tid], s = ss1[tid];
            lse_merge(mm, s, sm1[tid + stride], ss1[tid + stride]);
            sm1[tid] = mm; ss1[tid] = s;
            mm = sm2[tid]; s = ss2[tid];
            lse_merge(mm, s, sm2[tid + stride], ss2[tid + stride]);
            sm2[tid] = mm; ss2[tid] = s;
        }
        __syncthreads();
    }
    m1 = sm1[0]; s1 = ss1[0]; m2 = sm2[0]; s2 = ss2[0];
}

// record b <- (LSE pieces of a[b*chunk, (b+1)*chunk) and of twice those values)
__global__ void __launch_bounds__(kThreads)
lse_chunk_kernel(const double* __restrict__ a, int64_t n, Record* __restrict__ scratch)
{
    double m1 = -INFINITY, s1 = 0.0, m2 = -INFINITY, s2 = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kNoAllocChunk;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t j = base + (int64_t)i * kThreads + threadIdx.x;
        if (j < n) {
            const double v = a[j];
            push(m1, s1, v);
            push(m2, s2, 2.0 * v);
        }
    }
    block_merge(m1, s1, m2, s2);
    if (threadIdx.x == 0) scratch[blockIdx.x] = Record{m1, s1, m2, s2};
}

__global__ void __launch_bounds__(kThreads)
lse_records_kernel(const Record* __restrict__ scratch, int nrec, double* __restrict__ out)
{
    double m1 = -INFINITY, s1 = 0.0, m2 = -INFINITY, s2 = 0.0;
    for (int j = threadIdx.x; j < nrec; j += kThreads) {
        const Record r = scratch[j];
        lse_merge(m1, s1, r.m1, r.s1);
        lse_merge(m2, s2, r.m2, r.s2);
    }
    block_merge(m1, s1, m2, s2);
    if (threadIdx.x == 0) {
        out[0] = m1 + log(s1);
        out[1] = m2 + log(s2);
    }
}

static std::mutex g_mu;
static Record* g_addr[kMaxDevices] = {};
static_assert(kMaxN == OAIS_LOGSUMEXP_NOALLOC_MAX_N, "limit documented in oais.h");

} // namespace noalloc
} // namespace oais

extern "C" oais_status oais_logsumexp_noalloc(const double* d_a, int64_t n, double* d_out, void* stream)
{
    using namespace oais::noalloc;
    auto fail = [](oais_status st, const char* m) { return (oais_status)oais::fail_call(st, m); };
    if (!d_a || !d_out || n < 1) return fail(OAIS_EINVAL, "oais_logsumexp_noalloc: null pointer or n < 1");
    if (n > kMaxN)   // more inputs than the fixed scratch array covers; nothing is launched
        return fail(OAIS_EINVAL, "oais_logsumexp_noalloc: n above OAIS_LOGSUMEXP_NOALLOC_MAX_N");
    // an error left pending by an earlier, unrelated call is not this call's: clear it, so
    // that the checks after the launches below report only what they did
    (void)cudaGetLastError();
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(OAIS_ECUDA, "oais_logsumexp_noalloc: no usable current device");
    Record* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_lse);
            if (e != cudaSuccess || !p) return fail(OAIS_ECUDA, cudaGetErrorString(e));
            g_addr[dev] = static_cast<Record*>(p);
        }
        scratch = g_addr[dev];
    }
    const int nrec = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lse_chunk_kernel<<<nrec, kThreads, 0, s>>>(d_a, n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(OAIS_ECUDA, cudaGetErrorString(e));
    lse_records_kernel<<<1, kThreads, 0, s>>>(scratch, nrec, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(OAIS_ECUDA, cudaGetErrorString(e));
    return OAIS_OK;
}
