// internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include "sweep.cuh"

namespace oais {

// A target in the device layout the kernels read: X zero-padded to D columns
// (D = the compiled width), rows padded to a multiple of 4, fp64 for the
// Gaussian family and fp32 otherwise.
struct DevTarget {
    int kind = 0;
    int d = 0, D = 0, n = 0, n_pad = 0;
    double ref_scale = 1.0, p0 = 1.0;
    void* X = nullptr;   // GAUSS: double[D]; GMM: float[n][D]; rows: float[n_pad][D]
    void* y = nullptr;   // rows: float[n_pad]
};

// smallest compiled width >= d for the family, 0 if none
int padded_width(int kind, int d);

// launch the sweep for one family; grid = oais_sweep_blocks(P.N)
cudaError_t launch_sweep_gauss(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_logreg(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_gmm(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_linreg(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);

inline int sweep_grid(int64_t N) { return (int)((N + kSweepThreads - 1) / kSweepThreads); }

// generic launcher used by the per-family translation units
template <class Tgt, int MOVE, int D, typename R>
cudaError_t launch_one(const Tgt& tg, size_t smem, const SweepParams& P, cudaStream_t s)
{
    auto* k = &oais_sweep_kernel<Tgt, MOVE, D, R>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<sweep_grid(P.N), kSweepThreads, smem, s>>>(P, tg);
    return cudaGetLastError();
}

} // namespace oais
