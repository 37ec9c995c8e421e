// sweep_tcs_batch.cu -- many independent problems in one persistent launch of the streamed
// tensor-core sweep: the batched kernel and its launcher (a translation unit of its own so
// that it compiles beside the single-problem kernels).
#include "sweep_tcs.cuh"

namespace oais {
namespace tcs {

// Many independent problems in one persistent launch: each CTA takes (problem, tile) items
// from a queue ordered by decreasing cost (longest first) until it is empty.  All problems
// share the family; their widths may differ (the item picks the instantiation).  Every
// problem's Misc region sits at the same offset (the launch's largest).
// ALT: some problems run 128-row chunks (a separate instantiation, so that the default one
// keeps its register allocation)
template <int FAM, int H, bool ALT>
__global__ void __launch_bounds__(Roles<H>::threads(0), 1)
oais_sweep_tcs_batch_kernel(const Params* __restrict__ probs, const uint2* __restrict__ items, uint32_t n_items,
                            uint32_t* head, uint32_t off_misc)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    if (saddr(smem) & 1023u) {
        if (threadIdx.x == 0) atomicOr(probs[0].sp.status, 4u);
        return;
    }
    Misc* M = reinterpret_cast<Misc*>(smem + off_misc);
    Params& sP = M->prm;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        tmem_alloc(saddr(&M->tmem), 512);
        tmem_relinquish();
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(&M->tmem);
    int prev_stages = 0;   // thread 0 only
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t it = atomicAdd(head, 1u);
            M->item = it;
            if (it < n_items) {
                sP = probs[items[it].x];
                init_barriers(M, sP.stages, prev_stages, 0, Roles<H>::kEpiWarps);
                prev_stages = sP.stages;
            }
        }
        __syncthreads();
        const uint32_t it = M->item;
        if (it >= n_items) break;
        const uint32_t tile = items[it].y;
        const uint32_t tiles = (uint32_t)((sP.sp.N + kTile - 1) / kTile);
        // the item's width and chunk rows pick the instantiation: 64-row chunks, or (logistic,
        // d_pad <= 64, whose chunk images do not depend on the chunk size) 128-row chunks
        const int chr = sP.chunk;
        switch (sP.dp) {
        case 16:
            if constexpr (16 / H >= 8) {
                if constexpr (ALT && FAM == kLogreg) {
                    if (chr == 128) { run_tile<FAM, 16, 0, H, 128>(sP, tile, tiles, smem, tmem); break; }
                }
                run_tile<FAM, 16, 0, H>(sP, tile, tiles, smem, tmem);
            }
            break;
        case 32:
            if constexpr (32 / H >= 8) {
                if constexpr (ALT && FAM == kLogreg) {
                    if (chr == 128) { run_tile<FAM, 32, 0, H, 128>(sP, tile, tiles, smem, tmem); break; }
                }
                run_tile<FAM, 32, 0, H>(sP, tile, tiles, smem, tmem);
            }
            break;
        case 64:
            if constexpr (64 / H >= 8) {
                if constexpr (ALT && FAM == kLogreg) {
                    if (chr == 128) { run_tile<FAM, 64, 0, H, 128>(sP, tile, tiles, smem, tmem); break; }
                }
                run_tile<FAM, 64, 0, H>(sP, tile, tiles, smem, tmem);
            }
            break;
        case 128: if constexpr (H == 2) run_tile<FAM, 128, 0, H>(sP, tile, tiles, smem, tmem); break;
        default: if (threadIdx.x == 0) atomicOr(sP.sp.status, 8u);
        }
        // every role has finished the tile (its copies and MMAs complete) before the barriers
        // and the item slot are reused
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

} // namespace tcs

cudaError_t launch_sweep_tcs_batch(int kind, int h, const void* d_params, const void* d_items, uint32_t n_items,
                                   uint32_t* d_head, uint32_t off_misc, uint32_t smem, int grid, cudaStream_t s,
                                   bool alt_chunks)
{
    auto go = [&](auto kern, int threads) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, s>>>(static_cast<const tcs::Params*>(d_params),
                                         static_cast<const uint2*>(d_items), n_items, d_head, off_misc);
        return cudaGetLastError();
    };
    if (h != 2) return cudaErrorInvalidValue;
    if (kind == kLinreg) {
        if (alt_chunks) return cudaErrorInvalidValue;
        return go(tcs::oais_sweep_tcs_batch_kernel<kLinreg, 2, false>, tcs::Roles<2>::threads(0));
    }
    if (alt_chunks) return go(tcs::oais_sweep_tcs_batch_kernel<kLogreg, 2, true>, tcs::Roles<2>::threads(0));
    return go(tcs::oais_sweep_tcs_batch_kernel<kLogreg, 2, false>, tcs::Roles<2>::threads(0));
}

} // namespace oais
