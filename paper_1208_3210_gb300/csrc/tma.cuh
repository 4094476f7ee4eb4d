// TMA (tensor memory accelerator) helpers shared by the TMA-staged passes and
// the tensor-core pass: the 3D tile copy, the tile walk of a persistent CTA,
// bounded waits for a staged tile, and the host-side tensor-map encoding
// (3D FP32 maps, no swizzle) and persistent grid sizing.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "async.cuh"
#include "lindhard_internal.h"

namespace lh {

// Shared-memory layout of a pipelined CTA: [staging][FFT exchange][mbarrier].
// The staging buffer starts at the (128-byte aligned) dynamic base.
struct TmaSmem {
    size_t stage_bytes, fft_bytes;
    __host__ __device__ size_t total() const { return stage_bytes + fft_bytes + 16; }
};

// TMA copy of one 3D box into shared memory, completion counted on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_addr(bar))
        : "memory");
}

// Tiles of a persistent CTA: a contiguous run (neighbouring column tiles, whose
// row segments share DRAM lines, consumed back to back by one CTA: measured
// faster for the p_y forward pass on the 1024^2 x 512 grid) or every
// gridDim-th tile (neighbours processed at the same time by neighbouring CTAs:
// faster for the inverse and the product passes).
struct TileRun {
    int t, end, step;
    __device__ TileRun(int ntiles, bool contiguous)
    {
        if (contiguous) {
            const int per = (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
            t = min(ntiles, (int)blockIdx.x * per);
            end = min(ntiles, t + per);
            step = 1;
        } else {
            t = blockIdx.x;
            end = ntiles;
            step = gridDim.x;
        }
    }
};

// Records a timeout once; every thread of the CTA calls it with the same ok.
__device__ __forceinline__ bool tile_ready(unsigned long long *bar, unsigned parity, unsigned *status)
{
    const bool ok = mbar_wait_bounded(bar, parity);
    const int all = __syncthreads_and(ok ? 1 : 0);
    if (!all && threadIdx.x == 0) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ETIMEOUT);
    return all != 0;
}
// After a timeout: give the copy in flight (bounded) time to land before the
// CTA's shared memory is released.
__device__ __forceinline__ void drain(unsigned long long *bar, unsigned parity)
{
    if (threadIdx.x == 0) (void)mbar_wait_bounded(bar, parity);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Host side.

// Rows per box (at most 256, the TMA limit): the n rows split evenly into
// ceil(n / 256) boxes, so little staging goes to rows past the end.
inline int tma_box_rows(int n)
{
    const int nbox = (n + 255) / 256;
    return (n + nbox - 1) / nbox;
}
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// 3D FP32 tensor map: dims (fastest first) d0 x d1 x d2, byte strides s1, s2,
// box b0 x b1 x b2 (floats / rows).
inline cudaError_t make_map(CUtensorMap *m, const void *base, unsigned long long d0, unsigned long long d1,
                            unsigned long long d2, unsigned long long s1, unsigned long long s2, unsigned b0,
                            unsigned b1, unsigned b2)
{
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {s1, s2};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Persistent grid: every SM filled to its occupancy, no more CTAs than tiles.
template <typename K>
cudaError_t persistent_grid(K k, int T, size_t smem, int ntiles, int &grid)
{
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, T, smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    grid = std::min(ntiles, sms * per);
    return cudaSuccess;
}

}  // namespace lh
