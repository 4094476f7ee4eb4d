// Product pass (p_x forward of a^ and b^, conj(a^) b^, p_x inverse keeping the
// Q lags; Sec. 3's convolution theorem along p_x) on the pruned engine
// (fft_pruned.cuh), software-pipelined across column tiles.
//
// The plain pruned kernel (k_x_product_pr) loads a tile, transforms it and
// stores it; with one 512-thread CTA per SM (registers and shared memory admit
// no second one at L = 1536) the SM waits for every tile's loads with nothing
// else to issue.  Here persistent CTAs walk the tiles, and the loads of tile
// i + G (G = grid size) are in flight while tile i is inverse-transformed:
// after the product the b^ operand's registers are free, and the one-operand
// inverse exchange uses only the lower part of the shared memory the
// two-operand forward exchange needed.  KR of the 16 nonzero input rows of a
// thread go to those registers, the other 16 - KR by cp.async (16 bytes, L2
// only) into the unused upper part of shared memory.  TWS: the twiddle tables
// of the length are copied once into shared memory (padded rows) and read
// from there.
//
// Same layouts and results as k_x_product_pr: U2 [N][L][2 SP] -> U3 [Q][L][SP].
#include "pr_tiles.cuh"
#include "tma.cuh"

namespace lh {

template <int L, int CW_, int KR, bool TWS>
struct PrPipe {
    static constexpr int CW = CW_, T = CW * L / 24, KS = 16 - KR;
    using EF = PrEng<L, CW, T, false, 2, true, false, TWS>;
    using EI = PrEng<L, CW, T, true, 1, false, true, TWS>;
    static_assert(EF::VPT == 24 && EI::VPT == 24 && EF::RL == EI::R0, "one 24-value block per thread");
    static constexpr int UPPER = (EI::SMEM_ELEMS + 1) & ~1;   // first float2 of the prefetch region (16-byte aligned)
    static constexpr int XCH_ELEMS = ((EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS) + 1) & ~1;
    static_assert(UPPER + 2 * KS * T <= XCH_ELEMS, "prefetched rows must fit beside the inverse exchange");
    // TWS: the twiddle tables of length L follow the exchange buffer
    static constexpr int TW_ELEMS = TWS ? (pr_tws_entries(L) + 1) & ~1 : 0;
    static constexpr int SMEM_ELEMS = XCH_ELEMS + TW_ELEMS;
};

__device__ __forceinline__ float4 ld_stream_v4(const float2 *p)
{
    float4 q;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
                 : "l"(p));
    return q;
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// the global tables of length L, stages ST.. of one direction, into the padded
// shared-memory layout (pr_tws_offset)
template <int L, int T, bool INV, int ST>
__device__ __forceinline__ void pr_tws_copy(const float2 *__restrict__ ptw, float2 *stw)
{
    if constexpr (ST < pr_nstages(L)) {
        constexpr int Rs = pr_radix(L, ST, INV), n = pr_ns(L, ST, INV) * Rs;
        const float2 *src = ptw + pr_tw_offset(L, INV, ST);
        float2 *dst = stw + pr_tws_offset(L, INV, ST);
        for (int e = threadIdx.x; e < n; e += T) dst[(e / Rs) * (Rs + 2) + e % Rs] = __ldg(src + e);
        pr_tws_copy<L, T, INV, ST + 1>(ptw, stw);
    }
}

template <int L, int CW_, int KR, bool TWS, bool ODD>
__global__ void __launch_bounds__(PrPipe<L, CW_, KR, TWS>::T, PrCfg<L, CW_>::MINB)
k_x_product_pr_pipe(Geom g, const float2 *__restrict__ U2, float2 *__restrict__ U3, const float2 *__restrict__ ptw)
{
    using PP = PrPipe<L, CW_, KR, TWS>;
    using EF = typename PP::EF;
    using EI = typename PP::EI;
    constexpr int T = PP::T, CW = PP::CW, KS = PP::KS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM(PP::SMEM_ELEMS, float2)
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float4 *pre = reinterpret_cast<float4 *>(sm + PP::UPPER);   // [KS][T]
    const float2 *tw = ptw;
    if constexpr (TWS) {   // this length's tables into shared memory (read after the first exchange's barrier)
        float2 *stw = sm + PP::XCH_ELEMS;
        pr_tws_copy<L, T, false, 1>(ptw, stw);
        pr_tws_copy<L, T, true, 1>(ptw, stw);
        tw = stw;
    }

    const int tiles_x = (g.H + CW - 1) / CW, ntiles = tiles_x * g.P;
    const long long rs = g.xs2;                                    // U2 stride between i_x rows
    const long long rstep = (long long)(L / 24) * rs;              // between a thread's rows
    const int cl = EF::col(), j = EF::jb(0);
    const float2 zero = make_float2(0.f, 0.f);
    int t = blockIdx.x;
    if (t >= ntiles) return;

    float2 va[24], vb[24];
    {   // the first tile straight into registers
        const int c = (t % tiles_x) * CW + cl;
        const float2 *p = U2 + (long long)(t / tiles_x) * (2 * g.SP) + 2 * c + (long long)j * rs;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (c < g.H) pr_ld2<false>(p + r * rstep, va[r], vb[r]);
            else { va[r] = zero; vb[r] = zero; }
        }
    }
    for (;;) {
        const int ky = t / tiles_x, c = (t % tiles_x) * CW + cl;
        const int nt = t + (int)gridDim.x;
        EF::run(va, vb, sm, tw);                     // ends with a barrier: the exchange is read
#pragma unroll
        for (int i = 0; i < 24; ++i) va[i] = odd_part(cmulc(vb[i], va[i]), ODD);

        // next tile's inputs: in flight during the inverse below
        const int nc = (nt % tiles_x) * CW + cl;
        const bool nvalid = nt < ntiles && nc < g.H;
        float4 q[KR];
        if (nvalid) {
            const float2 *p = U2 + (long long)(nt / tiles_x) * (2 * g.SP) + 2 * nc + (long long)j * rs;
#pragma unroll
            for (int r = 0; r < KR; ++r) q[r] = ld_stream_v4(p + r * rstep);
#pragma unroll
            for (int r = 0; r < KS; ++r) cp_async16(pre + r * T + threadIdx.x, p + (KR + r) * rstep);
        } else {
#pragma unroll
            for (int r = 0; r < KR; ++r) q[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();

        EI::run(va, va, sm, tw);
        if (c < g.H) {
            float2 *dst = U3 + (long long)ky * g.SP + c;
            const long long os = g.xs3;
            pr_store_lags<L, EI>(va, [&](int l, float2 x) { dst[(long long)l * os] = x; });
        }
        if (nt >= ntiles) break;
        cp_async_wait_all();
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            va[r] = make_float2(q[r].x, q[r].y);
            vb[r] = make_float2(q[r].z, q[r].w);
        }
#pragma unroll
        for (int r = 0; r < KS; ++r) {
            const float4 x = nvalid ? pre[r * T + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
            va[KR + r] = make_float2(x.x, x.y);
            vb[KR + r] = make_float2(x.z, x.w);
        }
        __syncthreads();   // every thread has its prefetched rows before the next exchange overwrites them
        t = nt;
    }
}

template <int L, int CW, int KR, bool TWS>
static cudaError_t x_product_pr_pipe_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using PP = PrPipe<L, CW, KR, TWS>;
    const size_t smem = sizeof(float2) * PP::SMEM_ELEMS;
    const bool odd = g.quantity == LINDHARD_IMCHI_T;
    auto k = odd ? k_x_product_pr_pipe<L, CW, KR, TWS, true> : k_x_product_pr_pipe<L, CW, KR, TWS, false>;
    static const cudaError_t e0 = smem_attrs(k_x_product_pr_pipe<L, CW, KR, TWS, false>, smem);
    static const cudaError_t e1 = smem_attrs(k_x_product_pr_pipe<L, CW, KR, TWS, true>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    int grid = 0;
    const int ntiles = ((g.H + PP::CW - 1) / PP::CW) * g.P;
    cudaError_t e = persistent_grid(k, PP::T, smem, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PP::T, smem, s>>>(g, (const float2 *)w.Y, (float2 *)w.X, (const float2 *)w.ptw);
    return cudaGetLastError();
}

bool pr_fwd_applies(const Geom &g);
bool pr_inv_applies(const Geom &g);

// product variant 9: 8 of the 16 input rows by registers, 8 by cp.async,
// twiddles through the read-only cache; 10: the same with the twiddles in
// shared memory
cudaError_t launch_x_product_pr_pipe(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_fwd_applies(g) || !pr_inv_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 9 ? x_product_pr_pipe_t<L, 8, 8, false>(g, w, s) : x_product_pr_pipe_t<L, 8, 8, true>(g, w, s))
    switch (g.P) {
    case 384: return CALL(384);
    case 768: return CALL(768);
    case 1536: return CALL(1536);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace lh
