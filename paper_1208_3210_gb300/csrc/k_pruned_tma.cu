// TMA-staged persistent forms of the pruned momentum passes (FP32; the
// transforms of k_pruned.cu, the staging of k_tma.cu): persistent CTAs walk
// the column tiles, and while one tile is transformed on the pruned engine
// (fft_pruned.cuh) the tensor memory accelerator already copies the next
// tile's input columns into a shared-memory staging buffer (one buffer: the
// copy of tile i + 1 is issued once every thread has taken tile i's values).
// Waits are bounded (1 s of %globaltimer); a CTA that gives up records
// DEV_ETIMEOUT, lets its copy in flight land and leaves.  Tiles of CP = 4
// column pairs (64-byte row segments) on 256 threads, 24 values per thread.
#include <algorithm>

#include "pr_tiles.cuh"
#include "tma.cuh"

namespace lh {

constexpr int PT_CP = 4, PT_C = 2 * PT_CP;

template <int L>
struct PtFwd {   // one CTA per SM, registers to spare: packed complex sums
    static constexpr int T = PT_CP * L / 24;
    using E = PrEng<L, PT_CP, T, false, 2, true, false, false, true>;
};
template <int L>
struct PtInv {
    static constexpr int T = PT_CP * L / 24;
    using E = PrEng<L, PT_CP, T, true, 2, false, true, false, true>;
};
// Two CTAs per SM (128 registers a thread, plain complex sums): the staging
// buffer and the exchange share one region, so the next tile's copy is issued
// once the transform has left the shared memory (its global stores and the
// other CTA's tile overlap the copy, not the transform).
template <int L>
struct PtFwd2 {
    static constexpr int T = PT_CP * L / 24;
    using E = PrEng<L, PT_CP, T, false, 2, true, false, false, false>;
};
template <int L>
struct PtInv2 {
    static constexpr int T = PT_CP * L / 24;
    using E = PrEng<L, PT_CP, T, true, 2, false, true, false, false>;
};
// shared staging + exchange region, then the mbarrier
__host__ __device__ constexpr size_t pt_shared_bytes(size_t stage_bytes, size_t fft_bytes)
{
    return ((stage_bytes > fft_bytes ? stage_bytes : fft_bytes) + 15) / 16 * 16;
}

template <int L>
struct PtProd {
    static constexpr int FC = PT_CP;           // frequencies per tile: one (its a^, b^) per thread column
    static constexpr int T = FC * L / 24;
    using P = PrProduct<L, FC, T>;
};

// ---------------------------------------------------------------------------
// p_y forward: U1 [N][N][2 SP] -> U2 [N][L][2 SP]; tile = (PT_C columns, i_x),
// staging [NR][PT_C] (the N nonzero rows).
template <int L>
__global__ void __launch_bounds__(PtFwd<L>::T, 1)
k_fwd_y_pr_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U2,
               const float2 *__restrict__ ptw, unsigned *status, int box_rows)
{
    using E = typename PtFwd<L>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (g.N + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{(size_t)NR * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int W = 2 * g.SP, tiles_x = (W + PT_C - 1) / PT_C, ntiles = tiles_x * g.N;
    const unsigned tx = (unsigned)(NR * PT_C * sizeof(float2));
    auto issue = [&](int t) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * PT_C, &map, 2 * c0, q * box_rows, ix, bar);
    };
    const TileRun run(ntiles, true);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::col();
    for (int t = run.t; t < run.end; t += run.step) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / 24; ++b) {
            const float2 *s = stage + (size_t)E::jb(b) * PT_C + 2 * p;
#pragma unroll
            for (int r = 0; r < 16; ++r) {   // rows jb + r L/24 < N (the padding rows are not staged)
                const float4 q = *reinterpret_cast<const float4 *>(s + (size_t)(r * (L / 24)) * PT_C);
                va[24 * b + r] = make_float2(q.x, q.y);
                vb[24 * b + r] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();   // the staging buffer is free
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(va, vb, sm, ptw);
        const int c = c0 + 2 * p;
        if (c < W && ab_col_valid(c, g.H)) {   // (c, c + 1) = (a^, b^) of one frequency
            float2 *dst = U2 + (long long)ix * g.xs2 + c;
#pragma unroll
            for (int b = 0; b < E::VPT / E::RL; ++b) {
                float2 *q = dst + (long long)E::jb(b) * W;
#pragma unroll
                for (int r = 0; r < E::RL; ++r)
                    gst2(q + (long long)(r * (L / E::RL)) * W, va[b * E::RL + r], vb[b * E::RL + r]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// p_y inverse: U3 [Q][L][SP] (plane stride xs3) -> U4 [Q][Q][SP]; tile =
// (PT_C columns over [0, H), l_x), staging [NR][PT_C] (all L rows).
template <int L>
__global__ void __launch_bounds__(PtInv<L>::T, 1)
k_inv_y_pr_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U4,
               const float2 *__restrict__ ptw, unsigned *status, int box_rows)
{
    using E = typename PtInv<L>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (L + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{(size_t)NR * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int tiles_x = (g.H + PT_C - 1) / PT_C, ntiles = tiles_x * g.Q;
    const unsigned tx = (unsigned)(NR * PT_C * sizeof(float2));
    auto issue = [&](int t) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * PT_C, &map, 2 * c0, q * box_rows, lx, bar);
    };
    const TileRun run(ntiles, false);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::col();
    for (int t = run.t; t < run.end; t += run.step) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b) {
            const float2 *s = stage + (size_t)E::jb(b) * PT_C + 2 * p;
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                const float4 q = *reinterpret_cast<const float4 *>(s + (size_t)(r * (L / E::R0)) * PT_C);
                va[b * E::R0 + r] = make_float2(q.x, q.y);
                vb[b * E::R0 + r] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(va, vb, sm, ptw);
        const int c = c0 + 2 * p;
        if (c < g.H) {
            float2 *dst = U4 + (long long)lx * g.Q * g.SP + c;
            const int sp = g.SP;
#pragma unroll
            for (int b = 0; b < E::VPT / 24; ++b) {
                const int j = E::jb(b);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    gst2(dst + (long long)(j + r * (L / 24) + L / 3) * sp, va[24 * b + r], vb[24 * b + r]);
                    gst2(dst + (long long)(j + r * (L / 24)) * sp, va[24 * b + 16 + r], vb[24 * b + 16 + r]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same two passes, two CTAs per SM (PtFwd2, PtInv2).
template <int L>
__global__ void __launch_bounds__(PtFwd2<L>::T, 2)
k_fwd_y_pr_tma2(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U2,
                const float2 *__restrict__ ptw, unsigned *status, int box_rows)
{
    using E = typename PtFwd2<L>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (g.N + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const size_t buf = pt_shared_bytes((size_t)NR * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2));
    if (dyn_smem_bytes() < buf + 16) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = stage;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + buf);

    const int W = 2 * g.SP, tiles_x = (W + PT_C - 1) / PT_C, ntiles = tiles_x * g.N;
    const unsigned tx = (unsigned)(NR * PT_C * sizeof(float2));
    auto issue = [&](int t) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * PT_C, &map, 2 * c0, q * box_rows, ix, bar);
    };
    const TileRun run(ntiles, true);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::col();
    for (int t = run.t; t < run.end; t += run.step) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / 24; ++b) {
            const float2 *s = stage + (size_t)E::jb(b) * PT_C + 2 * p;
#pragma unroll
            for (int r = 0; r < 16; ++r) {   // rows jb + r L/24 < N (the padding rows are not staged)
                const float4 q = *reinterpret_cast<const float4 *>(s + (size_t)(r * (L / 24)) * PT_C);
                va[24 * b + r] = make_float2(q.x, q.y);
                vb[24 * b + r] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();   // the staging is read: the exchange may overwrite it
        E::run(va, vb, sm, ptw);   // ends with a barrier: the region is free
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        const int c = c0 + 2 * p;
        if (c < W && ab_col_valid(c, g.H)) {
            float2 *dst = U2 + (long long)ix * g.xs2 + c;
#pragma unroll
            for (int b = 0; b < E::VPT / E::RL; ++b) {
                float2 *q = dst + (long long)E::jb(b) * W;
#pragma unroll
                for (int r = 0; r < E::RL; ++r)
                    gst2(q + (long long)(r * (L / E::RL)) * W, va[b * E::RL + r], vb[b * E::RL + r]);
            }
        }
    }
}

template <int L>
__global__ void __launch_bounds__(PtInv2<L>::T, 2)
k_inv_y_pr_tma2(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U4,
                const float2 *__restrict__ ptw, unsigned *status, int box_rows)
{
    using E = typename PtInv2<L>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (L + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const size_t buf = pt_shared_bytes((size_t)NR * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2));
    if (dyn_smem_bytes() < buf + 16) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = stage;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + buf);

    const int tiles_x = (g.H + PT_C - 1) / PT_C, ntiles = tiles_x * g.Q;
    const unsigned tx = (unsigned)(NR * PT_C * sizeof(float2));
    auto issue = [&](int t) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * PT_C, &map, 2 * c0, q * box_rows, lx, bar);
    };
    const TileRun run(ntiles, false);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::col();
    for (int t = run.t; t < run.end; t += run.step) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * PT_C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b) {
            const float2 *s = stage + (size_t)E::jb(b) * PT_C + 2 * p;
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                const float4 q = *reinterpret_cast<const float4 *>(s + (size_t)(r * (L / E::R0)) * PT_C);
                va[b * E::R0 + r] = make_float2(q.x, q.y);
                vb[b * E::R0 + r] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();
        E::run(va, vb, sm, ptw);
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        const int c = c0 + 2 * p;
        if (c < g.H) {
            float2 *dst = U4 + (long long)lx * g.Q * g.SP + c;
            const int sp = g.SP;
#pragma unroll
            for (int b = 0; b < E::VPT / 24; ++b) {
                const int j = E::jb(b);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    gst2(dst + (long long)(j + r * (L / 24) + L / 3) * sp, va[24 * b + r], vb[24 * b + r]);
                    gst2(dst + (long long)(j + r * (L / 24)) * sp, va[24 * b + 16 + r], vb[24 * b + 16 + r]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// p_x product: U2 [N][L][2 SP] (plane stride xs2) -> U3 [Q][L][SP]; tile =
// (FC frequencies, k_y), staging [NR][FC][2] = (a^, b^) per frequency.
template <int L, bool ODD>
__global__ void __launch_bounds__(PtProd<L>::T, 1)
k_x_product_pr_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U3,
                   const float2 *__restrict__ ptw, unsigned *status, int box_rows)
{
    using EF = typename PtProd<L>::P::EF;
    using EI = typename PtProd<L>::P::EI;
    constexpr int FC = PtProd<L>::FC;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (g.N + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{2 * (size_t)NR * FC * sizeof(float2), (size_t)PtProd<L>::P::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int tiles_x = (g.H + FC - 1) / FC, ntiles = tiles_x * g.P;
    const unsigned tx = (unsigned)(2 * NR * FC * sizeof(float2));
    auto issue = [&](int t) {
        const int ky = t / tiles_x, c0 = (t % tiles_x) * FC;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q)
            tma_load_3d(stage + (size_t)q * box_rows * 2 * FC, &map, 4 * c0, ky, q * box_rows, bar);
    };
    const TileRun run(ntiles, false);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int col = EF::col();
    for (int t = run.t; t < run.end; t += run.step) {
        const int ky = t / tiles_x, c0 = (t % tiles_x) * FC;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[EF::VPT], vb[EF::VPT];
#pragma unroll
        for (int b = 0; b < EF::VPT / 24; ++b) {
            const float2 *s = stage + ((size_t)EF::jb(b) * FC + col) * 2;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float4 q = *reinterpret_cast<const float4 *>(s + (size_t)(r * (L / 24)) * FC * 2);
                va[24 * b + r] = make_float2(q.x, q.y);
                vb[24 * b + r] = make_float2(q.z, q.w);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        EF::run(va, vb, sm, ptw);
#pragma unroll
        for (int i = 0; i < EF::VPT; ++i) va[i] = odd_part(cmulc(vb[i], va[i]), ODD);   // conj(a^) b^
        EI::run(va, va, sm, ptw);
        const int c = c0 + col;
        if (c < g.H) {
            float2 *dst = U3 + (long long)ky * g.SP + c;
            const long long os = g.xs3;
            pr_store_lags<L, EI>(va, [&](int l, float2 x) { dst[(long long)l * os] = x; });
        }
    }
}

// ---------------------------------------------------------------------------
// Host side (maps as the TMA passes of k_tma.cu).
template <int L>
static cudaError_t fwd_y_pr_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using E = typename PtFwd<L>::E;
    const int box_rows = tma_box_rows(g.N), nbox = (g.N + box_rows - 1) / box_rows;
    const TmaSmem lay{(size_t)nbox * box_rows * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_fwd_y_pr_tma<L>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 4ull * g.SP, (unsigned long long)g.N, (unsigned long long)g.N, 16ull * g.SP,
                     16ull * g.SP * g.N, 2 * PT_C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((2 * g.SP + PT_C - 1) / PT_C) * g.N;
    if (e == cudaSuccess) e = persistent_grid(k, PtFwd<L>::T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PtFwd<L>::T, lay.total(), s>>>(g, map, (float2 *)w.Y, (const float2 *)w.ptw, w.status, box_rows);
    return cudaGetLastError();
}
template <int L>
static cudaError_t inv_y_pr_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using E = typename PtInv<L>::E;
    const int box_rows = tma_box_rows(L), nbox = (L + box_rows - 1) / box_rows;
    const TmaSmem lay{(size_t)nbox * box_rows * PT_C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_inv_y_pr_tma<L>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 2ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.Q, 8ull * g.SP,
                     8ull * (unsigned long long)g.xs3, 2 * PT_C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((g.H + PT_C - 1) / PT_C) * g.Q;
    if (e == cudaSuccess) e = persistent_grid(k, PtInv<L>::T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PtInv<L>::T, lay.total(), s>>>(g, map, (float2 *)w.Y, (const float2 *)w.ptw, w.status, box_rows);
    return cudaGetLastError();
}
template <int L>
static cudaError_t fwd_y_pr_tma2_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using E = typename PtFwd2<L>::E;
    const int box_rows = tma_box_rows(g.N), nbox = (g.N + box_rows - 1) / box_rows;
    const size_t smem = pt_shared_bytes((size_t)nbox * box_rows * PT_C * sizeof(float2),
                                        (size_t)E::SMEM_ELEMS * sizeof(float2)) + 16;
    auto k = k_fwd_y_pr_tma2<L>;
    cudaError_t e = smem_attrs(k, smem);
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 4ull * g.SP, (unsigned long long)g.N, (unsigned long long)g.N, 16ull * g.SP,
                     16ull * g.SP * g.N, 2 * PT_C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((2 * g.SP + PT_C - 1) / PT_C) * g.N;
    if (e == cudaSuccess) e = persistent_grid(k, PtFwd2<L>::T, smem, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PtFwd2<L>::T, smem, s>>>(g, map, (float2 *)w.Y, (const float2 *)w.ptw, w.status, box_rows);
    return cudaGetLastError();
}
template <int L>
static cudaError_t inv_y_pr_tma2_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using E = typename PtInv2<L>::E;
    const int box_rows = tma_box_rows(L), nbox = (L + box_rows - 1) / box_rows;
    const size_t smem = pt_shared_bytes((size_t)nbox * box_rows * PT_C * sizeof(float2),
                                        (size_t)E::SMEM_ELEMS * sizeof(float2)) + 16;
    auto k = k_inv_y_pr_tma2<L>;
    cudaError_t e = smem_attrs(k, smem);
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 2ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.Q, 8ull * g.SP,
                     8ull * (unsigned long long)g.xs3, 2 * PT_C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((g.H + PT_C - 1) / PT_C) * g.Q;
    if (e == cudaSuccess) e = persistent_grid(k, PtInv2<L>::T, smem, ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PtInv2<L>::T, smem, s>>>(g, map, (float2 *)w.Y, (const float2 *)w.ptw, w.status, box_rows);
    return cudaGetLastError();
}
template <int L>
static cudaError_t x_product_pr_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int FC = PtProd<L>::FC;
    const int box_rows = tma_box_rows(g.N), nbox = (g.N + box_rows - 1) / box_rows;
    const TmaSmem lay{2 * (size_t)nbox * box_rows * FC * sizeof(float2),
                      (size_t)PtProd<L>::P::SMEM_ELEMS * sizeof(float2)};
    const bool odd = g.quantity == LINDHARD_IMCHI_T;
    auto k = odd ? k_x_product_pr_tma<L, true> : k_x_product_pr_tma<L, false>;
    cudaError_t e = smem_attrs(k_x_product_pr_tma<L, true>, lay.total());
    if (e == cudaSuccess) e = smem_attrs(k_x_product_pr_tma<L, false>, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.Y, 4ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.N, 16ull * g.SP,
                     8ull * (unsigned long long)g.xs2, 4 * FC, 1, box_rows);
    int grid = 0;
    const int ntiles = ((g.H + FC - 1) / FC) * g.P;
    if (e == cudaSuccess) e = persistent_grid(k, PtProd<L>::T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, PtProd<L>::T, lay.total(), s>>>(g, map, (float2 *)w.X, (const float2 *)w.ptw, w.status, box_rows);
    return cudaGetLastError();
}

bool pr_fwd_applies(const Geom &g);
bool pr_inv_applies(const Geom &g);

#define LH_PT_SWITCH(L_, CALL)                                   \
    switch (L_) {                                                \
    case 384: return CALL(384);                                  \
    case 768: return CALL(768);                                  \
    case 1536: return CALL(1536);                                \
    default: return cudaErrorInvalidValue;                       \
    }
// p_y variant 10 (11: two CTAs per SM), product variant 8 (P in {384, 768, 1536})
cudaError_t launch_fwd_y_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_fwd_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 11 ? fwd_y_pr_tma2_t<L>(g, w, s) : fwd_y_pr_tma_t<L>(g, w, s))
    LH_PT_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_inv_y_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_inv_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 11 ? inv_y_pr_tma2_t<L>(g, w, s) : inv_y_pr_tma_t<L>(g, w, s))
    LH_PT_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_x_product_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    if (!pr_fwd_applies(g) || !pr_inv_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) x_product_pr_tma_t<L>(g, w, s)
    LH_PT_SWITCH(g.P, CALL)
#undef CALL
}

}  // namespace lh
