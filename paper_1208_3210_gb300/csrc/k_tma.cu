// TMA-staged, software-pipelined momentum passes (FP32).
//
// The same transforms as k_fwd_y2 / k_inv_y2 / k_x_product (Sec. 3: FFTs
// along p_y, the p_x product pass, the inverse along p_y), restructured for
// latency: persistent CTAs walk the column tiles, and while a CTA transforms
// one tile in registers, the tensor memory accelerator already copies the
// next tile's input columns from HBM into a shared-memory staging buffer
// (cp.async.bulk.tensor, completion counted on an mbarrier).  The copy of tile
// i + 1 is issued once every thread has moved tile i from the staging buffer
// into registers, so one buffer suffices; the FFT exchanges use a separate
// shared-memory region.  Waits are bounded (1 s of %globaltimer): a CTA that
// gives up records DEV_ETIMEOUT in the status word, waits (bounded) for its
// copy in flight and leaves.
//
// Tensor maps (3D, FP32 elements, no swizzle) are encoded on the host per
// launch from the workspace pointers; a complex value is two floats, so a
// column offset c is the float coordinate 2c (16-byte aligned for even c).
#include <algorithm>

#include "kernels.cuh"
#include "tma.cuh"

namespace lh {



// CTAs per SM the register budget is sized for: the tile config's own count,
// unless shared memory (staging for an estimated number of rows plus the FFT
// exchange) admits fewer.
__host__ __device__ constexpr int tma_minb(int minb, long long bytes)
{
    return bytes <= 0 ? minb : (225000 / bytes < 1 ? 1 : (225000 / bytes < minb ? (int)(225000 / bytes) : minb));
}
// Rows staged per tile in the usual geometry: N = 2P/3 for 3 * 2^k lengths
// (rounded up to 256-row boxes beyond 256), P otherwise.
__host__ __device__ constexpr long long tma_rows_est(int L, bool all_rows)
{
    return all_rows || fft_len_pow2(L) ? (L <= 256 ? L : (L + 255) / 256 * 256)
                                       : (2 * L / 3 <= 256 ? 2 * L / 3 : (2 * L / 3 + 255) / 256 * 256);
}
template <int L, typename Cfg, bool INV>
struct PairTmaBounds {
    using E = FftPair<float, L, Cfg::C, Cfg::T, INV>;
    static constexpr int MINB =
        tma_minb(Cfg::MINB, tma_rows_est(L, INV) * Cfg::C * 8 + (long long)E::SMEM_ELEMS * 8 + 16);
};
template <int L, typename Cfg>
struct XTmaBounds {
    using EF = FftPair<float, L, 2 * Cfg::C, Cfg::T, false>;
    static constexpr int MINB =
        tma_minb(Cfg::MINB, 2 * tma_rows_est(L, false) * Cfg::C * 8 + (long long)EF::SMEM_ELEMS * 8 + 16);
};

// ---------------------------------------------------------------------------
// p_y forward: U1 [N][N][2 SP] -> U2 [N][P][2 SP].  Tile = (column tile of C
// columns, i_x); staging [NR][C] (NR = N rounded up to the box height).
template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, (PairTmaBounds<L, Cfg, false>::MINB))
k_fwd_y_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U2,
            const float2 *__restrict__ tw, unsigned *status, int box_rows)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<float, L, C, T, false>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (g.N + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{(size_t)NR * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int W = 2 * g.SP, tiles_x = (W + C - 1) / C, ntiles = tiles_x * g.N;
    const unsigned tx = (unsigned)(nbox * box_rows * C * sizeof(float2));
    auto issue = [&](int t) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * C, &map, 2 * c0, q * box_rows, ix, bar);
    };
    const TileRun run(ntiles, true);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::pair();
    for (int t = run.t; t < run.end; t += run.step) {
        const int ix = t / tiles_x, c0 = (t % tiles_x) * C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                const int n = E::first_row(b, r);
                if (n < g.N) {
                    float4 q = *reinterpret_cast<const float4 *>(&stage[(size_t)n * C + 2 * p]);
                    va[b * E::R0 + r] = make_float2(q.x, q.y);
                    vb[b * E::R0 + r] = make_float2(q.z, q.w);
                } else {
                    va[b * E::R0 + r] = make_float2(0.f, 0.f);
                    vb[b * E::R0 + r] = make_float2(0.f, 0.f);
                }
            }
        __syncthreads();   // the staging buffer is free
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(va, vb, sm, tw);
        const int c = c0 + 2 * p;
        if (c < W && ab_col_valid(c, g.H)) {   // (c, c + 1) = (a^, b^) of one frequency
            float2 *dst = U2 + (long long)ix * g.xs2 + c;
#pragma unroll
            for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
                for (int r = 0; r < E::RL; ++r)
                    gst2(dst + (long long)E::last_row(b, r) * W, va[b * E::RL + r], vb[b * E::RL + r]);
        }
    }
}

// ---------------------------------------------------------------------------
// p_y inverse: U3 [Q][P][SP] (plane stride xs3) -> U4 [Q][Q][SP].  Tile =
// (column tile over [0, H), l_x); staging [NR][C], NR = P rounded up.
template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, (PairTmaBounds<L, Cfg, true>::MINB))
k_inv_y_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U4,
            const float2 *__restrict__ tw, unsigned *status, int box_rows)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    // packed complex sums where the launch leaves at least 192 registers a thread
    constexpr bool PK = 65536 / (T * PairTmaBounds<L, Cfg, true>::MINB) >= 192;
    using E = FftPair<float, L, C, T, true, PK>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (L + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{(size_t)NR * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int tiles_x = (g.H + C - 1) / C, ntiles = tiles_x * g.Q;
    const unsigned tx = (unsigned)(nbox * box_rows * C * sizeof(float2));
    auto issue = [&](int t) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * C, &map, 2 * c0, q * box_rows, lx, bar);
    };
    const TileRun run(ntiles, false);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int p = E::pair();
    for (int t = run.t; t < run.end; t += run.step) {
        const int lx = t / tiles_x, c0 = (t % tiles_x) * C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[E::VPT], vb[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                float4 q = *reinterpret_cast<const float4 *>(&stage[(size_t)E::first_row(b, r) * C + 2 * p]);
                va[b * E::R0 + r] = make_float2(q.x, q.y);
                vb[b * E::R0 + r] = make_float2(q.z, q.w);
            }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(va, vb, sm, tw);
        const int c = c0 + 2 * p;
        if (c < g.H) {
            float2 *dst = U4 + (long long)lx * g.Q * g.SP + c;
#pragma unroll
            for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
                for (int r = 0; r < E::RL; ++r) {
                    const int l = lag_index(E::last_row(b, r), g.P, g.Q);
                    if (l >= 0) gst2(dst + (long long)l * g.SP, va[b * E::RL + r], vb[b * E::RL + r]);
                }
        }
    }
}

// ---------------------------------------------------------------------------
// p_x pass with the conjugate product: U2 [N][P][2 SP] (plane stride xs2) ->
// U3 [Q][P][SP].  Tile = (column tile over [0, H), k_y); staging
// [NR][C][2] = (a^, b^) of each frequency (one box per row block), NR = N
// rounded up.
template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, (XTmaBounds<L, Cfg>::MINB))
k_x_product_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U3,
                const float2 *__restrict__ tw, unsigned *status, int box_rows)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using EF = FftPair<float, L, 2 * C, T, false>;
    using EI = Fft<float, L, C, T, MAP_COL, true>;
    static_assert(EF::RL == EI::R0 && EF::VPT == EI::VPT && EF::CP == C, "forward and inverse tiles must coincide");
    constexpr int FFT_ELEMS = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nbox = (g.N + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{2 * (size_t)NR * C * sizeof(float2), (size_t)FFT_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);   // [NR][C][2]: (a^, b^) per frequency
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const int tiles_x = (g.H + C - 1) / C, ntiles = tiles_x * g.P;
    const unsigned tx = (unsigned)(2 * nbox * box_rows * C * sizeof(float2));
    auto issue = [&](int t) {
        const int ky = t / tiles_x, c0 = (t % tiles_x) * C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) {
            tma_load_3d(stage + (size_t)q * box_rows * 2 * C, &map, 4 * c0, ky, q * box_rows, bar);
        }
    };
    const TileRun run(ntiles, false);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    const int col = (int)(threadIdx.x % C);
    const bool odd = g.quantity == LINDHARD_IMCHI_T;   // Im chi_T: the odd part P - conj(P)
    for (int t = run.t; t < run.end; t += run.step) {
        const int ky = t / tiles_x, c0 = (t % tiles_x) * C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 va[EF::VPT], vb[EF::VPT];
#pragma unroll
        for (int b = 0; b < EF::VPT / EF::R0; ++b)
#pragma unroll
            for (int r = 0; r < EF::R0; ++r) {
                const int n = EF::first_row(b, r);
                const bool ld = n < g.N;
                if (ld) {
                    const float4 q = *reinterpret_cast<const float4 *>(&stage[((size_t)n * C + col) * 2]);
                    va[b * EF::R0 + r] = make_float2(q.x, q.y);
                    vb[b * EF::R0 + r] = make_float2(q.z, q.w);
                } else {
                    va[b * EF::R0 + r] = make_float2(0.f, 0.f);
                    vb[b * EF::R0 + r] = make_float2(0.f, 0.f);
                }
            }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        EF::run(va, vb, sm, tw);
#pragma unroll
        for (int i = 0; i < EF::VPT; ++i) va[i] = odd_part(cmulc(vb[i], va[i]), odd);   // conj(a^) b^
        EI::run(va, sm, tw);
        const int c = c0 + col;
        if (c < g.H) {
            float2 *dst = U3 + (long long)ky * g.SP + c;
#pragma unroll
            for (int b = 0; b < EI::VPT / EI::RL; ++b)
#pragma unroll
                for (int r = 0; r < EI::RL; ++r) {
                    int cl, n;
                    EI::last_elem(b, r, cl, n);
                    const int l = lag_index(n, g.P, g.Q);
                    if (l >= 0) dst[(long long)l * g.xs3] = va[b * EI::RL + r];
                }
        }
    }
}


// ---------------------------------------------------------------------------
// Single-column forms of the two p_y passes (ColCfg tiles, 8-byte values):
// each thread transforms one column; same staging and pipeline as above.
template <int L, bool INV>
struct ColTmaBounds {
    using E = Fft<float, L, ColCfg<L>::C, ColCfg<L>::T, MAP_COL, INV>;
    static constexpr int MINB =
        tma_minb(ColCfg<L>::MINB, tma_rows_est(L, INV) * ColCfg<L>::C * 8 + (long long)E::SMEM_ELEMS * 8 + 16);
};

template <int L, bool INV>
__global__ void __launch_bounds__(ColCfg<L>::T, (ColTmaBounds<L, INV>::MINB))
k_y_col_tma(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ out,
            const float2 *__restrict__ tw, unsigned *status, int box_rows)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, INV>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int rows = INV ? L : g.N;   // input rows per column
    const int nbox = (rows + box_rows - 1) / box_rows, NR = nbox * box_rows;
    const TmaSmem lay{(size_t)NR * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    // forward: columns of U1 rows (2 SP wide), planes i_x; inverse: columns
    // [0, H) of U3 rows (SP wide), planes l_x
    const int W = INV ? g.SP : 2 * g.SP;
    const int tiles_x = INV ? (g.H + C - 1) / C : (W + C - 1) / C;
    const int ntiles = tiles_x * (INV ? g.Q : g.N);
    const unsigned tx = (unsigned)(nbox * box_rows * C * sizeof(float2));
    auto issue = [&](int t) {
        const int pl = t / tiles_x, c0 = (t % tiles_x) * C;
        mbar_expect_tx(bar, tx);
        for (int q = 0; q < nbox; ++q) tma_load_3d(stage + (size_t)q * box_rows * C, &map, 2 * c0, q * box_rows, pl, bar);
    };
    const TileRun run(ntiles, !INV);   // forward: contiguous runs, as the paired forward pass
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    unsigned parity = 0;
    for (int t = run.t; t < run.end; t += run.step) {
        const int pl = t / tiles_x, c0 = (t % tiles_x) * C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 v[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                int col, n;
                E::first_elem(b, r, col, n);
                v[b * E::R0 + r] = n < rows ? stage[(size_t)n * C + col] : make_float2(0.f, 0.f);
            }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(v, sm, tw);
        const int c = c0 + (int)(threadIdx.x % C);
        if (INV) {
            if (c < g.H) {
                float2 *dst = out + (long long)pl * g.Q * g.SP + c;
#pragma unroll
                for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
                    for (int r = 0; r < E::RL; ++r) {
                        int col, n;
                        E::last_elem(b, r, col, n);
                        const int l = lag_index(n, g.P, g.Q);
                        if (l >= 0) dst[(long long)l * g.SP] = v[b * E::RL + r];
                    }
            }
        } else if (c < W && ab_col_valid(c, g.H)) {
            float2 *dst = out + (long long)pl * g.xs2 + c;
#pragma unroll
            for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
                for (int r = 0; r < E::RL; ++r) {
                    int col, n;
                    E::last_elem(b, r, col, n);
                    dst[(long long)n * W] = v[b * E::RL + r];
                }
        }
    }
}


// ---------------------------------------------------------------------------
// Inverse energy pass (same transform as k_inv_energy): U4 [Q^2][SP] rows ->
// out [Q^2][n_omega].  Tile = C pairs of rows (2 C rows), staged by one box
// of a 3D view (row split into nbx chunks of bx columns) as plain
// [2 C][SP] complex.
template <int L>
__global__ void __launch_bounds__(LineCfg<L>::T)
k_inv_energy_tma(Geom g, const __grid_constant__ CUtensorMap map, float *__restrict__ out,
                 const float2 *__restrict__ tw, unsigned *status, int bx, int nbx)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_LINE, true>;
    constexpr int H = L / 2 + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const TmaSmem lay{(size_t)nbx * 2 * C * bx * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    if (dyn_smem_bytes() < lay.total()) return;
    float2 *stage = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + lay.stage_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem_raw + lay.stage_bytes + lay.fft_bytes);

    const long long npairs = (long long)g.Q * g.Q / 2;
    const int ntiles = (int)((npairs + C - 1) / C);
    const unsigned tx = (unsigned)(nbx * 2 * C * bx * sizeof(float2));
    const TileRun run(ntiles, false);
    auto issue = [&](int t) {
        mbar_expect_tx(bar, tx);
        tma_load_3d(stage, &map, 0, 0, 2 * t * C, bar);
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (run.t < run.end) issue(run.t);
    }
    __syncthreads();
    // element m of staged row rr
    const int SPs = nbx * bx;
    auto at = [&](int rr, int m) { return stage[(size_t)rr * SPs + m]; };
    unsigned parity = 0;
    const float sc = (float)g.scale;
    for (int t = run.t; t < run.end; t += run.step) {
        const long long f0 = (long long)t * C;
        if (!tile_ready(bar, parity, status)) { drain(bar, parity); return; }
        parity ^= 1u;
        float2 v[E::VPT];
#pragma unroll
        for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
            for (int r = 0; r < E::R0; ++r) {
                int col, n;
                E::first_elem(b, r, col, n);
                float2 x1, x2;
                if (n < H) { x1 = at(2 * col, n); x2 = at(2 * col + 1, n); }
                else { x1 = cconj(at(2 * col, L - n)); x2 = cconj(at(2 * col + 1, L - n)); }
                v[b * E::R0 + r] = make_float2(x1.x - x2.y, x1.y + x2.x);   // X1 + i X2
            }
        __syncthreads();
        if (threadIdx.x == 0 && t + run.step < run.end) {
            fence_proxy_async();
            issue(t + run.step);
        }
        E::run(v, sm, tw);
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int col, n;
                E::last_elem(b, r, col, n);
                const long long f = f0 + col;
                if (f < npairs && n < g.n_omega) {
                    const float2 w = v[b * E::RL + r];
                    out[(2 * f) * g.n_omega + n] = sc * w.x;
                    out[(2 * f + 1) * g.n_omega + n] = sc * w.y;
                }
            }
    }
}

// ---------------------------------------------------------------------------
// Host side.

template <int L, typename Cfg>
static cudaError_t launch_fwd_y_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<float, L, C, T, false>;
    const int box_rows = tma_box_rows(g.N), nbox = (g.N + box_rows - 1) / box_rows;
    const TmaSmem lay{(size_t)nbox * box_rows * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_fwd_y_tma<L, Cfg>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 4ull * g.SP, (unsigned long long)g.N, (unsigned long long)g.N, 16ull * g.SP,
                     16ull * g.SP * g.N, 2 * C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((2 * g.SP + C - 1) / C) * g.N;
    if (e == cudaSuccess) e = persistent_grid(k, T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, T, lay.total(), s>>>(g, map, (float2 *)w.Y, twiddles_for<float>(w, L), w.status, box_rows);
    return cudaGetLastError();
}

template <int L, typename Cfg>
static cudaError_t launch_inv_y_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<float, L, C, T, true>;
    const int box_rows = tma_box_rows(L), nbox = (L + box_rows - 1) / box_rows;
    const TmaSmem lay{(size_t)nbox * box_rows * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_inv_y_tma<L, Cfg>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.X, 2ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.Q, 8ull * g.SP,
                     8ull * (unsigned long long)g.xs3, 2 * C, box_rows, 1);
    int grid = 0;
    const int ntiles = ((g.H + C - 1) / C) * g.Q;
    if (e == cudaSuccess) e = persistent_grid(k, T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, T, lay.total(), s>>>(g, map, (float2 *)w.Y, twiddles_for<float>(w, L), w.status, box_rows);
    return cudaGetLastError();
}

template <int L, typename Cfg>
static cudaError_t launch_x_product_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using EF = FftPair<float, L, 2 * C, T, false>;
    using EI = Fft<float, L, C, T, MAP_COL, true>;
    constexpr int FFT_ELEMS = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
    const int box_rows = tma_box_rows(g.N), nbox = (g.N + box_rows - 1) / box_rows;
    const TmaSmem lay{2 * (size_t)nbox * box_rows * C * sizeof(float2), (size_t)FFT_ELEMS * sizeof(float2)};
    auto k = k_x_product_tma<L, Cfg>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    if (e == cudaSuccess)
        e = make_map(&map, w.Y, 4ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.N, 16ull * g.SP,
                     8ull * (unsigned long long)g.xs2, 4 * C, 1, box_rows);
    int grid = 0;
    const int ntiles = ((g.H + C - 1) / C) * g.P;
    if (e == cudaSuccess) e = persistent_grid(k, T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, T, lay.total(), s>>>(g, map, (float2 *)w.X, twiddles_for<float>(w, L), w.status, box_rows);
    return cudaGetLastError();
}


template <int L, bool INV>
static cudaError_t launch_y_col_tma_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, INV>;
    const int rows = INV ? L : g.N;
    const int box_rows = tma_box_rows(rows), nbox = (rows + box_rows - 1) / box_rows;
    const TmaSmem lay{(size_t)nbox * box_rows * C * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_y_col_tma<L, INV>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    int ntiles = 0;
    if (e == cudaSuccess) {
        if (INV) {
            e = make_map(&map, w.X, 2ull * g.SP, (unsigned long long)g.P, (unsigned long long)g.Q, 8ull * g.SP,
                         8ull * (unsigned long long)g.xs3, 2 * C, box_rows, 1);
            ntiles = ((g.H + C - 1) / C) * g.Q;
        } else {
            e = make_map(&map, w.X, 4ull * g.SP, (unsigned long long)g.N, (unsigned long long)g.N, 16ull * g.SP,
                         16ull * g.SP * g.N, 2 * C, box_rows, 1);
            ntiles = ((2 * g.SP + C - 1) / C) * g.N;
        }
    }
    int grid = 0;
    if (e == cudaSuccess) e = persistent_grid(k, T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, T, lay.total(), s>>>(g, map, (float2 *)w.Y, twiddles_for<float>(w, L), w.status, box_rows);
    return cudaGetLastError();
}


// Columns per box for rows of SP complex values: at most 128 (256 floats, the
// TMA box limit), dividing SP evenly into an even count.
static bool energy_boxes(int SP, int &bx, int &nbx)
{
    for (nbx = (2 * SP + 255) / 256; nbx <= SP; ++nbx)
        if (SP % nbx == 0 && (SP / nbx) % 2 == 0 && 2 * (SP / nbx) <= 256) {
            bx = SP / nbx;
            return true;
        }
    return false;
}

template <int L>
static cudaError_t launch_inv_energy_tma_t(const Geom &g, const Work<float> &w, float *out, cudaStream_t s)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_LINE, true>;
    int bx = 0, nbx = 0;
    if (!energy_boxes(g.SP, bx, nbx)) return cudaErrorNotSupported;
    const TmaSmem lay{(size_t)nbx * 2 * C * bx * sizeof(float2), (size_t)E::SMEM_ELEMS * sizeof(float2)};
    auto k = k_inv_energy_tma<L>;
    cudaError_t e = smem_attrs(k, lay.total());
    CUtensorMap map;
    const unsigned long long rows = (unsigned long long)g.Q * g.Q;
    // 3D view of the rows: (2 bx floats, nbx chunks, rows); one box = 2 C rows
    if (e == cudaSuccess)
        e = make_map(&map, w.Y, 2ull * bx, (unsigned long long)nbx, rows, 8ull * bx, 8ull * g.SP, 2 * bx, nbx, 2 * C);
    int grid = 0;
    const int ntiles = (int)(((long long)g.Q * g.Q / 2 + C - 1) / C);
    if (e == cudaSuccess) e = persistent_grid(k, T, lay.total(), ntiles, grid);
    if (e != cudaSuccess) return e;
    k<<<grid, T, lay.total(), s>>>(g, map, out, twiddles_for<float>(w, L), w.status, bx, nbx);
    return cudaGetLastError();
}

cudaError_t launch_inv_energy_tma(const Geom &g, const Work<float> &w, float *out, cudaStream_t s)
{
#define CALL(L) launch_inv_energy_tma_t<L>(g, w, out, s)
    LH_P_SWITCH(g.PE, CALL)
#undef CALL
}

// Entry points.  p_y passes: variant 3 = PairCfg tiles, 4 = PairCfg12 tiles,
// 5 = single-column ColCfg tiles;
// product pass: variant 2 = XCfg tiles, 3 = XCfg12 tiles.  Lengths >= 128.
template <int L>
static cudaError_t fwd_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if constexpr (L >= 128) {
        if (variant == 3) return launch_fwd_y_tma_t<L, PairCfg<L>>(g, w, s);
        if (variant == 5) return launch_y_col_tma_t<L, false>(g, w, s);
        if constexpr (fft_has_family1(L))
            if (variant == 4) return launch_fwd_y_tma_t<L, PairCfg12<L>>(g, w, s);
    }
    return cudaErrorInvalidValue;
}
template <int L>
static cudaError_t inv_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if constexpr (L >= 128) {
        if (variant == 3) return launch_inv_y_tma_t<L, PairCfg<L>>(g, w, s);
        if (variant == 5) return launch_y_col_tma_t<L, true>(g, w, s);
        if constexpr (fft_has_family1(L))
            if (variant == 4) return launch_inv_y_tma_t<L, PairCfg12<L>>(g, w, s);
    }
    return cudaErrorInvalidValue;
}
template <int L>
static cudaError_t x_product_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if constexpr (L >= 128) {
        if (variant == 2) return launch_x_product_tma_t<L, XCfg<L>>(g, w, s);
        if constexpr (fft_has_family1(L))
            if (variant == 3) return launch_x_product_tma_t<L, XCfg12<L>>(g, w, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
#define CALL(L) fwd_y_tma<L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_inv_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
#define CALL(L) inv_y_tma<L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_x_product_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
#define CALL(L) x_product_tma<L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}

}  // namespace lh
