// Inverse passes of the correlation.
//
//   k_inv_y      : inverse transform along p_y of the product spectrum, keeping
//                  the Q lags q_y.  U3 [Q][P][SP] -> U4 [Q][Q][SP].
//   k_inv_energy : inverse real transform along energy.  For fixed (q_x, q_y)
//                  the product spectrum is Hermitian in the energy frequency
//                  (the correlation is real), so two output lines share one
//                  complex inverse FFT: W(k) = X1(k) + i X2(k), with X(k) for
//                  k > PE/2 rebuilt as conj X(PE - k); Re w = line 1, Im w =
//                  line 2.  Keeps w_m = m de for m < n_omega and applies the
//                  prefactor of Eq. 9, -(de / 2 pi)(1 / npz^2), with the FFT
//                  normalisation 1 / (P P PE).  Writes out [Q][Q][n_omega].
#include "kernels.cuh"

namespace lh {

template <typename Real, int L>
__global__ void __launch_bounds__(ColCfg<L>::T, ColCfg<L>::MINB)
k_inv_y(Geom g, const cx<Real> *__restrict__ U3, cx<Real> *__restrict__ U4,
        const cx<Real> *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, true>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)

    const int lx = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < g.H;
    const Cx *src = U3 + (long long)lx * g.xs3 + c;
    Cx *dst = U4 + (long long)lx * g.Q * g.SP + c;

    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            v[b * E::R0 + r] = valid ? src[(long long)n * g.SP] : mk<Cx>((Real)0, (Real)0);
        }
    E::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int col, n;
                E::last_elem(b, r, col, n);
                int l = lag_index(n, g.P, g.Q);
                if (l >= 0) dst[(long long)l * g.SP] = v[b * E::RL + r];
            }
    }
}

// Paired-column version of the inverse p_y pass (L >= 128).
template <typename Real, int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_inv_y2(Geom g, const cx<Real> *__restrict__ U3, cx<Real> *__restrict__ U4,
         const cx<Real> *__restrict__ tw)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<Real, L, C, T, true>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)

    const int lx = blockIdx.y;
    const int c = blockIdx.x * C + 2 * E::pair();
    const bool valid = c < g.H;                   // c + 1 < SP: the pair stays in the row
    const Cx *src = U3 + (long long)lx * g.xs3 + c;
    Cx *dst = U4 + (long long)lx * g.Q * g.SP + c;
    const Cx zero = mk<Cx>((Real)0, (Real)0);

    Cx va[E::VPT], vb[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            if (valid) gld2(src + (long long)E::first_row(b, r) * g.SP, va[b * E::R0 + r], vb[b * E::R0 + r]);
            else { va[b * E::R0 + r] = zero; vb[b * E::R0 + r] = zero; }
        }
    E::run(va, vb, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int l = lag_index(E::last_row(b, r), g.P, g.Q);
                if (l >= 0) gst2(dst + (long long)l * g.SP, va[b * E::RL + r], vb[b * E::RL + r]);
            }
    }
}

// FP32, power-of-two lengths: at most 64 registers a thread (four 256-thread
// CTAs per SM at L = 512): the pass waits on its loads, and resident warps are
// what hides them (the FP64 and 3 * 2^k forms need more registers)
template <typename Real, int L>
struct InvEnergyBounds {
    static constexpr int MINB = (sizeof(Real) == 4 && fft_len_pow2(L)) ? 65536 / (LineCfg<L>::T * 64) : 1;
};
template <typename Real, typename OutT, int L>
__global__ void __launch_bounds__(LineCfg<L>::T, InvEnergyBounds<Real, L>::MINB)
k_inv_energy(Geom g, const cx<Real> *__restrict__ U4, OutT *__restrict__ out,
             const cx<Real> *__restrict__ tw)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, true>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)

    const long long npairs = (long long)g.Q * g.Q / 2;
    const long long f0 = (long long)blockIdx.x * C;
    constexpr int H = L / 2 + 1;                 // non-redundant frequencies (= g.H)
    constexpr int SP = (H + 7) / 8 * 8;          // row stride (= g.SP)

    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            long long f = f0 + col;
            Cx w = mk<Cx>((Real)0, (Real)0);
            if (f < npairs) {
                const Cx *row1 = U4 + (2 * f) * SP;
                const Cx *row2 = row1 + SP;
                Cx x1, x2;
                if (n < H) { x1 = row1[n]; x2 = row2[n]; }
                else { x1 = cconj(row1[L - n]); x2 = cconj(row2[L - n]); }
                w = mk<Cx>(x1.x - x2.y, x1.y + x2.x);   // X1 + i X2
            }
            v[b * E::R0 + r] = w;
        }
    E::run(v, sm, tw);
    const Real sc = (Real)g.scale;
#pragma unroll
    for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
        for (int r = 0; r < E::RL; ++r) {
            int col, n;
            E::last_elem(b, r, col, n);
            long long f = f0 + col;
            if (f < npairs && n < g.n_omega) {
                Cx w = v[b * E::RL + r];
                out[(2 * f) * g.n_omega + n] = (OutT)(sc * w.x);
                out[(2 * f + 1) * g.n_omega + n] = (OutT)(sc * w.y);
            }
        }
}

template <typename Real, int L, typename Cfg>
cudaError_t launch_inv_y2_t(const Geom &g, const Work<Real> &w, cudaStream_t s)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<Real, L, C, T, true>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = k_inv_y2<Real, L, Cfg>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.H + C - 1) / C, g.Q);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.X, (cx<Real> *)w.Y, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

// variant 0: single-column engine; 1: paired-column engine (L >= 128, FP32);
// 2: paired-column engine with 12 values per thread (3 * 2^k >= 192, FP32);
// 6: paired-column engine on tiles twice as wide (L >= 384, FP32)
template <typename Real, int L>
cudaError_t launch_inv_y_t(const Geom &g, const Work<Real> &w, cudaStream_t s, int variant)
{
    if constexpr (L >= 128 && sizeof(Real) == 4) {
        if (variant == 1) return launch_inv_y2_t<Real, L, PairCfg<L>>(g, w, s);
        if constexpr (fft_has_family1(L))
            if (variant == 2) return launch_inv_y2_t<Real, L, PairCfg12<L>>(g, w, s);
        if constexpr (L >= 384 && PairCfg<L>::T <= 512)
            if (variant == 6) return launch_inv_y2_t<Real, L, PairCfgW<L>>(g, w, s);
    }
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, true>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = k_inv_y<Real, L>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.H + C - 1) / C, g.Q);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.X, (cx<Real> *)w.Y, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

template <typename Real, typename OutT, int L>
cudaError_t launch_inv_energy_t(const Geom &g, const Work<Real> &w, OutT *out, cudaStream_t s)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, true>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = k_inv_energy<Real, OutT, L>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    long long npairs = (long long)g.Q * g.Q / 2;
    unsigned grid = (unsigned)((npairs + C - 1) / C);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.Y, out, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

cudaError_t launch_inv_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_y_tc(const Geom &g, const Work<float> &w, cudaStream_t s);
// variants 3, 4: the TMA-staged persistent kernels of k_tma.cu
cudaError_t launch_inv_y_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_y_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
// 8, 9: the pruned engine of k_pruned.cu (one-third padding); 10: its
// TMA-staged persistent form, 11 the same with two CTAs per SM
// (k_pruned_tma.cu)
cudaError_t launch_inv_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (variant == 10 || variant == 11) return launch_inv_y_pr_tma(g, w, s, variant);
    if (variant >= 3 && variant <= 5) return launch_inv_y_tma(g, w, s, variant);
    if (variant == 8 || variant == 9) return launch_inv_y_pr(g, w, s, variant);
    if (variant == 7) return launch_inv_y_tc(g, w, s);   // tensor-core stages (k_tc.cu)
#define CALL(L) launch_inv_y_t<float, L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_inv_y(const Geom &g, const Work<double> &w, cudaStream_t s, int variant)
{
#define CALL(L) launch_inv_y_t<double, L>(g, w, s, variant)
    LH_LEN_SWITCH_SMALL(g.P, CALL)
#undef CALL
}
cudaError_t launch_inv_energy_tma(const Geom &g, const Work<float> &w, float *out, cudaStream_t s);
cudaError_t launch_inv_energy_warp(const Geom &g, const Work<float> &w, float *out, cudaStream_t s);
// variant 1: the TMA-staged persistent kernel of k_tma.cu; 2: one warp per
// pair of output lines (k_energy.cu)
cudaError_t launch_inv_energy(const Geom &g, const Work<float> &w, float *out, cudaStream_t s, int variant)
{
    if (variant == 1) return launch_inv_energy_tma(g, w, out, s);
    if (variant == 2) return launch_inv_energy_warp(g, w, out, s);
#define CALL(L) launch_inv_energy_t<float, float, L>(g, w, out, s)
    LH_P_SWITCH(g.PE, CALL)
#undef CALL
}
cudaError_t launch_inv_energy(const Geom &g, const Work<double> &w, double *out, cudaStream_t s, int variant)
{
    (void)variant;
#define CALL(L) launch_inv_energy_t<double, double, L>(g, w, out, s)
    LH_LEN_SWITCH_SMALL(g.PE, CALL)
#undef CALL
}

}  // namespace lh
