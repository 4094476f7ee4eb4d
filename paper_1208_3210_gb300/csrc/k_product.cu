// The p_x pass: forward transform of both half spectra along p_x, their
// conjugate product (the convolution theorem of Sec. 3 turns the momentum and
// energy correlation of Eq. 9 into a pointwise product of transforms), and the
// inverse transform along p_x, keeping the Q lags q_x of the output.
//
// CTA = (column tile of energy frequencies, k_y).  Reads U2 [N][P][2 SP]
// (rows i_x < N; rows N..P-1 are the zero padding and are not stored), writes
// U3 [Q][P][SP]; both with the padded plane strides xs2 / xs3.  The forward and inverse transforms share the thread
// assignment of the last forward / first inverse stage, so the product
// conj(a^) b^ is formed in registers.
#include "kernels.cuh"

namespace lh {

// Engines of the product pass, shared by the kernel and its launcher.
// Forward: a^ and b^ of the same column as one pair (shared twiddles and
// barriers, two dependency chains per thread); inverse: the product alone.
template <typename Real, int L, typename Cfg>
struct XProduct {
    static constexpr int C = Cfg::C, T = Cfg::T;
    using EF = FftPair<Real, L, 2 * C, T, false>;
    using EI = Fft<Real, L, C, T, MAP_COL, true>;
    static_assert(EF::RL == EI::R0, "last forward radix must equal first inverse radix");
    static_assert(EF::VPT == EI::VPT && EF::CP == C, "forward pairs and inverse columns must coincide");
    static constexpr int SMEM_ELEMS = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
};

template <typename Real, int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_x_product(Geom g, const cx<Real> *__restrict__ U2, cx<Real> *__restrict__ U3,
            const cx<Real> *__restrict__ tw)
{
    using XP = XProduct<Real, L, Cfg>;
    constexpr int C = XP::C;
    using EF = typename XP::EF;
    using EI = typename XP::EI;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(XP::SMEM_ELEMS, Cx)

    const int W = 2 * g.SP;
    const int ky = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < g.H;
    const long long rstride = g.xs2;                  // U2 stride between i_x rows
    const Cx *src = U2 + (long long)ky * W + 2 * c;   // (a^, b^) of frequency c
    const Cx zero = mk<Cx>((Real)0, (Real)0);

    Cx va[EF::VPT], vb[EF::VPT];
#pragma unroll
    for (int b = 0; b < EF::VPT / EF::R0; ++b)
#pragma unroll
        for (int r = 0; r < EF::R0; ++r) {
            int n = EF::first_row(b, r);
            bool ld = valid && n < g.N;
            if (ld) gld2(src + (long long)n * rstride, va[b * EF::R0 + r], vb[b * EF::R0 + r]);
            else { va[b * EF::R0 + r] = zero; vb[b * EF::R0 + r] = zero; }
        }
    EF::run(va, vb, sm, tw);
    // conj(a^) * b^ : transform of the correlation C(q) = sum_p a(p) b(p + q);
    // for Im chi_T its odd part C(q) - C(-q), transform P - conj(P) = 2 i Im P
    const bool odd = g.quantity == LINDHARD_IMCHI_T;
#pragma unroll
    for (int i = 0; i < EF::VPT; ++i) va[i] = odd_part(cmulc(vb[i], va[i]), odd);
    EI::run(va, sm, tw);
    if (valid) {
        Cx *dst = U3 + (long long)ky * g.SP + c;
        const long long ostride = g.xs3;
#pragma unroll
        for (int b = 0; b < EI::VPT / EI::RL; ++b)
#pragma unroll
            for (int r = 0; r < EI::RL; ++r) {
                int col, n;
                EI::last_elem(b, r, col, n);
                int l = lag_index(n, g.P, g.Q);
                if (l >= 0) dst[(long long)l * ostride] = va[b * EI::RL + r];
            }
    }
}

template <typename Real, int L, typename Cfg>
cudaError_t launch_x_product_c(const Geom &g, const Work<Real> &w, cudaStream_t s)
{
    using XP = XProduct<Real, L, Cfg>;
    constexpr int C = XP::C, T = XP::T;
    size_t smem = sizeof(cx<Real>) * XP::SMEM_ELEMS;
    auto k = k_x_product<Real, L, Cfg>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.H + C - 1) / C, g.P);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.Y, (cx<Real> *)w.X, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

// variant 0: the tiles of XCfg; 1: 12 values per thread (3 * 2^k >= 192,
// FP32); 4: XCfg tiles with one more CTA per SM (FP32, L >= 128); 5: XCfg
// tiles twice as wide (FP32, L >= 384)
template <typename Real, int L>
cudaError_t launch_x_product_t(const Geom &g, const Work<Real> &w, cudaStream_t s, int variant)
{
    if constexpr (sizeof(Real) == 4 && fft_has_family1(L))
        if (variant == 1) return launch_x_product_c<Real, L, XCfg12<L>>(g, w, s);
    if constexpr (sizeof(Real) == 4 && L >= 128)
        if (variant == 4) return launch_x_product_c<Real, L, XCfgHi<L>>(g, w, s);
    if constexpr (sizeof(Real) == 4 && L >= 384 && XCfg<L>::T <= 256)
        if (variant == 5) return launch_x_product_c<Real, L, XCfgW<L>>(g, w, s);
    return launch_x_product_c<Real, L, XCfg<L>>(g, w, s);
}

cudaError_t launch_x_product_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_x_product_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_x_product_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s);
cudaError_t launch_x_product_pr_pipe(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
// variants 2, 3: the TMA-staged persistent kernels of k_tma.cu; 6, 7: the
// pruned engine of k_pruned.cu (one-third padding); 8: its TMA-staged
// persistent form (k_pruned_tma.cu); 9, 10: its software-pipelined persistent
// form (k_product_pipe.cu)
cudaError_t launch_x_product(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (variant == 8) return launch_x_product_pr_tma(g, w, s);
    if (variant == 9 || variant == 10) return launch_x_product_pr_pipe(g, w, s, variant);
    if (variant == 2 || variant == 3) return launch_x_product_tma(g, w, s, variant);
    if (variant == 6 || variant == 7) return launch_x_product_pr(g, w, s, variant);
#define CALL(L) launch_x_product_t<float, L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_x_product(const Geom &g, const Work<double> &w, cudaStream_t s, int variant)
{
#define CALL(L) launch_x_product_t<double, L>(g, w, s, variant)
    LH_LEN_SWITCH_SMALL(g.P, CALL)
#undef CALL
}

}  // namespace lh

namespace lh {
// Every momentum length's default tiles (the engines a plan runs without the
// autotuner) fit in the 227 KB of shared memory a CTA can have.
template <int L>
constexpr bool default_tiles_fit()
{
    constexpr size_t cap = 227 * 1024;
    using XP = XProduct<float, L, XCfg<L>>;
    constexpr size_t col = sizeof(float2) * Fft<float, L, ColCfg<L>::C, ColCfg<L>::T, MAP_COL, true>::SMEM_ELEMS;
    constexpr size_t x = sizeof(float2) * XP::SMEM_ELEMS;
    if constexpr (L >= 128) {
        constexpr size_t pair = sizeof(float2) * FftPair<float, L, PairCfg<L>::C, PairCfg<L>::T, false>::SMEM_ELEMS;
        return col <= cap && x <= cap && pair <= cap;
    }
    return col <= cap && x <= cap;
}
static_assert(default_tiles_fit<16>() && default_tiles_fit<32>() && default_tiles_fit<48>() &&
                  default_tiles_fit<64>() && default_tiles_fit<96>() && default_tiles_fit<128>() &&
                  default_tiles_fit<192>() && default_tiles_fit<256>() && default_tiles_fit<384>() &&
                  default_tiles_fit<512>() && default_tiles_fit<768>() && default_tiles_fit<1024>() &&
                  default_tiles_fit<1536>() && default_tiles_fit<2048>() && default_tiles_fit<4096>(),
              "a default tile exceeds the shared memory of a CTA");
}  // namespace lh
