// Momentum passes on the pruned engine (fft_pruned.cuh), for geometries whose
// momentum padding is exactly one third: L = 3N/2 (forward passes) and
// L = 3Q/2 (inverse passes), the default Q = N extended zone (Sec. 3's
// zero-padded convolution theorem; lags |s| <= N/2).
//
//   k_fwd_y_pr     : p_y forward of both half spectra, U1 [N][N][2 SP] ->
//                    U2 [N][L][2 SP]; the N nonzero input rows only.
//   k_x_product_pr : p_x forward of a^ and b^, conj(a^) b^ (Im chi_T: its odd
//                    part), p_x inverse, keeping the Q lags; U2 -> U3 [Q][L][SP].
//   k_inv_y_pr     : p_y inverse keeping the Q lags, U3 -> U4 [Q][Q][SP].
//
// The same transforms as k_fwd_y2 / k_x_product / k_inv_y2 (same layouts),
// with the zero rows neither loaded nor transformed in the first forward
// stage and the unkept lags not formed in the last inverse stage.
#include "pr_tiles.cuh"

namespace lh {

__global__ void k_pr_twiddles(float2 *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= pr_twiddle_entries()) return;
    for (int li = 0; li < 4; ++li)
        for (int d = 0; d < 2; ++d) {
            const int L = pr_len_of(li);
            for (int s = 1; s < pr_nstages(L); ++s) {
                const int off = pr_tables_before(li, d, s), n = pr_table_entries(L, d != 0, s);
                if (e >= off && e < off + n) {
                    const int Rs = pr_radix(L, s, d != 0), NR = pr_ns(L, s + 1, d != 0);
                    // row k holds w^1, w^2, ..., w^(Rs-1), w^0 (position p: power p + 1)
                    const int k = (e - off) / Rs, r = ((e - off) % Rs + 1) % Rs;
                    double sn, cs;
                    sincospi(-2.0 * (double)((k * r) % NR) / (double)NR, &sn, &cs);
                    out[e] = make_float2((float)cs, (float)sn);
                    return;
                }
            }
        }
}

cudaError_t launch_pr_twiddles(float2 *out, cudaStream_t s)
{
    const int n = pr_twiddle_entries();
    k_pr_twiddles<<<(n + 255) / 256, 256, 0, s>>>(out);
    return cudaGetLastError();
}
size_t pr_twiddle_bytes() { return (size_t)pr_twiddle_entries() * sizeof(float2); }

template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_fwd_y_pr(Geom g, const float2 *__restrict__ U1, float2 *__restrict__ U2, const float2 *__restrict__ ptw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM((PrEng<L, Cfg::C, Cfg::T, false, 2, true, false>::SMEM_ELEMS), float2)
    fwd_y_pr_tile<L, Cfg::C, Cfg::T, false>(g, U1, U2, ptw, reinterpret_cast<float2 *>(smem_raw), blockIdx.x,
                                            blockIdx.y);
}

template <int L, typename Cfg, bool ODD>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_x_product_pr(Geom g, const float2 *__restrict__ U2, float2 *__restrict__ U3, const float2 *__restrict__ ptw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM((PrProduct<L, Cfg::C, Cfg::T>::SMEM_ELEMS), float2)
    x_product_pr_tile<L, Cfg::C, Cfg::T, ODD, false>(g, U2, U3, ptw, reinterpret_cast<float2 *>(smem_raw),
                                                     blockIdx.x, blockIdx.y);
}

template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_inv_y_pr(Geom g, const float2 *__restrict__ U3, float2 *__restrict__ U4, const float2 *__restrict__ ptw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM((PrEng<L, Cfg::C, Cfg::T, true, 2, false, true>::SMEM_ELEMS), float2)
    inv_y_pr_tile<L, Cfg::C, Cfg::T, false>(g, U3, U4, ptw, reinterpret_cast<float2 *>(smem_raw), blockIdx.x,
                                            blockIdx.y);
}

// ---------------------------------------------------------------------------
// Launchers.  Variants: A = 8 columns (pairs) per tile, B = 4.
template <int L, int CW>
cudaError_t launch_fwd_y_pr_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using Cfg = PrCfg<L, CW>;
    using E = PrEng<L, CW, Cfg::T, false, 2, true, false>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    auto k = k_fwd_y_pr<L, Cfg>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((2 * g.SP + 2 * CW - 1) / (2 * CW), g.N);
    k<<<grid, Cfg::T, smem, s>>>(g, (const float2 *)w.X, (float2 *)w.Y, (const float2 *)w.ptw);
    return cudaGetLastError();
}

template <int L, int CW>
cudaError_t launch_x_product_pr_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using Cfg = PrCfg<L, CW>;
    using EF = PrEng<L, CW, Cfg::T, false, 2, true, false>;
    using EI = PrEng<L, CW, Cfg::T, true, 1, false, true>;
    size_t smem = sizeof(float2) * (EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS);
    const bool odd = g.quantity == LINDHARD_IMCHI_T;
    auto k = odd ? k_x_product_pr<L, Cfg, true> : k_x_product_pr<L, Cfg, false>;
    static const cudaError_t e0 = smem_attrs(k_x_product_pr<L, Cfg, false>, smem);
    static const cudaError_t e1 = smem_attrs(k_x_product_pr<L, Cfg, true>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    dim3 grid((g.H + CW - 1) / CW, g.P);
    k<<<grid, Cfg::T, smem, s>>>(g, (const float2 *)w.Y, (float2 *)w.X, (const float2 *)w.ptw);
    return cudaGetLastError();
}

template <int L, int CW>
cudaError_t launch_inv_y_pr_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    using Cfg = PrCfg<L, CW>;
    using E = PrEng<L, CW, Cfg::T, true, 2, false, true>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    auto k = k_inv_y_pr<L, Cfg>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.H + 2 * CW - 1) / (2 * CW), g.Q);
    k<<<grid, Cfg::T, smem, s>>>(g, (const float2 *)w.X, (float2 *)w.Y, (const float2 *)w.ptw);
    return cudaGetLastError();
}

// The pruned forms apply when the padding is exactly one third.
bool pr_fwd_applies(const Geom &g) { return pr_supported(g.P) && 3 * g.N == 2 * g.P && !g.periodic; }
bool pr_inv_applies(const Geom &g) { return pr_supported(g.P) && 3 * g.Q == 2 * g.P && !g.periodic; }

#define LH_PR_SWITCH(L_, CALL)                                   \
    switch (L_) {                                                \
    case 192: return CALL(192);                                  \
    case 384: return CALL(384);                                  \
    case 768: return CALL(768);                                  \
    case 1536: return CALL(1536);                                \
    default: return cudaErrorInvalidValue;                       \
    }

// variant 8: 8 column pairs per tile; 9: 4
cudaError_t launch_fwd_y_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_fwd_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 8 ? launch_fwd_y_pr_t<L, 8>(g, w, s) : launch_fwd_y_pr_t<L, 4>(g, w, s))
    LH_PR_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_inv_y_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_inv_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 8 ? launch_inv_y_pr_t<L, 8>(g, w, s) : launch_inv_y_pr_t<L, 4>(g, w, s))
    LH_PR_SWITCH(g.P, CALL)
#undef CALL
}
// variant 6: 8 columns per tile; 7: 4
cudaError_t launch_x_product_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (!pr_fwd_applies(g) || !pr_inv_applies(g) || !w.ptw) return cudaErrorInvalidValue;
#define CALL(L) (variant == 6 ? launch_x_product_pr_t<L, 8>(g, w, s) : launch_x_product_pr_t<L, 4>(g, w, s))
    LH_PR_SWITCH(g.P, CALL)
#undef CALL
}

}  // namespace lh
