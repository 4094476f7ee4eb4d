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
//   k_bw_product_pr: the adjoint's p_x products (k_backward.cu's
//                    k_bw_product on this engine), see below.
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

// The adjoint's products along p_x (k_bw_product, same layouts): W^ of the
// weights, a^ and b^ forward, h^ = W^ a^ and g^ = conj(W^) b^ (W^ - conj(W^)
// for Im chi_T) inverse, p_x < N kept, h over a^ and g over b^.  Both ends fit
// the pruned engine through a shift: the Q lag rows l (lag l - Q/2, at
// circular index l - Q/2) are loaded as rows [0, Q), so W^(k) = W_0(k)
// e^{2 pi i k (Q/2)/P} = W_0(k) w^k with w = e^{2 pi i/3} (Q/2 = P/3); and the
// inverse of X(k) w^k is x(m - 2P/3), so the kept rows of the pruned inverse
// (m' < P/3 and m' >= 2P/3) hold p_x = m' + P/3 mod P, exactly the rows
// [0, N) (the row map of pr_store_lags).  The frequency of forward output
// (b, r) is k = jb(b) + r L/RL, so k mod 3 = jb(b) mod 3 (L/RL a multiple of
// 3): one phase per butterfly.
template <int L, typename Cfg, bool ODD>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_bw_product_pr(Geom g, float2 *__restrict__ U2, const float2 *__restrict__ WU2, const float2 *__restrict__ ptw)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using EF2 = PrEng<L, C, T, false, 2, true, false>;
    using EF1 = PrEng<L, C, T, false, 1, true, false>;
    using EI = PrEng<L, C, T, true, 1, false, true>;
    static_assert(EF2::RL == EI::R0 && EF2::VPT == EI::VPT && EF2::VPT == 24 && (L / EF2::RL) % 3 == 0,
                  "forward outputs feed the inverse; one 24-value block per thread");
    // W^ waits in shared memory (each thread's own values) beside the
    // one-operand exchange while h^ is inverted and b^ transformed
    constexpr int PARK = (EI::SMEM_ELEMS + 1) & ~1;
    constexpr int SE = EF2::SMEM_ELEMS > PARK + 24 * T ? EF2::SMEM_ELEMS : PARK + 24 * T;
    static_assert(EF1::SMEM_ELEMS <= PARK, "the one-operand forward exchange stays below the parked W^");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM(SE, float2)
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *park = sm + PARK;
    const int ky = blockIdx.y;
    const int c = blockIdx.x * C + EF2::col();
    const bool valid = c < g.H;
    const long long rs = g.xs2, ws = g.xs3;
    float2 *colA = U2 + (long long)ky * (2 * g.SP) + 2 * c;   // a^, later h^
    float2 *colB = colA + 1;                                  // b^, later g^
    const float2 *colW = WU2 + (long long)ky * g.SP + c;
    const float2 zero = make_float2(0.f, 0.f);
    const int j = EF2::jb(0);
    // w^(k mod 3) of the frequencies of forward output butterfly b
    auto phase = [](int b) {
        const int k3 = EF2::jb(b) % 3;
        return k3 == 0 ? make_float2(1.f, 0.f)
                       : make_float2(-0.5f, k3 == 1 ? 0.866025403784438647f : -0.866025403784438647f);
    };

    float2 vw[24], v[24];
    {
        const float2 *pw = colW + (long long)j * ws, *pa = colA + (long long)j * rs;
        const long long dw = (long long)(L / 24) * ws, da = (long long)(L / 24) * rs;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            vw[r] = valid ? __ldg(pw + r * dw) : zero;
            v[r] = valid ? __ldg(pa + r * da) : zero;
        }
    }
    EF2::run(vw, v, sm, ptw);
#pragma unroll
    for (int b = 0; b < 24 / EF2::RL; ++b) {
        const float2 ph = phase(b);
#pragma unroll
        for (int r = 0; r < EF2::RL; ++r) {
            const int i = b * EF2::RL + r;
            float2 wt = cmul(vw[i], ph);                     // W^ at its true lags
            if (ODD) wt = make_float2(0.f, 2.f * wt.y);      // w(s) - w(-s)
            park[i * T + threadIdx.x] = wt;                  // (EF2 has left the shared memory)
            v[i] = cmul(cmul(wt, v[i]), ph);                 // h^, shifted for the kept rows
        }
    }
    EI::run(v, v, sm, ptw);
    if (valid) pr_store_lags<L, EI>(v, [&](int l, float2 x) { colA[(long long)l * rs] = x; });
    {
        const float2 *pb = colB + (long long)j * rs;
        const long long db = (long long)(L / 24) * rs;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = valid ? __ldg(pb + r * db) : zero;
    }
    EF1::run(v, v, sm, ptw);
#pragma unroll
    for (int b = 0; b < 24 / EF2::RL; ++b) {
        const float2 ph = phase(b);
#pragma unroll
        for (int r = 0; r < EF2::RL; ++r) {
            const int i = b * EF2::RL + r;
            v[i] = cmul(cmulc(v[i], park[i * T + threadIdx.x]), ph);   // g^ = conj(W^) b^, shifted
        }
    }
    EI::run(v, v, sm, ptw);
    if (valid) pr_store_lags<L, EI>(v, [&](int l, float2 x) { colB[(long long)l * rs] = x; });
}

template <int L>
cudaError_t launch_bw_product_pr_t(const Geom &g, float2 *U2, const float2 *WU2, const float2 *ptw, cudaStream_t s)
{
    using Cfg = PrCfg<L, 8>;
    using EF2 = PrEng<L, 8, Cfg::T, false, 2, true, false>;
    using EI = PrEng<L, 8, Cfg::T, true, 1, false, true>;
    constexpr int PARK = (EI::SMEM_ELEMS + 1) & ~1;
    const size_t smem = sizeof(float2) * (EF2::SMEM_ELEMS > PARK + 24 * Cfg::T ? EF2::SMEM_ELEMS : PARK + 24 * Cfg::T);
    const bool odd = g.quantity == LINDHARD_IMCHI_T;
    auto k = odd ? k_bw_product_pr<L, Cfg, true> : k_bw_product_pr<L, Cfg, false>;
    static const cudaError_t e0 = smem_attrs(k_bw_product_pr<L, Cfg, false>, smem);
    static const cudaError_t e1 = smem_attrs(k_bw_product_pr<L, Cfg, true>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    dim3 grid((g.H + 7) / 8, g.P);
    k<<<grid, Cfg::T, smem, s>>>(g, U2, WU2, ptw);
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
cudaError_t launch_bw_product_pr(const Geom &g, float2 *U2, const float2 *WU2, const float2 *ptw, cudaStream_t s)
{
    if (!pr_fwd_applies(g) || !pr_inv_applies(g) || !ptw) return cudaErrorInvalidValue;
#define CALL(L) launch_bw_product_pr_t<L>(g, U2, WU2, ptw, s)
    LH_PR_SWITCH(g.P, CALL)
#undef CALL
}

}  // namespace lh
