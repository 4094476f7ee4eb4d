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
#include "fft_pruned.cuh"
#include "kernels.cuh"

namespace lh {

// Tiles: A = CW 8 (128-byte row segments of the paired layouts), B = CW 4;
// both 24 values per thread per operand.
template <int L, int CW>
struct PrCfg {
    static constexpr int C = CW, T = CW * L / 24;
    static constexpr int MINB = 65536 / (T * 128) < 1 ? 1 : 65536 / (T * 128);   // <= 128 registers
};

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
                    const int k = (e - off) / Rs, r = (e - off) % Rs;
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

// ---------------------------------------------------------------------------
template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_fwd_y_pr(Geom g, const float2 *__restrict__ U1, float2 *__restrict__ U2, const float2 *__restrict__ ptw)
{
    constexpr int CP = Cfg::C;
    using E = PrEng<L, CP, Cfg::T, false, 2, true, false>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, float2)

    const int W = 2 * g.SP;                           // row width (a^ and b^)
    const int ix = blockIdx.y;
    const int c = blockIdx.x * (2 * CP) + 2 * E::col();  // (c, c + 1) = (a^, b^) of one frequency
    const bool valid = c < W && ab_col_valid(c, g.H);
    const float2 *src = U1 + (long long)ix * g.N * W + c;
    float2 *dst = U2 + (long long)ix * g.xs2 + c;
    const float2 zero = make_float2(0.f, 0.f);

    float2 va[E::VPT], vb[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / 24; ++b) {
        const float2 *p = src + (long long)E::jb(b) * W;
#pragma unroll
        for (int r = 0; r < 16; ++r) {   // rows jb + r L/24 < N; rows >= N are the padding
            if (valid) gld2(p + (long long)(r * (L / 24)) * W, va[24 * b + r], vb[24 * b + r]);
            else { va[24 * b + r] = zero; vb[24 * b + r] = zero; }
        }
    }
    E::run(va, vb, sm, ptw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b) {
            float2 *p = dst + (long long)E::jb(b) * W;
#pragma unroll
            for (int r = 0; r < E::RL; ++r) gst2(p + (long long)(r * (L / E::RL)) * W, va[b * E::RL + r], vb[b * E::RL + r]);
        }
    }
}

// Stores of the last inverse stage: outputs r < 8 are lags j + r L/24 + L/3,
// outputs r >= 16 lags j + (r - 16) L/24 (kept |s| <= L/3 = Q/2).
template <int L, typename E, typename St>
__device__ __forceinline__ void pr_store_lags(const float2 *v, St &&store)
{
#pragma unroll
    for (int b = 0; b < E::VPT / 24; ++b) {
        const int j = E::jb(b);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            store(j + r * (L / 24) + L / 3, v[24 * b + r]);
            store(j + r * (L / 24), v[24 * b + 16 + r]);
        }
    }
}

template <int L, typename Cfg, bool ODD>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_x_product_pr(Geom g, const float2 *__restrict__ U2, float2 *__restrict__ U3, const float2 *__restrict__ ptw)
{
    constexpr int C = Cfg::C;
    using EF = PrEng<L, C, Cfg::T, false, 2, true, false>;
    using EI = PrEng<L, C, Cfg::T, true, 1, false, true>;
    static_assert(EF::RL == EI::R0 && EF::VPT == EI::VPT, "last forward and first inverse stages must coincide");
    constexpr int SMEM = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    LH_REQUIRE_SMEM(SMEM, float2)

    const int ky = blockIdx.y;
    const int c = blockIdx.x * C + EF::col();
    const bool valid = c < g.H;
    const long long rs = g.xs2;                        // U2 stride between i_x rows
    const float2 *src = U2 + (long long)ky * (2 * g.SP) + 2 * c;   // (a^, b^) of frequency c
    const float2 zero = make_float2(0.f, 0.f);

    float2 va[EF::VPT], vb[EF::VPT];
#pragma unroll
    for (int b = 0; b < EF::VPT / 24; ++b) {
        const float2 *p = src + (long long)EF::jb(b) * rs;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (valid) gld2(p + (long long)(r * (L / 24)) * rs, va[24 * b + r], vb[24 * b + r]);
            else { va[24 * b + r] = zero; vb[24 * b + r] = zero; }
        }
    }
    EF::run(va, vb, sm, ptw);
    // conj(a^) b^: transform of C(q) = sum_p a(p) b(p + q); for Im chi_T its
    // odd part, P - conj(P) = 2 i Im P
#pragma unroll
    for (int i = 0; i < EF::VPT; ++i) va[i] = odd_part(cmulc(vb[i], va[i]), ODD);
    EI::run(va, va, sm, ptw);
    if (valid) {
        float2 *dst = U3 + (long long)ky * g.SP + c;
        const long long os = g.xs3;
        pr_store_lags<L, EI>(va, [&](int l, float2 x) { dst[(long long)l * os] = x; });
    }
}

template <int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_inv_y_pr(Geom g, const float2 *__restrict__ U3, float2 *__restrict__ U4, const float2 *__restrict__ ptw)
{
    constexpr int CP = Cfg::C;
    using E = PrEng<L, CP, Cfg::T, true, 2, false, true>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, float2)

    const int lx = blockIdx.y;
    const int c = blockIdx.x * (2 * CP) + 2 * E::col();
    const bool valid = c < g.H;                        // c + 1 < SP: the pair stays in the row
    const float2 *src = U3 + (long long)lx * g.xs3 + c;
    float2 *dst = U4 + (long long)lx * g.Q * g.SP + c;
    const float2 zero = make_float2(0.f, 0.f);

    float2 va[E::VPT], vb[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b) {
        const float2 *p = src + (long long)E::jb(b) * g.SP;
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            if (valid) gld2(p + (long long)(r * (L / E::R0)) * g.SP, va[b * E::R0 + r], vb[b * E::R0 + r]);
            else { va[b * E::R0 + r] = zero; vb[b * E::R0 + r] = zero; }
        }
    }
    E::run(va, vb, sm, ptw);
    if (valid) {
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
