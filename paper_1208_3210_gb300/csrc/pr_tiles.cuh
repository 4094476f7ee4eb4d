// Tile functions of the pruned momentum passes (fft_pruned.cuh engine),
// shared by the standalone kernels of k_pruned.cu and the persistent batch
// kernel of k_persist.cu.  Layouts as in k_pruned.cu.
#pragma once

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

// 16-byte load of columns (c, c + 1): streaming (COH = false), or through L2
// only (COH = true: data written earlier in the same launch by other CTAs,
// which a stale L1 line must not hide)
template <bool COH>
__device__ __forceinline__ void pr_ld2(const float2 *p, float2 &a, float2 &b)
{
    if constexpr (COH) {
        const float4 q = __ldcg(reinterpret_cast<const float4 *>(p));
        a = make_float2(q.x, q.y);
        b = make_float2(q.z, q.w);
    } else {
        gld2(p, a, b);
    }
}

// ---------------------------------------------------------------------------
// Tile functions (tile coordinates bx, by as the standalone kernels' block
// indices; T threads, shared memory sm), shared by the kernels below and the
// persistent batch kernel of k_persist.cu.
template <int L, int CP, int T, bool COH>
__device__ __forceinline__ void fwd_y_pr_tile(const Geom &g, const float2 *__restrict__ U1, float2 *__restrict__ U2,
                                              const float2 *__restrict__ ptw, float2 *sm, int bx, int by)
{
    using E = PrEng<L, CP, T, false, 2, true, false>;
    const int W = 2 * g.SP;                           // row width (a^ and b^)
    const int ix = by;
    const int c = bx * (2 * CP) + 2 * E::col();      // (c, c + 1) = (a^, b^) of one frequency
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
            if (valid) pr_ld2<COH>(p + (long long)(r * (L / 24)) * W, va[24 * b + r], vb[24 * b + r]);
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

template <int L, int C, int T>
struct PrProduct {
    using EF = PrEng<L, C, T, false, 2, true, false>;
    using EI = PrEng<L, C, T, true, 1, false, true>;
    static_assert(EF::RL == EI::R0 && EF::VPT == EI::VPT, "last forward and first inverse stages must coincide");
    static constexpr int SMEM_ELEMS = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
};

template <int L, int C, int T, bool ODD, bool COH>
__device__ __forceinline__ void x_product_pr_tile(const Geom &g, const float2 *__restrict__ U2,
                                                  float2 *__restrict__ U3, const float2 *__restrict__ ptw,
                                                  float2 *sm, int bx, int by)
{
    using EF = typename PrProduct<L, C, T>::EF;
    using EI = typename PrProduct<L, C, T>::EI;
    const int ky = by;
    const int c = bx * C + EF::col();
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
            if (valid) pr_ld2<COH>(p + (long long)(r * (L / 24)) * rs, va[24 * b + r], vb[24 * b + r]);
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

template <int L, int CP, int T, bool COH>
__device__ __forceinline__ void inv_y_pr_tile(const Geom &g, const float2 *__restrict__ U3, float2 *__restrict__ U4,
                                              const float2 *__restrict__ ptw, float2 *sm, int bx, int by)
{
    using E = PrEng<L, CP, T, true, 2, false, true>;
    const int lx = by;
    const int c = bx * (2 * CP) + 2 * E::col();
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
            if (valid) pr_ld2<COH>(p + (long long)(r * (L / E::R0)) * g.SP, va[b * E::R0 + r], vb[b * E::R0 + r]);
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

}  // namespace lh
