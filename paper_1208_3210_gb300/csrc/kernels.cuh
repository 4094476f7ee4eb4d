// Tile configurations and device helpers shared by the pass kernels.
#pragma once

#include "fft_engine.cuh"
#include "lindhard_internal.h"

namespace lh {

// Strided-axis passes (momentum axes): C columns x L rows per CTA, T threads,
// VPT = C L / T = 16 values per thread (32 registers of data per transform),
// 8 for L = 512 (radix 8 x 8 x 8), so several CTAs share an SM and hide each
// other's barrier and load latency.  MINB is the CTAs per SM the register
// budget aims at.
template <int L> struct ColCfg;
template <> struct ColCfg<16>   { static constexpr int C = 32, T = 32, MINB = 4, MINB_X = 4; };
template <> struct ColCfg<32>   { static constexpr int C = 32, T = 64, MINB = 4, MINB_X = 4; };
template <> struct ColCfg<64>   { static constexpr int C = 16, T = 64, MINB = 4, MINB_X = 4; };
template <> struct ColCfg<128>  { static constexpr int C = 16, T = 128, MINB = 4, MINB_X = 3; };
template <> struct ColCfg<256>  { static constexpr int C = 16, T = 256, MINB = 3, MINB_X = 2; };
template <> struct ColCfg<512>  { static constexpr int C = 8, T = 512, MINB = 2, MINB_X = 2; };  // VPT 8
template <> struct ColCfg<1024> { static constexpr int C = 8, T = 512, MINB = 2, MINB_X = 1; };
template <> struct ColCfg<2048> { static constexpr int C = 4, T = 512, MINB = 2, MINB_X = 1; };
template <> struct ColCfg<4096> { static constexpr int C = 4, T = 1024, MINB = 1, MINB_X = 1; };
// lengths 3 * 2^k: 24 values per thread (every radix of their schedules divides 24)
template <> struct ColCfg<48>   { static constexpr int C = 16, T = 32, MINB = 4, MINB_X = 4; };
template <> struct ColCfg<96>   { static constexpr int C = 16, T = 64, MINB = 4, MINB_X = 3; };
template <> struct ColCfg<192>  { static constexpr int C = 16, T = 128, MINB = 3, MINB_X = 2; };
template <> struct ColCfg<384>  { static constexpr int C = 16, T = 256, MINB = 2, MINB_X = 1; };
template <> struct ColCfg<768>  { static constexpr int C = 8, T = 256, MINB = 2, MINB_X = 1; };
template <> struct ColCfg<1536> { static constexpr int C = 4, T = 256, MINB = 2, MINB_X = 1; };

// Strided-axis passes on the paired-column engine (FftPair): C adjacent
// columns per CTA as C/2 pairs, VPT = (C/2) L / T = 16 values per thread per
// column (8 for L = 512).  Used for L >= 128.
template <int L> struct PairCfg;
// The p_x product pass (two operands per thread): its own tile sizes.
template <int L> struct XCfg { static constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T, MINB = ColCfg<L>::MINB_X; };
template <> struct XCfg<512> { static constexpr int C = 8, T = 256, MINB = 2; };   // VPT 16
template <> struct XCfg<384> { static constexpr int C = 8, T = 128, MINB = 3; };   // VPT 24
template <> struct XCfg<4096> { static constexpr int C = 2, T = 512, MINB = 1; };  // VPT 16, 139 KB

template <> struct PairCfg<128>  { static constexpr int C = 16, T = 64, MINB = 4; };
template <> struct PairCfg<256>  { static constexpr int C = 16, T = 128, MINB = 4; };
template <> struct PairCfg<512>  { static constexpr int C = 16, T = 512, MINB = 2; };  // VPT 8
template <> struct PairCfg<1024> { static constexpr int C = 16, T = 512, MINB = 1; };
template <> struct PairCfg<2048> { static constexpr int C = 8, T = 512, MINB = 1; };
template <> struct PairCfg<4096> { static constexpr int C = 4, T = 512, MINB = 1; };    // 139 KB of shared memory
template <> struct PairCfg<192>  { static constexpr int C = 16, T = 64, MINB = 4; };    // VPT 24
template <> struct PairCfg<384>  { static constexpr int C = 32, T = 256, MINB = 2; };
template <> struct PairCfg<768>  { static constexpr int C = 16, T = 256, MINB = 2; };
template <> struct PairCfg<1536> { static constexpr int C = 8, T = 256, MINB = 2; };

// Paired p_y tiles twice as wide (twice the columns and threads, one CTA per
// SM): 128-byte row segments at 1536.
template <int L> struct PairCfgW { static constexpr int C = 2 * PairCfg<L>::C, T = 2 * PairCfg<L>::T, MINB = 1; };

// Tiles with 12 values per thread per column (radix family 1) at the 3 * 2^k
// lengths from 192: half the registers of the 24-value tiles above (so no
// spills and up to twice the warps per SM), one or two more exchanges.
// Paired p_y passes: VPT = (C/2) L / T = 12.
template <int L> struct PairCfg12;
template <> struct PairCfg12<192>  { static constexpr int C = 16, T = 128, MINB = 4; };
template <> struct PairCfg12<384>  { static constexpr int C = 16, T = 256, MINB = 2; };
template <> struct PairCfg12<768>  { static constexpr int C = 16, T = 512, MINB = 1; };
template <> struct PairCfg12<1536> { static constexpr int C = 8, T = 512, MINB = 1; };
// Product pass, default tile with one more CTA per SM (registers capped
// accordingly; the autotuner weighs the spills against the extra warps).
template <int L> struct XCfgHi { static constexpr int C = XCfg<L>::C, T = XCfg<L>::T, MINB = XCfg<L>::MINB + 1; };
// Product pass, default tile twice as wide (twice the columns and threads,
// one CTA per SM): longer contiguous row segments on the strided planes.
template <int L> struct XCfgW { static constexpr int C = 2 * XCfg<L>::C, T = 2 * XCfg<L>::T, MINB = 1; };
// Product pass: VPT = C L / T = 12.
template <int L> struct XCfg12;
template <> struct XCfg12<192>  { static constexpr int C = 8, T = 128, MINB = 4; };
template <> struct XCfg12<384>  { static constexpr int C = 8, T = 256, MINB = 2; };
template <> struct XCfg12<768>  { static constexpr int C = 8, T = 512, MINB = 1; };
template <> struct XCfg12<1536> { static constexpr int C = 4, T = 512, MINB = 1; };

// Contiguous-axis passes (energy axis): C lines of length L per CTA.
template <int L> struct LineCfg;
template <> struct LineCfg<16>   { static constexpr int C = 64, T = 64; };
template <> struct LineCfg<32>   { static constexpr int C = 32, T = 64; };
template <> struct LineCfg<64>   { static constexpr int C = 16, T = 64; };
template <> struct LineCfg<128>  { static constexpr int C = 16, T = 128; };
template <> struct LineCfg<256>  { static constexpr int C = 16, T = 256; };
template <> struct LineCfg<512>  { static constexpr int C = 8, T = 256; };
template <> struct LineCfg<1024> { static constexpr int C = 8, T = 512; };
template <> struct LineCfg<2048> { static constexpr int C = 4, T = 512; };
template <> struct LineCfg<4096> { static constexpr int C = 4, T = 1024; };
// energy lengths 3 * 2^k (finite temperature pads the energy axis to
// n_eps + n_omega - 1): 24 values per thread
template <> struct LineCfg<48>   { static constexpr int C = 32, T = 64; };
template <> struct LineCfg<96>   { static constexpr int C = 16, T = 64; };
template <> struct LineCfg<192>  { static constexpr int C = 16, T = 128; };
template <> struct LineCfg<384>  { static constexpr int C = 16, T = 256; };
template <> struct LineCfg<768>  { static constexpr int C = 8, T = 256; };
template <> struct LineCfg<1536> { static constexpr int C = 4, T = 256; };

// Energy table entry: FP32 path stores e_j as an unevaluated sum hi + lo.
template <typename Real> struct EpsEntry;
template <> struct EpsEntry<float> { using type = float2; };
template <> struct EpsEntry<double> { using type = double; };

// Twiddle tables exp(-2 pi i n / L), n < L, one per supported length, stored
// contiguously: powers of two 16..4096 first (the length-L table at offset
// L - 16), then 3 * 2^k for 48..1536 (at 8176 + L - 48).
__host__ __device__ constexpr int twiddle_offset(int L)
{
    return fft_len_pow2(L) ? L - 16 : 8176 + L - 48;
}
__host__ __device__ constexpr int twiddle_entries() { return 8176 + 3024; }
template <typename Real>
__host__ __device__ inline const cx<Real> *twiddles_for(const Work<Real> &w, int L)
{
    return (const cx<Real> *)w.tw + twiddle_offset(L);
}

// Bytes of dynamic shared memory this launch was given.  Every FFT kernel
// compares it with what its engines address and returns before touching
// memory when it is short, so a launch configured with too little shared
// memory gives wrong results (caught by the tests) instead of an
// out-of-bounds access.
// Unevaluated FP32 pairs hi + lo (double-float arithmetic, Dekker 1971):
// error-free sums (Knuth's TwoSum), FMA-based error-free products, and their
// renormalisation.  Explicitly rounded intrinsics keep the compiler from
// contracting the additions into FMAs, which would break the error terms.
struct F2 { float h, l; };
__device__ __forceinline__ F2 f2_fast(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = __fadd_rn(a.h, b.h), bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    return f2_fast(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return f2_fast(p, e);
}

// Band energy xi_p = e0(p) - mu as an unevaluated FP32 pair (hi, lo), and the
// amplitude |M(p)|^2 gamma / pi, of the momentum point with axis entries
// (ax, ay) (Eqs. 4-5): double-float, about 1e-14 eV, in a chain of FP32
// operations of a few cycles each where FP64 operations cost about 60.
__device__ __forceinline__ void band_point_f32(const Band &band, const AxisTab &ax, const AxisTab &ay,
                                               const InstState *st, float &xhi, float &xlo, float &amp)
{
    F2 e0;
    if (band.band_kind == 1) {
        e0 = f2_add(F2{ax.p2h, ax.p2l}, F2{ay.p2h, ay.p2l});
        e0.h *= 0.5f;   // exact
        e0.l *= 0.5f;
    } else {
        const F2 cx{ax.c1h, ax.c1l}, cy{ay.c1h, ay.c1l};
        e0 = f2_add(f2_add(f2_mul(F2{band.k1[0], band.k1[1]}, f2_add(cx, cy)),
                           f2_mul(F2{band.k2[0], band.k2[1]}, f2_mul(cx, cy))),
                    f2_mul(F2{band.k3[0], band.k3[1]}, f2_add(F2{ax.c2h, ax.c2l}, F2{ay.c2h, ay.c2l})));
    }
    const F2 xi = f2_add(e0, F2{-st->mu_hi, -st->mu_lo});
    xhi = xi.h;
    xlo = xi.l;
    amp = ax.gf * ay.gf * band.gam_pi;
}

// Rows of the forward intermediates U1 and U2 (and of the adjoint's G3, G4)
// hold the two half spectra interleaved: column 2k is the first (a^, or h^ in
// the adjoint), column 2k + 1 the second (b^, or g^), k in [0, SP).  A tile
// of frequencies then reads both spectra from one contiguous row segment.
__host__ __device__ inline bool ab_col_valid(int c, int H) { return (c >> 1) < H; }

// Dynamic shared-memory limit of a kernel.  (The L1/shared carveout is left
// to the driver: pinning it to the largest shared share slowed the FFT passes,
// which read twiddles through L1, by 10-20%.)
template <typename K>
inline cudaError_t smem_attrs(K k, size_t dyn)
{
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

__device__ __forceinline__ unsigned dyn_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
#define LH_REQUIRE_SMEM(elems, Cx) \
    if (dyn_smem_bytes() < (unsigned)((elems) * sizeof(Cx))) return;

// Circular index n of an inverse transform of length P -> output lag index
// l in [0, Q), or -1 when the lag is not kept.
__device__ __forceinline__ int lag_index(int n, int P, int Q)
{
    int s = (n < P / 2) ? n : n - P;
    int l = s + Q / 2;
    return (l >= 0 && l < Q) ? l : -1;
}

}  // namespace lh

// Dispatch on a runtime FFT length to the compiled template instance.
#define LH_LEN_SWITCH(L_, CALL)                                   \
    switch (L_) {                                                 \
    case 16: return CALL(16);                                     \
    case 32: return CALL(32);                                     \
    case 64: return CALL(64);                                     \
    case 128: return CALL(128);                                   \
    case 256: return CALL(256);                                   \
    case 512: return CALL(512);                                   \
    case 1024: return CALL(1024);                                 \
    case 2048: return CALL(2048);                                 \
    case 4096: return CALL(4096);                                 \
    default: return cudaErrorInvalidValue;                        \
    }
// Momentum-axis lengths (FP32): powers of two and 3 * 2^k.
#define LH_P_SWITCH(L_, CALL)                                     \
    switch (L_) {                                                 \
    case 16: return CALL(16);                                     \
    case 32: return CALL(32);                                     \
    case 48: return CALL(48);                                     \
    case 64: return CALL(64);                                     \
    case 96: return CALL(96);                                     \
    case 128: return CALL(128);                                   \
    case 192: return CALL(192);                                   \
    case 256: return CALL(256);                                   \
    case 384: return CALL(384);                                   \
    case 512: return CALL(512);                                   \
    case 768: return CALL(768);                                   \
    case 1024: return CALL(1024);                                 \
    case 1536: return CALL(1536);                                 \
    case 2048: return CALL(2048);                                 \
    case 4096: return CALL(4096);                                 \
    default: return cudaErrorInvalidValue;                        \
    }
#define LH_LEN_SWITCH_SMALL(L_, CALL)                             \
    switch (L_) {                                                 \
    case 16: return CALL(16);                                     \
    case 32: return CALL(32);                                     \
    case 64: return CALL(64);                                     \
    case 128: return CALL(128);                                   \
    case 256: return CALL(256);                                   \
    default: return cudaErrorInvalidValue;                        \
    }

