// Tile functions of the warp-per-line energy passes (k_energy.cu), shared
// with the persistent batch kernel of k_persist.cu; per-stage twiddle table
// layout of those passes.
#pragma once

#include "kernels.cuh"

namespace lh {

// Lengths of the warp-per-line passes: 128, 256 and 512 (16 values per
// thread; also the lengths of the persistent batch kernel) and 384 and 768
// (24 values per thread: the energy axes that finite temperature pads to
// 3 * 2^k).
__host__ __device__ constexpr bool et_supported(int L) { return L == 128 || L == 256 || L == 512; }
__host__ __device__ constexpr bool et_len_supported(int L) { return et_supported(L) || L == 384 || L == 768; }
// Schedules: forward 128 = 4.4.8, 256 = 4.8.8, 512 = 8.8.8, 384 = 8.4.12,
// 768 = 8.8.12; inverse 128 = 8.4.4, 256 = 8.8.4, 512 = 8.8.8, 384 = 12.4.8,
// 768 = 12.8.8 (the forward ones reversed for 384 and 768)
__host__ __device__ constexpr int et_radix(int L, int s, bool inv = false)
{
    return inv ? (L == 768 ? (s == 0 ? 12 : 8) : L == 384 ? (s == 0 ? 12 : s == 1 ? 4 : 8)
                           : (s == 0 ? 8 : L == 512 ? 8 : L == 256 ? (s == 1 ? 8 : 4) : 4))
         : L == 768 ? (s == 2 ? 12 : 8)
         : L == 384 ? (s == 0 ? 8 : s == 1 ? 4 : 12)
                    : (s == 2 ? 8 : L == 512 ? 8 : L == 256 ? (s == 0 ? 4 : 8) : 4);
}
__host__ __device__ constexpr int et_ns(int L, int s, bool inv = false)
{
    return s == 0 ? 1 : et_ns(L, s - 1, inv) * et_radix(L, s - 1, inv);
}
// the i-th length with tables in direction d (0 past the last)
__host__ __device__ constexpr int et_len(int d, int i)
{
    return i == 0 ? 128 : i == 1 ? 256 : i == 2 ? 512 : i == 3 ? 384 : i == 4 ? 768 : 0;
}
// per-stage twiddle tables, rows [k], k < Ns, of Rs entries w^1, ...,
// w^(Rs-1), w^0, w = exp(-2 pi i k / (Ns Rs)), of stages 1 and 2 of each
// schedule: forward 128, 256, 512, 384, 768, then inverse the same
__host__ __device__ constexpr int et_table_offset(int L, int s, bool inv = false)
{
    int o = 0;
    for (int d = 0; d < 2; ++d)
        for (int i = 0; et_len(d, i) != 0; ++i)
            for (int st = 1; st <= 2; ++st) {
                if (et_len(d, i) == L && st == s && (d != 0) == inv) return o;
                o += et_ns(et_len(d, i), st + 1, d != 0);
            }
    return o;
}
__host__ __device__ constexpr int et_twiddle_entries() { return et_table_offset(0, 0); }

// Per warp: ET_LPW lines, LPI = 32 / TPL at a time (TPL = L / VPT threads per
// line, VPT values per thread); shared memory per warp LPI lines of L + L/16
// values.
constexpr int ET_LPW = 16, ET_WARPS = 4;
template <int L>
struct EtGeo {
    static constexpr int VPT = (L & (L - 1)) == 0 ? 16 : 24;
    static constexpr int TPL = L / VPT, LPI = 32 / TPL, LP = L + L / 16;
    static constexpr int R0 = et_radix(L, 0), R1 = et_radix(L, 1), R2 = et_radix(L, 2);
    static constexpr int N1 = et_ns(L, 1), N2 = et_ns(L, 2);
    static constexpr int WARP_ELEMS = LPI * LP;
    static_assert(R0 * R1 * R2 == L && VPT % R0 == 0 && VPT % R1 == 0 && VPT == 2 * R2, "schedule");
    static_assert((L / R1) % 16 == 0 && (L / R2) % 16 == 0 && N2 % 16 == 0 && ET_LPW % LPI == 0,
                  "compile-time padded offsets");
};
__host__ __device__ constexpr int et_pad(int n) { return n + n / 16; }

// 1/x as the hardware approximation (relative error about 2^-23; x lies in
// [gamma^2, 4 e_max^2 + gamma^2], away from zero, subnormals and overflow)
__device__ __forceinline__ float et_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Twiddles of one radix-R butterfly from its table row (w^1, ..., w^(R-1),
// w^0) applied to v[1..R) (conjugated with CONJ): one 16-byte load gives w and
// w^2, the other powers are products of them (at most three roundings deep).
template <int R, bool CONJ>
__device__ __forceinline__ void et_twiddle(float2 *v, const float4 *w4)
{
    static_assert(R == 4 || R == 8 || R == 12, "radices of the energy schedules");
    float2 w[R];
    const float4 q0 = __ldg(w4);
    w[1] = make_float2(q0.x, q0.y);
    w[2] = make_float2(q0.z, q0.w);
    w[3] = cmul(w[1], w[2]);
#pragma unroll
    for (int r = 4; r < R; ++r) w[r] = cmul(w[r / 2], w[r - r / 2]);   // w^4 = (w^2)^2, w^5 = w^2 w^3, ...
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = CONJ ? cmulc(v[r], w[r]) : cmul(v[r], w[r]);
}

// FULL: n_eps == L (no energy padding; occupied rows n < L/2).  GEN: A is
// generated (else read from the caller's A_in).  THERMAL: the finite-
// temperature weights (Appendix A, Eq. A1) instead of the T = 0 split: the
// occupied part A f and the empty part A (1 - f) of energy n, with (weight of
// the real part, weight of the imaginary part) read from wf[n] (a table the
// caller fills; et_fermi_weights).
// Tile function: tile `tile` holds lines [ET_WARPS ET_LPW tile, ...); smem:
// the tile's ET_WARPS * WARP_ELEMS values (shared by the kernel below and the
// persistent batch kernel of k_persist.cu).
template <int L, bool FULL, bool GEN, bool THERMAL = false>
__device__ __forceinline__ void energy_fwd_warp_tile(const Geom &g, const Band &band, const AxisTab *__restrict__ axis,
                                                     const float2 *__restrict__ eps, const InstState *__restrict__ st,
                                                     const float *__restrict__ A_in, float2 *__restrict__ U1,
                                                     const float2 *__restrict__ etw, float2 *smem, long long tile,
                                                     const float2 *wf = nullptr)
{
    using G = EtGeo<L>;
    constexpr int VPT = G::VPT, TPL = G::TPL, LPI = G::LPI, LP = G::LP, R0 = G::R0, R1 = G::R1, R2 = G::R2;
    constexpr int N1 = G::N1, N2 = G::N2, NB2 = L / R2;   // butterflies of the last stage
    const int lane = (int)threadIdx.x % 32, warp = (int)threadIdx.x / 32;
    const int sl = lane / TPL, u = lane % TPL;
    float2 *sm = smem + warp * G::WARP_ELEMS + sl * LP;
    const long long nlines = (long long)g.N * g.N;
    const long long line0 = (tile * ET_WARPS + warp) * ET_LPW;
    const float g2 = band.gam2;
    const float2 *tw1 = etw + et_table_offset(L, 1), *tw2 = etw + et_table_offset(L, 2);

    // band energy xi_p = e0(p) - mu (double-float) and |M(p)|^2 gamma / pi of
    // the warp's lines (Eqs. 4-5), one lane per line; the amplitude carries
    // the 1/2 of the a^ / b^ separation below (exact), and is 0 for lines
    // past the end (their values come out 0, no branch per value)
    float bx = 0.f, bl = 0.f, ba = 0.f;
    if (GEN && lane < ET_LPW && line0 + lane < nlines) {
        const long long line = line0 + lane;
        const int ix = (int)(line / g.N), iy = (int)(line - (long long)ix * g.N);
        band_point_f32(band, axis[ix], axis[iy], st, bx, bl, ba);
        ba *= 0.5f;
    }

    for (int it = 0; it < ET_LPW; it += LPI) {
        const long long line = line0 + it + sl;
        const bool live = line < nlines;
        const float xhi = __shfl_sync(0xffffffffu, bx, it + sl), xlo = __shfl_sync(0xffffffffu, bl, it + sl);
        const float amp = __shfl_sync(0xffffffffu, ba, it + sl);

        // stage 0: butterflies j = u + b TPL, rows j + r L/R0
        float2 v[VPT];
#pragma unroll
        for (int b = 0; b < VPT / R0; ++b) {
            const int j = u + b * TPL;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int n = j + r * (L / R0);
                float A;
                if constexpr (GEN) {
                    const float2 ej = __ldg(&eps[FULL ? n : min(n, g.n_eps - 1)]);
                    const float e = (ej.x - xhi) + (ej.y - xlo);
                    A = amp * et_rcp(fmaf(e, e, g2));
                    if (!FULL && n >= g.n_eps) A = 0.f;
                } else {
                    A = (live && (FULL || n < g.n_eps)) ? 0.5f * A_in[line * g.n_eps + n] : 0.f;
                }
                if constexpr (THERMAL) {
                    const float2 w = wf[n];
                    v[b * R0 + r] = make_float2(A * w.x, A * w.y);
                } else {
                    // occupied (e_n < 0) -> real part, empty -> imaginary part
                    const bool occ = FULL ? (r < R0 / 2) : (2 * n + 1 < g.n_eps);
                    v[b * R0 + r] = occ ? make_float2(A, 0.f) : make_float2(0.f, A);
                }
            }
            Dft<R0, false, float2>::run(v + b * R0);
        }
        // exchange 1 (outputs at j R0 + r) and stage 1: butterflies u + b TPL
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R0; ++b) {
            const int base = (u + b * TPL) * R0;
            const int pb = base + base / 16;
#pragma unroll
            for (int r = 0; r < R0; ++r) sm[pb + r] = v[b * R0 + r];
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R1; ++b) {
            const int j = u + b * TPL;
            const int pj = et_pad(j);
#pragma unroll
            for (int r = 0; r < R1; ++r) v[b * R1 + r] = sm[pj + et_pad(r * (L / R1))];
            et_twiddle<R1, false>(v + b * R1, reinterpret_cast<const float4 *>(tw1 + (j % N1) * R1));
            Dft<R1, false, float2>::run(v + b * R1);
        }
        // exchange 2 (outputs at (j / N1) N2 + j % N1 + r N1) and stage 2:
        // butterflies u and NB2 - u (u = 0: 0 and NB2/2 = TPL), so that Z(k)
        // and Z(L - k) end in the same thread
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R1; ++b) {
            const int j = u + b * TPL;
            const int base = (j / N1) * N2 + j % N1;   // base % 16 = j % N1 < N1
            const int pb = base + base / 16;
#pragma unroll
            for (int r = 0; r < R1; ++r) sm[pb + r * N1 + (r * N1) / 16] = v[b * R1 + r];
        }
        __syncwarp();
        const int j2[2] = {u, u == 0 ? TPL : NB2 - u};
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int pj = et_pad(j2[b]);
#pragma unroll
            for (int r = 0; r < R2; ++r) v[b * R2 + r] = sm[pj + et_pad(r * NB2)];
            et_twiddle<R2, false>(v + b * R2, reinterpret_cast<const float4 *>(tw2 + j2[b] * R2));   // j < N2
            Dft<R2, false, float2>::run(v + b * R2);
        }

        // Z(j + r NB2) in v[b R2 + r]; the partner Z(L - k) of (j2[0], r) is
        // (j2[1], R2 - 1 - r) for u > 0; of (0, r) it is (0, R2 - r), of
        // (NB2/2, r) it is (NB2/2, R2 - 1 - r)
        if (live) {
            float2 *row = U1 + line * (2LL * g.SP);
            // a^ = (Z(k) + conj Z(-k)) / 2, b^ = (Z(k) - conj Z(-k)) / 2i, the
            // 1/2 already in Z (the amplitude)
            auto put = [&](int k, float2 zk, float2 zm) {
                gst2(row + 2 * k, make_float2(zk.x + zm.x, zk.y - zm.y), make_float2(zk.y + zm.y, zm.x - zk.x));
            };
            const bool u0 = u == 0;
#pragma unroll
            for (int r = 0; r < R2 / 2; ++r) {
                put(j2[0] + r * NB2, v[r], u0 ? v[(R2 - r) % R2] : v[R2 + R2 - 1 - r]);
                put(j2[1] + r * NB2, v[R2 + r], u0 ? v[R2 + R2 - 1 - r] : v[R2 - 1 - r]);
            }
            if (u0) put(L / 2, v[R2 / 2], v[R2 / 2]);
        }
        __syncwarp();   // the next line's exchange overwrites this one's
    }
}

// The finite-temperature weights of energy n < L (Appendix A, Eq. A1) into
// wf[n] = (f, 1 - f), f = 1 / (exp(x) + 1), x = e_n / kT =
// (2 n + 1 - n_eps) x_step (the occupied weight multiplies the real part, the
// empty one the imaginary part), both from u = exp(-|x|) so that neither loses
// digits to 1 - f.  Entries t0, t0 + stride, ...
template <int L>
__device__ __forceinline__ void et_fermi_weights(const Geom &g, const Band &band, float2 *wf, int t0, int stride)
{
    for (int n = t0; n < L; n += stride) {
        const float x = (float)(2 * n + 1 - g.n_eps) * band.x_step;
        const float u = expf(-fabsf(x));
        const float big = 1.f / (1.f + u), small = u * big;
        wf[n] = x < 0 ? make_float2(big, small) : make_float2(small, big);
    }
}

// ---------------------------------------------------------------------------
// Inverse energy pass, one warp per pair of output lines (the transform of
// k_inv_energy): for the lines (2f, 2f + 1) of U4 [Q^2][SP], W(k) = X1(k) +
// i X2(k) over k in [0, L), with X(k) = conj X(L - k) above L/2 (the product
// spectrum of the real correlation is Hermitian in the energy frequency), one
// complex inverse FFT, Re w -> line 2f, Im w -> line 2f + 1, the transfers
// m < n_omega, times the Eq. 9 prefactor with the FFT normalisation.  In the
// first stage a thread owns butterflies j and L/8 - j: it loads X(k) once for
// k <= L/2 and forms both W(k) and W(L - k) = conj X1(k) + i conj X2(k).
// HALF: n_omega == L/2 (the outputs of the last stage's first R2/2 rows).
template <int L>
__host__ __device__ constexpr int et_inv_smem_elems() { return ET_WARPS * EtGeo<L>::LPI * EtGeo<L>::LP; }
// Tile function (pairs [ET_WARPS ET_LPW tile, ...)); COH: read U4 through L2
// only (written earlier in the same launch by other CTAs).
template <int L, bool HALF, bool COH>
__device__ __forceinline__ void inv_energy_warp_tile(const Geom &g, const float2 *__restrict__ U4,
                                                     float *__restrict__ out, const float2 *__restrict__ etw,
                                                     float2 *smem, long long tile)
{
    using G = EtGeo<L>;
    constexpr int VPT = G::VPT, TPL = G::TPL, LPI = G::LPI, LP = G::LP;
    constexpr int R0 = et_radix(L, 0, true), R1 = et_radix(L, 1, true), R2 = et_radix(L, 2, true);
    constexpr int N1 = et_ns(L, 1, true), N2 = et_ns(L, 2, true), NB0 = L / R0;   // first-stage butterflies
    constexpr int H = L / 2 + 1, SP = (H + 7) / 8 * 8;
    static_assert(VPT == 2 * R0 && R0 * R1 * R2 == L && VPT % R1 == 0 && VPT % R2 == 0 && NB0 == 2 * TPL,
                  "schedule");
    static_assert((L / R1) % 16 == 0 && (L / R2) % 16 == 0 && N1 % 4 == 0 && ET_LPW % LPI == 0,
                  "compile-time padded offsets");
    const int lane = (int)threadIdx.x % 32, warp = (int)threadIdx.x / 32;
    const int sl = lane / TPL, u = lane % TPL;
    float2 *sm = smem + (warp * LPI + sl) * LP;
    const long long npairs = (long long)g.Q * g.Q / 2;
    const long long pair0 = (tile * ET_WARPS + warp) * ET_LPW;
    const float2 *tw1 = etw + et_table_offset(L, 1, true), *tw2 = etw + et_table_offset(L, 2, true);
    const float sc = (float)g.scale;
    const int j0[2] = {u, u == 0 ? TPL : NB0 - u};

    for (int it = 0; it < ET_LPW; it += LPI) {
        const long long f = pair0 + it + sl;
        const bool live = f < npairs;
        const float2 *row1 = U4 + (live ? 2 * f : 0) * SP, *row2 = row1 + SP;
        // stage 0: rows j + r NB0 of butterflies j0[0] and j0[1]; the rows
        // above L/2 of one are the conjugate mirrors of the other's
        float2 v[VPT];
        const float2 zero = make_float2(0.f, 0.f);
        auto ldx = [](const float2 *p) { return COH ? __ldcg(p) : __ldg(p); };
        auto w_of = [](float2 x1, float2 x2) { return make_float2(x1.x - x2.y, x1.y + x2.x); };       // X1 + i X2
        auto w_conj = [](float2 x1, float2 x2) { return make_float2(x1.x + x2.y, x2.x - x1.y); };     // conj X1 + i conj X2
#pragma unroll
        for (int r = 0; r < R0 / 2; ++r) {
            const float2 a1 = live ? ldx(row1 + j0[0] + r * NB0) : zero;
            const float2 a2 = live ? ldx(row2 + j0[0] + r * NB0) : zero;
            const float2 b1 = live ? ldx(row1 + j0[1] + r * NB0) : zero;
            const float2 b2 = live ? ldx(row2 + j0[1] + r * NB0) : zero;
            v[r] = w_of(a1, a2);
            v[R0 + r] = w_of(b1, b2);
            // u > 0: L - (j0[0] + r NB0) = j0[1] + (R0 - 1 - r) NB0 and the other way round
            v[R0 - 1 - r] = w_conj(b1, b2);
            v[R0 + R0 - 1 - r] = w_conj(a1, a2);
        }
        if (u == 0) {
            // j0[0] = 0: rows r NB0 mirror (R0 - r) NB0; row L/2 is its own mirror
            const float2 c1 = live ? ldx(row1 + L / 2) : zero, c2 = live ? ldx(row2 + L / 2) : zero;
            v[R0 / 2] = w_of(c1, c2);
#pragma unroll
            for (int r = 1; r < R0 / 2; ++r) {
                const float2 x1 = live ? ldx(row1 + r * NB0) : zero, x2 = live ? ldx(row2 + r * NB0) : zero;
                v[R0 - r] = w_conj(x1, x2);
            }
            // j0[1] = NB0/2: rows NB0/2 + r NB0 mirror NB0/2 + (R0 - 1 - r) NB0
#pragma unroll
            for (int r = 0; r < R0 / 2; ++r) {
                const float2 x1 = live ? ldx(row1 + TPL + r * NB0) : zero;
                const float2 x2 = live ? ldx(row2 + TPL + r * NB0) : zero;
                v[R0 + R0 - 1 - r] = w_conj(x1, x2);
            }
        }
        Dft<R0, true, float2>::run(v);
        Dft<R0, true, float2>::run(v + R0);
        // exchange 1 (outputs at j R0 + r) and stage 1: butterflies u + b TPL
        __syncwarp();
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int base = j0[b] * R0;
#pragma unroll
            for (int r = 0; r < R0; ++r) sm[et_pad(base + r)] = v[b * R0 + r];
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R1; ++b) {
            const int j = u + b * TPL;
            const int pj = et_pad(j);
#pragma unroll
            for (int r = 0; r < R1; ++r) v[b * R1 + r] = sm[pj + et_pad(r * (L / R1))];
            et_twiddle<R1, true>(v + b * R1, reinterpret_cast<const float4 *>(tw1 + (j % N1) * R1));
            Dft<R1, true, float2>::run(v + b * R1);
        }
        // exchange 2 (outputs at (j / N1) N2 + j % N1 + r N1) and stage 2
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R1; ++b) {
            const int j = u + b * TPL;
            const int base = (j / N1) * N2 + j % N1;
#pragma unroll
            for (int r = 0; r < R1; ++r) sm[et_pad(base + r * N1)] = v[b * R1 + r];
        }
        __syncwarp();
#pragma unroll
        for (int b = 0; b < VPT / R2; ++b) {
            const int j = u + b * TPL;
            const int pj = et_pad(j);
#pragma unroll
            for (int r = 0; r < R2; ++r) v[b * R2 + r] = sm[pj + et_pad(r * (L / R2))];
            et_twiddle<R2, true>(v + b * R2, reinterpret_cast<const float4 *>(tw2 + j * R2));   // j < N2
            Dft<R2, true, float2>::run(v + b * R2);
        }
        // outputs m = j + r L/R2; Re -> line 2f, Im -> line 2f + 1
        if (live) {
            float *o1 = out + 2 * f * g.n_omega, *o2 = o1 + g.n_omega;
#pragma unroll
            for (int b = 0; b < VPT / R2; ++b) {
                const int j = u + b * TPL;
#pragma unroll
                for (int r = 0; r < (HALF ? R2 / 2 : R2); ++r) {
                    const int m = j + r * (L / R2);
                    if (HALF || m < g.n_omega) {
                        o1[m] = sc * v[b * R2 + r].x;
                        o2[m] = sc * v[b * R2 + r].y;
                    }
                }
            }
        }
        __syncwarp();   // the next pair's exchange overwrites this one's
    }
}

}  // namespace lh
