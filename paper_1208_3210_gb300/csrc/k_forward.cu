// Forward passes of the correlation (Sec. 3: Fourier transforms of the
// occupied and empty parts of A).
//
//   k_fwd_energy : generates A(p, e) for a tile of momentum points (Eqs. 4-5),
//                  splits it at e = 0 into the occupied part a and the empty
//                  part b (T = 0 split, Appendix A Eq. A3; at temperature
//                  kT > 0, a = A f and b = A (1 - f), Eq. A1), transforms
//                  z = a + i b along energy, and separates the two transforms
//                  a^(k) = (Z(k) + conj Z(-k)) / 2, b^(k) = (Z(k) - conj Z(-k)) / 2i
//                  for the non-redundant frequencies k in [0, PE/2].
//   k_fwd_y      : transforms both half spectra along p_y, zero-padded from N
//                  to P points.
#include "kernels.cuh"

namespace lh {

// ---------------------------------------------------------------------------
// Energy pass.  One CTA = C momentum points (lines), output U1 layout
// [N*N lines][SP][2] complex: (a^(k), b^(k)) interleaved.
// THERMAL: the finite-temperature weights (band.kT > 0) instead of the split.
template <typename Real, int L, bool THERMAL>
__global__ void __launch_bounds__(LineCfg<L>::T)
k_fwd_energy(Geom g, Band band, const AxisTab *__restrict__ axis,
             const typename EpsEntry<Real>::type *__restrict__ eps,
             const InstState *__restrict__ st, const Real *__restrict__ A_in,
             cx<Real> *__restrict__ U1, const cx<Real> *__restrict__ tw)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, false>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)
    __shared__ Real s_xhi[C], s_xlo[C], s_amp[C];

    const long long nlines = (long long)g.N * g.N;
    const long long line0 = (long long)blockIdx.x * C;

    if constexpr (THERMAL) {
        // finite temperature (Appendix A, Eq. A1): the occupied part is A f, the
        // empty part A (1 - f), f = 1 / (exp(x) + 1), x = e_n / kT; both weights
        // from u = exp(-|x|) so that neither loses digits to 1 - f.  They depend
        // on the energy only: tabulated once per CTA in the transform's shared
        // memory (read before the transform writes it; barrier below) as
        // (weight of the real part, weight of the imaginary part).
        for (int n = threadIdx.x; n < L; n += T) {
            Real x, u;
            if constexpr (sizeof(Real) == 4) {
                x = (Real)(2 * n + 1 - g.n_eps) * band.x_step;
                u = expf(-fabsf(x));
            } else {
                x = (Real)(2 * n + 1 - g.n_eps) * (Real)band.x_step64;
                u = exp(-fabs(x));
            }
            const Real big = (Real)1 / ((Real)1 + u), small = u * big;
            sm[n] = x < 0 ? mk<Cx>(big, small) : mk<Cx>(small, big);
        }
    }
    if (A_in == nullptr && threadIdx.x < C) {
        // band energy xi_p = e0(p) - mu and |M(p)|^2 gamma / pi of this line's
        // momentum point (Eqs. 4-5)
        long long line = line0 + threadIdx.x;
        if (line < nlines) {
            int ix = (int)(line / g.N), iy = (int)(line % g.N);
            const AxisTab &ax = axis[ix], &ay = axis[iy];
            if constexpr (sizeof(Real) == 4) {
                // double-float: FP64 operations would hold the CTA at the barrier below
                band_point_f32(band, ax, ay, st, s_xhi[threadIdx.x], s_xlo[threadIdx.x], s_amp[threadIdx.x]);
            } else {
                double e0;
                if (band.band_kind == 1)
                    e0 = 0.5 * (ax.p2 + ay.p2);
                else
                    e0 = -2.0 * band.t * (ax.c1 + ay.c1) - 4.0 * band.tp * ax.c1 * ay.c1
                         - 2.0 * band.tpp * (ax.c2 + ay.c2);
                double xi = e0 - st->mu;
                s_xhi[threadIdx.x] = (Real)xi;
                s_xlo[threadIdx.x] = (Real)(xi - (double)(Real)xi);
                s_amp[threadIdx.x] = (Real)(ax.g * ay.g * band.gamma / 3.14159265358979323846);
            }
        }
    }
    __syncthreads();

    const Real g2 = (Real)(band.gamma * band.gamma);
    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b) {
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            long long line = line0 + col;
            Real A = 0;
            if (n < g.n_eps && line < nlines) {
                if (A_in != nullptr) {
                    A = A_in[line * g.n_eps + n];
                } else {
                    Real e;
                    if constexpr (sizeof(Real) == 4) {
                        float2 ej = eps[n];
                        e = (ej.x - s_xhi[col]) + (ej.y - s_xlo[col]);
                    } else {
                        e = eps[n] - s_xhi[col];
                    }
                    Real d = e * e + g2;
                    // FP32: the hardware reciprocal (2 ulp; d lies in [gamma^2, 4 e_max^2])
                    if constexpr (sizeof(Real) == 4) A = __fdividef(s_amp[col], d);
                    else A = s_amp[col] / d;
                }
            }
            if constexpr (THERMAL) {
                const Cx wf = sm[n];   // the Fermi weights of energy n (table above)
                v[b * E::R0 + r] = mk<Cx>(A * wf.x, A * wf.y);
            } else {
                // occupied (e_n < 0) -> real part, empty -> imaginary part
                v[b * E::R0 + r] = (n < g.J0) ? mk<Cx>(A, (Real)0) : mk<Cx>((Real)0, A);
            }
        }
    }

    if constexpr (THERMAL) __syncthreads();   // the weight table is read: the transform may overwrite it
    E::run(v, sm, tw);

    // natural-order spectrum to shared memory, then separate a^ and b^
#pragma unroll
    for (int b = 0; b < E::VPT / E::RL; ++b) {
#pragma unroll
        for (int r = 0; r < E::RL; ++r) {
            int col, n;
            E::last_elem(b, r, col, n);
            sm[E::saddr(col, n)] = v[b * E::RL + r];
        }
    }
    __syncthreads();
    const Real half = (Real)0.5;
    constexpr int H = L / 2 + 1;                 // non-redundant frequencies (= g.H)
    constexpr int SP = (H + 7) / 8 * 8;          // row stride (= g.SP)
    // a^ = (Z(k) + conj Z(-k)) / 2 ; b^ = (Z(k) - conj Z(-k)) / 2i, stored as
    // the adjacent pair (a^(k), b^(k)): one 16-byte store per frequency, a
    // warp's stores one contiguous run
    // one warp per line, lanes over the frequencies (no index division)
    for (int col = threadIdx.x >> 5; col < C; col += T >> 5) {
        const long long line = line0 + col;
        if (line >= nlines) continue;
        Cx *row = U1 + line * (2LL * SP);
#pragma unroll 2
        for (int k = threadIdx.x & 31; k < H; k += 32) {
            Cx zk = sm[E::saddr(col, k)];
            Cx zm = sm[E::saddr(col, k == 0 ? 0 : L - k)];
            Cx ah = mk<Cx>(half * (zk.x + zm.x), half * (zk.y - zm.y));
            Cx bh = mk<Cx>(half * (zk.y + zm.y), -half * (zk.x - zm.x));
            gst2(row + 2 * k, ah, bh);
        }
    }
}

// ---------------------------------------------------------------------------
// p_y pass.  CTA = (column tile, ix).  U1 [N][N][2 SP] -> U2 [N][P][2 SP].
template <typename Real, int L>
__global__ void __launch_bounds__(ColCfg<L>::T, ColCfg<L>::MINB)
k_fwd_y(Geom g, const cx<Real> *__restrict__ U1, cx<Real> *__restrict__ U2,
        const cx<Real> *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, false>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)

    const int W = 2 * g.SP;                       // row width (a^ and b^)
    const int ix = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < W && ab_col_valid(c, g.H);
    const Cx *src = U1 + (long long)ix * g.N * W + c;
    Cx *dst = U2 + (long long)ix * g.xs2 + c;

    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            v[b * E::R0 + r] = (valid && n < g.N) ? src[(long long)n * W] : mk<Cx>((Real)0, (Real)0);
        }
    E::run(v, sm, tw);
    if (valid) {
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

// Paired-column version of the p_y pass (L >= 128): each thread moves the two
// adjacent columns (c, c + 1) with 16-byte accesses.
template <typename Real, int L, typename Cfg>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB)
k_fwd_y2(Geom g, const cx<Real> *__restrict__ U1, cx<Real> *__restrict__ U2,
         const cx<Real> *__restrict__ tw)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<Real, L, C, T, false>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)

    const int W = 2 * g.SP;                       // row width (a^ and b^)
    const int ix = blockIdx.y;
    const int c = blockIdx.x * C + 2 * E::pair(); // first column of the pair
    const bool valid = c < W && ab_col_valid(c, g.H); // (c, c + 1) = (a^, b^) of one frequency
    const Cx *src = U1 + (long long)ix * g.N * W + c;
    Cx *dst = U2 + (long long)ix * g.xs2 + c;
    const Cx zero = mk<Cx>((Real)0, (Real)0);

    Cx va[E::VPT], vb[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int n = E::first_row(b, r);
            if (valid && n < g.N) gld2(src + (long long)n * W, va[b * E::R0 + r], vb[b * E::R0 + r]);
            else { va[b * E::R0 + r] = zero; vb[b * E::R0 + r] = zero; }
        }
    E::run(va, vb, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r)
                gst2(dst + (long long)E::last_row(b, r) * W, va[b * E::RL + r], vb[b * E::RL + r]);
    }
}

// ---------------------------------------------------------------------------
// Launchers.
template <typename Real, int L>
cudaError_t launch_fwd_energy_t(const Geom &g, const Band &band, const Work<Real> &w,
                                const Real *A_in, cudaStream_t s)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, false>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = band.kT > 0 ? k_fwd_energy<Real, L, true> : k_fwd_energy<Real, L, false>;
    static const cudaError_t e0 = smem_attrs(k_fwd_energy<Real, L, false>, smem);
    static const cudaError_t e1 = smem_attrs(k_fwd_energy<Real, L, true>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    long long nlines = (long long)g.N * g.N;
    unsigned grid = (unsigned)((nlines + C - 1) / C);
    k<<<grid, T, smem, s>>>(g, band, w.axis, (const typename EpsEntry<Real>::type *)w.eps, w.state, A_in,
                            (cx<Real> *)w.X, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

template <typename Real, int L, typename Cfg>
cudaError_t launch_fwd_y2_t(const Geom &g, const Work<Real> &w, cudaStream_t s)
{
    constexpr int C = Cfg::C, T = Cfg::T;
    using E = FftPair<Real, L, C, T, false>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = k_fwd_y2<Real, L, Cfg>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((2 * g.SP + C - 1) / C, g.N);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.X, (cx<Real> *)w.Y, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

// variant 0: single-column engine; 1: paired-column engine (L >= 128, FP32);
// 2: paired-column engine with 12 values per thread (3 * 2^k >= 192, FP32);
// 6: paired-column engine on tiles twice as wide (L >= 384, FP32)
template <typename Real, int L>
cudaError_t launch_fwd_y_t(const Geom &g, const Work<Real> &w, cudaStream_t s, int variant)
{
    if constexpr (L >= 128 && sizeof(Real) == 4) {
        if (variant == 1) return launch_fwd_y2_t<Real, L, PairCfg<L>>(g, w, s);
        if constexpr (fft_has_family1(L))
            if (variant == 2) return launch_fwd_y2_t<Real, L, PairCfg12<L>>(g, w, s);
        if constexpr (L >= 384 && PairCfg<L>::T <= 512)
            if (variant == 6) return launch_fwd_y2_t<Real, L, PairCfgW<L>>(g, w, s);
    }
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, false>;
    size_t smem = sizeof(cx<Real>) * E::SMEM_ELEMS;
    auto k = k_fwd_y<Real, L>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((2 * g.SP + C - 1) / C, g.N);
    k<<<grid, T, smem, s>>>(g, (const cx<Real> *)w.X, (cx<Real> *)w.Y, twiddles_for<Real>(w, L));
    return cudaGetLastError();
}

bool et_applies(const Geom &g, const Band &band);
cudaError_t launch_fwd_energy_col(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                                  cudaStream_t s);
// FP32: lengths 128, 256 and 512 at T = 0 take the lines-across-lanes pass of
// k_energy.cu when the plan has its twiddle tables
cudaError_t launch_fwd_energy(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                              cudaStream_t s)
{
    if (w.etw && et_applies(g, band)) return launch_fwd_energy_col(g, band, w, A_in, s);
#define CALL(L) launch_fwd_energy_t<float, L>(g, band, w, A_in, s)
    LH_P_SWITCH(g.PE, CALL)
#undef CALL
}
cudaError_t launch_fwd_energy(const Geom &g, const Band &band, const Work<double> &w, const double *A_in,
                              cudaStream_t s)
{
#define CALL(L) launch_fwd_energy_t<double, L>(g, band, w, A_in, s)
    LH_LEN_SWITCH_SMALL(g.PE, CALL)
#undef CALL
}
cudaError_t launch_fwd_y_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_fwd_y_pr(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_fwd_y_pr_tma(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
// variants 3, 4, 5: the TMA-staged persistent kernels of k_tma.cu; 8, 9: the
// pruned engine of k_pruned.cu (one-third padding); 10: its TMA-staged
// persistent form, 11 the same with two CTAs per SM (k_pruned_tma.cu)
cudaError_t launch_fwd_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant)
{
    if (variant == 10 || variant == 11) return launch_fwd_y_pr_tma(g, w, s, variant);
    if (variant >= 3 && variant <= 5) return launch_fwd_y_tma(g, w, s, variant);
    if (variant == 8 || variant == 9) return launch_fwd_y_pr(g, w, s, variant);
#define CALL(L) launch_fwd_y_t<float, L>(g, w, s, variant)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_fwd_y(const Geom &g, const Work<double> &w, cudaStream_t s, int variant)
{
#define CALL(L) launch_fwd_y_t<double, L>(g, w, s, variant)
    LH_LEN_SWITCH_SMALL(g.P, CALL)
#undef CALL
}

}  // namespace lh
