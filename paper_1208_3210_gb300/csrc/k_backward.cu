// Adjoint of the forward call for L = sum_{l,m} w(q_l, w_m) Im chi(q_l, w_m).
//
// Eq. 9 is bilinear in the occupied part a and the empty part b of A, so
//   dL/da(p, e_j)  = -c sum_{s,m} w(s, m) b(p + s, e_{j+m})   (correlation with w)
//   dL/db(p, e_j)  = -c sum_{s,m} w(s, m) a(p - s, e_{j-m})   (convolution with w)
// and both are products of transforms again:
//   g^ = conj(W^) b^,  h^ = W^ a^,  dL/dA = -c (g on occupied cells, h on empty cells).
// The forward passes k_fwd_energy / k_fwd_y supply a^ and b^ (transformed
// along energy and p_y); these kernels transform w the same way, form both
// products along p_x, and invert.  The wrap-around argument of the forward
// call (P >= N + Q/2, PE >= n_eps) also covers these lags.
//
// Finite temperature (Appendix A, Eq. A1): a = A f and b = A (1 - f) on every
// cell, and the correlation C(q, w) = sum a(p, e) b(p + q, e + w) enters
// Im chi_T as C(q, w) - C(-q, -w) and S(q, w) as C(q, w).  For Im chi_T the
// adjoint of C therefore sees w(q, w) - w(-q, -w), whose transform is the odd
// part W^ - conj(W^) = 2i Im W^ (the forward's odd_part, applied to W^); for
// S it sees w.  dL/dA = scale (f g + (1 - f) h) with the same Fermi weights as
// the forward energy pass.
//
//   k_w_energy      : w [Q][Q][n_omega] (real) -> half spectra along energy,
//                     two lines per complex FFT.                WU1 [Q][Q][SP]
//   k_w_y           : FFT along q_y, lags placed at their circular index.
//                                                              WU2 [Q][P][SP]
//   k_bw_product    : FFT along p_x of W^, a^, b^; h^ = W^ a^, g^ = conj(W^) b^;
//                     inverse along p_x, keep p_x < N.  Written over U2 in
//                     place (each CTA reads its column tile fully before it
//                     writes it): G3 [N][P][SP][2] = (h^, g^) interleaved.
//   k_bw_inv_y      : inverse along p_y, keep p_y < N.         G4 [N][N][SP][2]
//   k_bw_inv_energy : inverse real FFT along energy of g and h together
//                     (g + i h), dL/dA = scale * (Re on occupied cells, Im on
//                     empty ones); optionally the chain rule through Eqs. 4-5
//                     to (t, t', t'', mu, gamma), reduced per CTA in FP64.
#include "kernels.cuh"

namespace lh {

// --- w along energy -----------------------------------------------------------
template <typename Real, int L>
__global__ void __launch_bounds__(LineCfg<L>::T)
k_w_energy(Geom g, const Real *__restrict__ w, cx<Real> *__restrict__ WU1, const cx<Real> *__restrict__ tw)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, false>;
    using Cx = cx<Real>;
    constexpr int H = L / 2 + 1, SP = (H + 7) / 8 * 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)
    const long long npairs = (long long)g.Q * g.Q / 2;
    const long long f0 = (long long)blockIdx.x * C;

    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            long long f = f0 + col;
            Real x1 = 0, x2 = 0;
            if (f < npairs && n < g.n_omega) {
                x1 = w[(2 * f) * g.n_omega + n];
                x2 = w[(2 * f + 1) * g.n_omega + n];
            }
            v[b * E::R0 + r] = mk<Cx>(x1, x2);
        }
    E::run(v, sm, tw);
#pragma unroll
    for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
        for (int r = 0; r < E::RL; ++r) {
            int col, n;
            E::last_elem(b, r, col, n);
            sm[E::saddr(col, n)] = v[b * E::RL + r];
        }
    __syncthreads();
    const Real half = (Real)0.5;
    for (int idx = threadIdx.x; idx < C * H; idx += T) {
        int col = idx / H, k = idx % H;
        long long f = f0 + col;
        if (f >= npairs) continue;
        Cx zk = sm[E::saddr(col, k)];
        Cx zm = sm[E::saddr(col, k == 0 ? 0 : L - k)];   // Z(L - k), any length
        Cx w1 = mk<Cx>(half * (zk.x + zm.x), half * (zk.y - zm.y));
        Cx dd = mk<Cx>(zk.x - zm.x, zk.y + zm.y);
        Cx w2 = mk<Cx>(half * dd.y, -half * dd.x);
        WU1[(2 * f) * SP + k] = w1;
        WU1[(2 * f + 1) * SP + k] = w2;
    }
}

// --- w along q_y ----------------------------------------------------------------
template <typename Real, int L>
__global__ void __launch_bounds__(ColCfg<L>::T, ColCfg<L>::MINB)
k_w_y(Geom g, const cx<Real> *__restrict__ WU1, cx<Real> *__restrict__ WU2, const cx<Real> *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, false>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)
    const int lx = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < g.H;
    const Cx *src = WU1 + (long long)lx * g.Q * g.SP + c;
    Cx *dst = WU2 + (long long)lx * g.xs3 + c;
    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            int l = lag_index(n, g.P, g.Q);
            v[b * E::R0 + r] = (valid && l >= 0) ? src[(long long)l * g.SP] : mk<Cx>((Real)0, (Real)0);
        }
    E::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int col, n;
                E::last_elem(b, r, col, n);
                dst[(long long)n * g.SP] = v[b * E::RL + r];
            }
    }
}

// --- products along p_x -----------------------------------------------------------
template <typename Real, int L>
__global__ void __launch_bounds__(ColCfg<L>::T, 1)
k_bw_product(Geom g, cx<Real> *__restrict__ U2, const cx<Real> *__restrict__ WU2, const cx<Real> *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using EF = Fft<Real, L, C, T, MAP_COL, false>;
    using EI = Fft<Real, L, C, T, MAP_COL, true>;
    static_assert(EF::RL == EI::R0, "last forward radix must equal first inverse radix");
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM((EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS), Cx)
    const int W2 = 2 * g.SP;
    const int ky = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < g.H;
    const long long rstride = g.xs2;
    Cx *colA = U2 + (long long)ky * W2 + 2 * c;    // a^ column, later h^
    Cx *colB = colA + 1;                            // b^ column, later g^ (interleaved)
    const Cx *colW = WU2 + (long long)ky * g.SP + c;
    const long long wstride = g.xs3;
    const Cx zero = mk<Cx>((Real)0, (Real)0);

    Cx vw[EF::VPT], v[EF::VPT];
#pragma unroll
    for (int b = 0; b < EF::VPT / EF::R0; ++b)
#pragma unroll
        for (int r = 0; r < EF::R0; ++r) {
            int col, n;
            EF::first_elem(b, r, col, n);
            int l = lag_index(n, g.P, g.Q);
            vw[b * EF::R0 + r] = (valid && l >= 0) ? colW[(long long)l * wstride] : zero;
            v[b * EF::R0 + r] = (valid && n < g.N) ? colA[(long long)n * rstride] : zero;
        }
    EF::run(vw, sm, tw);
    if (g.quantity == LINDHARD_IMCHI_T) {   // w(q, w) - w(-q, -w): W^ - conj(W^)
#pragma unroll
        for (int i = 0; i < EF::VPT; ++i) vw[i] = mk<Cx>((Real)0, (Real)2 * vw[i].y);
    }
    EF::run(v, sm, tw);
#pragma unroll
    for (int i = 0; i < EF::VPT; ++i) v[i] = cmul(vw[i], v[i]);          // h^ = W^ a^
    EI::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < EI::VPT / EI::RL; ++b)
#pragma unroll
            for (int r = 0; r < EI::RL; ++r) {
                int col, n;
                EI::last_elem(b, r, col, n);
                if (n < g.N) colA[(long long)n * rstride] = v[b * EI::RL + r];
            }
    }
#pragma unroll
    for (int b = 0; b < EF::VPT / EF::R0; ++b)
#pragma unroll
        for (int r = 0; r < EF::R0; ++r) {
            int col, n;
            EF::first_elem(b, r, col, n);
            v[b * EF::R0 + r] = (valid && n < g.N) ? colB[(long long)n * rstride] : zero;
        }
    EF::run(v, sm, tw);
#pragma unroll
    for (int i = 0; i < EF::VPT; ++i) v[i] = cmulc(v[i], vw[i]);         // g^ = conj(W^) b^
    EI::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < EI::VPT / EI::RL; ++b)
#pragma unroll
            for (int r = 0; r < EI::RL; ++r) {
                int col, n;
                EI::last_elem(b, r, col, n);
                if (n < g.N) colB[(long long)n * rstride] = v[b * EI::RL + r];
            }
    }
}

// --- inverse along p_y -------------------------------------------------------------
template <typename Real, int L>
__global__ void __launch_bounds__(ColCfg<L>::T, ColCfg<L>::MINB)
k_bw_inv_y(Geom g, const cx<Real> *__restrict__ G3, cx<Real> *__restrict__ G4, const cx<Real> *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_COL, true>;
    using Cx = cx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)
    const int W2 = 2 * g.SP;
    const int px = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < W2 && ab_col_valid(c, g.H);
    const Cx *src = G3 + (long long)px * g.xs2 + c;
    Cx *dst = G4 + (long long)px * g.N * W2 + c;
    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            v[b * E::R0 + r] = valid ? src[(long long)n * W2] : mk<Cx>((Real)0, (Real)0);
        }
    E::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int col, n;
                E::last_elem(b, r, col, n);
                if (n < g.N) dst[(long long)n * W2] = v[b * E::RL + r];
            }
    }
}

// --- inverse along energy, dL/dA and dL/dtheta -----------------------------------
// partial[blockIdx.x][5] receives this CTA's FP64 sums of dL/dA * dA/dtheta.
template <typename Real, int L>
__global__ void __launch_bounds__(LineCfg<L>::T, (L & (L - 1)) == 0 ? 3 : 1)   // 16-value tiles: three CTAs per SM
k_bw_inv_energy(Geom g, Band band, const AxisTab *__restrict__ axis,
                const typename EpsEntry<Real>::type *__restrict__ eps, const InstState *__restrict__ st,
                const cx<Real> *__restrict__ G4, Real *__restrict__ dA, double *__restrict__ partial,
                const cx<Real> *__restrict__ tw)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<Real, L, C, T, MAP_LINE, true>;
    using Cx = cx<Real>;
    constexpr int H = L / 2 + 1, SP = (H + 7) / 8 * 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx *sm = reinterpret_cast<Cx *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, Cx)
    __shared__ Real s_xhi[C], s_xlo[C], s_amp[C], s_f[C][4];
    __shared__ double s_red[T / 32][5];
    const long long nlines = (long long)g.N * g.N;
    const long long line0 = (long long)blockIdx.x * C;
    const bool want_params = partial != nullptr;

    if (want_params && threadIdx.x < C) {
        long long line = line0 + threadIdx.x;
        if (line < nlines) {
            int ix = (int)(line / g.N), iy = (int)(line % g.N);
            AxisTab ax = axis[ix], ay = axis[iy];
            double e0;
            if (band.band_kind == 1) e0 = 0.5 * (ax.p2 + ay.p2);
            else e0 = -2.0 * band.t * (ax.c1 + ay.c1) - 4.0 * band.tp * ax.c1 * ay.c1
                      - 2.0 * band.tpp * (ax.c2 + ay.c2);
            double xi = e0 - st->mu;
            s_xhi[threadIdx.x] = (Real)xi;
            s_xlo[threadIdx.x] = (Real)(xi - (double)(Real)xi);
            s_amp[threadIdx.x] = (Real)(ax.g * ay.g * band.gamma / 3.14159265358979323846);
            // d xi / d(t, t', t''); d xi / d mu = -1
            bool tb = band.band_kind != 1;
            s_f[threadIdx.x][0] = tb ? (Real)(-2.0 * (ax.c1 + ay.c1)) : (Real)0;
            s_f[threadIdx.x][1] = tb ? (Real)(-4.0 * ax.c1 * ay.c1) : (Real)0;
            s_f[threadIdx.x][2] = tb ? (Real)(-2.0 * (ax.c2 + ay.c2)) : (Real)0;
            s_f[threadIdx.x][3] = (Real)-1;
        }
    }
    __syncthreads();

    Cx v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            long long line = line0 + col;
            Cx x = mk<Cx>((Real)0, (Real)0);
            if (line < nlines) {
                const Cx *row = G4 + line * (2LL * SP);    // (h^, g^) interleaved
                Cx xg, xh;
                if (n < H) { xh = row[2 * n]; xg = row[2 * n + 1]; }
                else { xh = cconj(row[2 * (L - n)]); xg = cconj(row[2 * (L - n) + 1]); }
                x = mk<Cx>(xg.x - xh.y, xg.y + xh.x);      // g^ + i h^
            }
            v[b * E::R0 + r] = x;
        }
    E::run(v, sm, tw);   // ends with __syncthreads: s_* visible

    const Real sc = (Real)g.scale;
    const Real gam = (Real)band.gamma, g2 = gam * gam, igam = (Real)1 / gam;
    Real acc_xi[4] = {0, 0, 0, 0}, acc_g = 0;
#pragma unroll
    for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
        for (int r = 0; r < E::RL; ++r) {
            int col, n;
            E::last_elem(b, r, col, n);
            long long line = line0 + col;
            if (line < nlines && n < g.n_eps) {
                Cx x = v[b * E::RL + r];
                Real d;                                       // dL/dA(p, e_n)
                if (band.kT > 0) {
                    // Fermi weights of e_n as the forward energy pass forms them
                    Real xe, u;
                    if constexpr (sizeof(Real) == 4) {
                        xe = (Real)(2 * n + 1 - g.n_eps) * band.x_step;
                        u = expf(-fabsf(xe));
                    } else {
                        xe = (Real)(2 * n + 1 - g.n_eps) * (Real)band.x_step64;
                        u = exp(-fabs(xe));
                    }
                    const Real big = (Real)1 / ((Real)1 + u), small = u * big;
                    d = xe < 0 ? sc * (big * x.x + small * x.y) : sc * (small * x.x + big * x.y);
                } else {
                    d = sc * ((n < g.J0) ? x.x : x.y);
                }
                if (dA) dA[line * g.n_eps + n] = d;
                if (want_params) {
                    Real e;
                    if constexpr (sizeof(Real) == 4) {
                        float2 ej = eps[n];
                        e = (ej.x - s_xhi[col]) + (ej.y - s_xlo[col]);
                    } else {
                        e = eps[n] - s_xhi[col];
                    }
                    Real D = e * e + g2;
                    Real iD;
                    if constexpr (sizeof(Real) == 4) {
                        // the hardware reciprocal (relative error about 2^-23;
                        // D lies in [gamma^2, 4 e_max^2 + gamma^2])
                        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iD) : "f"(D));
                    } else {
                        iD = (Real)1 / D;
                    }
                    Real A = s_amp[col] * iD;
                    Real dxi = d * (2 * e * A * iD);                  // dL/dA * dA/dxi
                    Real dg = d * (s_amp[col] * igam) * (e * e - g2) * iD * iD;   // dL/dA * dA/dgamma
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc_xi[q] += dxi * s_f[col][q];
                    acc_g += dg;
                }
            }
        }
    if (want_params) {
        double vals[5] = {acc_xi[0], acc_xi[1], acc_xi[2], acc_xi[3], acc_g};
#pragma unroll
        for (int q = 0; q < 5; ++q)
            for (int o = 16; o > 0; o >>= 1) vals[q] += __shfl_down_sync(0xffffffffu, vals[q], o);
        if ((threadIdx.x & 31) == 0)
            for (int q = 0; q < 5; ++q) s_red[threadIdx.x >> 5][q] = vals[q];
        __syncthreads();
        if (threadIdx.x < 5) {
            double t = 0;
            for (int wv = 0; wv < T / 32; ++wv) t += s_red[wv][threadIdx.x];
            partial[(size_t)blockIdx.x * 5 + threadIdx.x] = t;
        }
    }
}

// Final sum of the per-CTA partials [nblocks][5] in a fixed order
// (deterministic), in two levels: KRP_G CTAs each sum one fixed contiguous
// range into level[g][5], then one CTA sums the KRP_G rows.  In a CTA, 1020
// threads sweep the range coalesced, thread t always on component t % 5 (the
// stride 1020 keeps it), eight independent chains each; then each
// component's 204 thread sums are added in thread order.
constexpr int KRP_T = 1020, KRP_G = 64;
__device__ __forceinline__ void krp_sum(const double *__restrict__ src, long long n, double *s, double *dst)
{
    const int t = threadIdx.x;
    if (t < KRP_T) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        long long i = t;
        for (; i + 7 * KRP_T < n; i += 8 * KRP_T)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += src[i + u * KRP_T];
        for (; i < n; i += KRP_T) acc[0] += src[i];
        s[t] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
    __syncthreads();
    if (t < 5) {
        double acc = 0;
        for (int k = t; k < KRP_T; k += 5) acc += s[k];
        dst[t] = acc;
    }
}
__global__ void __launch_bounds__(1024) k_reduce_params1(const double *__restrict__ partial, int nblocks,
                                                         double *__restrict__ level)
{
    __shared__ double s[KRP_T];
    const long long per = (nblocks + KRP_G - 1) / KRP_G;
    const long long b0 = min((long long)nblocks, per * blockIdx.x), b1 = min((long long)nblocks, b0 + per);
    krp_sum(partial + 5 * b0, 5 * (b1 - b0), s, level + 5 * blockIdx.x);
}
__global__ void __launch_bounds__(1024) k_reduce_params2(const double *__restrict__ level, double *__restrict__ out)
{
    __shared__ double s[KRP_T];
    krp_sum(level, 5LL * KRP_G, s, out);
}

// --- launchers ------------------------------------------------------------------
template <typename K>
static cudaError_t set_smem(K k, size_t smem)
{
    return smem_attrs(k, smem);
}

template <int L>
cudaError_t launch_w_energy_t(const Geom &g, const float *w, float2 *WU1, const float2 *tw, int tw_len,
                              cudaStream_t s)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_LINE, false>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    static const cudaError_t e = set_smem(k_w_energy<float, L>, smem);
    if (e != cudaSuccess) return e;
    long long npairs = (long long)g.Q * g.Q / 2;
    k_w_energy<float, L><<<(unsigned)((npairs + C - 1) / C), T, smem, s>>>(g, w, WU1, tw + twiddle_offset(L));
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_w_y_t(const Geom &g, const float2 *WU1, float2 *WU2, const float2 *tw, int tw_len,
                         cudaStream_t s)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, false>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    static const cudaError_t e = set_smem(k_w_y<float, L>, smem);
    if (e != cudaSuccess) return e;
    k_w_y<float, L><<<dim3((g.H + C - 1) / C, g.Q), T, smem, s>>>(g, WU1, WU2, tw + twiddle_offset(L));
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_bw_product_t(const Geom &g, float2 *U2, const float2 *WU2, const float2 *tw, int tw_len,
                                cudaStream_t s)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using EF = Fft<float, L, C, T, MAP_COL, false>;
    using EI = Fft<float, L, C, T, MAP_COL, true>;
    constexpr int elems = EF::SMEM_ELEMS > EI::SMEM_ELEMS ? EF::SMEM_ELEMS : EI::SMEM_ELEMS;
    size_t smem = sizeof(float2) * elems;
    static const cudaError_t e = set_smem(k_bw_product<float, L>, smem);
    if (e != cudaSuccess) return e;
    k_bw_product<float, L><<<dim3((g.H + C - 1) / C, g.P), T, smem, s>>>(g, U2, WU2, tw + twiddle_offset(L));
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_bw_inv_y_t(const Geom &g, const float2 *G3, float2 *G4, const float2 *tw, int tw_len,
                              cudaStream_t s)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, true>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    static const cudaError_t e = set_smem(k_bw_inv_y<float, L>, smem);
    if (e != cudaSuccess) return e;
    k_bw_inv_y<float, L><<<dim3((2 * g.SP + C - 1) / C, g.N), T, smem, s>>>(g, G3, G4, tw + twiddle_offset(L));
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_bw_inv_energy_t(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                                   const InstState *st, const float2 *G4, float *dA, double *partial,
                                   const float2 *tw, int tw_len, cudaStream_t s)
{
    constexpr int C = LineCfg<L>::C, T = LineCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_LINE, true>;
    size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    static const cudaError_t e = set_smem(k_bw_inv_energy<float, L>, smem);
    if (e != cudaSuccess) return e;
    long long nlines = (long long)g.N * g.N;
    k_bw_inv_energy<float, L><<<(unsigned)((nlines + C - 1) / C), T, smem, s>>>(g, band, axis, eps, st, G4, dA,
                                                                              partial, tw + twiddle_offset(L));
    return cudaGetLastError();
}

// energy lengths: powers of two and, at finite temperature, 3 * 2^k
cudaError_t launch_w_energy(const Geom &g, const float *w, float2 *WU1, const float2 *tw, int tw_len,
                            cudaStream_t s)
{
#define CALL(L) launch_w_energy_t<L>(g, w, WU1, tw, tw_len, s)
    LH_P_SWITCH(g.PE, CALL)
#undef CALL
}
cudaError_t launch_w_y(const Geom &g, const float2 *WU1, float2 *WU2, const float2 *tw, int tw_len, cudaStream_t s)
{
#define CALL(L) launch_w_y_t<L>(g, WU1, WU2, tw, tw_len, s)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
bool pr_fwd_applies(const Geom &g);
bool pr_inv_applies(const Geom &g);
cudaError_t launch_bw_product_pr(const Geom &g, float2 *U2, const float2 *WU2, const float2 *ptw, cudaStream_t s);
// the pruned engine (k_pruned.cu) where the padding is exactly one third
cudaError_t launch_bw_product(const Geom &g, float2 *U2, const float2 *WU2, const float2 *tw, int tw_len,
                              const float2 *ptw, cudaStream_t s)
{
    if (ptw && pr_fwd_applies(g) && pr_inv_applies(g)) return launch_bw_product_pr(g, U2, WU2, ptw, s);
#define CALL(L) launch_bw_product_t<L>(g, U2, WU2, tw, tw_len, s)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_bw_inv_y(const Geom &g, const float2 *G3, float2 *G4, const float2 *tw, int tw_len,
                            cudaStream_t s)
{
#define CALL(L) launch_bw_inv_y_t<L>(g, G3, G4, tw, tw_len, s)
    LH_P_SWITCH(g.P, CALL)
#undef CALL
}
cudaError_t launch_bw_inv_energy(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                                 const InstState *st, const float2 *G4, float *dA, double *partial,
                                 const float2 *tw, int tw_len, cudaStream_t s)
{
#define CALL(L) launch_bw_inv_energy_t<L>(g, band, axis, eps, st, G4, dA, partial, tw, tw_len, s)
    LH_P_SWITCH(g.PE, CALL)
#undef CALL
}
int bw_energy_blocks(const Geom &g)
{
    int C = 0;
    switch (g.PE) {
    case 16: C = LineCfg<16>::C; break;
    case 32: C = LineCfg<32>::C; break;
    case 48: C = LineCfg<48>::C; break;
    case 64: C = LineCfg<64>::C; break;
    case 96: C = LineCfg<96>::C; break;
    case 128: C = LineCfg<128>::C; break;
    case 192: C = LineCfg<192>::C; break;
    case 256: C = LineCfg<256>::C; break;
    case 384: C = LineCfg<384>::C; break;
    case 512: C = LineCfg<512>::C; break;
    case 768: C = LineCfg<768>::C; break;
    case 1024: C = LineCfg<1024>::C; break;
    case 1536: C = LineCfg<1536>::C; break;
    case 2048: C = LineCfg<2048>::C; break;
    default: C = LineCfg<4096>::C; break;
    }
    long long nlines = (long long)g.N * g.N;
    return (int)((nlines + C - 1) / C);
}
// rows the reduction's first level adds after the nblocks x 5 sums
int bw_partial_extra_rows() { return KRP_G; }
// partial holds nblocks x 5 sums followed by room for KRP_G x 5
cudaError_t launch_reduce_params(const double *partial, int nblocks, double *out, cudaStream_t s)
{
    double *level = const_cast<double *>(partial) + 5LL * nblocks;
    k_reduce_params1<<<KRP_G, 1024, 0, s>>>(partial, nblocks, level);
    k_reduce_params2<<<1, 1024, 0, s>>>(level, out);
    return cudaGetLastError();
}

}  // namespace lh
