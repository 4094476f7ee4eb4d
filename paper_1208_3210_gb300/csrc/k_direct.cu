// The energy-direct form of the correlation: the paper's own arrangement
// (Sec. 3).  The momentum convolution of Eq. 9 becomes a product of 2D
// transforms over momentum, one per energy plane (the real-space B(r, e) of
// Sec. 3), and the energy integral stays a sum, done directly for every
// momentum frequency k:
//
//   C(k, w_m) = sum_j conj(a^_j(k)) b^_{j+m}(k),  j < J0 <= j + m < n_eps,
//   Im chi(q, w_m) = -c / P^2 sum_k exp(i k q) C(k, w_m).
//
//   k_direct_planes : A(p, e) of the occupied plane t and the empty plane
//                     J0 + t packed as z_t = a_t + i b_{J0+t} (one complex
//                     transform for two real planes), columns of [N][N][2 SPt]
//   (p_y forward pass of the 3D form on those columns)
//   k_outer_fft     : transform along p_x (forward, all P frequencies) or
//                     along k_x (inverse, keeping the Q lags)
//   k_direct_corr   : for a frequency k and its mirror -k, separates a^_t and
//                     b^_{J0+t} from z^_t(k) and z^_t(-k) and sums the energy
//                     correlation at every transfer; C(-k) = conj C(k)
//   (p_y inverse pass of the 3D form on the transfer columns)
//   k_direct_out    : real part with the prefactor, [Q][Q][n_omega]
#include "kernels.cuh"

namespace lh {

// ---------------------------------------------------------------------------
// Planes.  CTA = 8 momentum points (lines) x the 2 SPt columns of each.
constexpr int kPlaneLines = 8;

__global__ void __launch_bounds__(256)
k_direct_planes(Geom g, int T, int W, Band band, const AxisTab *__restrict__ axis, const float2 *__restrict__ eps,
                const InstState *__restrict__ st, const float *__restrict__ A_in, float2 *__restrict__ U1)
{
    __shared__ float s_xhi[kPlaneLines], s_xlo[kPlaneLines], s_amp[kPlaneLines];
    const long long nlines = (long long)g.N * g.N;
    const long long line0 = (long long)blockIdx.x * kPlaneLines;
    if (A_in == nullptr && threadIdx.x < kPlaneLines) {
        const long long line = line0 + threadIdx.x;
        if (line < nlines) {
            const int ix = (int)(line / g.N), iy = (int)(line % g.N);
            band_point_f32(band, axis[ix], axis[iy], st, s_xhi[threadIdx.x], s_xlo[threadIdx.x], s_amp[threadIdx.x]);
        }
    }
    __syncthreads();
    const float g2 = (float)(band.gamma * band.gamma);
    auto spectral = [&](int col, long long line, int j) -> float {
        if (j >= g.n_eps) return 0.f;
        if (A_in != nullptr) return A_in[line * g.n_eps + j];
        const float2 ej = eps[j];
        const float e = (ej.x - s_xhi[col]) + (ej.y - s_xlo[col]);
        return __fdividef(s_amp[col], e * e + g2);
    };
    for (int idx = threadIdx.x; idx < kPlaneLines * W; idx += blockDim.x) {
        const int col = idx / W, t = idx % W;
        const long long line = line0 + col;
        if (line >= nlines) continue;
        float2 z = make_float2(0.f, 0.f);
        if (t < T) {
            z.x = t < g.J0 ? spectral(col, line, t) : 0.f;   // occupied plane t
            z.y = spectral(col, line, g.J0 + t);              // empty plane J0 + t
        }
        U1[line * W + t] = z;
    }
}

// ---------------------------------------------------------------------------
// Transform along the outer axis of a [rows][inner][width] layout, one CTA per
// (column tile, inner index).  Forward: rows n < nin (zero beyond), all L
// outputs; inverse: all L rows in, the Q lags out.
template <int L, bool INV>
__global__ void __launch_bounds__(ColCfg<L>::T, ColCfg<L>::MINB)
k_outer_fft(int ncols, int nin, int Q, long long istride, int iw, long long ostride, int ow,
            const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, INV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    LH_REQUIRE_SMEM(E::SMEM_ELEMS, float2)

    const int y = blockIdx.y;
    const int c = blockIdx.x * C + (int)(threadIdx.x % C);
    const bool valid = c < ncols;
    const float2 *src = in + (long long)y * iw + c;
    float2 *dst = out + (long long)y * ow + c;
    float2 v[E::VPT];
#pragma unroll
    for (int b = 0; b < E::VPT / E::R0; ++b)
#pragma unroll
        for (int r = 0; r < E::R0; ++r) {
            int col, n;
            E::first_elem(b, r, col, n);
            v[b * E::R0 + r] = (valid && n < nin) ? src[(long long)n * istride] : make_float2(0.f, 0.f);
        }
    E::run(v, sm, tw);
    if (valid) {
#pragma unroll
        for (int b = 0; b < E::VPT / E::RL; ++b)
#pragma unroll
            for (int r = 0; r < E::RL; ++r) {
                int col, n;
                E::last_elem(b, r, col, n);
                const int l = INV ? lag_index(n, L, Q) : n;
                if (l >= 0) dst[(long long)l * ostride] = v[b * E::RL + r];
            }
    }
}

// ---------------------------------------------------------------------------
// Energy correlation per momentum frequency.  One warp per frequency pair
// (k, -k): k_x in (0, P/2) with every k_y, and k_x in {0, P/2} with
// k_y in [0, P/2] (those pairs' mirrors lie in the same columns).  Lane l sums
// the transfers m = l R .. l R + R - 1; a window of 2R values of b^ slides
// along j, so each step loads one value of a^ (a broadcast) and one of b^
// per R^2 complex products.
constexpr int kCorrWarps = 8;

__host__ __device__ inline long long corr_pairs(int P) { return 2LL * (P / 2 + 1) + (long long)(P / 2 - 1) * P; }
// shared float2s of one warp: a^ (J0 rounded up to R, and to 2 so that every
// warp's arrays start on 16 bytes) and b^ (that + 32 R)
__host__ __device__ inline int corr_a_len(int J0, int R)
{
    const int q = R < 2 ? 2 : R;
    return (J0 + q - 1) / q * q;
}

template <int R>
__global__ void __launch_bounds__(kCorrWarps * 32)
k_direct_corr(Geom g, int T, int W, long long zs, int SPo, long long cs, const float2 *__restrict__ Z,
              float2 *__restrict__ Cout)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int J0 = g.J0, P = g.P;
    const int AL = corr_a_len(J0, R), BL = AL + 32 * R;
    if (dyn_smem_bytes() < (unsigned)(kCorrWarps * (AL + BL) * sizeof(float2))) return;
    float2 *as = reinterpret_cast<float2 *>(smem_raw) + (size_t)warp * (AL + BL);
    float2 *bs = as + AL;

    const long long pair = (long long)blockIdx.x * kCorrWarps + warp;
    if (pair >= corr_pairs(P)) return;
    int kx, ky;
    if (pair < P / 2 + 1) { kx = 0; ky = (int)pair; }
    else if (pair < 2 * (P / 2 + 1)) { kx = P / 2; ky = (int)(pair - (P / 2 + 1)); }
    else {
        const long long r = pair - 2 * (P / 2 + 1);
        kx = 1 + (int)(r / P);
        ky = (int)(r % P);
    }
    const int mx = (P - kx) % P, my = (P - ky) % P;
    const bool self = mx == kx && my == ky;
    const float2 *zk = Z + (long long)kx * zs + (long long)ky * W;
    const float2 *zm = Z + (long long)mx * zs + (long long)my * W;

    for (int i = lane; i < AL; i += 32) as[i] = make_float2(0.f, 0.f);
    for (int i = lane; i < BL; i += 32) bs[i] = make_float2(0.f, 0.f);
    __syncwarp();
    for (int t = lane; t < T; t += 32) {
        const float2 p = zk[t], q = zm[t];
        // a^ = (z^(k) + conj z^(-k)) / 2, stored conjugated; b^ = (z^(k) - conj z^(-k)) / 2i
        if (t < J0) as[t] = make_float2(0.5f * (p.x + q.x), -0.5f * (p.y - q.y));
        if (J0 + t < BL) bs[J0 + t] = make_float2(0.5f * (p.y + q.y), -0.5f * (p.x - q.x));
    }
    __syncwarp();

    const int m0 = lane * R;
    float2 acc[R], w[2 * R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r] = make_float2(0.f, 0.f);
        w[r] = bs[m0 + r];
    }
    for (int j0 = 0; j0 < AL; j0 += R) {
        float2 a[R];
        if constexpr (R % 2 == 0) {
            // j0 and m0 are multiples of R: every pair below starts on 16 bytes
            const float4 *b4 = reinterpret_cast<const float4 *>(bs + j0 + R + m0);
            const float4 *a4 = reinterpret_cast<const float4 *>(as + j0);
#pragma unroll
            for (int i = 0; i < R / 2; ++i) {
                const float4 q = b4[i], u = a4[i];
                w[R + 2 * i] = make_float2(q.x, q.y);
                w[R + 2 * i + 1] = make_float2(q.z, q.w);
                a[2 * i] = make_float2(u.x, u.y);
                a[2 * i + 1] = make_float2(u.z, u.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) {
                w[R + i] = bs[j0 + R + m0 + i];
                a[i] = as[j0 + i];
            }
        }
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 b = w[jj + r];
                acc[r].x = fmaf(a[jj].x, b.x, fmaf(-a[jj].y, b.y, acc[r].x));
                acc[r].y = fmaf(a[jj].x, b.y, fmaf(a[jj].y, b.x, acc[r].y));
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) w[i] = w[R + i];
    }
    float2 *ck = Cout + (long long)kx * cs + (long long)ky * SPo;
    float2 *cm = Cout + (long long)mx * cs + (long long)my * SPo;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int m = m0 + r;
        if (m < g.n_omega) {
            ck[m] = acc[r];
            if (!self) cm[m] = make_float2(acc[r].x, -acc[r].y);
        }
    }
}

// ---------------------------------------------------------------------------
// Output: Im chi = scale * Re of the inverse transform, [Q][Q][n_omega].
__global__ void __launch_bounds__(256)
k_direct_out(int Q, int n_omega, int SPo, double scale, const float2 *__restrict__ U4, float *__restrict__ out)
{
    const long long n = (long long)Q * Q * n_omega;
    const float sc = (float)scale;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long l = i / n_omega;
        const int m = (int)(i % n_omega);
        out[i] = sc * U4[l * SPo + m].x;
    }
}

// ---------------------------------------------------------------------------
// Launchers.
template <int L, bool INV>
static cudaError_t launch_outer_t(int ncols, int nin, int Q, int ninner, long long istride, int iw,
                                  long long ostride, int ow, const float2 *in, float2 *out, const float2 *tw,
                                  cudaStream_t s)
{
    constexpr int C = ColCfg<L>::C, T = ColCfg<L>::T;
    using E = Fft<float, L, C, T, MAP_COL, INV>;
    const size_t smem = sizeof(float2) * E::SMEM_ELEMS;
    auto k = k_outer_fft<L, INV>;
    static const cudaError_t e = smem_attrs(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((ncols + C - 1) / C, ninner);
    k<<<grid, T, smem, s>>>(ncols, nin, Q, istride, iw, ostride, ow, in, out, tw);
    return cudaGetLastError();
}

template <bool INV>
static cudaError_t launch_outer(int L, int ncols, int nin, int Q, int ninner, long long istride, int iw,
                                long long ostride, int ow, const float2 *in, float2 *out, const Work<float> &w,
                                cudaStream_t s)
{
#define CALL(L) launch_outer_t<L, INV>(ncols, nin, Q, ninner, istride, iw, ostride, ow, in, out, \
                                       twiddles_for<float>(w, L), s)
    LH_P_SWITCH(L, CALL)
#undef CALL
}

template <int R>
static cudaError_t launch_corr_t(const Geom &g, const DirectGeom &d, const float2 *Z, float2 *C, cudaStream_t s)
{
    const int AL = corr_a_len(g.J0, R), BL = AL + 32 * R;
    const size_t smem = sizeof(float2) * (size_t)kCorrWarps * (AL + BL);
    auto k = k_direct_corr<R>;
    // the limit for the largest geometry the form takes (J0 <= 512), set once
    static const cudaError_t e = smem_attrs(k, sizeof(float2) * (size_t)kCorrWarps * (2 * 512 + 32 * R));
    if (e != cudaSuccess) return e;
    const long long blocks = (corr_pairs(g.P) + kCorrWarps - 1) / kCorrWarps;
    k<<<(unsigned)blocks, kCorrWarps * 32, smem, s>>>(g, d.T, 2 * d.t.SP, d.zs, d.o.SP, d.cs, Z, C);
    return cudaGetLastError();
}

cudaError_t launch_fwd_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);

// Whether the direct form takes this geometry (the transfers per lane and the
// shared memory of the correlation kernel bound n_omega and n_eps).
bool direct_supported(const Geom &g) { return g.n_omega <= 512 && g.n_eps <= 1024; }

// The passes after the set-up: planes, p_y, p_x, energy correlation, k_x
// inverse, k_y inverse, output (stage = 0: planes; 1: p_y forward; 2: p_x
// forward, correlation and k_x inverse; 3: k_y inverse; 4: output).
cudaError_t launch_direct_stage(int stage, const Geom &g, const Band &band, const Work<float> &w,
                                const float *A_in, float *out, cudaStream_t s)
{
    const DirectGeom d = direct_geom(g);
    float2 *X = (float2 *)w.X, *Y = (float2 *)w.Y;
    const int Wt = 2 * d.t.SP;
    switch (stage) {
    case 0: {
        const long long nlines = (long long)g.N * g.N;
        k_direct_planes<<<(unsigned)((nlines + kPlaneLines - 1) / kPlaneLines), 256, 0, s>>>(
            g, d.T, Wt, band, w.axis, (const float2 *)w.eps, w.state, A_in, X);
        return cudaGetLastError();
    }
    case 1:   // X [N][N][2 SPt] -> Y [N][P][2 SPt]
        return launch_fwd_y(d.t, w, s, g.P >= 128 ? 1 : 0);
    case 2: {
        // Y [N (x)][P][2 SPt] -> X: Z [P (k_x)][P][2 SPt]
        cudaError_t e = launch_outer<false>(g.P, Wt, g.N, g.Q, g.P, d.t.xs2, Wt, d.zs, Wt, Y, X, w, s);
        // X: Z -> Y: C [P][P][SPo]
        if (e == cudaSuccess) {
            const int n = g.n_omega;
            e = n <= 32 ? launch_corr_t<1>(g, d, X, Y, s)
              : n <= 64 ? launch_corr_t<2>(g, d, X, Y, s)
              : n <= 128 ? launch_corr_t<4>(g, d, X, Y, s)
              : n <= 256 ? launch_corr_t<8>(g, d, X, Y, s)
                         : launch_corr_t<16>(g, d, X, Y, s);
        }
        // Y: C -> X: [Q (l_x)][P][SPo]
        if (e == cudaSuccess)
            e = launch_outer<true>(g.P, g.n_omega, g.P, g.Q, g.P, d.cs, d.o.SP, d.o.xs3, d.o.SP, Y, X, w, s);
        return e;
    }
    case 3:   // X [Q][P][SPo] -> Y [Q][Q][SPo]
        return launch_inv_y(d.o, w, s, 0);
    default: {
        const double scale = g.scale * g.PE;   // -(de / 2 pi) / npz^2 / P^2: no energy transform
        const long long n = (long long)g.Q * g.Q * g.n_omega;
        const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
        k_direct_out<<<blocks, 256, 0, s>>>(g.Q, g.n_omega, d.o.SP, scale, Y, out);
        return cudaGetLastError();
    }
    }
}

}  // namespace lh
