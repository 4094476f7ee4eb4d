// FP64 sum-rule reductions (a check of a computed output, not part of the
// forward call).  Summing Eq. 9 over every lag q factorises (and so do the
// finite-temperature quantities, with Fermi weights: see k_dos_corr):
//   sum_q Im chi(q, w_m) = -c sum_j D_a(e_j) D_b(e_{j+m}),
//   D_a(e) = sum_p a(p, e),  D_b(e) = sum_p b(p, e),
// (swap the order of the momentum sums), which holds exactly on the grid when
// the output keeps every lag (Q = N in the reduced zone, Q = 2N in the
// extended zone).  The left side reduces the output, the right side the
// spectral function; both in FP64.
#include "kernels.cuh"

namespace lh {

// D(e_j) = sum_p A(p, e_j): A generated as in k_fwd_energy (or read from
// A_in); one CTA per chunk of momentum points, FP64 atomics into D.
__global__ void k_dos(Geom g, Band band, const AxisTab *__restrict__ axis, const float2 *__restrict__ eps,
                      const InstState *__restrict__ st, const float *__restrict__ A_in, double *D)
{
    extern __shared__ double s_d[];   // [n_eps]
    for (int j = threadIdx.x; j < g.n_eps; j += blockDim.x) s_d[j] = 0.0;
    __syncthreads();
    const long long nlines = (long long)g.N * g.N;
    const float g2 = (float)(band.gamma * band.gamma);
    for (long long line = blockIdx.x; line < nlines; line += gridDim.x) {
        float xhi = 0.f, xlo = 0.f, amp = 0.f;
        if (A_in == nullptr) {
            int ix = (int)(line / g.N), iy = (int)(line % g.N);
            AxisTab ax = axis[ix], ay = axis[iy];
            double e0 = (band.band_kind == 1) ? 0.5 * (ax.p2 + ay.p2)
                        : -2.0 * band.t * (ax.c1 + ay.c1) - 4.0 * band.tp * ax.c1 * ay.c1
                              - 2.0 * band.tpp * (ax.c2 + ay.c2);
            double xi = e0 - st->mu;
            xhi = (float)xi;
            xlo = (float)(xi - (double)xhi);
            amp = (float)(ax.g * ay.g * band.gamma / 3.14159265358979323846);
        }
        for (int j = threadIdx.x; j < g.n_eps; j += blockDim.x) {
            float A;
            if (A_in != nullptr) {
                A = A_in[line * g.n_eps + j];
            } else {
                float2 ej = eps[j];
                float e = (ej.x - xhi) + (ej.y - xlo);
                A = amp * __frcp_rn(e * e + g2);
            }
            s_d[j] += (double)A;   // each thread owns its own j entries
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < g.n_eps; j += blockDim.x) atomicAdd(&D[j], s_d[j]);
}

// dos_corr[m] = -c sum_j D_a(e_j) D_b(e_{j+m}), c = de/(2 pi)/npz^2.  At
// temperature kT > 0 (a = A f, b = A (1 - f), Eq. A1) the same exchange of
// sums gives
//   Im chi_T: -c sum_j D(e_j) D(e_{j+m}) [f(e_j) - f(e_{j+m})],
//   S:     (c/pi) sum_j D(e_j) D(e_{j+m}) f(e_j) [1 - f(e_{j+m})],
// f(e_j) = 1 / (exp((2j + 1 - n_eps) x_step) + 1) in FP64.
__global__ void k_dos_corr(Geom g, double x_step, const double *__restrict__ D, double *dos_corr)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.n_omega) return;
    const double pi = 3.14159265358979323846;
    const double c = (g.de / (2.0 * pi)) / ((double)g.npz * g.npz);
    auto occ = [&](int j) { return 1.0 / (exp((double)(2 * j + 1 - g.n_eps) * x_step) + 1.0); };
    auto emp = [&](int j) { return 1.0 / (exp(-(double)(2 * j + 1 - g.n_eps) * x_step) + 1.0); };
    double s = 0.0;
    for (int j = 0; j + m < g.n_eps; ++j) {
        if (g.quantity == LINDHARD_IMCHI_T) s += D[j] * D[j + m] * (occ(j) - occ(j + m));
        else if (g.quantity == LINDHARD_SQW) s += D[j] * D[j + m] * (occ(j) * emp(j + m));
        else if (j < g.J0 && j + m >= g.J0) s += D[j] * D[j + m];
    }
    dos_corr[m] = g.quantity == LINDHARD_SQW ? c / pi * s : -c * s;
}

// sum_q[m] = sum over all lags of out[l_x][l_y][m], FP64.
__global__ void k_sum_q(Geom g, const float *__restrict__ out, double *sum_q)
{
    extern __shared__ double s_q[];   // [n_omega]
    for (int m = threadIdx.x; m < g.n_omega; m += blockDim.x) s_q[m] = 0.0;
    __syncthreads();
    const long long rows = (long long)g.Q * g.Q;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x)
        for (int m = threadIdx.x; m < g.n_omega; m += blockDim.x) s_q[m] += (double)out[r * g.n_omega + m];
    __syncthreads();
    for (int m = threadIdx.x; m < g.n_omega; m += blockDim.x) atomicAdd(&sum_q[m], s_q[m]);
}

// dmu/d(t, t', t'', gamma) at fixed filling (the rigid band of Sec. 3): the
// filling n = (2/npz^2) sum_k [1/2 - atan(xi_k/gamma)/pi] over the first-zone
// grid is held fixed, so dmu/dtheta = -(dn/dtheta) / (dn/dmu).  Per state,
// with D = xi^2 + gamma^2: dn/dmu ~ gamma/(pi D); dn/dtheta ~ -gamma/(pi D)
// dxi/dtheta, dxi/d(t, t', t'') = (-2 (cos px + cos py), -4 cos px cos py,
// -2 (cos 2px + cos 2py)) (0 for free electrons); dn/dgamma ~ xi/(pi D).
// Each CTA reduces its share of the npz^2 states in FP64 (fixed-order tree)
// into part[blockIdx.x][5]; the host adds the CTAs in order.
constexpr int DMU_THREADS = 256;
__global__ void __launch_bounds__(DMU_THREADS)
k_dmu_partials(int kind, double t, double tp, double tpp, double gamma, int npz, double mu, double *part)
{
    extern __shared__ double sd[];                  // c1[npz], c2[npz], p2[npz], red[5][DMU_THREADS]
    double *c1 = sd, *c2 = sd + npz, *p2 = sd + 2 * npz, *red = sd + 3 * npz;
    const double pi = 3.14159265358979323846, dp = 2.0 * pi / npz;
    for (int i = threadIdx.x; i < npz; i += blockDim.x) {
        const double p = (double)(i - npz / 2) * dp;
        c1[i] = cos(p);
        c2[i] = cos(2.0 * p);
        p2[i] = p * p;
    }
    __syncthreads();
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)npz * npz;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(idx / npz), iy = (int)(idx % npz);
        const double e0 = kind == 1 ? 0.5 * (p2[ix] + p2[iy])
                                    : -2.0 * t * (c1[ix] + c1[iy]) - 4.0 * tp * c1[ix] * c1[iy]
                                          - 2.0 * tpp * (c2[ix] + c2[iy]);
        const double xi = e0 - mu, D = xi * xi + gamma * gamma, w = gamma / (pi * D);
        acc[0] += w;
        if (kind == 0) {
            acc[1] += w * 2.0 * (c1[ix] + c1[iy]);
            acc[2] += w * 4.0 * c1[ix] * c1[iy];
            acc[3] += w * 2.0 * (c2[ix] + c2[iy]);
        }
        acc[4] += xi / (pi * D);
    }
    for (int r = 0; r < 5; ++r) red[r * DMU_THREADS + threadIdx.x] = acc[r];
    __syncthreads();
    for (int h = DMU_THREADS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int r = 0; r < 5; ++r) red[r * DMU_THREADS + threadIdx.x] += red[r * DMU_THREADS + threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x * DMU_THREADS];
}

cudaError_t launch_dmu_partials(int kind, double t, double tp, double tpp, double gamma, int npz, double mu,
                                double *part, int blocks, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (3 * (size_t)npz + 5 * DMU_THREADS);
    static const cudaError_t e0 = smem_attrs(k_dmu_partials, sizeof(double) * (3 * 4096 + 5 * DMU_THREADS));
    if (e0 != cudaSuccess) return e0;
    k_dmu_partials<<<blocks, DMU_THREADS, smem, s>>>(kind, t, tp, tpp, gamma, npz, mu, part);
    return cudaGetLastError();
}

cudaError_t launch_sum_rule(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                            const InstState *st, const float *A_in, const float *out, double *D, double *sum_q,
                            double *dos_corr, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(D, 0, sizeof(double) * g.n_eps, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum_q, 0, sizeof(double) * g.n_omega, s);
    if (e != cudaSuccess) return e;
    int T = 256;
    k_dos<<<1024, T, sizeof(double) * g.n_eps, s>>>(g, band, axis, eps, st, A_in, D);
    k_dos_corr<<<(g.n_omega + 127) / 128, 128, 0, s>>>(g, band.x_step64, D, dos_corr);
    k_sum_q<<<1024, T, sizeof(double) * g.n_omega, s>>>(g, out, sum_q);
    return cudaGetLastError();
}

}  // namespace lh
