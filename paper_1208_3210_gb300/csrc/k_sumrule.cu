// FP64 sum-rule reductions (a check of a computed output, not part of the
// forward call).  Summing Eq. 9 over every lag q factorises:
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

// dos_corr[m] = -c sum_j D_a(e_j) D_b(e_{j+m}), c = de/(2 pi)/npz^2.
__global__ void k_dos_corr(Geom g, const double *__restrict__ D, double *dos_corr)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.n_omega) return;
    const double c = (g.de / (2.0 * 3.14159265358979323846)) / ((double)g.npz * g.npz);
    double s = 0.0;
    for (int j = 0; j + m < g.n_eps; ++j)
        if (j < g.J0 && j + m >= g.J0) s += D[j] * D[j + m];
    dos_corr[m] = -c * s;
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

cudaError_t launch_sum_rule(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                            const InstState *st, const float *A_in, const float *out, double *D, double *sum_q,
                            double *dos_corr, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(D, 0, sizeof(double) * g.n_eps, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum_q, 0, sizeof(double) * g.n_omega, s);
    if (e != cudaSuccess) return e;
    int T = 256;
    k_dos<<<1024, T, sizeof(double) * g.n_eps, s>>>(g, band, axis, eps, st, A_in, D);
    k_dos_corr<<<(g.n_omega + 127) / 128, 128, 0, s>>>(g, D, dos_corr);
    k_sum_q<<<1024, T, sizeof(double) * g.n_omega, s>>>(g, out, sum_q);
    return cudaGetLastError();
}

}  // namespace lh
