// Set-up kernels: twiddle tables, per-axis momentum tables, the energy grid,
// and the rigid-band chemical potential (Sec. 3: the Fermi level is shifted to
// hold the requested electron count).
#include <math.h>

#include "kernels.cuh"

namespace lh {

// Every twiddle table (see twiddle_offset), FP64 sincospi.
__global__ void k_twiddles(int max_len, float2 *tw32, double2 *tw64)
{
    (void)max_len;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= twiddle_entries()) return;
    int L, n;
    if (idx < 8176) {                       // powers of two
        L = 16;
        while (2 * L - 16 <= idx) L *= 2;   // the table that holds idx
        n = idx - (L - 16);
    } else {                                // 3 * 2^k
        int r = idx - 8176;
        L = 48;
        while (2 * L - 48 <= r) L *= 2;
        n = r - (L - 48);
    }
    double s, c;
    sincospi(-2.0 * (double)n / (double)L, &s, &c);
    tw32[idx] = make_float2((float)c, (float)s);
    tw64[idx] = make_double2(c, s);
}

// Per-axis tables at p_i = (i - N/2) 2 pi / npz and the energy grid
// e_j = -e_max + (j + 1/2) de, all in FP64.  The FP32 path stores e_j as an
// unevaluated pair hi + lo so that e_j - xi_p keeps full precision near the
// Lorentzian peak.
__global__ void k_tables(Geom g, Band band, AxisTab *axis, float2 *eps32, double *eps64)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.N) {
        double u = 2.0 * (double)(i - g.N / 2) / (double)g.npz;   // p_i / pi
        double p = u * 3.14159265358979323846;
        AxisTab a;
        a.c1 = cospi(u);
        a.c2 = cospi(2.0 * u);
        a.g = (band.ff_a == 0.0) ? 1.0 : exp(-p * p * band.ff_a * band.ff_a / 8.0);
        a.p2 = p * p;
        a.c1f = (float)a.c1;
        a.c2f = (float)a.c2;
        a.p2f = (float)a.p2;
        a.pad = 0.f;
        axis[i] = a;
    }
    if (i < g.n_eps) {
        double e = -g.e_max + ((double)i + 0.5) * g.de;
        if (eps32) {
            float hi = (float)e;
            eps32[i] = make_float2(hi, (float)(e - (double)hi));
        }
        if (eps64) eps64[i] = e;
    }
}

// ---------------------------------------------------------------------------
// Chemical potential.  n(mu) = (2/npz^2) sum_k [1/2 - atan((e0_k - mu)/gamma)/pi]
// over the first-zone grid (the Lorentzian occupation of Eq. 5 below the Fermi
// level).  n is strictly increasing in mu.  Five small launches of G CTAs:
//   3 passes of MU_SECT-point multisection in FP32 shrink the bracket
//   [-B-3, B+3] eV (B bounds |e0|) by (MU_SECT-1)^3 to tens of micro-eV;
//   every thread owns one candidate and a share of the points;
//   2 Newton steps in FP64 from the bracket midpoint reach FP64 precision
//   (the error after a step is about |F''/2F'| times the step squared).
// Each launch ends the same way: every CTA stores its partial sums, and the
// last CTA to finish (an atomic counter, which it resets) adds them in a fixed
// order and publishes the new bracket or mu for the next launch.  No CTA ever
// waits for another.
constexpr int MU_SECT = 64;
constexpr int MU_THREADS = 256;
constexpr int MU_FP32_PASSES = 3;
constexpr int MU_NEWTON = 2;
constexpr int MU_SECT_CTAS = 152;  // CTAs of a multisection pass
constexpr int MU_RES = 16;   // result slots at the start of acc

// Layout of acc: [MU_RES] results (3 per multisection pass from 0, 2 per
// Newton step from 10), then [MU_FP32_PASSES][G][MU_SECT], then
// [MU_NEWTON][G][2] doubles.
size_t mu_acc_doubles(int G) { return MU_RES + (size_t)G * (MU_FP32_PASSES * MU_SECT + MU_NEWTON * 2); }
size_t mu_barrier_words() { return 32; }   // the arrival counter (one 128-byte line)

__device__ __forceinline__ double band_e0(const Band &b, const AxisTab &ax, const AxisTab &ay)
{
    if (b.band_kind == 1) return 0.5 * (ax.p2 + ay.p2);
    return -2.0 * b.t * (ax.c1 + ay.c1) - 4.0 * b.tp * ax.c1 * ay.c1 - 2.0 * b.tpp * (ax.c2 + ay.c2);
}
// The first-zone axis values a CTA needs, staged once in shared memory
// (pts_per_zone <= 512 for the filling solve).
constexpr int MU_MAXZ = 512;
struct ZoneAxis {
    float c1[MU_MAXZ], c2[MU_MAXZ], p2[MU_MAXZ];
};
__device__ __forceinline__ void stage_zone_axis(const Geom &g, const AxisTab *__restrict__ axis, ZoneAxis &z)
{
    const int base = g.N / 2 - g.npz / 2;
    for (int i = threadIdx.x; i < g.npz; i += blockDim.x) {
        z.c1[i] = axis[base + i].c1f;
        z.c2[i] = axis[base + i].c2f;
        z.p2[i] = axis[base + i].p2f;
    }
    __syncthreads();
}
// FP32 band energy of first-zone point (i, j); t32 = (t, t', t'') in FP32.
__device__ __forceinline__ float band_e0f(int kind, const float *t32, const ZoneAxis &z, int i, int j)
{
    if (kind == 1) return 0.5f * (z.p2[i] + z.p2[j]);
    return -2.0f * t32[0] * (z.c1[i] + z.c1[j]) - 4.0f * t32[1] * z.c1[i] * z.c1[j]
           - 2.0f * t32[2] * (z.c2[i] + z.c2[j]);
}

// True in every thread of the CTA that finishes last; that CTA resets the
// counter for the next launch.  Partial sums written before the call are
// visible to it.
__device__ __forceinline__ bool last_cta(unsigned *counter)
{
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
        if (s_last) *counter = 0;   // no other CTA touches it again in this launch
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

__device__ __forceinline__ double mu_bracket_B(const Band &band)
{
    return (band.band_kind == 1) ? 9.869604401089358 : 4.0 * (fabs(band.t) + fabs(band.tp) + fabs(band.tpp));
}

// One multisection pass: candidates mu_c = lo + c (hi - lo)/(MU_SECT - 1).
__global__ void __launch_bounds__(MU_THREADS)
k_mu_sect(Geom g, Band band, const AxisTab *__restrict__ axis, double *acc, unsigned *counter, int pass)
{
    const int G = gridDim.x;
    const int npts = g.npz * g.npz;
    const double target = band.filling * 0.5 * (double)npts;  // sum of occupations
    double *res = acc;
    double *part = acc + MU_RES + (size_t)pass * G * MU_SECT;
    double lo, hi;
    if (pass == 0) {
        lo = -mu_bracket_B(band) - 3.0;
        hi = -lo;
    } else {
        if (res[3 * (pass - 1) + 2] != 0.0) return;   // not bracketed: nothing to refine
        lo = res[3 * (pass - 1) + 0];
        hi = res[3 * (pass - 1) + 1];
    }
    constexpr int NGRP = MU_THREADS / MU_SECT;
    __shared__ double s_tot[NGRP][MU_SECT];
    __shared__ int s_first;
    const int cand = threadIdx.x % MU_SECT, grp = threadIdx.x / MU_SECT;
    const int pg = blockIdx.x * NGRP + grp, npg = G * NGRP;
    const float gam = (float)band.gamma;
    const float inv_pi = 0.318309886183790672f;
    const float t32[3] = {(float)band.t, (float)band.tp, (float)band.tpp};
    const double h = (hi - lo) / (MU_SECT - 1);
    const float mu_c = (float)(lo + cand * h);
    const float inv_gam = 1.0f / gam;
    __shared__ ZoneAxis za;
    stage_zone_axis(g, axis, za);
    float sum = 0.f;
#pragma unroll 4
    for (int k = pg; k < npts; k += npg) {
        int i = k / g.npz, j = k % g.npz;
        sum += 0.5f - atanf((band_e0f(band.band_kind, t32, za, i, j) - mu_c) * inv_gam) * inv_pi;
    }
    s_tot[grp][cand] = sum;
    __syncthreads();
    if (threadIdx.x < MU_SECT) {
        double t = 0;
        for (int q = 0; q < NGRP; ++q) t += s_tot[q][threadIdx.x];
        part[(size_t)blockIdx.x * MU_SECT + threadIdx.x] = t;
    }
    if (!last_cta(counter)) return;
    // last CTA: totals per candidate in a fixed order, first one >= target
    if (threadIdx.x == 0) s_first = MU_SECT;
    double t = 0;
#pragma unroll 16
    for (int q = grp; q < G; q += NGRP) t += __ldcg(&part[(size_t)q * MU_SECT + cand]);
    __syncthreads();
    s_tot[grp][cand] = t;
    __syncthreads();
    if (threadIdx.x < MU_SECT) {
        double tt = 0;
        for (int q = 0; q < NGRP; ++q) tt += s_tot[q][threadIdx.x];
        if (tt >= target) atomicMin(&s_first, (int)threadIdx.x);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int i = s_first;
        double flag = 0.0;
        if (pass == 0 && (i == 0 || i == MU_SECT)) flag = 1.0;   // filling not bracketed
        if (i == 0) i = 1;
        if (i == MU_SECT) i = MU_SECT - 1;
        res[3 * pass + 0] = lo + (i - 1) * h;
        res[3 * pass + 1] = lo + i * h;
        res[3 * pass + 2] = flag;
    }
}

// One Newton step in FP64; the last step also publishes mu.
__global__ void __launch_bounds__(MU_THREADS)
k_mu_newton(Geom g, Band band, const AxisTab *__restrict__ axis, InstState *st, double *acc, unsigned *counter,
            int it, unsigned *status, double *mu_out)
{
    const int G = gridDim.x;
    const int npts = g.npz * g.npz;
    const int base = g.N / 2 - g.npz / 2;
    const double target = band.filling * 0.5 * (double)npts;
    double *res = acc;
    double *part = acc + MU_RES + (size_t)MU_FP32_PASSES * G * MU_SECT + (size_t)it * G * 2;
    if (res[2] != 0.0) {   // the filling was not bracketed
        if (it == MU_NEWTON - 1 && blockIdx.x == 0 && threadIdx.x == 0)
            atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
        return;
    }
    const double mu = (it == 0) ? 0.5 * (res[3 * (MU_FP32_PASSES - 1) + 0] + res[3 * (MU_FP32_PASSES - 1) + 1])
                                : res[10 + 2 * (it - 1)];
    const double gd = band.gamma, ipi = 0.31830988618379067154;
    constexpr int NW = MU_THREADS / 32;
    __shared__ double s_red[2][NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double f = 0.0, fp = 0.0;
    // points interleaved over the CTAs, so every SM's FP64 units share the work
    for (int k = threadIdx.x * G + blockIdx.x; k < npts; k += G * MU_THREADS) {
        int ix = base + k / g.npz, iy = base + k % g.npz;
        double xi = band_e0(band, axis[ix], axis[iy]) - mu;
        f += 0.5 - atan(xi / gd) * ipi;
        fp += gd * ipi / (xi * xi + gd * gd);
    }
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_down_sync(0xffffffffu, f, o);
        fp += __shfl_down_sync(0xffffffffu, fp, o);
    }
    if (lane == 0) { s_red[0][warp] = f; s_red[1][warp] = fp; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < NW; ++w) { a += s_red[0][w]; b += s_red[1][w]; }
        part[(size_t)blockIdx.x * 2 + 0] = a;
        part[(size_t)blockIdx.x * 2 + 1] = b;
    }
    if (!last_cta(counter)) return;
    double F = 0, Fp = 0;
    for (int q = threadIdx.x; q < G; q += MU_THREADS) {
        F += __ldcg(&part[(size_t)q * 2 + 0]);
        Fp += __ldcg(&part[(size_t)q * 2 + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        F += __shfl_down_sync(0xffffffffu, F, o);
        Fp += __shfl_down_sync(0xffffffffu, Fp, o);
    }
    __syncthreads();
    if (lane == 0) { s_red[0][warp] = F; s_red[1][warp] = Fp; }
    __syncthreads();
    if (threadIdx.x == 0) {
        F = 0;
        Fp = 0;
        for (int w = 0; w < NW; ++w) { F += s_red[0][w]; Fp += s_red[1][w]; }
        const double step = (F - target) / Fp;   // d/dmu of sum_k occ = sum_k Lorentzian
        res[10 + 2 * it] = mu - step;
        res[11 + 2 * it] = step;
        if (it == MU_NEWTON - 1) {
            st->mu = mu - step;
            st->last_step = fabs(step);
            if (mu_out) *mu_out = mu - step;
            // a last step below 1e-7 eV leaves an error of order 1e-12 eV
            if (!(fabs(step) < 1e-7)) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
        }
    }
}

// mu given by the caller.
__global__ void k_mu_given(double mu, InstState *st, double *mu_out)
{
    st->mu = mu;
    st->last_step = 0.0;
    if (mu_out) *mu_out = mu;
}

cudaError_t launch_twiddles(int len, float2 *tw32, double2 *tw64, cudaStream_t s)
{
    k_twiddles<<<(twiddle_entries() + 255) / 256, 256, 0, s>>>(len, tw32, tw64);
    return cudaGetLastError();
}

cudaError_t launch_tables(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                          cudaStream_t s)
{
    int n = g.N > g.n_eps ? g.N : g.n_eps;
    k_tables<<<(n + 127) / 128, 128, 0, s>>>(g, band, axis, eps32, eps64);
    return cudaGetLastError();
}

// CTAs of each chemical-potential launch: one per SM.
int mu_grid_size(int num_sms, int npts)
{
    (void)npts;
    return num_sms < 1 ? 1 : num_sms;   // one CTA per SM
}

cudaError_t launch_solve_mu(const Geom &g, const Band &band, const AxisTab *axis, InstState *st, double *acc,
                            unsigned *bar, unsigned *status, double *mu_out, int G, cudaStream_t s)
{
    if (!band.solve_mu) {
        k_mu_given<<<1, 1, 0, s>>>(band.mu, st, mu_out);
        return cudaGetLastError();
    }
    const int Gs = G < MU_SECT_CTAS ? G : MU_SECT_CTAS;
    for (int pass = 0; pass < MU_FP32_PASSES; ++pass)
        k_mu_sect<<<Gs, MU_THREADS, 0, s>>>(g, band, axis, acc, bar, pass);
    for (int it = 0; it < MU_NEWTON; ++it)
        k_mu_newton<<<G, MU_THREADS, 0, s>>>(g, band, axis, st, acc, bar, it, status, mu_out);
    return cudaGetLastError();
}

}  // namespace lh
