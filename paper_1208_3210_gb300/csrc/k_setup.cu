// Set-up kernels: twiddle tables, per-axis momentum tables, the energy grid,
// and the rigid-band chemical potential (Sec. 3: the Fermi level is shifted to
// hold the requested electron count).
#include <math.h>

#include "kernels.cuh"

namespace lh {

// exp(-2 pi i n / len) for n in [0, len), evaluated in FP64 with sincospi.
__global__ void k_twiddles(int len, float2 *tw32, double2 *tw64)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= len) return;
    double s, c;
    sincospi(-2.0 * (double)n / (double)len, &s, &c);
    tw32[n] = make_float2((float)c, (float)s);
    tw64[n] = make_double2(c, s);
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
// level).  n is strictly increasing.  One cooperative launch of G CTAs (one
// per SM):
//   MU_FP32_PASSES passes of MU_SECT-point multisection in FP32 shrink the
//   bracket [-B-3, B+3] eV (B bounds |e0|) by (MU_SECT-1)^passes; every thread
//   owns one candidate and a share of the points;
//   MU_NEWTON Newton steps in FP64 from the bracket midpoint reach FP64
//   precision.
// After each pass the last CTA to arrive at the grid barrier adds the per-CTA
// partial sums in a fixed order, publishes the new bracket (or mu) and then
// releases the others, so the result does not depend on scheduling.
constexpr int MU_SECT = 128;
constexpr int MU_THREADS = 256;
constexpr int MU_FP32_PASSES = 2;
constexpr int MU_NEWTON = 3;
constexpr int MU_RES = 16;   // result slots at the start of acc
constexpr int MU_BAR_GEN = 32, MU_BAR_FAIL = 64, MU_BAR_WORDS = 96;   // barrier word offsets

// Layout of acc: [MU_RES] results, then [MU_FP32_PASSES][G][MU_SECT], then [MU_NEWTON][G][2] doubles.
size_t mu_acc_doubles(int G) { return MU_RES + (size_t)G * (MU_FP32_PASSES * MU_SECT + MU_NEWTON * 2); }
size_t mu_barrier_words() { return MU_BAR_WORDS; }

__device__ __forceinline__ double band_e0(const Band &b, const AxisTab &ax, const AxisTab &ay)
{
    if (b.band_kind == 1) return 0.5 * (ax.p2 + ay.p2);
    return -2.0 * b.t * (ax.c1 + ay.c1) - 4.0 * b.tp * ax.c1 * ay.c1 - 2.0 * b.tpp * (ax.c2 + ay.c2);
}
// FP32 band energy from the FP32 table copies; t32 = (t, t', t'') in FP32.
__device__ __forceinline__ float band_e0f(int kind, const float *t32, const AxisTab *__restrict__ axis, int ix,
                                          int iy)
{
    const float4 ax = *reinterpret_cast<const float4 *>(&axis[ix].c1f);
    const float4 ay = *reinterpret_cast<const float4 *>(&axis[iy].c1f);
    if (kind == 1) return 0.5f * (ax.z + ay.z);
    return -2.0f * t32[0] * (ax.x + ay.x) - 4.0f * t32[1] * ax.x * ay.x - 2.0f * t32[2] * (ax.y + ay.y);
}

// Grid barrier whose last arriving CTA first runs `on_last` (with all its
// threads) and then releases the others.  bar[0] counts arrivals, bar[32] is
// the generation, bar[64] a failure flag (separate 128-byte lines, so that
// the waiters' polling does not slow the arrivals' atomics); all are zeroed
// before the launch.  A waiting CTA records the generation before it arrives; the
// release (generation + 1) cannot happen before its arrival.  The wait is
// bounded (about 1 s): on timeout the failure flag and the plan's status word
// are set, and this and every later barrier of the launch return false.
template <typename F>
__device__ bool grid_sync_reduce(unsigned *bar, unsigned *status, F &&on_last)
{
    __shared__ int s_last, s_fail;
    __shared__ unsigned s_gen;
    volatile unsigned *vgen = bar + MU_BAR_GEN;
    volatile unsigned *vfail = bar + MU_BAR_FAIL;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = *vfail != 0;
        s_last = 0;
        if (!s_fail) {
            s_gen = *vgen;
            __threadfence();
            s_last = atomicAdd(bar, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (s_fail) return false;
    if (s_last) {
        __threadfence();
        on_last();
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + MU_BAR_GEN, 1u);
        }
    } else if (threadIdx.x == 0) {
        long long t0 = clock64();
        while (*vgen == s_gen) {
            if (*vfail != 0) { s_fail = 1; break; }
            __nanosleep(20);
            if (clock64() - t0 > 2000000000LL) {
                atomicExch(bar + MU_BAR_FAIL, 1u);
                atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ETIMEOUT);
                s_fail = 1;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_fail == 0;
}

__global__ void __launch_bounds__(MU_THREADS)
k_solve_mu(Geom g, Band band, const AxisTab *__restrict__ axis, InstState *st, double *acc,
           unsigned *bar, unsigned *status, double *mu_out)
{
    if (!band.solve_mu) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->mu = band.mu;
            st->last_step = 0.0;
            if (mu_out) *mu_out = band.mu;
        }
        return;
    }
    const int G = gridDim.x;
    const int npts = g.npz * g.npz;
    const int base = g.N / 2 - g.npz / 2;       // first-zone indices on the grid
    const double target = band.filling * 0.5 * (double)npts;  // sum of occupations
    const double B = (band.band_kind == 1) ? 9.869604401089358
                     : 4.0 * (fabs(band.t) + fabs(band.tp) + fabs(band.tpp));
    volatile double *res = acc;                 // result slots
    double *part32 = acc + MU_RES;
    double *part64 = part32 + (size_t)MU_FP32_PASSES * G * MU_SECT;
    constexpr int NGRP = MU_THREADS / MU_SECT;
    constexpr int NW = MU_THREADS / 32;
    __shared__ float s_part[NGRP][MU_SECT];
    __shared__ double s_red2[2][NW];
    __shared__ int s_first;

    double lo = -B - 3.0, hi = B + 3.0;
    const int cand = threadIdx.x % MU_SECT, grp = threadIdx.x / MU_SECT;
    const int pg = blockIdx.x * NGRP + grp, npg = G * NGRP;
    const float gam = (float)band.gamma;
    const float inv_pi = 0.318309886183790672f;
    const float t32[3] = {(float)band.t, (float)band.tp, (float)band.tpp};
    __shared__ double s_tot[NGRP][MU_SECT];
    __shared__ double s_nw[2][NW];

    // --- FP32 multisection ---------------------------------------------------
    for (int pass = 0; pass < MU_FP32_PASSES; ++pass) {
        const double h = (hi - lo) / (MU_SECT - 1);
        const float mu_c = (float)(lo + cand * h);
        float sum = 0.f;
#pragma unroll 4
        for (int k = pg; k < npts; k += npg) {
            int ix = base + k / g.npz, iy = base + k % g.npz;
            sum += 0.5f - atanf((band_e0f(band.band_kind, t32, axis, ix, iy) - mu_c) / gam) * inv_pi;
        }
        s_part[grp][cand] = sum;
        __syncthreads();
        if (threadIdx.x < MU_SECT) {
            double t = 0;
            for (int q = 0; q < NGRP; ++q) t += s_part[q][threadIdx.x];
            part32[((size_t)pass * G + blockIdx.x) * MU_SECT + threadIdx.x] = t;
        }
        bool ok = grid_sync_reduce(bar, status, [&] {
            if (threadIdx.x == 0) s_first = MU_SECT;
            // every thread adds a fixed subset of the CTA partials of its
            // candidate (loads unrolled so they overlap), then two halves
            double t = 0;
#pragma unroll 16
            for (int q = grp; q < G; q += NGRP) t += __ldcg(&part32[((size_t)pass * G + q) * MU_SECT + cand]);
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
        });
        if (!ok) return;
        if (res[3 * pass + 2] != 0.0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
            return;
        }
        lo = res[3 * pass + 0];
        hi = res[3 * pass + 1];
    }

    // --- FP64 Newton ---------------------------------------------------------
    double mu = 0.5 * (lo + hi), step = 0.0;
    const double gd = band.gamma, ipi = 0.31830988618379067154;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = 0; it < MU_NEWTON; ++it) {
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
        if (lane == 0) { s_red2[0][warp] = f; s_red2[1][warp] = fp; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int w = 0; w < NW; ++w) { a += s_red2[0][w]; b += s_red2[1][w]; }
            part64[((size_t)it * G + blockIdx.x) * 2 + 0] = a;
            part64[((size_t)it * G + blockIdx.x) * 2 + 1] = b;
        }
        bool ok = grid_sync_reduce(bar, status, [&] {
            // a fixed reduction tree over the CTA partials
            double F = 0, Fp = 0;
            for (int q = threadIdx.x; q < G; q += MU_THREADS) {
                F += __ldcg(&part64[((size_t)it * G + q) * 2 + 0]);
                Fp += __ldcg(&part64[((size_t)it * G + q) * 2 + 1]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                F += __shfl_down_sync(0xffffffffu, F, o);
                Fp += __shfl_down_sync(0xffffffffu, Fp, o);
            }
            if (lane == 0) { s_nw[0][warp] = F; s_nw[1][warp] = Fp; }
            __syncthreads();
            if (threadIdx.x == 0) {
                F = 0;
                Fp = 0;
                for (int w = 0; w < NW; ++w) { F += s_nw[0][w]; Fp += s_nw[1][w]; }
                double stp = (F - target) / Fp;     // d/dmu of sum_k occ = sum_k Lorentzian
                res[8 + 2 * it] = mu - stp;
                res[9 + 2 * it] = stp;
            }
        });
        if (!ok) return;
        mu = res[8 + 2 * it];
        step = res[9 + 2 * it];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->mu = mu;
        st->last_step = fabs(step);
        if (mu_out) *mu_out = mu;
        if (!(fabs(step) < 1e-9)) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
    }
}

cudaError_t launch_twiddles(int len, float2 *tw32, double2 *tw64, cudaStream_t s)
{
    k_twiddles<<<(len + 255) / 256, 256, 0, s>>>(len, tw32, tw64);
    return cudaGetLastError();
}

cudaError_t launch_tables(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                          cudaStream_t s)
{
    int n = g.N > g.n_eps ? g.N : g.n_eps;
    k_tables<<<(n + 127) / 128, 128, 0, s>>>(g, band, axis, eps32, eps64);
    return cudaGetLastError();
}

// CTAs of the cooperative chemical-potential launch: at most one per SM.
int mu_grid_size(int num_sms, int npts)
{
    (void)npts;
    return num_sms < 1 ? 1 : num_sms;   // one CTA per SM
}

cudaError_t launch_solve_mu(const Geom &g, const Band &band, const AxisTab *axis, InstState *st, double *acc,
                            unsigned *bar, unsigned *status, double *mu_out, int G, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, MU_BAR_WORDS * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(band.solve_mu ? G : 1);
    cfg.blockDim = dim3(MU_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_mu, g, band, axis, st, acc, bar, status, mu_out);
}

}  // namespace lh
