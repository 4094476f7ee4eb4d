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
// level).  n is strictly increasing.  One cooperative launch of G CTAs:
//   3 passes of 64-point multisection in FP32 shrink the bracket
//   [-B-3, B+3] eV (B bounds |e0|) by 63^3;
//   3 Newton steps in FP64 from the bracket midpoint reach FP64 precision.
// Per-CTA partial sums go to `acc`; after a grid barrier every CTA adds them
// in the same order, so all CTAs take identical decisions and the result does
// not depend on scheduling.
constexpr int MU_SECT = 64;
constexpr int MU_THREADS = 256;
constexpr int MU_FP32_PASSES = 3;
constexpr int MU_NEWTON = 3;
constexpr int MU_MAXP = 8;   // first-zone points held per thread

// Layout of acc: [MU_FP32_PASSES][G][MU_SECT] then [MU_NEWTON][G][2] doubles.
size_t mu_acc_doubles(int G) { return (size_t)G * (MU_FP32_PASSES * MU_SECT + MU_NEWTON * 2); }

__device__ __forceinline__ double band_e0(const Band &b, const AxisTab &ax, const AxisTab &ay)
{
    if (b.band_kind == 1) return 0.5 * (ax.p2 + ay.p2);
    return -2.0 * b.t * (ax.c1 + ay.c1) - 4.0 * b.tp * ax.c1 * ay.c1 - 2.0 * b.tpp * (ax.c2 + ay.c2);
}

// Grid-wide barrier with a bounded wait (about 1 s).  bar[0] counts arrivals,
// bar[1] is the generation, bar[2] a failure flag for this launch (all three
// zeroed before the launch).  On timeout the flag and the plan's status word
// are set, and every wait and later barrier of the launch returns false.
__device__ bool grid_sync(unsigned *bar, unsigned *status)
{
    __syncthreads();
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile unsigned *vfail = bar + 2;
        s_fail = *vfail != 0;
        if (!s_fail) {
            unsigned gen = *vgen;
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                long long t0 = clock64();
                while (*vgen == gen) {
                    if (*vfail != 0) { s_fail = 1; break; }
                    if (clock64() - t0 > 2000000000LL) {
                        atomicExch(bar + 2, 1u);
                        atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ETIMEOUT);
                        s_fail = 1;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
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
    double lo = -B - 3.0, hi = B + 3.0;
    constexpr int NW = MU_THREADS / 32;
    __shared__ float s_sect[NW][MU_SECT];
    __shared__ double s_red2[2][NW];
    __shared__ int s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // this thread's first-zone points (usually at most one): band energies once, in FP64
    constexpr int MAXP = MU_MAXP;
    double e0[MAXP];
    int np = 0;
    for (int k = blockIdx.x * MU_THREADS + threadIdx.x; k < npts && np < MAXP; k += G * MU_THREADS) {
        int ix = base + k / g.npz, iy = base + k % g.npz;
        e0[np++] = band_e0(band, axis[ix], axis[iy]);
    }
    // (the launch uses G >= npts / (MU_MAXP * MU_THREADS), so every point is covered)

    // --- FP32 multisection ---------------------------------------------------
    const float gam = (float)band.gamma;
    const float inv_pi = 0.318309886183790672f;
    for (int pass = 0; pass < MU_FP32_PASSES; ++pass) {
        const double h = (hi - lo) / (MU_SECT - 1);
        for (int c = 0; c < MU_SECT; ++c) {
            float mu_c = (float)(lo + c * h), sum = 0.f;
            for (int q = 0; q < np; ++q) sum += 0.5f - atanf(((float)e0[q] - mu_c) / gam) * inv_pi;
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (lane == 0) s_sect[warp][c] = sum;
        }
        __syncthreads();
        if (threadIdx.x < MU_SECT) {
            double t = 0;
            for (int w = 0; w < NW; ++w) t += s_sect[w][threadIdx.x];
            acc[((size_t)pass * G + blockIdx.x) * MU_SECT + threadIdx.x] = t;
        }
        if (threadIdx.x == 0) s_first = MU_SECT;
        if (!grid_sync(bar, status)) return;
        // every CTA: total occupation at each candidate, first candidate >= target
        if (threadIdx.x < MU_SECT) {
            double t = 0;
            for (int q = 0; q < G; ++q) t += __ldcg(&acc[((size_t)pass * G + q) * MU_SECT + threadIdx.x]);
            if (t >= target) atomicMin(&s_first, (int)threadIdx.x);
        }
        __syncthreads();
        int i = s_first;
        if (pass == 0 && (i == 0 || i == MU_SECT)) {
            // the filling is not bracketed by [-B-3, B+3] eV
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
            return;
        }
        if (i == 0) i = 1;
        if (i == MU_SECT) i = MU_SECT - 1;
        double nlo = lo + (i - 1) * h, nhi = lo + i * h;
        lo = nlo;
        hi = nhi;
        __syncthreads();
    }

    // --- FP64 Newton ---------------------------------------------------------
    double mu = 0.5 * (lo + hi), step = 0.0;
    const double gd = band.gamma, ipi = 0.31830988618379067154;
    for (int it = 0; it < MU_NEWTON; ++it) {
        double f = 0.0, fp = 0.0;
        for (int q = 0; q < np; ++q) {
            double xi = e0[q] - mu;
            f += 0.5 - atan(xi / gd) * ipi;
            fp += gd * ipi / (xi * xi + gd * gd);
        }
        for (int o = 16; o > 0; o >>= 1) {
            f += __shfl_down_sync(0xffffffffu, f, o);
            fp += __shfl_down_sync(0xffffffffu, fp, o);
        }
        if (lane == 0) { s_red2[0][warp] = f; s_red2[1][warp] = fp; }
        __syncthreads();
        double *slot = acc + (size_t)G * MU_FP32_PASSES * MU_SECT + ((size_t)it * G + blockIdx.x) * 2;
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int w = 0; w < NW; ++w) { a += s_red2[0][w]; b += s_red2[1][w]; }
            slot[0] = a;
            slot[1] = b;
        }
        if (!grid_sync(bar, status)) return;
        double F = 0, Fp = 0;
        const double *all = acc + (size_t)G * MU_FP32_PASSES * MU_SECT + (size_t)it * G * 2;
        for (int q = 0; q < G; ++q) { F += __ldcg(&all[2 * q]); Fp += __ldcg(&all[2 * q + 1]); }
        step = (F - target) / Fp;          // d/dmu of sum_k occ = sum_k Lorentzian
        mu -= step;
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
    // one point per thread where the SMs allow, at most MU_MAXP
    int want = (npts + MU_THREADS - 1) / MU_THREADS;
    int need = (npts + MU_MAXP * MU_THREADS - 1) / (MU_MAXP * MU_THREADS);
    if (want > num_sms) want = num_sms;
    if (want < need) want = need;
    return want < 1 ? 1 : want;
}

cudaError_t launch_solve_mu(const Geom &g, const Band &band, const AxisTab *axis, InstState *st, double *acc,
                            unsigned *bar, unsigned *status, double *mu_out, int G, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), s);
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
