// Set-up kernels: twiddle tables, per-axis momentum tables, the energy grid,
// and the rigid-band chemical potential (Sec. 3: the Fermi level is shifted to
// hold the requested electron count).
#include <math.h>
#include <stddef.h>

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

// ---------------------------------------------------------------------------
// Set-up and chemical potential.
//
// Tables: per-axis values at p_i = (i - N/2) 2 pi / npz and the energy grid
// e_j = -e_max + (j + 1/2) de, all in FP64.  The FP32 path stores e_j as an
// unevaluated pair hi + lo so that e_j - xi_p keeps full precision near the
// Lorentzian peak.
//
// Chemical potential (Sec. 3: the Fermi level is placed to hold the requested
// electron count).  n(mu) = (2/npz^2) sum_k occ(e0_k - mu) with the Lorentzian
// occupation occ(xi) = 1/2 - atan(xi/gamma)/pi of Eq. 5 below the Fermi level,
// summed over the first-zone grid p = 2 pi r / npz, r in [-npz/2, npz/2).
// n is strictly increasing in mu.  Both band kinds depend on p_x and p_y only
// through even functions (cos p, cos 2p, p^2) and are symmetric under
// p_x <-> p_y, so the sum runs over the classes m = |r| in [0, npz/2] with
// weights w(0) = w(npz/2) = 1, w(m) = 2 otherwise, and over pairs
// m_x <= m_y (twice for m_x < m_y): (npz/2 + 1)(npz/2 + 2)/2 terms instead of
// npz^2 (561 instead of 4096 at npz = 64).
//
// Launches (no CTA ever waits for another; zones of at most 98 points per
// axis instead solve in one CTA of k_setup by a bracketed Newton iteration,
// see mu_solve_one_cta):
//   k_setup     multisection pass 0 over [-B-3, B+3] eV on G CTAs, and the
//               tables on further CTAs of the same launch (their FP64 cospi and
//               exp chains run beside the multisection, not before it)
//   k_mu_sect   further multisection passes (one, or two when gamma < 0.02 eV)
//   k_mu_halley one FP64 Halley step from the midpoint of the last bracket
// A multisection pass samples NC = 8 G candidates (G CTAs, eight candidates
// each) in FP32.  Every CTA sums the whole zone for its own candidates (the
// pairs' band energies and weights staged in shared memory, lane % 8 picks
// the candidate), so no cross-CTA reduction is needed; it records the first
// of its candidates whose total reaches the target, and the next launch's CTAs
// each take the minimum over the G records.  Two passes shrink the bracket by
// (NC - 1)^2 (to about 1e-5 eV), three to below FP32 resolution; FP32
// rounding moves the sampled n(mu) by the equivalent of some 1e-7 eV at most.
// The Halley step (cubic convergence; its error is of order (d/gamma)^2 d for
// a distance d to the root) then lands at FP64 precision.  Its per-CTA sums of
// n (FP64), gamma n' and gamma^2 n'' (FP32 terms: they only scale the step)
// are stored, and the last CTA to finish (an atomic counter) adds them in a
// fixed tree order and forms the step.
//
// On this GPU a dependent FP64 operation takes about 60 cycles, an FP64
// division about 450 and an FP64 atan about 1900, so the few FP64 steps on
// the critical path use constants computed on the host.
constexpr int MU_THREADS = 512;      // multisection CTAs
constexpr int MU_NT_THREADS = 128;   // Halley CTAs (at most; one warp when the pairs fit)
constexpr int MU_TAB_THREADS = 32;   // table entries per table CTA
constexpr int MU_NCPT = 8;           // candidates per CTA
constexpr int MU_MAX_PASSES = 3;
constexpr int MU_RES = 16;           // doubles of results at the start of acc
constexpr int MU_MAXC = 2049;        // classes for npz <= 4096
constexpr int MU_CHUNK = 2048;       // pairs staged per round
constexpr float MU_SECT_SCALE = 4294967296.0f;   // 2^32

// Layout of acc: res[3 p + 0, 1, 2] = (lo, hi, not-bracketed flag) of the
// interval pass p sampled (p = passes: that of the Halley step); then
// [G][4] doubles of per-CTA Halley sums; then [MU_MAX_PASSES][G] int first
// crossings (index in the CTA's candidates, MU_NCPT = none).
size_t mu_acc_doubles(int G) { return MU_RES + 4 * (size_t)G + ((size_t)MU_MAX_PASSES * G + 1) / 2; }
size_t mu_barrier_words() { return 32; }   // the arrival counter (one 128-byte line)

// CTAs of each chemical-potential launch: one per SM.
int mu_grid_size(int num_sms, int npts)
{
    (void)npts;
    return num_sms < 1 ? 1 : num_sms;
}

// Host-computed constants of one solve.
struct MuConst {
    double inv_nc1;      // 1 / (NC - 1)
    double inv_gam;      // 1 / gamma
    double target;       // filling npz^2 / 2 (sum of occupations)
    long long target32;  // the same in 2^-32 fixed point
    double B;            // bracket half-width - 3 eV
    int NC, passes;
    int single;          // the whole solve in one CTA of the set-up launch
};

// Zones small enough for the one-CTA solve: every pass and the Halley step in
// one CTA of the set-up launch, beside the table CTAs, and no further launch
// (npz <= 98).  The multi-CTA passes cost two more launches and their
// grid-wide exchanges, which dominate at these sizes.
constexpr int MU_SINGLE_MAX_PAIRS = 1300;
constexpr int MU_SINGLE_MAX_H = 49;  // (h + 1)(h + 2) / 2 <= 1300
__host__ __device__ inline bool mu_single(const Geom &g)
{
    const int h = g.npz / 2;
    return (h + 1) * (h + 2) / 2 <= MU_SINGLE_MAX_PAIRS;
}

__device__ __forceinline__ int *mu_cross(double *acc, int G, int pass)
{
    return (int *)(acc + MU_RES + 4 * (size_t)G) + (size_t)pass * G;
}

__device__ __forceinline__ double band_e0(const Band &b, const AxisTab &ax, const AxisTab &ay)
{
    if (b.band_kind == 1) return 0.5 * (ax.p2 + ay.p2);
    return -2.0 * b.t * (ax.c1 + ay.c1) - 4.0 * b.tp * ax.c1 * ay.c1 - 2.0 * b.tpp * (ax.c2 + ay.c2);
}

// The same from FP64 class values (cos p, cos 2p, p^2 of the two axes).
__device__ __forceinline__ double band_e0_cls(const Band &b, double c1a, double c1b, double c2a, double c2b,
                                              double p2a, double p2b)
{
    if (b.band_kind == 1) return 0.5 * (p2a + p2b);
    return -2.0 * b.t * (c1a + c1b) - 4.0 * b.tp * c1a * c1b - 2.0 * b.tpp * (c2a + c2b);
}

// Pair index k in [0, (h+1)(h+2)/2) -> classes (a, b), 0 <= a <= b <= h, row
// a holding b = a..h; row a starts at a (2h + 3 - a) / 2.
__device__ __forceinline__ void tri_pair(int k, int h, int &a, int &b)
{
    const float c = 2.0f * (float)h + 3.0f;
    int x = (int)((c - sqrtf(c * c - 8.0f * (float)k)) * 0.5f);
    x = max(0, min(x, h));
    while (x < h && (x + 1) * (2 * h + 2 - x) / 2 <= k) ++x;
    while (x > 0 && x * (2 * h + 3 - x) / 2 > k) --x;
    a = x;
    b = x + (k - x * (2 * h + 3 - x) / 2);
}
// Multiplicity of pair (a, b): w(a) w(b), twice when a != b.
__device__ __forceinline__ int pair_weight(int a, int b, int h)
{
    int wa = (a == 0 || a == h) ? 1 : 2, wb = (b == 0 || b == h) ? 1 : 2;
    return wa * wb * (a == b ? 1 : 2);
}

struct MuBracket {
    int wmin[MU_THREADS / 32];
    double lo, hi, step;
    int flag;
    int wmin_done;   // one-CTA solve: the search has converged
};
struct MuShared {
    float c1[MU_MAXC], c2[MU_MAXC], p2[MU_MAXC];   // class values in FP32
    float2 ew[MU_CHUNK];                           // (band energy, weight) of staged pairs
    long long red[MU_THREADS / 32][MU_NCPT];
    float mu_c[MU_NCPT];
    MuBracket br;
};

// Class values at p = 2 pi m / npz, FP32 (the multisection only needs them to
// about 1e-7).
__device__ __forceinline__ void stage_classes(const Geom &g, MuShared &sh)
{
    const int h = g.npz / 2;
    const float inv = 2.0f / (float)g.npz;
    for (int m = threadIdx.x; m <= h; m += blockDim.x) {
        float u = (float)m * inv;                  // p / pi
        float p = u * 3.14159265358979f;
        sh.c1[m] = cospif(u);
        sh.c2[m] = cospif(2.0f * u);
        sh.p2[m] = p * p;
    }
}

// Bracket from the first-crossing records of pass p: sh.lo, sh.hi, sh.flag
// (read after the next __syncthreads).  Every thread takes part.
__device__ __forceinline__ void bracket_from(const double *res, const int *cross_p, const MuConst &mc, int p,
                                             MuBracket &sh)
{
    const int G = mc.NC / MU_NCPT;
    double plo = 0.0, phi = 0.0, pflag = 0.0;
    if (threadIdx.x == 0) {   // issued together with the records' loads
        plo = __ldcg(res + 3 * p);
        phi = __ldcg(res + 3 * p + 1);
        pflag = __ldcg(res + 3 * p + 2);
    }
    int first = mc.NC;
    for (int j = threadIdx.x; j < G; j += blockDim.x) {
        int q = __ldcg(cross_p + j);
        if (q < MU_NCPT) first = min(first, MU_NCPT * j + q);
    }
    first = (int)__reduce_min_sync(0xffffffffu, (unsigned)first);
    if ((threadIdx.x & 31) == 0) sh.wmin[threadIdx.x >> 5] = first;
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = mc.NC;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c = min(c, sh.wmin[w]);
        sh.flag = pflag != 0.0 || (p == 0 && (c == 0 || c == mc.NC));
        c = max(1, min(c, mc.NC - 1));
        const double step = (phi - plo) * mc.inv_nc1;
        sh.lo = plo + (double)(c - 1) * step;
        sh.hi = sh.lo + step;
    }
}

// One multisection pass over [sh.br.lo, sh.br.hi] (set by thread 0 before the
// call): this CTA's candidates; records the first one whose total reaches
// the target in cross[blockIdx.x].
// Band energies and weights of pairs [base, base + n) into sh.ew (FP32).
__device__ __forceinline__ void stage_pairs(const Geom &g, const Band &band, MuShared &sh, int base, int n)
{
    const int h = g.npz / 2;
    const float t = (float)band.t, tp = (float)band.tp, tpp = (float)band.tpp;
    const bool free_e = band.band_kind == 1;
    for (int k = threadIdx.x; k < n; k += MU_THREADS) {
        int a, b;
        tri_pair(base + k, h, a, b);
        const float e = free_e ? 0.5f * (sh.p2[a] + sh.p2[b])
                               : -2.0f * t * (sh.c1[a] + sh.c1[b]) - 4.0f * tp * sh.c1[a] * sh.c1[b]
                                     - 2.0f * tpp * (sh.c2[a] + sh.c2[b]);
        sh.ew[k] = make_float2(e, (float)pair_weight(a, b, h));
    }
}

// prestaged: the first chunk of pairs is already in sh.ew (staged before the
// bracket was known; the classes must then have been staged and synchronised)
__device__ __forceinline__ void sect_pass(const Geom &g, const Band &band, const MuConst &mc, MuShared &sh,
                                          int *cross, bool prestaged = false)
{
    const int h = g.npz / 2;
    const int npairs = (h + 1) * (h + 2) / 2;
    const int c0 = MU_NCPT * blockIdx.x;
    if (threadIdx.x == 0) sh.br.step = (sh.br.hi - sh.br.lo) * mc.inv_nc1;
    __syncthreads();
    if (threadIdx.x < MU_NCPT) sh.mu_c[threadIdx.x] = (float)(sh.br.lo + (double)(c0 + (int)threadIdx.x) * sh.br.step);
    const float inv_gam = (float)mc.inv_gam, inv_pi = 0.318309886183790672f;
    const int q = threadIdx.x % MU_NCPT;        // this thread's candidate
    constexpr int LANES = MU_THREADS / MU_NCPT;  // threads per candidate
    long long acc = 0;
    for (int base = 0; base < npairs; base += MU_CHUNK) {
        const int n = min(MU_CHUNK, npairs - base);
        __syncthreads();   // previous chunk consumed; mu_c written
        if (!(prestaged && base == 0)) stage_pairs(g, band, sh, base, n);
        __syncthreads();
        const float mu = sh.mu_c[q];
        float s[4] = {0.f, 0.f, 0.f, 0.f};   // four chains; at most MU_CHUNK / LANES terms of at most 8
        int k = threadIdx.x / MU_NCPT;
        for (; k + 3 * LANES < n; k += 4 * LANES) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 ew = sh.ew[k + u * LANES];
                s[u] += ew.y * (0.5f - atanf((ew.x - mu) * inv_gam) * inv_pi);
            }
        }
        for (; k < n; k += LANES) {
            const float2 ew = sh.ew[k];
            s[0] += ew.y * (0.5f - atanf((ew.x - mu) * inv_gam) * inv_pi);
        }
        acc += __float2ll_rn(((s[0] + s[1]) + (s[2] + s[3])) * MU_SECT_SCALE);
    }
    // lanes l, l ^ 8, l ^ 16, l ^ 24 share a candidate
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < MU_NCPT) sh.red[warp][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long tsum = 0;
        if (lane < MU_NCPT)
            for (int w = 0; w < MU_THREADS / 32; ++w) tsum += sh.red[w][lane];
        unsigned hit = __ballot_sync(0xffffffffu, lane < MU_NCPT && tsum >= mc.target32);
        if (lane == 0) cross[blockIdx.x] = hit ? __ffs(hit) - 1 : MU_NCPT;
    }
    (void)c0;
}

// One-CTA solve (mu_single): a bracketed Newton iteration in FP32 (each step
// sums n and dn/dmu over the pairs, one or two per thread, in a fixed order;
// a step that leaves the bracket, or a flat n, falls back to bisection) from
// the full bracket until the step is below 1e-6 eV, then the FP64 Halley step
// of k_mu_halley from there.  n is increasing, so the bracket always holds the
// root; the first evaluation checks that both ends straddle the filling.
constexpr int MU_NEWTON_MAX = 64;    // bisection alone reaches 1e-6 eV in 24 steps
__device__ void mu_solve_one_cta(const Geom &g, const Band &band, const MuConst &mc, MuShared &sh, InstState *st,
                                 unsigned *status, double *mu_out)
{
    constexpr int NW = MU_THREADS / 32;
    // 8-byte scratch lives in sh.c1 (offset 0 of MuShared, so 8-byte aligned;
    // sh.c2 and sh.p2 start at 4 mod 8): the per-warp sums of the search,
    // then 3 (h + 1) class values and [NW][3] Halley sums
    static_assert(offsetof(MuShared, c1) == 0 && alignof(MuShared) >= 8, "sh.c1 must be 8-byte aligned");
    static_assert((3 * (MU_SINGLE_MAX_H + 1) + 3 * NW) * sizeof(double) <= sizeof(sh.c1) &&
                      2 * NW * sizeof(float) <= sizeof(sh.c1),
                  "scratch fits in the class table");
    const int h = g.npz / 2, npairs = (h + 1) * (h + 2) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    stage_pairs(g, band, sh, 0, npairs);                        // npairs <= MU_CHUNK
    if (threadIdx.x == 0) {
        sh.br.lo = -mc.B - 3.0;
        sh.br.hi = mc.B + 3.0;
        sh.br.step = 0.0;                                       // the current estimate
        sh.br.flag = 0;
    }
    __syncthreads();
    float *red = reinterpret_cast<float *>(sh.c1);             // [NW][2]
    const float inv_gam = (float)mc.inv_gam, inv_pi = 0.318309886183790672f;
    const float target = (float)mc.target;
    // it = 0: n at both ends of the bracket; it >= 1: n and dn/dmu at the estimate
    for (int it = 0; it < MU_NEWTON_MAX; ++it) {
        const float m0 = (float)(it == 0 ? sh.br.lo : sh.br.step), m1 = (float)sh.br.hi;
        float n0 = 0.f, n1 = 0.f;   // it = 0: n(lo), n(hi); else n(mu), gamma dn/dmu
        for (int k = threadIdx.x; k < npairs; k += MU_THREADS) {
            const float2 ew = sh.ew[k];
            const float x = (ew.x - m0) * inv_gam;
            n0 += ew.y * (0.5f - atanf(x) * inv_pi);
            if (it == 0) n1 += ew.y * (0.5f - atanf((ew.x - m1) * inv_gam) * inv_pi);
            else n1 += ew.y * (inv_pi / (1.0f + x * x));
        }
        for (int o = 16; o > 0; o >>= 1) {
            n0 += __shfl_down_sync(0xffffffffu, n0, o);
            n1 += __shfl_down_sync(0xffffffffu, n1, o);
        }
        if (lane == 0) { red[2 * warp] = n0; red[2 * warp + 1] = n1; }
        __syncthreads();
        int done = 0;
        if (threadIdx.x == 0) {
            float N0 = 0.f, N1 = 0.f;
            for (int w = 0; w < NW; ++w) { N0 += red[2 * w]; N1 += red[2 * w + 1]; }
            if (it == 0) {
                if (!(N0 < target && N1 >= target)) { sh.br.flag = 1; done = 1; }   // not bracketed
                sh.br.step = 0.5 * (sh.br.lo + sh.br.hi);
            } else {
                // FP32 step (an FP64 division costs some 450 cycles on this critical path)
                const double mu = sh.br.step;
                const float F = N0 - target, slope = N1 * inv_gam;   // n - target, dn/dmu
                if (F < 0.f) sh.br.lo = mu; else sh.br.hi = mu;
                double nxt = slope > 0.f ? mu - (double)(F / slope) : sh.br.lo - 1.0;
                if (!(nxt > sh.br.lo && nxt < sh.br.hi)) nxt = 0.5 * (sh.br.lo + sh.br.hi);
                done = fabs(nxt - mu) < 1e-6 || sh.br.hi - sh.br.lo < 1e-6;
                sh.br.step = nxt;
            }
            sh.br.wmin_done = done;
        }
        __syncthreads();
        if (sh.br.wmin_done) break;
    }
    const double mu = sh.br.step;
    if (sh.br.flag) {   // the filling was not bracketed
        if (threadIdx.x == 0) {
            atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
            set_mu(st, mu);
            st->last_step = INFINITY;
            if (mu_out) *mu_out = mu;
        }
        return;
    }
    // FP64 class values, the same expressions as the axis tables at p_i = -2 pi m / npz
    // (in sh.c1, the one 8-byte aligned scratch of MuShared; the search sums are consumed)
    double *d1 = reinterpret_cast<double *>(sh.c1), *d2 = d1 + (h + 1), *dp = d2 + (h + 1);
    for (int m = threadIdx.x; m <= h; m += blockDim.x) {
        const double u = 2.0 * (double)(-m) / (double)g.npz;
        const double p = u * 3.14159265358979323846;
        d1[m] = cospi(u);
        d2[m] = cospi(2.0 * u);
        dp[m] = p * p;
    }
    __syncthreads();
    const double igam = mc.inv_gam, ipi = 0.31830988618379067154;
    double f = 0.0;
    float f1 = 0.f, f2 = 0.f;
    for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
        int a, b;
        tri_pair(k, h, a, b);
        const int w = pair_weight(a, b, h);
        const double x = (band_e0_cls(band, d1[a], d1[b], d2[a], d2[b], dp[a], dp[b]) - mu) * igam;
        f += (double)w * (0.5 - atan(x) * ipi);
        const float xf = (float)x, r = 1.0f / (1.0f + xf * xf);
        f1 += (float)w * r * (float)ipi;
        f2 += (float)w * 2.0f * xf * r * r * (float)ipi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_down_sync(0xffffffffu, f, o);
        f1 += __shfl_down_sync(0xffffffffu, f1, o);
        f2 += __shfl_down_sync(0xffffffffu, f2, o);
    }
    double *hs = dp + (h + 1);   // [NW][3], after the class values
    if (lane == 0) { hs[3 * warp] = f; hs[3 * warp + 1] = f1; hs[3 * warp + 2] = f2; }
    __syncthreads();
    if (warp == 0) {
        // the NW warp sums by a shuffle tree (a chain of NW dependent FP64 adds
        // would cost some 60 cycles each)
        double F = lane < NW ? hs[3 * lane] : 0.0, F1 = lane < NW ? hs[3 * lane + 1] : 0.0,
               F2 = lane < NW ? hs[3 * lane + 2] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            F += __shfl_down_sync(0xffffffffu, F, o);
            F1 += __shfl_down_sync(0xffffffffu, F1, o);
            F2 += __shfl_down_sync(0xffffffffu, F2, o);
        }
        if (lane != 0) return;
        const double d = F - mc.target;
        const double dd1 = F1 * igam, dd2 = F2 * igam * igam;
        const double stp = 2.0 * d * dd1 / (2.0 * dd1 * dd1 - d * dd2);
        const double mu_new = mu - stp;
        set_mu(st, mu_new);
        st->last_step = fabs(stp);
        if (mu_out) *mu_out = mu_new;
        // the FP32 search stops within about 1e-6 eV of the root: a larger
        // FP64 correction means it went wrong
        if (!(fabs(stp) <= 1e-4)) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
    }
}

// Set-up launch.  CTAs [0, G): multisection pass 0 (mu from the filling);
// CTAs [G, G + GT): the per-axis tables and the energy grid, one entry per
// thread of their first warp; without a filling solve only the table CTAs run
// and the first of them records the given mu.
__global__ void __launch_bounds__(MU_THREADS, 2)
k_setup(Geom g, Band band, AxisTab *axis, float2 *eps32, double *eps64, InstState *st, double *acc,
        unsigned *counter, unsigned *status, double *mu_out, MuConst mc, int G, Band *band_out)
{
    if (band_out && blockIdx.x == 0 && threadIdx.x == 0) *band_out = band;   // the call's band, for later launches
    if ((int)blockIdx.x >= G) {
        const int tb = blockIdx.x - G;
        if (!band.solve_mu && tb == 0 && threadIdx.x == 0) {
            set_mu(st, band.mu);
            st->last_step = 0.0;
            if (mu_out) *mu_out = band.mu;
        }
        const int i = tb * MU_TAB_THREADS + threadIdx.x;
        if (threadIdx.x >= MU_TAB_THREADS) return;
        if (i < g.N) {
            double u = 2.0 * (double)(i - g.N / 2) / (double)g.npz;   // p_i / pi
            double p = u * 3.14159265358979323846;
            AxisTab a;
            a.c1 = cospi(u);
            a.c2 = cospi(2.0 * u);
            a.g = (band.ff_a == 0.0) ? 1.0 : exp(-p * p * band.ff_a * band.ff_a / 8.0);
            a.p2 = p * p;
            a.c1h = (float)a.c1;
            a.c1l = (float)(a.c1 - (double)a.c1h);
            a.c2h = (float)a.c2;
            a.c2l = (float)(a.c2 - (double)a.c2h);
            a.p2h = (float)a.p2;
            a.p2l = (float)(a.p2 - (double)a.p2h);
            a.gf = (float)a.g;
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
        return;
    }
    __shared__ MuShared sh;
    stage_classes(g, sh);
    if (mc.single) {
        __syncthreads();
        mu_solve_one_cta(g, band, mc, sh, st, status, mu_out);
        return;
    }
    if (threadIdx.x == 0) {
        sh.br.lo = -mc.B - 3.0;
        sh.br.hi = mc.B + 3.0;
        if (blockIdx.x == 0) {
            acc[0] = sh.br.lo;
            acc[1] = sh.br.hi;
            acc[2] = 0.0;
            *counter = 0;
        }
    }
    sect_pass(g, band, mc, sh, mu_cross(acc, G, 0));
}

// Multisection pass `pass` >= 1.
__global__ void __launch_bounds__(MU_THREADS, 2)
k_mu_sect(Geom g, Band band, double *acc, int pass, MuConst mc)
{
    __shared__ MuShared sh;
    const int G = gridDim.x;
    stage_classes(g, sh);
    __syncthreads();
    // the first chunk of pair energies does not depend on the bracket
    const int h = g.npz / 2, npairs = (h + 1) * (h + 2) / 2;
    stage_pairs(g, band, sh, 0, min(MU_CHUNK, npairs));
    bracket_from(acc, mu_cross(acc, G, pass - 1), mc, pass - 1, sh.br);
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        acc[3 * pass + 0] = sh.br.lo;
        acc[3 * pass + 1] = sh.br.hi;
        acc[3 * pass + 2] = sh.br.flag;
    }
    __syncthreads();
    if (sh.br.flag) return;   // the filling was not bracketed
    sect_pass(g, band, mc, sh, mu_cross(acc, G, pass), true);
}

// Halley step in FP64 from the midpoint of the last bracket; publishes mu.
__global__ void __launch_bounds__(MU_NT_THREADS)
k_mu_halley(Geom g, Band band, const AxisTab *__restrict__ axis, InstState *st, double *acc, unsigned *counter,
            unsigned *status, double *mu_out, MuConst mc)
{
    const int P = mc.passes, G = gridDim.x;
    __shared__ struct { MuBracket br; } sh;
    __shared__ double s_red[MU_NT_THREADS / 32][3];
    double *part = acc + MU_RES;   // [G][4]
    const int h = g.npz / 2, npairs = (h + 1) * (h + 2) / 2, c = g.N / 2;
    // the band energy of this thread's first pair does not depend on mu: its
    // loads and FP64 chain overlap the bracket search
    const int k0 = blockIdx.x + G * threadIdx.x;
    double e0_first = 0.0;
    int w_first = 0;
    if (k0 < npairs) {
        int a, b;
        tri_pair(k0, h, a, b);
        w_first = pair_weight(a, b, h);
        e0_first = band_e0(band, axis[c - a], axis[c - b]);
    }
    bracket_from(acc, mu_cross(acc, G, P - 1), mc, P - 1, sh.br);
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        acc[3 * P + 0] = sh.br.lo;
        acc[3 * P + 1] = sh.br.hi;
        acc[3 * P + 2] = sh.br.flag;
    }
    __syncthreads();
    const double mu = 0.5 * (sh.br.lo + sh.br.hi);
    if (sh.br.flag) {   // the filling was not bracketed
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
            set_mu(st, mu);
            st->last_step = INFINITY;
            if (mu_out) *mu_out = mu;
        }
        return;
    }
    const double igam = mc.inv_gam, ipi = 0.31830988618379067154;
    double f = 0.0;
    float f1 = 0.f, f2 = 0.f;
    // pairs interleaved over the CTAs first, so every SM's FP64 units share the work
    for (int k = k0; k < npairs; k += G * (int)blockDim.x) {
        double e0 = e0_first;
        int w = w_first;
        if (k != k0) {
            int a, b;
            tri_pair(k, h, a, b);
            w = pair_weight(a, b, h);
            e0 = band_e0(band, axis[c - a], axis[c - b]);
        }
        const double x = (e0 - mu) * igam;                                       // xi / gamma
        f += (double)w * (0.5 - atan(x) * ipi);                                   // occupation
        const float xf = (float)x, r = 1.0f / (1.0f + xf * xf);                    // gamma^2 / (xi^2 + gamma^2)
        f1 += (float)w * r * (float)ipi;                                           // gamma d occ / d mu
        f2 += (float)w * 2.0f * xf * r * r * (float)ipi;                           // gamma^2 d^2 occ / d mu^2
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_down_sync(0xffffffffu, f, o);
        f1 += __shfl_down_sync(0xffffffffu, f1, o);
        f2 += __shfl_down_sync(0xffffffffu, f2, o);
    }
    if (lane == 0) { s_red[warp][0] = f; s_red[warp][1] = f1; s_red[warp][2] = f2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double F = 0, F1 = 0, F2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { F += s_red[w][0]; F1 += s_red[w][1]; F2 += s_red[w][2]; }
        part[4 * (size_t)blockIdx.x + 0] = F;
        part[4 * (size_t)blockIdx.x + 1] = F1;
        part[4 * (size_t)blockIdx.x + 2] = F2;
    }
    // the last CTA to finish adds the partial sums in a fixed order
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
        if (s_last) *counter = 0;   // no other CTA touches it again in this launch
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double F = 0.0, F1 = 0.0, F2 = 0.0;
    for (int q = threadIdx.x; q < G; q += (int)blockDim.x) {
        F += __ldcg(part + 4 * (size_t)q + 0);
        F1 += __ldcg(part + 4 * (size_t)q + 1);
        F2 += __ldcg(part + 4 * (size_t)q + 2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        F += __shfl_down_sync(0xffffffffu, F, o);
        F1 += __shfl_down_sync(0xffffffffu, F1, o);
        F2 += __shfl_down_sync(0xffffffffu, F2, o);
    }
    __syncthreads();
    if (lane == 0) { s_red[warp][0] = F; s_red[warp][1] = F1; s_red[warp][2] = F2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        F = F1 = F2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { F += s_red[w][0]; F1 += s_red[w][1]; F2 += s_red[w][2]; }
        const double d = F - mc.target;                   // n - target
        const double d1 = F1 * igam, d2 = F2 * igam * igam;  // dn/dmu, d2n/dmu2
        const double step = 2.0 * d * d1 / (2.0 * d1 * d1 - d * d2);
        const double mu_new = mu - step;
        set_mu(st, mu_new);
        st->last_step = fabs(step);
        if (mu_out) *mu_out = mu_new;
        // the root lies within the last bracket up to FP32 noise (below
        // 1e-6 eV); a larger step means the multisection went wrong
        if (!(fabs(step) <= 2.0 * (sh.br.hi - sh.br.lo) + 1e-5))
            atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ENOCONV);
    }
}

static MuConst mu_const(const Geom &g, const Band &band, int G)
{
    MuConst mc;
    mc.NC = MU_NCPT * G;
    mc.passes = band.gamma < 0.02 ? 3 : 2;
    mc.single = mu_single(g) ? 1 : 0;
    mc.inv_nc1 = 1.0 / (double)(mc.NC - 1);
    mc.inv_gam = 1.0 / band.gamma;
    mc.target = band.filling * 0.5 * (double)g.npz * (double)g.npz;
    mc.target32 = llrint(mc.target * (double)MU_SECT_SCALE);
    mc.B = (band.band_kind == 1) ? 9.869604401089358 : 4.0 * (fabs(band.t) + fabs(band.tp) + fabs(band.tpp));
    return mc;
}

cudaError_t launch_twiddles(int len, float2 *tw32, double2 *tw64, cudaStream_t s)
{
    k_twiddles<<<(twiddle_entries() + 255) / 256, 256, 0, s>>>(len, tw32, tw64);
    return cudaGetLastError();
}

// Tables plus the first chemical-potential launch (multisection pass 0, or
// the given mu).
// band_out (device, or null): receives the call's band for later launches.
cudaError_t launch_setup_band(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                              InstState *st, double *acc, unsigned *bar, unsigned *status, double *mu_out, int G,
                              Band *band_out, cudaStream_t s)
{
    const int ntab = g.N > g.n_eps ? g.N : g.n_eps;
    const int GT = (ntab + MU_TAB_THREADS - 1) / MU_TAB_THREADS;
    const int Gs = band.solve_mu ? (mu_single(g) ? 1 : G) : 0;
    k_setup<<<Gs + GT, MU_THREADS, 0, s>>>(g, band, axis, eps32, eps64, st, acc, bar, status, mu_out,
                                           mu_const(g, band, G), Gs, band_out);
    return cudaGetLastError();
}
cudaError_t launch_setup(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                         InstState *st, double *acc, unsigned *bar, unsigned *status, double *mu_out, int G,
                         cudaStream_t s)
{
    return launch_setup_band(g, band, axis, eps32, eps64, st, acc, bar, status, mu_out, G, nullptr, s);
}

// Whether the chemical potential is solved inside the set-up launch.
bool mu_solve_in_setup(const Geom &g) { return mu_single(g); }

// The remaining chemical-potential launches (none for a given mu).
cudaError_t launch_solve_mu(const Geom &g, const Band &band, const AxisTab *axis, InstState *st, double *acc,
                            unsigned *bar, unsigned *status, double *mu_out, int G, cudaStream_t s)
{
    if (!band.solve_mu || mu_single(g)) return cudaSuccess;   // solved in the set-up launch
    const MuConst mc = mu_const(g, band, G);
    for (int pass = 1; pass < mc.passes; ++pass) k_mu_sect<<<G, MU_THREADS, 0, s>>>(g, band, acc, pass, mc);
    // one warp per CTA when every CTA has at most 32 pairs (the FP64 chains
    // then run side by side and the reductions are short)
    const int h = g.npz / 2, npairs = (h + 1) * (h + 2) / 2;
    const int T = npairs <= 32 * G ? 32 : MU_NT_THREADS;
    k_mu_halley<<<G, T, 0, s>>>(g, band, axis, st, acc, bar, status, mu_out, mc);
    return cudaGetLastError();
}

}  // namespace lh
