// Register-resident Stockham FFT engine for one CTA (sm_103a).
//
// A CTA transforms C independent lines of length L (powers of two 16..4096,
// and 3 * 2^k from 48 to 1536).
// Each stage is a radix-R butterfly held in registers; between stages the
// values go through shared memory once (the Stockham exchange), so an L-point
// transform with S stages touches shared memory 2(S-1) times per point and
// global memory only in the caller's load (first stage) and store (last
// stage).  Two thread mappings:
//   MAP_COL  : lanes run across the C lines first.  Used when the lines are
//              the strided axis of a row-major array (C neighbouring columns
//              form contiguous segments), so loads/stores of one warp cover
//              C*sizeof(complex) contiguous bytes per row.
//   MAP_LINE : lanes run along a line.  Used when each line is contiguous.
// Shared memory layouts keep each exchange free of bank conflicts for
// 8-byte elements: [L][C] for MAP_COL, [C][L + L/16] with one pad element per
// 16 for MAP_LINE (the stride-R writes of the first exchange then spread over
// all banks).
//
// Conventions: forward = sum_n x_n exp(-2 pi i n k / L), inverse uses the
// opposite sign, neither is scaled.  The inverse runs the forward radix
// schedule in reverse order, so that the last forward stage and the first
// inverse stage have the same radix and the same element-to-thread
// assignment: a pointwise operation between them (the conjugate product of
// the correlation) needs no data exchange.
#pragma once

#include <cuda_runtime.h>

namespace lh {

template <typename R> struct cpx_of;
template <> struct cpx_of<float> { using type = float2; };
template <> struct cpx_of<double> { using type = double2; };
template <typename R> using cx = typename cpx_of<R>::type;

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) { return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } // a * conj(b)
// Complex sums of the butterflies under a policy PK: FP32 complex sums as
// packed f32x2 instructions (one instruction for both parts; the same IEEE
// results as two scalar additions) when PK, else scalar.  Packing pays where
// the kernel has registers to spare (the pair operands must sit in aligned
// register pairs); kernels at 128 registers per thread run slower with it.
template <bool PK, typename C> __device__ __forceinline__ C padd(C a, C b)
{
    if constexpr (PK && sizeof(C) == 8) return __fadd2_rn(a, b);
    else return cadd(a, b);
}
template <bool PK, typename C> __device__ __forceinline__ C psub(C a, C b)
{
    if constexpr (PK && sizeof(C) == 8) {
        C c;
        asm("{\n\t.reg .b64 pa, pb, pc;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
            "sub.rn.f32x2 pc, pa, pb;\n\tmov.b64 {%0, %1}, pc;\n\t}"
            : "=f"(c.x), "=f"(c.y)
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
        return c;
    } else {
        return csub(a, b);
    }
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// odd ? p - conj(p) = 2 i Im p : p (the transform of the odd part of a real sequence)
template <typename C> __device__ __forceinline__ C odd_part(C p, bool odd)
{
    return odd ? mk<C>(decltype(p.x)(0), p.y + p.y) : p;
}
template <typename C> __device__ __forceinline__ C mul_i(C a) { return mk<C>(-a.y, a.x); }   //  i * a
template <typename C> __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }  // -i * a

// ---------------------------------------------------------------------------
// Radix schedules (forward order).  L = prod radix(L, s, F).  Two families:
//   F = 0: few stages with large radices (8, 16, 24) for powers of two up to
//          4096 and 3 * 2^k from 48 to 1536 (momentum axes padded to exactly
//          1.5 N); tiles hold a multiple of 8, 16 or 24 values per thread.
//   F = 1: radices dividing 12 (6, 12, 4) for 192, 384, 768 and 1536: one or
//          two more stages, but tiles of 12 values per thread, half the
//          registers of the 24-value tiles.
// An engine takes family 0 when its values per thread allow it, else 1.
__host__ __device__ constexpr bool fft_len_pow2(int L) { return (L & (L - 1)) == 0; }
__host__ __device__ constexpr bool fft_has_family1(int L) { return L == 192 || L == 384 || L == 768 || L == 1536; }
__host__ __device__ constexpr int fft_nstages(int L, int F = 0)
{
    return F == 1 ? (L == 192 ? 3 : (L == 1536 ? 5 : 4))
         : fft_len_pow2(L) ? (L <= 16 ? 1 : (L <= 256 ? 2 : 3)) : (L <= 96 ? 2 : 3);
}
__host__ __device__ constexpr int fft_fwd_radix(int L, int s, int F = 0)
{
    return F == 1 ? (s == 0 ? (L == 192 || L == 768 ? 12 : 6) : 4)
         : L == 16 ? 16
         : L == 32 ? (s == 0 ? 8 : 4)
         : L == 64 ? 8
         : L == 128 ? (s == 0 ? 16 : 8)
         : L == 256 ? 16
         : L == 512 ? 8
         : L == 1024 ? (s == 0 ? 16 : 8)
         : L == 2048 ? (s < 2 ? 16 : 8)
         : L == 4096 ? 16
         : L == 48 ? (s == 0 ? 8 : 6)
         : L == 96 ? (s == 0 ? 8 : 12)
         : L == 192 ? (s < 2 ? 8 : 3)
         : L == 384 ? (s < 2 ? 8 : 6)
         : L == 768 ? (s < 2 ? 8 : 12)
         : /* 1536 */ (s < 2 ? 8 : 24);
}
__host__ __device__ constexpr int fft_radix(int L, int s, bool inv, int F = 0)
{
    return inv ? fft_fwd_radix(L, fft_nstages(L, F) - 1 - s, F) : fft_fwd_radix(L, s, F);
}
__host__ __device__ constexpr int fft_ns_before(int L, int s, bool inv, int F = 0)
{
    return s == 0 ? 1 : fft_ns_before(L, s - 1, inv, F) * fft_radix(L, s - 1, inv, F);
}
__host__ __device__ constexpr int fft_sched_len(int L, int F, int s = 0)
{
    return s >= fft_nstages(L, F) ? 1 : fft_fwd_radix(L, s, F) * fft_sched_len(L, F, s + 1);
}
// every radix of family F's schedule divides v (values per thread)
__host__ __device__ constexpr bool fft_radices_divide(int L, int v, int F = 0, int s = 0)
{
    return (F == 1 && !fft_has_family1(L)) ? false
         : s >= fft_nstages(L, F) ? true
         : (v % fft_fwd_radix(L, s, F) == 0 && fft_radices_divide(L, v, F, s + 1));
}
__host__ __device__ constexpr int fft_family(int L, int v) { return fft_radices_divide(L, v, 0) ? 0 : 1; }

// ---------------------------------------------------------------------------
// Exact small DFTs in registers.  cos(2 pi m / 48) for m = 0..12 (multiples of
// 7.5 degrees), which covers every radix used (2, 3, 4, 6, 8, 12, 16, 24).
__host__ __device__ constexpr double cos48_q(int m)
{
    return m == 0 ? 1.0 : m == 1 ? 0.99144486137381041114 : m == 2 ? 0.96592582628906828675
         : m == 3 ? 0.92387953251128675613 : m == 4 ? 0.86602540378443864676
         : m == 5 ? 0.79335334029123516458 : m == 6 ? 0.70710678118654752440
         : m == 7 ? 0.60876142900872063942 : m == 8 ? 0.5
         : m == 9 ? 0.38268343236508977173 : m == 10 ? 0.25881904510252076235
         : m == 11 ? 0.13052619222005159155 : 0.0;
}
__host__ __device__ constexpr double cos48(int m)
{
    // cos(2 pi m / 48) for any m >= 0, from the first-quadrant values
    return (m % 48) <= 12 ? cos48_q(m % 48)
         : (m % 48) <= 24 ? -cos48_q(24 - m % 48)
         : (m % 48) <= 36 ? -cos48_q(m % 48 - 24)
         : cos48_q(48 - m % 48);
}
__host__ __device__ constexpr double sin48(int m) { return cos48(m + 36); }  // sin x = cos(x - pi/2)

// x * exp(-+ 2 pi i K / R) with compile-time R | 48 (INV flips the sign).
template <int R, int K, bool INV, typename C>
__device__ __forceinline__ C twc(C x)
{
    constexpr int k = ((K % R) + R) % R;
    constexpr int k48 = k * (48 / R);
    using T = decltype(C::x);
    if constexpr (k48 == 0) return x;
    else if constexpr (k48 == 24) return mk<C>(-x.x, -x.y);
    else if constexpr (k48 == 12) return INV ? mul_i(x) : mul_mi(x);
    else if constexpr (k48 == 36) return INV ? mul_mi(x) : mul_i(x);
    else {
        constexpr T cr = (T)cos48(k48);
        constexpr T ci = INV ? (T)sin48(k48) : (T)-sin48(k48);
        return mk<C>(x.x * cr - x.y * ci, x.x * ci + x.y * cr);
    }
}

template <int R, bool INV, typename C, bool PK = false> struct Dft;

template <bool INV, typename C, bool PK> struct Dft<1, INV, C, PK> {
    __device__ __forceinline__ static void run(C *) {}
};
template <bool INV, typename C, bool PK> struct Dft<2, INV, C, PK> {
    __device__ __forceinline__ static void run(C *v)
    {
        C a = v[0], b = v[1];
        v[0] = padd<PK>(a, b);
        v[1] = psub<PK>(a, b);
    }
};
template <bool INV, typename C, bool PK> struct Dft<4, INV, C, PK> {
    __device__ __forceinline__ static void run(C *v)
    {
        C t0 = padd<PK>(v[0], v[2]), t1 = psub<PK>(v[0], v[2]);
        C t2 = padd<PK>(v[1], v[3]), t3 = psub<PK>(v[1], v[3]);
        t3 = INV ? mul_i(t3) : mul_mi(t3);
        v[0] = padd<PK>(t0, t2);
        v[2] = psub<PK>(t0, t2);
        v[1] = padd<PK>(t1, t3);
        v[3] = psub<PK>(t1, t3);
    }
};
// Radix 8 and 16: decimation in time into two halves of radix R/2.
template <int R, bool INV, typename C, int K, bool PK = false>
__device__ __forceinline__ void dit_combine(C *v, const C *e, const C *o)
{
    if constexpr (K < R / 2) {
        C t = twc<R, K, INV>(o[K]);
        v[K] = padd<PK>(e[K], t);
        v[K + R / 2] = psub<PK>(e[K], t);
        dit_combine<R, INV, C, K + 1, PK>(v, e, o);
    }
}
template <bool INV, typename C, bool PK> struct Dft<8, INV, C, PK> {
    __device__ __forceinline__ static void run(C *v)
    {
        C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV, C, PK>::run(e);
        Dft<4, INV, C, PK>::run(o);
        dit_combine<8, INV, C, 0, PK>(v, e, o);
    }
};
template <bool INV, typename C, bool PK> struct Dft<3, INV, C, PK> {
    __device__ __forceinline__ static void run(C *v)
    {
        using T = decltype(C::x);
        constexpr T s3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
        C t1 = padd<PK>(v[1], v[2]);
        C t2 = mk<C>(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        C d = psub<PK>(v[1], v[2]);
        C t3 = mk<C>(s3 * d.x, s3 * d.y);
        v[0] = padd<PK>(v[0], t1);
        // forward: y1 = t2 - i t3, y2 = t2 + i t3 (inverse: the other way round)
        v[1] = INV ? padd<PK>(t2, mul_i(t3)) : padd<PK>(t2, mul_mi(t3));
        v[2] = INV ? padd<PK>(t2, mul_mi(t3)) : padd<PK>(t2, mul_i(t3));
    }
};
// Radix 6, 12 and 24: decimation in time into two halves.
template <int R, bool INV, typename C, bool PK = false> struct DftDit {
    __device__ __forceinline__ static void run(C *v)
    {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
        Dft<R / 2, INV, C, PK>::run(e);
        Dft<R / 2, INV, C, PK>::run(o);
        dit_combine<R, INV, C, 0, PK>(v, e, o);
    }
};
template <bool INV, typename C, bool PK> struct Dft<6, INV, C, PK> : DftDit<6, INV, C, PK> {};
template <bool INV, typename C, bool PK> struct Dft<12, INV, C, PK> : DftDit<12, INV, C, PK> {};
template <bool INV, typename C, bool PK> struct Dft<24, INV, C, PK> : DftDit<24, INV, C, PK> {};

template <bool INV, typename C, bool PK> struct Dft<16, INV, C, PK> {
    __device__ __forceinline__ static void run(C *v)
    {
        C e[8], o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
        Dft<8, INV, C, PK>::run(e);
        Dft<8, INV, C, PK>::run(o);
        dit_combine<16, INV, C, 0, PK>(v, e, o);
    }
};

// The twiddles w^r = tw[r m], r < R, of one butterfly from the length-L table
// (m = k L / (Ns R)): for R = 2, 4, 8 and 16 only w is loaded and its powers
// formed as products (at most four roundings deep), instead of R - 1 loads.
template <int R, typename Cx>
__device__ __forceinline__ void stage_twiddles(const Cx *__restrict__ tw, int m, Cx *w)
{
    if constexpr (R == 2 || R == 4 || R == 8 || R == 16) {
        w[1] = __ldg(&tw[m]);
#pragma unroll
        for (int r = 2; r < R; ++r) w[r] = cmul(w[r / 2], w[r - r / 2]);
    } else {
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = __ldg(&tw[r * m]);
    }
}

enum { MAP_COL = 0, MAP_LINE = 1 };

// ---------------------------------------------------------------------------
// The engine.  VPT = C*L/T values per thread, stored as v[b*R + r] for the
// b-th butterfly of the current stage.
template <typename Real, int L, int C, int T, int MAP, bool INV>
struct Fft {
    using Cx = cx<Real>;
    static constexpr int VPT = C * L / T;
    static constexpr int F = fft_family(L, VPT);             // radix schedule family
    static constexpr int NS = fft_nstages(L, F);
    static constexpr int LP = L + L / 16;                    // padded line (MAP_LINE)
    static constexpr int R0 = fft_radix(L, 0, INV, F);
    static constexpr int RL = fft_radix(L, NS - 1, INV, F);
    // MAP_COL rows: one empty row after every R0 rows, so that the first
    // exchange's writes (rows R0 apart) fall into different banks
    static constexpr int SMEM_ELEMS = (MAP == MAP_COL) ? (L + L / R0) * C : C * LP;
    static_assert((C * L) % T == 0, "tile must split evenly over threads");
    static_assert(fft_radices_divide(L, VPT, F), "values per thread must be a multiple of every radix");
    static_assert(fft_sched_len(L, F) == L, "radix schedule must multiply to L");
    static_assert(MAP == MAP_LINE || T % C == 0, "column map needs T % C == 0");

    __device__ __forceinline__ static int saddr(int col, int n)
    {
        return MAP == MAP_COL ? (n + n / R0) * C + col : col * LP + n + (n >> 4);
    }
    // butterfly index -> (line, j) for a stage of radix Rs
    template <int Rs>
    __device__ __forceinline__ static void map(int beta, int &col, int &j)
    {
        if constexpr (MAP == MAP_COL) { col = beta % C; j = beta / C; }
        else { col = beta / (L / Rs); j = beta % (L / Rs); }
    }
    // element held in v[b*R0 + r] before the first stage
    __device__ __forceinline__ static void first_elem(int b, int r, int &col, int &n)
    {
        int j;
        map<R0>(threadIdx.x + b * T, col, j);
        n = j + r * (L / R0);
    }
    // element held in v[b*RL + r] after the last stage
    __device__ __forceinline__ static void last_elem(int b, int r, int &col, int &n)
    {
        int j;
        map<RL>(threadIdx.x + b * T, col, j);
        n = j + r * (L / RL);
    }

    template <int S>
    __device__ __forceinline__ static void stage_rest(Cx *v, Cx *sm, const Cx *__restrict__ tw)
    {
        if constexpr (S < NS) {
            constexpr int Rp = fft_radix(L, S - 1, INV, F);
            constexpr int Nsp = fft_ns_before(L, S - 1, INV, F);
            constexpr int Rs = fft_radix(L, S, INV, F);
            constexpr int Ns = Nsp * Rp;
            // write the previous stage's outputs (Stockham order)
#pragma unroll
            for (int b = 0; b < VPT / Rp; ++b) {
                int col, j;
                map<Rp>(threadIdx.x + b * T, col, j);
                int idxD = (j / Nsp) * Nsp * Rp + (j % Nsp);
#pragma unroll
                for (int r = 0; r < Rp; ++r) sm[saddr(col, idxD + r * Nsp)] = v[b * Rp + r];
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < VPT / Rs; ++b) {
                int col, j;
                map<Rs>(threadIdx.x + b * T, col, j);
#pragma unroll
                for (int r = 0; r < Rs; ++r) v[b * Rs + r] = sm[saddr(col, j + r * (L / Rs))];
                int k = j % Ns;
                // twiddle exp(-+ 2 pi i k r / (Ns Rs)) from the length-L table exp(-2 pi i n / L)
                Cx w[Rs];
                stage_twiddles<Rs>(tw, k * (L / (Ns * Rs)), w);
#pragma unroll
                for (int r = 1; r < Rs; ++r) v[b * Rs + r] = INV ? cmulc(v[b * Rs + r], w[r]) : cmul(v[b * Rs + r], w[r]);
                Dft<Rs, INV, Cx>::run(v + b * Rs);
            }
            __syncthreads();
            stage_rest<S + 1>(v, sm, tw);
        }
    }

    // Transform the tile in place: v holds the first-stage inputs (see
    // first_elem) on entry and the outputs (see last_elem) on exit.  sm must
    // hold SMEM_ELEMS elements; tw is the length-L table exp(-2 pi i n / L);
    // the call ends with a __syncthreads().
    __device__ __forceinline__ static void run(Cx *v, Cx *sm, const Cx *__restrict__ tw)
    {
#pragma unroll
        for (int b = 0; b < VPT / R0; ++b) Dft<R0, INV, Cx>::run(v + b * R0);
        stage_rest<1>(v, sm, tw);
    }
};

}  // namespace lh

namespace lh {

// ---------------------------------------------------------------------------
// Column engine with paired columns: each thread transforms two adjacent
// columns (2p, 2p + 1) of a C-column tile with the same butterfly indices, so
// every twiddle is loaded once for both, global and shared-memory accesses
// move 16 bytes (both columns of a row) per instruction, and each thread has
// two independent dependency chains in flight.  Layout and Stockham ordering
// as in Fft<..., MAP_COL, ...>: shared memory [L][C].
// VPT = (C/2) L / T values per thread per column.
// PK: packed f32x2 complex sums in the butterflies (padd/psub).
template <typename Real, int L, int C, int T, bool INV, bool PK = false>
struct FftPair {
    using Cx = cx<Real>;
    static constexpr int CP = C / 2;                 // column pairs per tile
    static constexpr int VPT = CP * L / T;
    static constexpr int F = fft_family(L, VPT);     // radix schedule family
    static constexpr int NS = fft_nstages(L, F);
    static constexpr int R0 = fft_radix(L, 0, INV, F);
    static constexpr int RL = fft_radix(L, NS - 1, INV, F);
    // Rows of C complex values.  With at least 8 pairs per row every 16-byte
    // access phase of a warp (8 threads) lies in one 128-byte row segment, so
    // rows are stored back to back (addresses linear in the row: no per-value
    // index arithmetic); narrower tiles get one empty row after every R0 rows
    // so that the first exchange's writes (rows R0 apart) fall into different
    // banks.
    static constexpr bool LIN = CP >= 8;
    static constexpr int SMEM_ELEMS = LIN ? L * C : (L + L / R0) * C;
    static_assert(C % 2 == 0 && T % CP == 0 && (CP * L) % T == 0, "tile must split evenly over threads");
    static_assert(fft_radices_divide(L, VPT, F), "values per thread must be a multiple of every radix");
    static_assert(fft_sched_len(L, F) == L, "radix schedule must multiply to L");

    // the thread's column pair (columns 2p and 2p + 1 of the tile)
    __device__ __forceinline__ static int pair() { return threadIdx.x % CP; }
    // row of the b-th butterfly's r-th element before the first stage
    __device__ __forceinline__ static int first_row(int b, int r)
    {
        return (threadIdx.x + b * T) / CP + r * (L / R0);
    }
    // row of v[b*RL + r] after the last stage
    __device__ __forceinline__ static int last_row(int b, int r)
    {
        return (threadIdx.x + b * T) / CP + r * (L / RL);
    }

    __device__ __forceinline__ static int srow(int row) { return LIN ? row * C : (row + row / R0) * C; }
    __device__ __forceinline__ static void st2(Cx *sm, int row, int p, Cx a, Cx b)
    {
        if constexpr (sizeof(Real) == 4) {
            *reinterpret_cast<float4 *>(&sm[srow(row) + 2 * p]) = make_float4(a.x, a.y, b.x, b.y);
        } else {
            sm[srow(row) + 2 * p] = a;
            sm[srow(row) + 2 * p + 1] = b;
        }
    }
    __device__ __forceinline__ static void ld2(const Cx *sm, int row, int p, Cx &a, Cx &b)
    {
        if constexpr (sizeof(Real) == 4) {
            float4 q = *reinterpret_cast<const float4 *>(&sm[srow(row) + 2 * p]);
            a = mk<Cx>(q.x, q.y);
            b = mk<Cx>(q.z, q.w);
        } else {
            a = sm[srow(row) + 2 * p];
            b = sm[srow(row) + 2 * p + 1];
        }
    }

    template <int S>
    __device__ __forceinline__ static void stage_rest(Cx *va, Cx *vb, Cx *sm, const Cx *__restrict__ tw)
    {
        if constexpr (S < NS) {
            constexpr int Rp = fft_radix(L, S - 1, INV, F);
            constexpr int Nsp = fft_ns_before(L, S - 1, INV, F);
            constexpr int Rs = fft_radix(L, S, INV, F);
            constexpr int Ns = Nsp * Rp;
            const int p = pair();
#pragma unroll
            for (int b = 0; b < VPT / Rp; ++b) {
                int j = (threadIdx.x + b * T) / CP;
                int idxD = (j / Nsp) * Nsp * Rp + (j % Nsp);
#pragma unroll
                for (int r = 0; r < Rp; ++r) st2(sm, idxD + r * Nsp, p, va[b * Rp + r], vb[b * Rp + r]);
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < VPT / Rs; ++b) {
                int j = (threadIdx.x + b * T) / CP;
#pragma unroll
                for (int r = 0; r < Rs; ++r) ld2(sm, j + r * (L / Rs), p, va[b * Rs + r], vb[b * Rs + r]);
                int k = j % Ns;
                Cx w[Rs];
                stage_twiddles<Rs>(tw, k * (L / (Ns * Rs)), w);
#pragma unroll
                for (int r = 1; r < Rs; ++r) {
                    va[b * Rs + r] = INV ? cmulc(va[b * Rs + r], w[r]) : cmul(va[b * Rs + r], w[r]);
                    vb[b * Rs + r] = INV ? cmulc(vb[b * Rs + r], w[r]) : cmul(vb[b * Rs + r], w[r]);
                }
                Dft<Rs, INV, Cx, PK>::run(va + b * Rs);
                Dft<Rs, INV, Cx, PK>::run(vb + b * Rs);
            }
            __syncthreads();
            stage_rest<S + 1>(va, vb, sm, tw);
        }
    }

    // Transform both columns in place (inputs per first_row, outputs per
    // last_row); ends with a __syncthreads().
    __device__ __forceinline__ static void run(Cx *va, Cx *vb, Cx *sm, const Cx *__restrict__ tw)
    {
#pragma unroll
        for (int b = 0; b < VPT / R0; ++b) {
            Dft<R0, INV, Cx, PK>::run(va + b * R0);
            Dft<R0, INV, Cx, PK>::run(vb + b * R0);
        }
        stage_rest<1>(va, vb, sm, tw);
    }
};

// 16-byte access to columns (c, c + 1) of a row of complex values.
template <typename Cx>
__device__ __forceinline__ void gld2(const Cx *p, Cx &a, Cx &b)
{
    if constexpr (sizeof(Cx) == 8) {
        float4 q = __ldcs(reinterpret_cast<const float4 *>(p));
        a = mk<Cx>(q.x, q.y);
        b = mk<Cx>(q.z, q.w);
    } else {
        a = p[0];
        b = p[1];
    }
}
template <typename Cx>
__device__ __forceinline__ void gst2(Cx *p, Cx a, Cx b)
{
    if constexpr (sizeof(Cx) == 8) {
        *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        p[0] = a;
        p[1] = b;
    }
}

}  // namespace lh
