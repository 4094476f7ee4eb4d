// Pruned Stockham engine for the momentum passes whose padding is exactly
// one third (sm_103a, FP32).
//
// With the default Q = N lags the momentum axes are padded from N to
// L = N + Q/2 = 3N/2 points (no wrap-around of the lags |s| <= Q/2, Sec. 3's
// convolution theorem on a zero-padded grid).  This engine puts a radix-24
// stage at the padded end of each transform:
//   forward, first stage: rows j + (L/24) r, r in [0, 24); the rows with
//     r >= 16 are the zero padding (>= 2L/3 = N), so 16 inputs are loaded and
//     the 24-point DFT runs as three 8-point DFTs over pre-combined pairs;
//   inverse, last stage (the forward schedule reversed): outputs
//     j + (L/24) r; the kept lags |s| <= L/3 are r < 8 (s >= 0) and r >= 16
//     (s < 0), so only 16 of the 24 outputs are formed.
// Schedules (forward order): 192 = 24.8, 384 = 24.4.4, 768 = 24.8.4,
// 1536 = 24.8.8.
//
// Thread map: a tile of CW columns (or column pairs) x L rows, T threads;
// thread t owns column (pair) t % CW and, in a stage of radix R, the
// butterflies j = t / CW + b (T / CW), b < VPT / R.  Every shared-memory and
// global address is a per-butterfly base plus compile-time offsets, and the
// twiddles of a butterfly come from a per-stage table [k][R] (k = j mod Ns)
// as 16-byte loads.  Rows narrower than 128 bytes get one empty row after
// every R0 rows (R0 = the first stage's radix), so that the first exchange's
// writes, R0 rows apart, spread over the banks; offsets stay compile-time
// because every access offset is a multiple of R0 or lies inside one block.
#pragma once

#include "fft_engine.cuh"

namespace lh {

__host__ __device__ constexpr bool pr_supported(int L) { return L == 192 || L == 384 || L == 768 || L == 1536; }
__host__ __device__ constexpr int pr_nstages(int L) { return L == 192 ? 2 : 3; }
__host__ __device__ constexpr int pr_fwd_radix(int L, int s)
{
    return s == 0 ? 24 : L == 1536 ? 8 : L == 768 ? (s == 1 ? 8 : 4) : L == 384 ? 4 : 8;
}
__host__ __device__ constexpr int pr_radix(int L, int s, bool inv)
{
    return inv ? pr_fwd_radix(L, pr_nstages(L) - 1 - s) : pr_fwd_radix(L, s);
}
// product of the radices before stage s
__host__ __device__ constexpr int pr_ns(int L, int s, bool inv)
{
    return s == 0 ? 1 : pr_ns(L, s - 1, inv) * pr_radix(L, s - 1, inv);
}

// Per-stage twiddle tables: for stage s >= 1 of a schedule, rows [k], k < Ns,
// of Rs entries w^1, w^2, ..., w^(Rs-1), w^0, w = exp(-2 pi i k / (Ns Rs))
// (forward sign; the inverse engine multiplies by the conjugate): a butterfly's
// w and w^2 are one 16-byte load.  Tables of L in {192, 384, 768, 1536},
// forward then inverse schedule, stages in order, back to back.
__host__ __device__ constexpr int pr_len_index(int L) { return L == 192 ? 0 : L == 384 ? 1 : L == 768 ? 2 : 3; }
__host__ __device__ constexpr int pr_len_of(int i) { return 192 << i; }
__host__ __device__ constexpr int pr_table_entries(int L, bool inv, int s) { return pr_ns(L, s + 1, inv); }
__host__ __device__ constexpr int pr_tables_before(int li, int inv, int s)
{
    // entries of every table that precedes (length index li, direction inv, stage s)
    int n = 0;
    for (int l = 0; l < 4; ++l)
        for (int d = 0; d < 2; ++d)
            for (int st = 1; st < pr_nstages(pr_len_of(l)); ++st) {
                if (l == li && d == inv && st == s) return n;
                n += pr_table_entries(pr_len_of(l), d != 0, st);
            }
    return n;
}
__host__ __device__ constexpr int pr_twiddle_entries() { return pr_tables_before(4, 0, 1); }
__host__ __device__ constexpr int pr_tw_offset(int L, bool inv, int s) { return pr_tables_before(pr_len_index(L), inv, s); }

// ---------------------------------------------------------------------------
// 24-point DFTs with a pruned end (sign by INV as in Dft<>).
// Inputs v[16..23] zero: y[3 k2 + k1] = DFT8_k2( w^(r1 k1) (v[r1] + W3^k1 v[r1 + 8]) ),
// w = exp(-+2 pi i / 24), W3 = w^8.
template <bool INV, bool PK = false>
__device__ __forceinline__ void dft24_in16(float2 *v)
{
    constexpr float s3 = 0.86602540378443864676f;   // sin(2 pi / 3)
    float2 u0[8], u1[8], u2[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float2 a = v[r], c = v[r + 8];
        u0[r] = padd<PK>(a, c);
        const float2 t = make_float2(fmaf(-0.5f, c.x, a.x), fmaf(-0.5f, c.y, a.y));
        const float2 q = make_float2(s3 * c.x, s3 * c.y);
        // a + W3 c = t -+ i q, a + W3^2 c = t +- i q (forward: W3 = -1/2 - i s3)
        u1[r] = INV ? padd<PK>(t, mul_i(q)) : padd<PK>(t, mul_mi(q));
        u2[r] = INV ? padd<PK>(t, mul_mi(q)) : padd<PK>(t, mul_i(q));
    }
    u1[1] = twc<24, 1, INV>(u1[1]); u1[2] = twc<24, 2, INV>(u1[2]); u1[3] = twc<24, 3, INV>(u1[3]);
    u1[4] = twc<24, 4, INV>(u1[4]); u1[5] = twc<24, 5, INV>(u1[5]); u1[6] = twc<24, 6, INV>(u1[6]);
    u1[7] = twc<24, 7, INV>(u1[7]);
    u2[1] = twc<24, 2, INV>(u2[1]); u2[2] = twc<24, 4, INV>(u2[2]); u2[3] = twc<24, 6, INV>(u2[3]);
    u2[4] = twc<24, 8, INV>(u2[4]); u2[5] = twc<24, 10, INV>(u2[5]); u2[6] = twc<24, 12, INV>(u2[6]);
    u2[7] = twc<24, 14, INV>(u2[7]);
    Dft<8, INV, float2, PK>::run(u0);
    Dft<8, INV, float2, PK>::run(u1);
    Dft<8, INV, float2, PK>::run(u2);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[3 * k] = u0[k];
        v[3 * k + 1] = u1[k];
        v[3 * k + 2] = u2[k];
    }
}

// Outputs y[0..7] and y[16..23] only (v[8..15] are left undefined):
// y[k1 + 8 k2] = sum_i2 W3^(i2 k2) w^(i2 k1) DFT8_k1(v[3 i1 + i2]).
template <bool INV, bool PK = false>
__device__ __forceinline__ void dft24_out16(float2 *v)
{
    constexpr float s3 = 0.86602540378443864676f;
    float2 y0[8], y1[8], y2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        y0[i] = v[3 * i];
        y1[i] = v[3 * i + 1];
        y2[i] = v[3 * i + 2];
    }
    Dft<8, INV, float2, PK>::run(y0);
    Dft<8, INV, float2, PK>::run(y1);
    Dft<8, INV, float2, PK>::run(y2);
    y1[1] = twc<24, 1, INV>(y1[1]); y1[2] = twc<24, 2, INV>(y1[2]); y1[3] = twc<24, 3, INV>(y1[3]);
    y1[4] = twc<24, 4, INV>(y1[4]); y1[5] = twc<24, 5, INV>(y1[5]); y1[6] = twc<24, 6, INV>(y1[6]);
    y1[7] = twc<24, 7, INV>(y1[7]);
    y2[1] = twc<24, 2, INV>(y2[1]); y2[2] = twc<24, 4, INV>(y2[2]); y2[3] = twc<24, 6, INV>(y2[3]);
    y2[4] = twc<24, 8, INV>(y2[4]); y2[5] = twc<24, 10, INV>(y2[5]); y2[6] = twc<24, 12, INV>(y2[6]);
    y2[7] = twc<24, 14, INV>(y2[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 s = padd<PK>(y1[k], y2[k]), d = psub<PK>(y1[k], y2[k]);
        v[k] = padd<PK>(y0[k], s);
        const float2 t = make_float2(fmaf(-0.5f, s.x, y0[k].x), fmaf(-0.5f, s.y, y0[k].y));
        const float2 q = make_float2(s3 * d.x, s3 * d.y);
        // W3^2 z1 + W3 z2 = -s/2 -+ i s3 d (forward: W3 = -1/2 - i s3)
        v[k + 16] = INV ? padd<PK>(t, mul_mi(q)) : padd<PK>(t, mul_i(q));
    }
}

// ---------------------------------------------------------------------------
// The engine.  NOPS = 2: two operands per thread (va, vb) that share every
// twiddle, stored side by side (16 bytes) in rows of CW pairs; NOPS = 1: one
// operand, rows of CW values.  PIN: inputs at rows >= 2L/3 are zero (forward
// first stage); POUT: only the kept lags of the last stage are formed.
// TWS (PrEng): the twiddle tables of length L are in shared memory at tw
// (the padded layout of pr_tws_offset), read with ld.shared, instead of in
// global memory read through the read-only cache.
__device__ __forceinline__ float4 lds_f4(const float4 *p)
{
    float4 q;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return q;
}
// The shared-memory copy of one length's tables: forward stages, then inverse
// stages, each row [k] padded by 16 bytes (Rs + 2 entries) so that the 16-byte
// twiddle loads of the four consecutive butterflies of a warp fall in
// different banks.
__host__ __device__ constexpr int pr_tws_row(int L, bool inv, int s) { return pr_radix(L, s, inv) + 2; }
__host__ __device__ constexpr int pr_tws_offset(int L, bool inv, int s)
{
    int n = 0;
    for (int d = 0; d < 2; ++d)
        for (int st = 1; st < pr_nstages(L); ++st) {
            if (d == (int)inv && st == s) return n;
            n += pr_ns(L, st, d != 0) * pr_tws_row(L, d != 0, st);
        }
    return n;   // past the last table: the total
}
__host__ __device__ constexpr int pr_tws_entries(int L) { return pr_tws_offset(L, true, pr_nstages(L)); }

// PK: packed f32x2 complex sums in the butterflies (padd/psub).
template <int L, int CW, int T, bool INV, int NOPS, bool PIN, bool POUT, bool TWS = false, bool PK = false>
struct PrEng {
    using Cx = float2;
    static constexpr int S = pr_nstages(L);
    static constexpr int VPT = CW * L / T;          // values per thread per operand
    static constexpr int RPT = T / CW;              // butterfly stride of one thread
    static constexpr int R0 = pr_radix(L, 0, INV);
    static constexpr int RL = pr_radix(L, S - 1, INV);
    static constexpr int ROW_BYTES = CW * NOPS * 8;
    static constexpr bool PAD = ROW_BYTES < 128;
    static constexpr int ROWS = PAD ? L + L / R0 : L;
    static constexpr int SMEM_ELEMS = ROWS * CW * NOPS;
    static_assert(pr_supported(L), "no pruned schedule for this length");
    static_assert(T % CW == 0 && (CW * L) % T == 0, "tile must split evenly over threads");
    static_assert(VPT % 24 == 0, "values per thread must be a multiple of every radix (24, 8, 4)");
    static_assert(!PIN || (!INV && R0 == 24), "pruned inputs: forward schedule, radix-24 first stage");
    static_assert(!POUT || (INV && RL == 24), "pruned outputs: inverse schedule, radix-24 last stage");

    __device__ __forceinline__ static int col() { return (int)threadIdx.x % CW; }
    __device__ __forceinline__ static int jb(int b) { return (int)threadIdx.x / CW + b * RPT; }
    // padded row of base + off, where off is a multiple of R0 or base is and off < R0
    __host__ __device__ static constexpr int poff(int off) { return PAD ? off + off / R0 : off; }
    __device__ __forceinline__ static int pbase(int base) { return PAD ? base + base / R0 : base; }

    __device__ __forceinline__ static void st(Cx *sm, int prow, Cx a, Cx b)
    {
        if constexpr (NOPS == 2)
            *reinterpret_cast<float4 *>(&sm[prow * (2 * CW) + 2 * col()]) = make_float4(a.x, a.y, b.x, b.y);
        else
            sm[prow * CW + col()] = a;
    }
    __device__ __forceinline__ static void ld(const Cx *sm, int prow, Cx &a, Cx &b)
    {
        if constexpr (NOPS == 2) {
            const float4 q = *reinterpret_cast<const float4 *>(&sm[prow * (2 * CW) + 2 * col()]);
            a = make_float2(q.x, q.y);
            b = make_float2(q.z, q.w);
        } else {
            a = sm[prow * CW + col()];
        }
    }

    __device__ __forceinline__ static float4 tw_ld(const float4 *p) { return TWS ? lds_f4(p) : __ldg(p); }
    // The twiddles w^r, r < R, of one butterfly (w = exp(-2 pi i k / (Ns R))),
    // from its table row (w^1, w^2, ..., w^(R-1), w^0): one 16-byte load gives
    // w and w^2, the other powers are products (for R = 24 also w^7, w^8 and
    // w^15, w^16 are loaded); at most three roundings deep, a few ulp.  The
    // 16-byte table loads, not the multiplications, were what the twiddles
    // cost in these passes.
    template <int R>
    __device__ __forceinline__ static void twiddle_set(const float4 *w4, Cx *w)
    {
        auto lo = [](float4 q) { return make_float2(q.x, q.y); };
        auto hi = [](float4 q) { return make_float2(q.z, q.w); };
        static_assert(R == 4 || R == 8 || R == 24, "radices of the pruned schedules");
        const float4 q0 = tw_ld(w4);
        w[1] = lo(q0);
        w[2] = hi(q0);
        w[3] = cmul(w[1], w[2]);
        if constexpr (R >= 8) {
            w[4] = cmul(w[2], w[2]);
            w[5] = cmul(w[2], w[3]);
            w[6] = cmul(w[3], w[3]);
        }
        if constexpr (R == 8) w[7] = cmul(w[3], w[4]);
        if constexpr (R == 24) {
            const float4 q3 = tw_ld(w4 + 3), q7 = tw_ld(w4 + 7);
            w[7] = lo(q3);
            w[8] = hi(q3);
            w[15] = lo(q7);
            w[16] = hi(q7);
#pragma unroll
            for (int r = 1; r < 7; ++r) w[8 + r] = cmul(w[8], w[r]);
#pragma unroll
            for (int r = 1; r < 8; ++r) w[16 + r] = cmul(w[16], w[r]);
        }
    }

    template <int R, bool FIRST, bool LAST>
    __device__ __forceinline__ static void dft(Cx *v)
    {
        if constexpr (R == 24 && FIRST && PIN) dft24_in16<INV, PK>(v);
        else if constexpr (R == 24 && LAST && POUT) dft24_out16<INV, PK>(v);
        else Dft<R, INV, Cx, PK>::run(v);
    }

    template <int SS>
    __device__ __forceinline__ static void stage_rest(Cx *va, Cx *vb, Cx *sm, const Cx *__restrict__ tw)
    {
        if constexpr (SS < S) {
            constexpr int Rp = pr_radix(L, SS - 1, INV), Nsp = pr_ns(L, SS - 1, INV);
            constexpr int Rs = pr_radix(L, SS, INV), Ns = pr_ns(L, SS, INV);
            static_assert(Nsp == 1 || Nsp % R0 == 0, "exchange offsets must stay compile-time");
            static_assert((L / Rs) % R0 == 0, "read offsets must stay compile-time");
            const Cx *tws = tw + (TWS ? pr_tws_offset(L, INV, SS) : pr_tw_offset(L, INV, SS));
            constexpr int TWROW = TWS ? Rs + 2 : Rs;
            // the previous stage's outputs, Stockham order: idxD + r Nsp
#pragma unroll
            for (int b = 0; b < VPT / Rp; ++b) {
                const int j = jb(b);
                const int base = pbase((j / Nsp) * Nsp * Rp + j % Nsp);
#pragma unroll
                for (int r = 0; r < Rp; ++r) st(sm, base + poff(r * Nsp), va[b * Rp + r], vb[b * Rp + r]);
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < VPT / Rs; ++b) {
                const int j = jb(b);
                const int base = pbase(j);
#pragma unroll
                for (int r = 0; r < Rs; ++r) ld(sm, base + poff(r * (L / Rs)), va[b * Rs + r], vb[b * Rs + r]);
                // twiddles exp(-+2 pi i k r / (Ns Rs)), k = j mod Ns, entries [k][0..Rs)
                const float4 *w4 = reinterpret_cast<const float4 *>(tws + (j % Ns) * TWROW);
                Cx w[Rs];
                twiddle_set<Rs>(w4, w);
#pragma unroll
                for (int r = 1; r < Rs; ++r) {
                    va[b * Rs + r] = INV ? cmulc(va[b * Rs + r], w[r]) : cmul(va[b * Rs + r], w[r]);
                    if constexpr (NOPS == 2) vb[b * Rs + r] = INV ? cmulc(vb[b * Rs + r], w[r]) : cmul(vb[b * Rs + r], w[r]);
                }
                dft<Rs, false, SS == S - 1>(va + b * Rs);
                if constexpr (NOPS == 2) dft<Rs, false, SS == S - 1>(vb + b * Rs);
            }
            __syncthreads();
            stage_rest<SS + 1>(va, vb, sm, tw);
        }
    }

    // In place: inputs v[b R0 + r] = row jb(b) + r (L / R0) on entry (rows
    // >= 2L/3 ignored with PIN), outputs v[b RL + r] = row jb(b) + r (L / RL)
    // on exit (with POUT only the kept r < 8, r >= 16).  tw: the per-stage
    // tables (pr_tw_offset).  Ends with a __syncthreads().
    __device__ __forceinline__ static void run(Cx *va, Cx *vb, Cx *sm, const Cx *__restrict__ tw)
    {
#pragma unroll
        for (int b = 0; b < VPT / R0; ++b) {
            dft<R0, true, S == 1>(va + b * R0);
            if constexpr (NOPS == 2) dft<R0, true, S == 1>(vb + b * R0);
        }
        stage_rest<1>(va, vb, sm, tw);
    }
};

}  // namespace lh
