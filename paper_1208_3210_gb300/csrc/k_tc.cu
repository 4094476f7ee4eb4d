// Tensor-core form of the inverse p_y pass (precision LINDHARD_SPLITBF16_TC).
//
// The same transform as k_inv_y / k_inv_y2 (Sec. 3: inverse Fourier transform
// of the product spectrum along p_y, keeping the Q lags q_y), with both DFT
// stages of a two-stage decomposition P = R1 * R2 run as dense matrix
// products on the fifth-generation tensor cores (tcgen05.mma, accumulators in
// tensor memory):
//
//   n = n1 + R1 n2,  m = m2 + R2 m1,
//   y(m) = sum_n1 e^{+2 pi i n1 m1 / R1} [ e^{+2 pi i n1 m2 / P}
//                 sum_n2 e^{+2 pi i n2 m2 / R2} x(n1 + R1 n2) ].
//
// Stage 1 is a product [C R1 lines x 2 R2] . [2 R2 x 2 R2]^T with the DFT of
// size R2 embedded as a real matrix (re/im interleaved along K and N); the
// twiddle e^{+2 pi i n1 m2 / P} is applied in FP32 registers between the
// stages; stage 2 is [C R2 lines x 2 R1] . [2 R1 x 2 R1]^T.  Operands are
// split into BF16 hi + lo parts (x = hi + lo to about 2^-16 relative) and
// each product takes three terms, hi.hi + lo.hi + hi.lo, accumulated in FP32
// in tensor memory.  The DFT matrices are built once per plan in FP64 and
// split on the device (k_tc_mats).
//
// Persistent CTAs walk tiles of C columns of one q_x plane; the TMA copies
// the next tile's P x C input into a shared-memory staging buffer while the
// current one is transformed.  Thread t owns line t of stage 1 (n1 = t / C,
// column t % C) and line t of stage 2 (m2 = t / C); tensor-memory lane =
// t % 128, row block t / 128 in its own columns.  One thread issues the MMAs
// (descriptors precomputed, loops unrolled) and commits them to an mbarrier;
// every wait is bounded (1 s of %globaltimer) and a CTA that gives up records
// DEV_ETIMEOUT, lets its copy in flight land, frees its tensor memory and
// returns.
#include "kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace lh {

// ---------------------------------------------------------------------------
// Decompositions P = R1 * R2 and columns per CTA (C R1 and C R2 multiples of
// 128, the M of one MMA; R1, R2 multiples of 8, so that 2 R is a multiple of
// the K = 16 of one instruction).
__host__ __device__ constexpr int tc_r1(int P)
{
    return P == 128 ? 8 : P == 192 ? 8 : P == 256 ? 16 : P == 384 ? 16 : P == 512 ? 16 : P == 768 ? 16 : P == 1024 ? 32
         : P == 1536 ? 32 : 0;
}
__host__ __device__ constexpr int tc_cols(int P)
{
    return P == 128 ? 16 : P == 192 ? 16 : P == 256 ? 8 : P == 384 ? 16 : P == 512 ? 8 : P == 768 ? 8 : P == 1024 ? 4
         : P == 1536 ? 8 : 0;
}
bool tc_supported(int P) { return tc_r1(P) != 0; }

// Shared memory of one persistent CTA: [staging P x C complex][A][B1 hi][B1 lo]
// [B2 hi][B2 lo][two mbarriers][tensor-memory address].  The TMA copies each
// tile's input into the staging buffer one tile ahead.  A holds one stage's
// operand, hi and lo parts side by side, or (SEQ, where both would not fit
// next to the staging buffer) one part at a time: the hi products first, then
// the lo part written over it.
template <int R1, int R2, int C, bool SEQ>
struct TcInvY {
    static constexpr int P = R1 * R2;
    static constexpr int ROWS1 = C * R1, ROWS2 = C * R2;
    static constexpr int NB1 = ROWS1 / 128, NB2 = ROWS2 / 128;
    static constexpr int T = 128 * (NB1 > NB2 ? NB1 : NB2);
    static constexpr int K1 = 2 * R2, K2 = 2 * R1;                    // K = N of each stage
    static constexpr int SBO1 = K1 / 8 * 128, SBO2 = K2 / 8 * 128;    // bytes per 8-row group
    static constexpr int ABYTES = ROWS1 * K1 * 2;                      // one part; = ROWS2 * K2 * 2
    static constexpr int B1BYTES = K1 * K1 * 2, B2BYTES = K2 * K2 * 2;
    static constexpr int NBOX = (P + 255) / 256, BOX = P / NBOX;       // TMA boxes of <= 256 rows
    static constexpr int STAGE = P * C * 8;
    static constexpr int OFF_A = STAGE, OFF_ALO = OFF_A + ABYTES;
    static constexpr int OFF_B1 = OFF_A + (SEQ ? 1 : 2) * ABYTES, OFF_B2 = OFF_B1 + 2 * B1BYTES;
    static constexpr int MAT_BYTES = 2 * B1BYTES + 2 * B2BYTES;
    static constexpr int OFF_BAR = OFF_B1 + MAT_BYTES;
    static constexpr int SMEM = OFF_BAR + 32;
    // stage-2 accumulators in their own columns: a tile's results are read
    // out while the next tile's stage-1 products run (and SEQ re-reads the
    // stage-1 accumulators for the lo part)
    static constexpr int D2COL = NB1 * K1;
    static constexpr int DCOLS = NB1 * K1 + NB2 * K2;
    static constexpr int COLS = DCOLS <= 32 ? 32 : DCOLS <= 64 ? 64 : DCOLS <= 128 ? 128 : DCOLS <= 256 ? 256 : 512;
    // CTAs per SM (up to 4) that shared memory (228 KB, 1 KB reserved per
    // CTA), tensor memory (512 columns) and the registers a thread keeps live
    // (2 max(R1, R2) values and addressing) admit
    static constexpr bool fits(int m)
    {
        return m * (SMEM + 1024) <= 228 * 1024 && m * COLS <= 512 && (2 * (R1 > R2 ? R1 : R2) + 32) * m * T <= 65536;
    }
    static constexpr int MINB = fits(4) ? 4 : fits(3) ? 3 : fits(2) ? 2 : 1;
    static_assert(ROWS1 % 128 == 0 && ROWS2 % 128 == 0, "stage rows must fill whole M = 128 blocks");
    static_assert(R1 % 8 == 0 && R2 % 8 == 0, "2 R must be a multiple of K = 16");
    static_assert(ROWS1 * K1 == ROWS2 * K2, "both stages hold C P complex values");
    static_assert(P % NBOX == 0 && (2 * C * 4) % 16 == 0, "whole TMA boxes of 16-byte rows");
    static_assert(DCOLS <= 512 && SMEM <= 227 * 1024, "tensor or shared memory");
};
// The plain layout where it fits, else SEQ
// (staging 8 C P + hi and lo operands 8 C P + matrices 16 (R1^2 + R2^2) bytes).
template <int R1, int R2, int C>
constexpr bool tc_seq() { return 16 * C * R1 * R2 + 16 * (R1 * R1 + R2 * R2) + 32 > 227 * 1024; }

// Byte offset of length P's matrices in the table built by k_tc_mats (the
// shared-memory image [B1 hi][B1 lo][B2 hi][B2 lo] of TcInvY).
__host__ __device__ constexpr int tc_mats_bytes_of(int P)
{
    return tc_r1(P) == 0 ? 0 : 16 * ((P / tc_r1(P)) * (P / tc_r1(P)) + tc_r1(P) * tc_r1(P));
}
__host__ __device__ constexpr int tc_mats_offset(int P)
{
    return P == 128 ? 0
         : P == 192 ? tc_mats_offset(128) + tc_mats_bytes_of(128)
         : P == 256 ? tc_mats_offset(192) + tc_mats_bytes_of(192)
         : P == 384 ? tc_mats_offset(256) + tc_mats_bytes_of(256)
         : P == 512 ? tc_mats_offset(384) + tc_mats_bytes_of(384)
         : P == 768 ? tc_mats_offset(512) + tc_mats_bytes_of(512)
         : P == 1024 ? tc_mats_offset(768) + tc_mats_bytes_of(768)
         : P == 1536 ? tc_mats_offset(1024) + tc_mats_bytes_of(1024)
         : tc_mats_offset(1536) + tc_mats_bytes_of(1536);   // total
}
size_t tc_mats_bytes() { return (size_t)tc_mats_offset(0); }

// The real embedding of the inverse DFT of size R, split into BF16 hi and lo:
// row 2m + o (output m, o = re/im), column 2r + i (input r, i = re/im) of
//   [[cos t, -sin t], [sin t, cos t]],  t = 2 pi r m / R,
// written as a K-major operand (tc_koff, sbo = 2R / 8 * 128).
__global__ void k_tc_mats(unsigned char *out)
{
    const int lens[8] = {128, 192, 256, 384, 512, 768, 1024, 1536};
    const int P = lens[blockIdx.y];
    const int R1 = tc_r1(P), R2 = P / R1;
    unsigned char *base = out + tc_mats_offset(P);
    const int e1 = 4 * R2 * R2, e2 = 4 * R1 * R1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < e1 + e2; i += gridDim.x * blockDim.x) {
        const bool st1 = i < e1;
        const int R = st1 ? R2 : R1, j = st1 ? i : i - e1;
        const int row = j / (2 * R), col = j % (2 * R);
        const int m = row / 2, o = row % 2, r = col / 2, ii = col % 2;
        double s, c;
        sincospi(2.0 * (double)((r * m) % R) / (double)R, &s, &c);
        const double v = (o == ii) ? c : (o == 0 ? -s : s);
        const __nv_bfloat16 hi = __double2bfloat16(v);
        const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        const int bytes = 4 * R * R * 2;                  // one matrix, hi or lo
        unsigned char *mat = base + (st1 ? 0 : 2 * (4 * R2 * R2 * 2));
        const unsigned off = tc_koff(row, col, 2 * R / 8 * 128);
        *reinterpret_cast<__nv_bfloat16 *>(mat + off) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(mat + bytes + off) = lo;
    }
}

cudaError_t launch_tc_mats(void *buf, cudaStream_t s)
{
    k_tc_mats<<<dim3(8, 8), 256, 0, s>>>(static_cast<unsigned char *>(buf));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Products of one stage (thread 0): for each 128-line block b,
//   MODE 0: D = A hi . B hi + A lo . B hi + A hi . B lo
//   MODE 1: D = A . B hi + A . B lo          (A holds the hi part)
//   MODE 2: D += A . B hi                    (A holds the lo part)
// Descriptors of one operand differ only in the start address (bits 0-13,
// address / 16), so each is its base descriptor plus a compile-time offset.
template <int NB, int K, int SBO, int ALO, int BLO, int MODE>
__device__ __forceinline__ void tc_stage_products(unsigned d, unsigned long long a0, unsigned long long b0)
{
    constexpr unsigned IDESC = tc_idesc_bf16(128, K);
    constexpr int NT = MODE == 0 ? 3 : MODE == 1 ? 2 : 1;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int term = 0; term < NT; ++term) {
            const int aoff = (MODE == 0 && term == 1) ? ALO : 0;
            const int boff = ((MODE == 0 && term == 2) || (MODE == 1 && term == 1)) ? BLO : 0;
#pragma unroll
            for (int ks = 0; ks < K / 16; ++ks)
                tc_mma(d + b * K, a0 + (unsigned long long)((aoff + b * 16 * SBO + ks * 256) >> 4),
                       b0 + (unsigned long long)((boff + ks * 256) >> 4), IDESC, MODE == 2 || term > 0 || ks > 0);
        }
}

// ---------------------------------------------------------------------------
// The pass.  U3 [Q][P][SP] (plane stride xs3) -> U4 [Q][Q][SP].  Persistent
// CTAs walk the tiles (C columns of one q_x plane); while a tile is on the
// tensor cores the TMA copies the next tile's P x C input into the staging
// buffer (issued as soon as the staged tile has been turned into operands).
template <int R1, int R2, int C, bool SEQ>
__global__ void __launch_bounds__(TcInvY<R1, R2, C, SEQ>::T, TcInvY<R1, R2, C, SEQ>::MINB)
k_inv_y_tc(Geom g, const __grid_constant__ CUtensorMap map, float2 *__restrict__ U4, const float2 *__restrict__ tw,
           const uint4 *__restrict__ mats, unsigned *status)
{
    using S = TcInvY<R1, R2, C, SEQ>;
    extern __shared__ __align__(1024) unsigned char smem[];
    if (dyn_smem_bytes() < (unsigned)S::SMEM) return;
    const float2 *stage = reinterpret_cast<const float2 *>(smem);
    unsigned char *A = smem + S::OFF_A;
    unsigned long long *bar_t = reinterpret_cast<unsigned long long *>(smem + S::OFF_BAR);
    unsigned long long *bar_m = bar_t + 1;
    unsigned *slot = reinterpret_cast<unsigned *>(smem + S::OFF_BAR + 16);
    const int t = threadIdx.x, warp = t >> 5, c = t % C;
    const unsigned long long dA1 = tc_desc(smem_addr(A), 128, S::SBO1), dA2 = tc_desc(smem_addr(A), 128, S::SBO2);
    const unsigned long long dB1 = tc_desc(smem_addr(smem + S::OFF_B1), 128, S::SBO1);
    const unsigned long long dB2 = tc_desc(smem_addr(smem + S::OFF_B2), 128, S::SBO2);
    const int tiles_x = (g.H + C - 1) / C, ntiles = tiles_x * g.Q;
    auto issue = [&](int tile) {
        const int lx = tile / tiles_x, c0 = (tile % tiles_x) * C;
        mbar_expect_tx(bar_t, (unsigned)S::STAGE);
        for (int q = 0; q < S::NBOX; ++q)
            tma_load_3d(smem + q * S::BOX * C * 8, &map, 2 * c0, q * S::BOX, lx, bar_t);
    };
    const TileRun run(ntiles, false);

    // both stages' DFT matrices: a straight copy of their shared-memory image
    for (int i = t; i < S::MAT_BYTES / 16; i += S::T) reinterpret_cast<uint4 *>(smem + S::OFF_B1)[i] = mats[i];
    if (t == 0) {
        mbar_init(bar_t, 1);
        mbar_init(bar_m, 1);
        if (run.t < run.end) issue(run.t);
    }
    if (warp == 0) tc_alloc(slot, S::COLS);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot;
    unsigned pt = 0, pm = 0;       // mbarrier phases
    bool inflight = run.t < run.end, ok = true;

    // generic smem writes of this thread -> visible to the tensor cores, CTA in step
    auto publish = [&]() {
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    };
    auto products_done = [&]() {
        ok = tile_ready(bar_m, pm, status);
        pm ^= 1u;
        tc_fence_after();
        return ok;
    };
    // stage-1 operand: line t = (n1, c) holds x(n1 + R1 n2), n2 < R2
    // (part 0: hi and lo side by side; 1: hi; 2: lo, in the A region)
    auto operand1 = [&](int part) {
        if (t < S::ROWS1) {
            const int n1 = t / C;
            float2 x[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) x[n2] = stage[(n1 + R1 * n2) * C + c];
            unsigned char *row = A + tc_koff(t, 0, S::SBO1);
#pragma unroll
            for (int j = 0; j < R2 / 4; ++j) {
                unsigned h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) bf16_split(x[4 * j + q], h[q], l[q]);
                if (part != 2) *reinterpret_cast<uint4 *>(row + j * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                if (part != 1)
                    *reinterpret_cast<uint4 *>(row + (part == 0 ? S::ABYTES : 0) + j * 128) =
                        make_uint4(l[0], l[1], l[2], l[3]);
            }
        }
    };
    // stage-2 operand from the stage-1 accumulators: twiddle e^{+2 pi i n1 m2 / P}
    // in FP32, split, scatter to line (m2, c) = m2 C + c at K position 2 n1.
    // The twiddles are powers of w = e^{-2 pi i n1 / P}: read from the table
    // every 8th power and advanced by one complex product in between (at
    // most 7 roundings, about 1e-6, well below the BF16 split's 2^-16), so
    // that a tile waits on 3 table reads per line instead of R2 - 1.
    auto operand2 = [&](int part) {
        if (t < S::ROWS1) {
            const int n1 = t / C, b = warp / 4;
            const float2 w1 = __ldg(&tw[n1]);
            float d[S::K1];
            tc_ld<S::K1>(tmem + ((unsigned)((warp % 4) * 32) << 16) + (unsigned)(b * S::K1), d);
            float2 wp = make_float2(1.f, 0.f);
#pragma unroll
            for (int m2 = 0; m2 < R2; ++m2) {
                float2 z = make_float2(d[2 * m2], d[2 * m2 + 1]);
                if (m2 > 0) {
                    wp = (m2 % 8 == 0) ? __ldg(&tw[n1 * m2]) : cmul(wp, w1);
                    z = cmulc(z, wp);
                }
                unsigned h, l;
                bf16_split(z, h, l);
                const unsigned off = tc_koff(m2 * C + c, 2 * n1, S::SBO2);
                if (part != 2) *reinterpret_cast<unsigned *>(A + off) = h;
                if (part != 1) *reinterpret_cast<unsigned *>(A + (part == 0 ? S::ABYTES : 0) + off) = l;
            }
        }
    };

    // outputs y(m2 + R2 m1), m1 < R1, of line (m2, c) of a finished tile; keep the Q lags
    auto outputs = [&](int tile) {
        const int lx = tile / tiles_x, c0 = (tile % tiles_x) * C;
        if (t < S::ROWS2) {
            const int m2 = t / C, b = warp / 4;
            float d[S::K2];
            tc_ld<S::K2>(tmem + ((unsigned)((warp % 4) * 32) << 16) + (unsigned)(S::D2COL + b * S::K2), d);
            if (c0 + c < g.H) {
                float2 *dst = U4 + (long long)lx * g.Q * g.SP + c0 + c;
#pragma unroll
                for (int m1 = 0; m1 < R1; ++m1) {
                    const int l = lag_index(m2 + R2 * m1, S::P, g.Q);
                    if (l >= 0) __stcs(dst + (long long)l * g.SP, make_float2(d[2 * m1], d[2 * m1 + 1]));
                }
            }
        }
        tc_fence_before();
    };

    int prev = -1;   // tile whose stage-2 results wait in tensor memory
    for (int tile = run.t; tile < run.end; tile += run.step) {
        if (!tile_ready(bar_t, pt, status)) { ok = false; break; }
        pt ^= 1u;
        inflight = false;
        const bool more = tile + run.step < run.end;
        // stage 1
        operand1(SEQ ? 1 : 0);
        publish();
        if (t == 0) {
            if (!SEQ && more) { issue(tile + run.step); }
            tc_stage_products<S::NB1, S::K1, S::SBO1, S::ABYTES, S::B1BYTES, SEQ ? 1 : 0>(tmem, dA1, dB1);
            tc_commit(bar_m);
        }
        if (!SEQ) inflight = more;
        // the previous tile's results leave while these products run
        if (prev >= 0) outputs(prev);
        prev = -1;
        if (!products_done()) break;
        if constexpr (SEQ) {
            operand1(2);
            publish();
            if (t == 0) {
                if (more) issue(tile + run.step);
                tc_stage_products<S::NB1, S::K1, S::SBO1, S::ABYTES, S::B1BYTES, 2>(tmem, dA1, dB1);
                tc_commit(bar_m);
            }
            inflight = more;
            if (!products_done()) break;
        }
        // stage 2
        operand2(SEQ ? 1 : 0);
        publish();
        if (t == 0) {
            tc_stage_products<S::NB2, S::K2, S::SBO2, S::ABYTES, S::B2BYTES, SEQ ? 1 : 0>(tmem + S::D2COL, dA2, dB2);
            tc_commit(bar_m);
        }
        if (!products_done()) break;
        if constexpr (SEQ) {
            operand2(2);
            publish();
            if (t == 0) {
                tc_stage_products<S::NB2, S::K2, S::SBO2, S::ABYTES, S::B2BYTES, 2>(tmem + S::D2COL, dA2, dB2);
                tc_commit(bar_m);
            }
            if (!products_done()) break;
        }
        prev = tile;
    }
    if (ok && prev >= 0) outputs(prev);
    // a copy still in flight after a timeout lands before the CTA leaves
    if (!ok && inflight) drain(bar_t, pt);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, S::COLS);
}

template <int P>
cudaError_t launch_inv_y_tc_t(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    constexpr int R1 = tc_r1(P), R2 = P / R1, C = tc_cols(P);
    constexpr bool SEQ = tc_seq<R1, R2, C>();
    using S = TcInvY<R1, R2, C, SEQ>;
    auto k = k_inv_y_tc<R1, R2, C, SEQ>;
    static const cudaError_t e0 = smem_attrs(k, (size_t)S::SMEM);
    if (e0 != cudaSuccess) return e0;
    if (w.tc == nullptr) return cudaErrorInvalidValue;
    CUtensorMap map;
    cudaError_t e = make_map(&map, w.X, 2ull * g.SP, (unsigned long long)P, (unsigned long long)g.Q, 8ull * g.SP,
                             8ull * (unsigned long long)g.xs3, 2 * C, S::BOX, 1);
    int grid = 0;
    const int ntiles = ((g.H + C - 1) / C) * g.Q;
    // one CTA per SM per MINB: the residency the tile was sized for (shared,
    // tensor memory and registers; the occupancy query reports one CTA less
    // for these kernels on this part)
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = std::min(ntiles, sms * S::MINB);
    }
    if (e != cudaSuccess) return e;
    k<<<grid, S::T, S::SMEM, s>>>(g, map, (float2 *)w.Y, twiddles_for<float>(w, P),
                                 reinterpret_cast<const uint4 *>(static_cast<const unsigned char *>(w.tc) +
                                                                 tc_mats_offset(P)),
                                 w.status);
    return cudaGetLastError();
}

cudaError_t launch_inv_y_tc(const Geom &g, const Work<float> &w, cudaStream_t s)
{
    switch (g.P) {
    case 128: return launch_inv_y_tc_t<128>(g, w, s);
    case 192: return launch_inv_y_tc_t<192>(g, w, s);
    case 256: return launch_inv_y_tc_t<256>(g, w, s);
    case 384: return launch_inv_y_tc_t<384>(g, w, s);
    case 512: return launch_inv_y_tc_t<512>(g, w, s);
    case 768: return launch_inv_y_tc_t<768>(g, w, s);
    case 1024: return launch_inv_y_tc_t<1024>(g, w, s);
    case 1536: return launch_inv_y_tc_t<1536>(g, w, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lh
