// Real part of the Lindhard susceptibility by the Kramers-Kronig relation and
// the RPA susceptibility (Sec. 4: "the real part of the Lindhard
// susceptibility ... by applying Kramers-Kronig relation";
// chi_RPA = chi_L / (1 - V_q chi_L) with V_q decaying as 1 / q^2).
//
// For every lag q the transfers w_m = m de, m < n_omega, carry Im chi; with
// Im chi odd in w (chi(-q) = chi(q) for the inversion-symmetric bands of this
// problem) and zero beyond the computed window, Maclaurin's rule for the
// principal value gives a dense linear map along w:
//
//   Re chi_m = sum_k W(m, k) Im chi_k,  W(m, k) = (4/pi) k / (k^2 - m^2)
//              for k >= 1 with k - m odd, 0 otherwise.
//
// Split by parity, the even outputs take the odd inputs and the odd outputs
// the even inputs: two products [lines x n_omega/2] . [n_omega/2 x n_omega/2]^T.
//
//   k_kk_tc   : the far field |k - m| >= 8 on the tensor cores (tcgen05,
//               BF16 hi + lo operands, three products, FP32 accumulation in
//               tensor memory, 128 lines per block), the near band
//               |k - m| < 8 (the largest weights, where a BF16 split would
//               cost most of the accuracy) in FP32 in the epilogue, then
//               chi_RPA.  n_omega <= 256.
//   k_kk_simt : the whole sum in FP32 SIMT (every weight from an FP32 table),
//               then chi_RPA.  n_omega <= 1536.
//
// V_q = v0 / |q|^2 at q = ((l_x - Q/2) dp, (l_y - Q/2) dp); at q = 0 chi_RPA
// takes its limit 0 (v0 = 0: chi_RPA = chi everywhere).  The weight tables
// are built once per plan in FP64 (k_kk_tables).
#include "kernels.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace lh {

constexpr int KK_BAND = 8;        // |k - m| < KK_BAND: near band, FP32
constexpr int KK_MAX_TC = 256;    // longest n_omega of the tensor-core form
constexpr int KK_MAX_SIMT = 1536;

// padded half width of the tensor-core operands (a multiple of the MMA's K = 16)
__host__ __device__ constexpr int kk_kp(int nw)
{
    return (nw + 1) / 2 <= 16 ? 16 : (nw + 1) / 2 <= 32 ? 32 : (nw + 1) / 2 <= 64 ? 64 : 128;
}
// Weight table of one n_omega: [tensor-core Be hi][Be lo][Bo hi][Bo lo] (BF16,
// K-major operands of KP x KP, n_omega <= 256 only), [near band: n_omega x 8
// FP32], [SIMT: ceil(n_omega / 2) x n_omega FP32].  Byte offsets:
__host__ __device__ constexpr size_t kk_tc_bytes(int nw) { return nw <= KK_MAX_TC ? 8ull * kk_kp(nw) * kk_kp(nw) : 0; }
__host__ __device__ constexpr size_t kk_band_off(int nw) { return kk_tc_bytes(nw); }
__host__ __device__ constexpr size_t kk_simt_off(int nw) { return kk_band_off(nw) + 32ull * nw; }
size_t kk_table_bytes(int nw) { return kk_simt_off(nw) + 4ull * ((nw + 1) / 2) * nw; }

__host__ __device__ inline double kk_weight(int m, int k, int nw)
{
    if (k < 1 || k >= nw || m >= nw || ((k - m) & 1) == 0) return 0.0;
    return 4.0 / 3.14159265358979323846 * (double)k / ((double)k * k - (double)m * m);
}

__global__ void k_kk_tables(int nw, unsigned char *tab)
{
    const int KP = kk_kp(nw), H = (nw + 1) / 2;
    const long long n_tc = nw <= KK_MAX_TC ? 2LL * KP * KP : 0, n_band = 8LL * nw, n_simt = (long long)H * nw;
    const int sbo = KP / 8 * 128;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_tc + n_band + n_simt;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n_tc) {
            // Be (p = 0): output m = 2r, input k = 2c + 1; Bo (p = 1): m = 2r + 1, k = 2c
            const int p = (int)(i / ((long long)KP * KP)), e = (int)(i % ((long long)KP * KP));
            const int r = e / KP, c = e % KP;
            const int m = 2 * r + p, k = 2 * c + 1 - p;
            const double w = (abs(k - m) >= KK_BAND) ? kk_weight(m, k, nw) : 0.0;
            const __nv_bfloat16 hi = __double2bfloat16(w);
            const __nv_bfloat16 lo = __double2bfloat16(w - (double)__bfloat162float(hi));
            unsigned char *mat = tab + (size_t)p * 4 * KP * KP;
            const unsigned off = tc_koff(r, c, sbo);
            *reinterpret_cast<__nv_bfloat16 *>(mat + off) = hi;
            *reinterpret_cast<__nv_bfloat16 *>(mat + 2 * KP * KP + off) = lo;
        } else if (i < n_tc + n_band) {
            const int e = (int)(i - n_tc), m = e / 8, d = e % 8;
            reinterpret_cast<float *>(tab + kk_band_off(nw))[e] = (float)kk_weight(m, m + 2 * d - (KK_BAND - 1), nw);
        } else {
            const int e = (int)(i - n_tc - n_band), j = e / nw, m = e % nw;
            reinterpret_cast<float *>(tab + kk_simt_off(nw))[e] = (float)kk_weight(m, 2 * j + 1 - (m & 1), nw);
        }
    }
}

cudaError_t launch_kk_tables(int nw, void *tab, cudaStream_t s)
{
    k_kk_tables<<<64, 256, 0, s>>>(nw, static_cast<unsigned char *>(tab));
    return cudaGetLastError();
}

// chi_RPA from chi = (r, x) at one transfer; V = 0 returns chi unchanged.
// The reciprocal of |1 - V chi|^2 is the hardware approximation (2 ulp),
// far inside the FP32 bar of chi_RPA.
__device__ __forceinline__ float2 kk_rpa(float r, float x, float V, bool zero)
{
    if (zero) return make_float2(0.f, 0.f);
    const float dr = 1.f - V * r, di = -V * x;
    const float inv = __fdividef(1.f, dr * dr + di * di);
    return make_float2((r * dr + x * di) * inv, (x * dr - r * di) * inv);
}
// V_q of lag line l = l_x Q + l_y; *zero when q = 0 with an interaction
__device__ __forceinline__ float kk_vq(long long l, int Q, double dp, double v0, bool *zero)
{
    const double qx = (double)(l / Q - Q / 2) * dp, qy = (double)(l % Q - Q / 2) * dp, q2 = qx * qx + qy * qy;
    *zero = (q2 == 0.0 && v0 != 0.0);
    return (v0 == 0.0 || q2 == 0.0) ? 0.f : (float)(v0 / q2);
}

// ---------------------------------------------------------------------------
// Tensor-core form.  One CTA of 256 threads per block of 128 lines (persistent
// over blocks).  Shared memory: [work][Be hi][Be lo][Bo hi][Bo lo][mbarrier]
// [tensor-memory address]; the work region holds one parity's operand (hi,
// lo: 128 lines x KP) while the products run, then the epilogue's chunks.
//   operand: each warp reads whole rows of Im chi (32 consecutive transfers
//            per load, coalesced) and pairs neighbouring elements of one
//            parity with a shuffle before the BF16 split;
//   epilogue, per chunk of 32 transfers: the accumulators of the 128 lines go
//            to shared memory (transposed), the chunk's Im chi with a halo
//            of 8 is loaded row by row, and the lanes run along the
//            transfers for the near band, chi_RPA and the stores (coalesced).
// The next block's rows are prefetched into L2 (cp.async.bulk.prefetch).
template <int KP>
struct KkTc {
    static constexpr int T = 256, CH = 32, HALO = 8;
    static constexpr int SBO = KP / 8 * 128;
    static constexpr int ABYTES = 128 * KP * 2, BBYTES = KP * KP * 2;
    static constexpr int RE_LD = CH + 1, IM_LD = CH + 2 * HALO + 1;       // padded rows of the epilogue tiles
    static constexpr int EPI = 128 * (RE_LD + IM_LD + 1) * 4;       // + V_q of each line
    // both parities' operands side by side when they fit beside two CTAs per SM
    static constexpr bool BOTH = KP <= 64;
    static constexpr int AREG = (BOTH ? 4 : 2) * ABYTES;
    static constexpr int WORK = AREG > EPI ? AREG : EPI;
    static constexpr int OFF_B = (WORK + 1023) / 1024 * 1024, OFF_BAR = OFF_B + 4 * BBYTES;
    static constexpr int SMEM = OFF_BAR + 16;
    static constexpr int COLS = 2 * KP <= 32 ? 32 : 2 * KP <= 64 ? 64 : 2 * KP <= 128 ? 128 : 256;
    static constexpr bool fits(int m) { return m * (SMEM + 1024) <= 228 * 1024 && m * COLS <= 512 && m * T * 128 <= 65536; }
    static constexpr int MINB = fits(2) ? 2 : 1;
};

__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int KP>
__global__ void __launch_bounds__(256, KkTc<KP>::MINB)
k_kk_tc(long long nlines, int nw, int Q, double dp, double v0, const float *__restrict__ im, float *__restrict__ re,
        float2 *__restrict__ rpa, const uint4 *__restrict__ mats, const float *__restrict__ band,
        unsigned *status)
{
    using S = KkTc<KP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    if (dyn_smem_bytes() < (unsigned)S::SMEM) return;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + S::OFF_BAR);
    unsigned *slot = reinterpret_cast<unsigned *>(smem + S::OFF_BAR + 8);
    float *reT = reinterpret_cast<float *>(smem);                    // [128][RE_LD]
    float *imS = reT + 128 * S::RE_LD;                               // [128][IM_LD]
    float *vS = imS + 128 * S::IM_LD;                                // [128] V_q (NaN: chi_RPA = 0)
    const int t = threadIdx.x, warp = t >> 5, ln = t & 31;
    constexpr unsigned IDESC = tc_idesc_bf16(128, KP);

    for (int i = t; i < 4 * S::BBYTES / 16; i += S::T) reinterpret_cast<uint4 *>(smem + S::OFF_B)[i] = mats[i];
    if (t == 0) mbar_init(bar, 1);
    if (warp == 0) tc_alloc(slot, S::COLS);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot;
    const unsigned long long dA = tc_desc(smem_addr(smem), 128, S::SBO);
    const unsigned long long dB = tc_desc(smem_addr(smem + S::OFF_B), 128, S::SBO);
    const unsigned lane = (unsigned)((warp % 4) * 32) << 16;
    unsigned pm = 0;
    bool ok = true;
    // near-band weights of this lane's transfer in each chunk are loaded per chunk
    const long long nblk = (nlines + 127) / 128;
    auto prefetch = [&](long long blk) {
        if (blk >= nblk) return;
        const long long l0 = blk * 128, nl = min(128LL, nlines - l0);
        // the 16-byte aligned part of the block's rows (the instance's block may
        // start anywhere in the caller's output)
        const unsigned long long a = reinterpret_cast<unsigned long long>(im + l0 * nw);
        const unsigned long long b = a + (unsigned long long)(nl * nw) * 4ull;
        const unsigned long long a16 = (a + 15) & ~15ull, b16 = b & ~15ull;
        if (b16 > a16) prefetch_l2(reinterpret_cast<const void *>(a16), (unsigned)(b16 - a16));
    };
    if (t == 0) prefetch(blockIdx.x);

    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long l0 = blk * 128;
        if (t == 0) prefetch(blk + gridDim.x);
        // p = 0: even outputs from the odd inputs (Be); p = 1: odd outputs from the even inputs (Bo)
        // Operand of parity p (its hi part at aoff(p), lo at aoff(p) + ABYTES):
        // element j of a row is x(2j + 1 - p); lane k of a 32-transfer load pairs
        // with lane k + 2 (element j + 1), and lanes with (k - (1 - p)) % 4 == 0
        // store.  The warp's 16 rows are loaded back to back (16 loads in flight
        // per lane).  BOTH: one pass over the rows builds both parities.
        auto aoff = [](int p) { return S::BOTH ? 2 * p * S::ABYTES : 0; };
        auto build = [&](int p0, int p1) {
#pragma unroll 1
            for (int c = 0; c < KP / 16; ++c) {
                const int k = 32 * c + ln;
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const long long line = l0 + warp * 16 + i;
                    v[i] = (line < nlines && k < nw) ? __ldg(im + line * nw + k) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float w = __shfl_down_sync(0xffffffffu, v[i], 2);
                    for (int p = p0; p <= p1; ++p)
                        if (((ln - (1 - p)) & 3) == 0) {
                            unsigned h, l;
                            bf16_split(make_float2(v[i], w), h, l);
                            const unsigned off = aoff(p) + tc_koff(warp * 16 + i, (k - (1 - p)) >> 1, S::SBO);
                            *reinterpret_cast<unsigned *>(smem + off) = h;
                            *reinterpret_cast<unsigned *>(smem + S::ABYTES + off) = l;
                        }
                }
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        };
        // products of parity p into accumulator columns p KP (thread 0)
        auto products = [&](int p) {
            const unsigned long long a0 = dA + (unsigned long long)(aoff(p) >> 4);
            const unsigned long long b0 = dB + (unsigned long long)((2 * p * S::BBYTES) >> 4);
#pragma unroll
            for (int term = 0; term < 3; ++term) {
                const unsigned long long a = a0 + (unsigned long long)(((term == 1) ? S::ABYTES : 0) >> 4);
                const unsigned long long b = b0 + (unsigned long long)(((term == 2) ? S::BBYTES : 0) >> 4);
#pragma unroll
                for (int ks = 0; ks < KP / 16; ++ks)
                    tc_mma(tmem + p * KP, a + (unsigned long long)((ks * 256) >> 4),
                           b + (unsigned long long)((ks * 256) >> 4), IDESC, term > 0 || ks > 0);
            }
        };
        if constexpr (S::BOTH) {
            build(0, 1);
            if (t == 0) {
                products(0);
                products(1);
                tc_commit(bar);
            }
            ok = tile_ready(bar, pm, status);
            pm ^= 1u;
            tc_fence_after();
        } else {
            for (int p = 0; p < 2 && ok; ++p) {
                build(p, p);
                if (t == 0) {
                    products(p);
                    tc_commit(bar);
                }
                ok = tile_ready(bar, pm, status);
                pm ^= 1u;
                tc_fence_after();
            }
        }
        if (!ok) break;
        // epilogue, chunks of 32 transfers m0 .. m0 + 31
#pragma unroll 1
        for (int m0 = 0; m0 < nw; m0 += S::CH) {
            {   // accumulators -> reT[line][q]: warps 0-3 the even transfers, 4-7 the odd ones
                float d[16];
                tc_ld<16>(tmem + lane + (unsigned)((warp < 4 ? 0 : KP) + m0 / 2), d);
                const int li = (warp % 4) * 32 + ln;
#pragma unroll
                for (int q = 0; q < 16; ++q) reT[li * S::RE_LD + 2 * q + (warp < 4 ? 0 : 1)] = d[q];
            }
            if (m0 == 0 && t < 128) {    // V_q of the block's lines, once (an FP64 division each)
                bool zero;
                const float V = kk_vq(l0 + t, Q, dp, v0, &zero);
                vS[t] = zero ? __int_as_float(0x7fc00000) : V;
            }
            {   // Im chi of the chunk with a halo of 8 on each side: the warp's 16 rows,
                // all loads issued before the first store
                const int k0 = m0 - S::HALO + ln, k1 = k0 + 32;
                float a[16], b[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const long long line = l0 + warp * 16 + i;
                    const float *row = im + line * nw;
                    a[i] = (line < nlines && k0 >= 0 && k0 < nw) ? __ldg(row + k0) : 0.f;
                    b[i] = (line < nlines && ln < 2 * S::HALO && k1 < nw) ? __ldg(row + k1) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    imS[(warp * 16 + i) * S::IM_LD + ln] = a[i];
                    if (ln < 2 * S::HALO) imS[(warp * 16 + i) * S::IM_LD + 32 + ln] = b[i];
                }
            }
            __syncthreads();
            // lanes along the transfers: near band in FP32, Re chi, chi_RPA, coalesced stores
            const int m = m0 + ln;
            float wb[KK_BAND];
#pragma unroll
            for (int d = 0; d < KK_BAND; ++d) wb[d] = (m < nw) ? __ldg(band + m * KK_BAND + d) : 0.f;
            if (m < nw) {
                const int nli = (int)min(16LL, nlines - (l0 + warp * 16));   // lines of this warp in range
                float *ro = re + (l0 + warp * 16) * nw + m;
                float2 *po = rpa ? rpa + (l0 + warp * 16) * nw + m : nullptr;
#pragma unroll 4
                for (int i = 0; i < nli; ++i) {
                    const int li = warp * 16 + i;
                    const float *xs = imS + li * S::IM_LD + ln + S::HALO;     // xs[o] = Im chi(m + o)
                    float r = reT[li * S::RE_LD + ln];
#pragma unroll
                    for (int d = 0; d < KK_BAND; ++d) r = fmaf(wb[d], xs[2 * d - (KK_BAND - 1)], r);
                    ro[(size_t)i * nw] = r;
                    if (po) {
                        const float V = vS[li];
                        po[(size_t)i * nw] = kk_rpa(r, xs[0], isnan(V) ? 0.f : V, isnan(V));
                    }
                }
            }
            __syncthreads();
        }
        tc_fence_before();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, S::COLS);
}

// ---------------------------------------------------------------------------
// FP32 SIMT form: LB lines per CTA of 256 threads staged in shared memory
// (rows padded with one zero to nw + 1 floats), V_q per line beside them.
// Warp w takes lines w LPW .. w LPW + LPW - 1 and its lanes run along the
// transfers: each weight W(m, k) is read once per warp step (coalesced) and
// applied to the warp's LPW lines from registers; stores are coalesced.
constexpr int KK_SIMT_LPW = 8;
__host__ __device__ constexpr int kk_simt_lines(int nw)
{
    // 8 warps x up to 8 lines, at most ~96 KB of rows (two CTAs per SM)
    return (96 * 1024) / (4 * (nw + 1)) >= 64 ? 64 : ((96 * 1024) / (4 * (nw + 1))) / 8 * 8 < 8 ? 8
         : ((96 * 1024) / (4 * (nw + 1))) / 8 * 8;
}

__global__ void __launch_bounds__(256)
k_kk_simt(long long nlines, int nw, int Q, double dp, double v0, const float *__restrict__ im, float *__restrict__ re,
          float2 *__restrict__ rpa, const float *__restrict__ hs, int LB)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *rows = reinterpret_cast<float *>(smem_raw);          // [LB][nw + 1]
    float *vS = rows + LB * (nw + 1);                           // [LB] V_q (NaN: chi_RPA = 0)
    if (dyn_smem_bytes() < (unsigned)((LB * (nw + 1) + LB) * 4)) return;
    const long long l0 = (long long)blockIdx.x * LB;
#pragma unroll 8
    for (int i = threadIdx.x; i < LB * (nw + 1); i += blockDim.x) {
        const int l = i / (nw + 1), k = i % (nw + 1);
        rows[i] = (k < nw && l0 + l < nlines) ? im[(l0 + l) * nw + k] : 0.f;
    }
    if (threadIdx.x < LB) {
        bool zero;
        const float V = kk_vq(l0 + threadIdx.x, Q, dp, v0, &zero);
        vS[threadIdx.x] = zero ? __int_as_float(0x7fc00000) : V;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31, lpw = LB / 8;
    const int H = (nw + 1) / 2;
    for (int m0 = 0; m0 < nw; m0 += 32) {
        const int m = m0 + ln, k0 = 1 - (m & 1);
        float s[KK_SIMT_LPW];
#pragma unroll
        for (int i = 0; i < KK_SIMT_LPW; ++i) s[i] = 0.f;
#pragma unroll 4
        for (int j = 0; j < H; ++j) {
            const float h = (m < nw) ? __ldg(hs + (size_t)j * nw + m) : 0.f;
            const int k = 2 * j + k0;                           // <= nw: the padding zero
#pragma unroll
            for (int i = 0; i < KK_SIMT_LPW; ++i)
                if (i < lpw) s[i] = fmaf(h, rows[(warp * lpw + i) * (nw + 1) + k], s[i]);
        }
        if (m < nw) {
#pragma unroll
            for (int i = 0; i < KK_SIMT_LPW; ++i) {
                const int l = warp * lpw + i;
                if (i >= lpw || l0 + l >= nlines) continue;
                re[(l0 + l) * nw + m] = s[i];
                if (rpa) {
                    const float V = vS[l];
                    rpa[(l0 + l) * nw + m] = kk_rpa(s[i], rows[l * (nw + 1) + m], isnan(V) ? 0.f : V, isnan(V));
                }
            }
        }
    }
}

// variant 0: tensor cores (n_omega <= 256); 1: FP32 SIMT (n_omega <= 1536)
template <int KP>
static cudaError_t launch_kk_tc_t(const Geom &g, const float *im, float *re, float2 *rpa, const void *tab,
                                  double v0, unsigned *status, cudaStream_t s)
{
    using S = KkTc<KP>;
    auto k = k_kk_tc<KP>;
    static const cudaError_t e0 = smem_attrs(k, (size_t)S::SMEM);
    if (e0 != cudaSuccess) return e0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long nlines = (long long)g.Q * g.Q, nblk = (nlines + 127) / 128;
    const int grid = (int)std::min<long long>(nblk, (long long)sms * S::MINB);
    const unsigned char *t8 = static_cast<const unsigned char *>(tab);
    k<<<grid, S::T, S::SMEM, s>>>(nlines, g.n_omega, g.Q, g.dp, v0, im, re, rpa, reinterpret_cast<const uint4 *>(t8),
                                  reinterpret_cast<const float *>(t8 + kk_band_off(g.n_omega)), status);
    return cudaGetLastError();
}

cudaError_t launch_kk_rpa(const Geom &g, const float *im, float *re, float2 *rpa, const void *tab, double v0,
                          int variant, unsigned *status, cudaStream_t s)
{
    const int nw = g.n_omega;
    if (variant == 0) {
        if (nw > KK_MAX_TC) return cudaErrorNotSupported;
        switch (kk_kp(nw)) {
        case 16: return launch_kk_tc_t<16>(g, im, re, rpa, tab, v0, status, s);
        case 32: return launch_kk_tc_t<32>(g, im, re, rpa, tab, v0, status, s);
        case 64: return launch_kk_tc_t<64>(g, im, re, rpa, tab, v0, status, s);
        default: return launch_kk_tc_t<128>(g, im, re, rpa, tab, v0, status, s);
        }
    }
    if (variant != 1 || nw > KK_MAX_SIMT) return cudaErrorNotSupported;
    const int LB = kk_simt_lines(nw);
    const size_t smem = (size_t)(LB * (nw + 1) + LB) * 4;
    static const cudaError_t e0 = smem_attrs(k_kk_simt, 100 * 1024);
    if (e0 != cudaSuccess) return e0;
    const long long nlines = (long long)g.Q * g.Q;
    const int grid = (int)((nlines + LB - 1) / LB);
    k_kk_simt<<<grid, 256, smem, s>>>(nlines, nw, g.Q, g.dp, v0, im, re, rpa,
                                     reinterpret_cast<const float *>(static_cast<const unsigned char *>(tab) +
                                                                     kk_simt_off(nw)),
                                     LB);
    return cudaGetLastError();
}

}  // namespace lh
