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
__device__ __forceinline__ float2 kk_rpa(float r, float x, float V, bool zero)
{
    if (zero) return make_float2(0.f, 0.f);
    const float dr = 1.f - V * r, di = -V * x;
    const float inv = 1.f / (dr * dr + di * di);
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
// Tensor-core form.  Shared memory: [A hi][A lo] (one parity's operand, 128
// lines x KP) [Be hi][Be lo][Bo hi][Bo lo] [mbarrier][tensor-memory address].
template <int KP>
struct KkTc {
    static constexpr int T = 128;
    static constexpr int SBO = KP / 8 * 128;
    static constexpr int ABYTES = 128 * KP * 2, BBYTES = KP * KP * 2;
    static constexpr int OFF_B = 2 * ABYTES, OFF_BAR = OFF_B + 4 * BBYTES;
    static constexpr int SMEM = OFF_BAR + 16;
    static constexpr int COLS = 2 * KP <= 32 ? 32 : 2 * KP <= 64 ? 64 : 2 * KP <= 128 ? 128 : 256;
    static constexpr bool fits(int m) { return m * (SMEM + 1024) <= 228 * 1024 && m * COLS <= 512 && m * T * 168 <= 65536; }
    static constexpr int MINB = fits(3) ? 3 : fits(2) ? 2 : 1;
};

template <int KP>
__global__ void __launch_bounds__(128, KkTc<KP>::MINB)
k_kk_tc(long long nlines, int nw, int Q, double dp, double v0, const float *__restrict__ im, float *__restrict__ re,
        float2 *__restrict__ rpa, const uint4 *__restrict__ mats, const float *__restrict__ band,
        unsigned *status)
{
    using S = KkTc<KP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    if (dyn_smem_bytes() < (unsigned)S::SMEM) return;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + S::OFF_BAR);
    unsigned *slot = reinterpret_cast<unsigned *>(smem + S::OFF_BAR + 8);
    const int t = threadIdx.x, warp = t >> 5;
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

    const long long nblk = (nlines + 127) / 128;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long line = blk * 128 + t;
        const bool valid = line < nlines;
        const float *row = im + line * nw;
        // p = 0: even outputs from the odd inputs (Be); p = 1: odd outputs from the even inputs (Bo)
        for (int p = 0; p < 2 && ok; ++p) {
            // operand row t: element j is x(2j + 1 - p); one 16-byte chunk holds j..j+7
            unsigned char *arow = smem + tc_koff(t, 0, S::SBO);
#pragma unroll 1
            for (int j8 = 0; j8 < KP / 8; ++j8) {
                unsigned h[4], l[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k0 = 2 * (8 * j8 + 2 * q) + 1 - p, k1 = k0 + 2;
                    const float2 x = make_float2(valid && k0 < nw ? __ldg(row + k0) : 0.f,
                                                 valid && k1 < nw ? __ldg(row + k1) : 0.f);
                    bf16_split(x, h[q], l[q]);
                }
                *reinterpret_cast<uint4 *>(arow + j8 * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4 *>(arow + S::ABYTES + j8 * 128) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (t == 0) {
                const unsigned long long b0 = dB + (unsigned long long)((2 * p * S::BBYTES) >> 4);
#pragma unroll
                for (int term = 0; term < 3; ++term) {
                    const unsigned long long a = dA + (unsigned long long)(((term == 1) ? S::ABYTES : 0) >> 4);
                    const unsigned long long b = b0 + (unsigned long long)(((term == 2) ? S::BBYTES : 0) >> 4);
#pragma unroll
                    for (int ks = 0; ks < KP / 16; ++ks)
                        tc_mma(tmem + p * KP, a + (unsigned long long)((ks * 256) >> 4),
                               b + (unsigned long long)((ks * 256) >> 4), IDESC, term > 0 || ks > 0);
                }
                tc_commit(bar);
            }
            ok = tile_ready(bar, pm, status);
            pm ^= 1u;
            tc_fence_after();
        }
        if (!ok) break;
        // epilogue: far field from tensor memory + near band in FP32, Re chi and chi_RPA
        bool zero;
        const float V = kk_vq(line, Q, dp, v0, &zero);
#pragma unroll 1
        for (int i0 = 0; i0 < KP; i0 += 16) {
            float de[16], dq[16];
            tc_ld<16>(tmem + lane + (unsigned)i0, de);        // m = 2 (i0 + q)
            tc_ld<16>(tmem + lane + (unsigned)(KP + i0), dq); // m = 2 (i0 + q) + 1
            if (valid) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int m = 2 * i0 + q;
                    if (m >= nw) break;
                    float r = (q & 1) ? dq[q >> 1] : de[q >> 1];
#pragma unroll
                    for (int d = 0; d < KK_BAND; ++d) {
                        const int k = m + 2 * d - (KK_BAND - 1);
                        if (k >= 1 && k < nw) r = fmaf(__ldg(band + m * KK_BAND + d), __ldg(row + k), r);
                    }
                    re[line * nw + m] = r;
                    if (rpa) rpa[line * nw + m] = kk_rpa(r, __ldg(row + m), V, zero);
                }
            }
        }
        tc_fence_before();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, S::COLS);
}

// ---------------------------------------------------------------------------
// FP32 SIMT form: LB lines per CTA staged in shared memory (rows padded to
// nw + 1 floats), one thread per line, the weights of a transfer read once
// per warp from the table (the same address for every lane).
__global__ void __launch_bounds__(128)
k_kk_simt(long long nlines, int nw, int Q, double dp, double v0, const float *__restrict__ im, float *__restrict__ re,
          float2 *__restrict__ rpa, const float *__restrict__ hs, int LB)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *rows = reinterpret_cast<float *>(smem_raw);
    if (dyn_smem_bytes() < (unsigned)(LB * (nw + 1) * 4)) return;
    const long long l0 = (long long)blockIdx.x * LB;
    for (int i = threadIdx.x; i < LB * nw; i += blockDim.x) {
        const int l = i / nw, k = i % nw;
        rows[l * (nw + 1) + k] = (l0 + l < nlines) ? im[(l0 + l) * nw + k] : 0.f;
    }
    __syncthreads();
    const int t = threadIdx.x;
    const long long line = l0 + t;
    if (t >= LB || line >= nlines) return;
    const float *x = rows + t * (nw + 1);
    bool zero;
    const float V = kk_vq(line, Q, dp, v0, &zero);
    const int H = (nw + 1) / 2;
    for (int m = 0; m < nw; ++m) {
        float s = 0.f;
        const int k0 = 1 - (m & 1);
        for (int j = 0; j < H; ++j) {
            const int k = 2 * j + k0;
            if (k < nw) s = fmaf(__ldg(hs + (size_t)j * nw + m), x[k], s);
        }
        re[line * nw + m] = s;
        if (rpa) rpa[line * nw + m] = kk_rpa(s, x[m], V, zero);
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
    const int LB = nw <= 384 ? 128 : 32;
    const size_t smem = (size_t)LB * (nw + 1) * 4;
    static const cudaError_t e0 = smem_attrs(k_kk_simt, std::max<size_t>(128ull * 385 * 4, 32ull * (KK_MAX_SIMT + 1) * 4));
    if (e0 != cudaSuccess) return e0;
    const long long nlines = (long long)g.Q * g.Q;
    const int grid = (int)((nlines + LB - 1) / LB);
    k_kk_simt<<<grid, LB, smem, s>>>(nlines, nw, g.Q, g.dp, v0, im, re, rpa,
                                     reinterpret_cast<const float *>(static_cast<const unsigned char *>(tab) +
                                                                     kk_simt_off(nw)),
                                     LB);
    return cudaGetLastError();
}

}  // namespace lh
