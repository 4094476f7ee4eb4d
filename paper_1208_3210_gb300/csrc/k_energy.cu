// Energy passes with one warp per momentum point (FP32).
//
// Forward: the same transform as k_fwd_energy (Eqs. 4-5 generated on chip,
// split into the occupied and the empty part (Sec. 3 / Appendix A: Eq. A3 at
// T = 0, the Fermi weights of Eq. A1 at T > 0), z = a + i b transformed along
// energy, a^ and b^ separated for the non-redundant frequencies k <= L/2),
// arranged so that
//   * the TPL = L/VPT threads of one line (momentum point) sit in one warp (a
//     warp holds 32 / TPL lines at a time): every exchange of a line stays in
//     its warp (__syncwarp, no CTA barrier), the warp's lines' band energies
//     are computed by one lane each and broadcast by shuffles, and every
//     thread keeps its line's band energy and amplitude in registers;
//   * every shared-memory address is a per-butterfly base plus compile-time
//     offsets (one pad value every 16 spreads the Stockham writes over the
//     banks), the twiddles 16-byte loads from per-stage tables;
//   * in the last stage a thread owns butterflies j and L/R2 - j, so it holds
//     Z(k) and Z(L - k) together and separates a^(k) = (Z(k) + conj Z(L - k))/2
//     and b^(k) = (Z(k) - conj Z(L - k))/2i in registers (no natural-order
//     copy of the spectrum); a warp's stores of one line are contiguous.
// Inverse: one warp per pair of (q_x, q_y) lines, the mirror image (a thread's
// first-stage butterflies j and L/R0 - j form W(k) and W(L - k) from the
// stored half spectra).
// Schedules (et_tiles.cuh): VPT = 16 values per thread at 128, 256 and 512,
// 24 at 384 and 768.  Output U1 [N*N lines][SP][2] as k_fwd_energy writes it.
#include "et_tiles.cuh"

namespace lh {

__global__ void k_et_twiddles(float2 *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= et_twiddle_entries()) return;
    for (int d = 0; d < 2; ++d)
        for (int i = 0; et_len(d, i) != 0; ++i)
        for (int s = 1; s <= 2; ++s) {
            const int L = et_len(d, i);
            const int off = et_table_offset(L, s, d != 0), n = et_ns(L, s + 1, d != 0), Rs = et_radix(L, s, d != 0);
            if (e >= off && e < off + n) {
                // row k holds w^1, ..., w^(Rs-1), w^0 (position p: power p + 1)
                const int k = (e - off) / Rs, r = ((e - off) % Rs + 1) % Rs;
                double sn, cs;
                sincospi(-2.0 * (double)((k * r) % n) / (double)n, &sn, &cs);
                out[e] = make_float2((float)cs, (float)sn);
                return;
            }
        }
}
cudaError_t launch_et_twiddles(float2 *out, cudaStream_t s)
{
    k_et_twiddles<<<(et_twiddle_entries() + 255) / 256, 256, 0, s>>>(out);
    return cudaGetLastError();
}
size_t et_twiddle_bytes() { return (size_t)et_twiddle_entries() * sizeof(float2); }
// the warp-per-line forward pass: T = 0 at 128, 256 and 512 energies, finite
// temperature (whose energy axes are padded to 3 * 2^k) also at 384 and 768
bool et_applies(const Geom &g, const Band &band)
{
    return band.kT > 0 ? et_len_supported(g.PE) : et_supported(g.PE);
}

// THERMAL: the CTA tabulates the Fermi weights of its energies once, after the
// warps' exchange areas, before the tile
template <int L, bool FULL, bool GEN, bool THERMAL>
__global__ void __launch_bounds__(32 * ET_WARPS)
k_fwd_energy_warp(Geom g, Band band, const AxisTab *__restrict__ axis, const float2 *__restrict__ eps,
                  const InstState *__restrict__ st, const float *__restrict__ A_in, float2 *__restrict__ U1,
                  const float2 *__restrict__ etw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM(ET_WARPS * EtGeo<L>::WARP_ELEMS + (THERMAL ? L : 0), float2)
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    float2 *wf = sm + ET_WARPS * EtGeo<L>::WARP_ELEMS;
    if constexpr (THERMAL) {
        et_fermi_weights<L>(g, band, wf, (int)threadIdx.x, 32 * ET_WARPS);
        __syncthreads();
    }
    energy_fwd_warp_tile<L, FULL, GEN, THERMAL>(g, band, axis, eps, st, A_in, U1, etw, sm, blockIdx.x, wf);
}

template <int L, bool HALF>
__global__ void __launch_bounds__(32 * ET_WARPS)
k_inv_energy_warp(Geom g, const float2 *__restrict__ U4, float *__restrict__ out, const float2 *__restrict__ etw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM(et_inv_smem_elems<L>(), float2)
    inv_energy_warp_tile<L, HALF, false>(g, U4, out, etw, reinterpret_cast<float2 *>(smem_raw), blockIdx.x);
}

template <int L>
cudaError_t launch_inv_energy_warp_t(const Geom &g, const Work<float> &w, float *out, cudaStream_t s)
{
    const long long npairs = (long long)g.Q * g.Q / 2;
    const long long per = (long long)ET_WARPS * ET_LPW;
    const unsigned grid = (unsigned)((npairs + per - 1) / per);
    const size_t smem = sizeof(float2) * et_inv_smem_elems<L>();
    static const cudaError_t e0 = smem_attrs(k_inv_energy_warp<L, true>, smem);
    static const cudaError_t e1 = smem_attrs(k_inv_energy_warp<L, false>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    auto k = 2 * g.n_omega == L ? k_inv_energy_warp<L, true> : k_inv_energy_warp<L, false>;
    k<<<grid, 32 * ET_WARPS, smem, s>>>(g, (const float2 *)w.Y, out, (const float2 *)w.etw);
    return cudaGetLastError();
}

// the warp-per-pair inverse pass: every length of the warp-per-line passes
bool et_inv_applies(const Geom &g) { return et_len_supported(g.PE) && g.Q % 2 == 0; }
cudaError_t launch_inv_energy_warp(const Geom &g, const Work<float> &w, float *out, cudaStream_t s)
{
    if (!w.etw || !et_inv_applies(g)) return cudaErrorInvalidValue;
    switch (g.PE) {
    case 128: return launch_inv_energy_warp_t<128>(g, w, out, s);
    case 256: return launch_inv_energy_warp_t<256>(g, w, out, s);
    case 512: return launch_inv_energy_warp_t<512>(g, w, out, s);
    case 384: return launch_inv_energy_warp_t<384>(g, w, out, s);
    case 768: return launch_inv_energy_warp_t<768>(g, w, out, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int L, bool THERMAL>
cudaError_t launch_fwd_energy_col_tt(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                                     cudaStream_t s)
{
    const long long nlines = (long long)g.N * g.N;
    const long long per = (long long)ET_WARPS * ET_LPW;
    const unsigned grid = (unsigned)((nlines + per - 1) / per);
    const size_t smem = sizeof(float2) * (ET_WARPS * EtGeo<L>::WARP_ELEMS + (THERMAL ? L : 0));
    static const cudaError_t e0 = smem_attrs(k_fwd_energy_warp<L, true, true, THERMAL>, smem);
    static const cudaError_t e1 = smem_attrs(k_fwd_energy_warp<L, false, true, THERMAL>, smem);
    static const cudaError_t e2 = smem_attrs(k_fwd_energy_warp<L, true, false, THERMAL>, smem);
    static const cudaError_t e3 = smem_attrs(k_fwd_energy_warp<L, false, false, THERMAL>, smem);
    if (e0 != cudaSuccess) return e0;
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    if (e3 != cudaSuccess) return e3;
    const bool full = g.n_eps == L;
    auto k = A_in ? (full ? k_fwd_energy_warp<L, true, false, THERMAL> : k_fwd_energy_warp<L, false, false, THERMAL>)
                  : (full ? k_fwd_energy_warp<L, true, true, THERMAL> : k_fwd_energy_warp<L, false, true, THERMAL>);
    k<<<grid, 32 * ET_WARPS, smem, s>>>(g, band, w.axis, (const float2 *)w.eps, w.state, A_in, (float2 *)w.X,
                                        (const float2 *)w.etw);
    return cudaGetLastError();
}
template <int L>
cudaError_t launch_fwd_energy_col_t(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                                    cudaStream_t s)
{
    if constexpr (et_supported(L)) {
        if (!(band.kT > 0)) return launch_fwd_energy_col_tt<L, false>(g, band, w, A_in, s);
    }
    return launch_fwd_energy_col_tt<L, true>(g, band, w, A_in, s);
}

cudaError_t launch_fwd_energy_col(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                                  cudaStream_t s)
{
    if (!w.etw) return cudaErrorInvalidValue;
    switch (g.PE) {
    case 128: return launch_fwd_energy_col_t<128>(g, band, w, A_in, s);
    case 256: return launch_fwd_energy_col_t<256>(g, band, w, A_in, s);
    case 512: return launch_fwd_energy_col_t<512>(g, band, w, A_in, s);
    case 384: return launch_fwd_energy_col_t<384>(g, band, w, A_in, s);
    case 768: return launch_fwd_energy_col_t<768>(g, band, w, A_in, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lh
