// Persistent batch scheduler: one launch runs the five transform passes of
// every instance of a batch (Sec. 3's FFT correlation, per instance: the
// energy forward pass with A generated on chip, p_y forward, the p_x product
// pass, p_y inverse, the energy inverse pass with the Eq. 9 prefactor).
//
// Work items are (instance, pass, tile) triples in one queue, pass-major:
// every tile of pass 0 of every instance, then pass 1, and so on.  Each CTA
// claims the next item with an atomic counter; an item of pass k > 0 waits
// until its instance's pass k - 1 has completed all its tiles (a per-instance
// per-pass counter).  Because items are claimed in queue order and every
// dependency lies earlier in the queue, the earliest claimed but unfinished
// item has all its dependencies finished, so the launch always progresses,
// whatever number of CTAs is resident.  The waits are bounded (a host-set
// limit, %globaltimer): a CTA that gives up records DEV_ETIMEOUT and every
// CTA stops at its next claim.  Tiles are the tile functions of the pruned
// momentum passes (pr_tiles.cuh, 256-thread tiles of 6144 / P columns) and of
// the warp-per-line energy passes (et_tiles.cuh); data written earlier in the
// launch is read through L2 only.  The chemical-potential solve and the
// tables run before the launch (their own launches per instance).
#include "async.cuh"
#include "et_tiles.cuh"
#include "pr_tiles.cuh"

namespace lh {

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

constexpr int PS_T = 256;
constexpr int PS_PASSES = 5;
constexpr int PS_EG = 2;   // energy-pass units per queue item
// An energy unit is what the CTA's PS_EW warps cover in one call of an energy
// tile function: PS_EW / ET_WARPS consecutive tiles (the tile functions place
// warp w at line (tile ET_WARPS + w) ET_LPW, so warps past ET_WARPS take the
// next tiles' lines).
constexpr int PS_EW = PS_T / 32;

// Per-instance constants of a persistent plan (device array).
struct PInst {
    Geom g;
    float2 *X, *Y;             // the instance's workspace slot
    const AxisTab *axis;
    const float2 *eps;
    const InstState *st;
    const Band *band;          // written by the instance's set-up launch of each call
    long long out_off;         // offset of the instance's output in the call's out
    int ntiles[PS_PASSES];     // tiles of each pass
    int gx[PS_PASSES];         // tiles along x of each pass's 2D tile grid
};
// Queue segment: items [start, start + ntiles) are the tiles of (inst, pass).
struct PSeg {
    int inst, pass, start, ntiles;
};

template <int P>
struct PsCfg {
    static constexpr int CW = 6144 / P;   // columns (pairs) of a 256-thread tile, 24 values per thread
    static constexpr int SMEM = cmax(cmax(PrEng<P, CW, PS_T, false, 2, true, false>::SMEM_ELEMS,
                                          PrEng<P, CW, PS_T, true, 2, false, true>::SMEM_ELEMS),
                                     PrProduct<P, CW, PS_T>::SMEM_ELEMS);
};
static_assert(PS_EW % ET_WARPS == 0, "whole energy tiles per unit");
// shared memory of the energy tiles for all PS_EW warps of the CTA
__host__ __device__ constexpr int ps_energy_smem_elems()
{
    return (PS_EW / ET_WARPS) * cmax(ET_WARPS * EtGeo<512>::WARP_ELEMS, et_inv_smem_elems<512>());
}
__host__ __device__ constexpr int ps_smem_elems()
{
    return cmax(cmax(cmax(PsCfg<192>::SMEM, PsCfg<384>::SMEM), cmax(PsCfg<768>::SMEM, PsCfg<1536>::SMEM)),
                ps_energy_smem_elems());
}
// shared memory a plan's launch needs: the largest tile of its instances
int ps_inst_smem_elems(const Geom &g)
{
    const int pr = g.P == 192 ? PsCfg<192>::SMEM : g.P == 384 ? PsCfg<384>::SMEM
                 : g.P == 768 ? PsCfg<768>::SMEM : PsCfg<1536>::SMEM;
    return cmax(pr, ps_energy_smem_elems());
}
size_t ps_smem_bytes() { return sizeof(float2) * ps_smem_elems(); }

bool ps_supported(const Geom &g)
{
    return g.quantity == LINDHARD_IMCHI && !g.periodic && pr_supported(g.P) && 3 * g.N == 2 * g.P &&
           3 * g.Q == 2 * g.P && et_supported(g.PE) && g.Q % 2 == 0;
}
// tiles of each pass (x extent in gx for the 2D grids)
void ps_tiles(const Geom &g, int *ntiles, int *gx)
{
    const int CW = 6144 / g.P;
    const long long per = (long long)PS_EW * ET_LPW;   // lines (pairs) of one energy unit
    gx[0] = gx[4] = 0;
    ntiles[0] = (int)(((long long)g.N * g.N + per * PS_EG - 1) / (per * PS_EG));
    gx[1] = (2 * g.SP + 2 * CW - 1) / (2 * CW);
    ntiles[1] = gx[1] * g.N;
    gx[2] = (g.H + CW - 1) / CW;
    ntiles[2] = gx[2] * g.P;
    gx[3] = (g.H + 2 * CW - 1) / (2 * CW);
    ntiles[3] = gx[3] * g.Q;
    ntiles[4] = (int)(((long long)g.Q * g.Q / 2 + per * PS_EG - 1) / (per * PS_EG));
}

// Counter value with a bounded wait (thread 0 of the CTA): false when the
// limit ran out first.
__device__ __forceinline__ bool ps_wait(const unsigned *cnt, unsigned need, unsigned long long wait_ns)
{
    if (*(volatile const unsigned *)cnt >= need) return true;
    const unsigned long long t0 = global_ns();
    while (*(volatile const unsigned *)cnt < need) {
        if (global_ns() - t0 > wait_ns) return false;
        __nanosleep(64);
    }
    return true;
}

// One tile of each pass, dispatched on the instance's transform lengths.
__device__ __noinline__ void ps_energy_fwd(const PInst &in, long long t, const float2 *etw, float2 *sm)
{
    const Geom g = in.g;   // registers (the constant fields the tile reads)
    float2 *U1 = in.X;
    const bool full = g.n_eps == g.PE;
#define ET_CASE(L)                                                                                                 \
    case L:                                                                                                        \
        if (full) energy_fwd_warp_tile<L, true, true>(g, *in.band, in.axis, in.eps, in.st, nullptr, U1, etw, sm, t); \
        else energy_fwd_warp_tile<L, false, true>(g, *in.band, in.axis, in.eps, in.st, nullptr, U1, etw, sm, t);    \
        break;
    switch (g.PE) { ET_CASE(128) ET_CASE(256) ET_CASE(512) }
#undef ET_CASE
}
__device__ __noinline__ void ps_fwd_y(const PInst &in, int t, const float2 *ptw, float2 *sm)
{
    const int bx = t % in.gx[1], by = t / in.gx[1];
    const Geom g = in.g;
#define PR_CASE(P)                                                                                  \
    case P: fwd_y_pr_tile<P, PsCfg<P>::CW, PS_T, true>(g, in.X, in.Y, ptw, sm, bx, by); break;
    switch (g.P) { PR_CASE(192) PR_CASE(384) PR_CASE(768) PR_CASE(1536) }
#undef PR_CASE
}
__device__ __noinline__ void ps_product(const PInst &in, int t, const float2 *ptw, float2 *sm)
{
    const int bx = t % in.gx[2], by = t / in.gx[2];
    const Geom g = in.g;
#define PR_CASE(P)                                                                                          \
    case P: x_product_pr_tile<P, PsCfg<P>::CW, PS_T, false, true>(g, in.Y, in.X, ptw, sm, bx, by); break;
    switch (g.P) { PR_CASE(192) PR_CASE(384) PR_CASE(768) PR_CASE(1536) }
#undef PR_CASE
}
__device__ __noinline__ void ps_inv_y(const PInst &in, int t, const float2 *ptw, float2 *sm)
{
    const int bx = t % in.gx[3], by = t / in.gx[3];
    const Geom g = in.g;
#define PR_CASE(P)                                                                                  \
    case P: inv_y_pr_tile<P, PsCfg<P>::CW, PS_T, true>(g, in.X, in.Y, ptw, sm, bx, by); break;
    switch (g.P) { PR_CASE(192) PR_CASE(384) PR_CASE(768) PR_CASE(1536) }
#undef PR_CASE
}
__device__ __noinline__ void ps_energy_inv(const PInst &in, long long t, float *out, const float2 *etw, float2 *sm)
{
    const Geom g = in.g;
    float *o = out + in.out_off;
    const bool half = 2 * g.n_omega == g.PE;
#define ET_CASE(L)                                                                       \
    case L:                                                                              \
        if (half) inv_energy_warp_tile<L, true, true>(g, in.Y, o, etw, sm, t);          \
        else inv_energy_warp_tile<L, false, true>(g, in.Y, o, etw, sm, t);              \
        break;
    switch (g.PE) { ET_CASE(128) ET_CASE(256) ET_CASE(512) }
#undef ET_CASE
}

constexpr int PS_CHUNK = 4;   // items claimed per atomic

__global__ void __launch_bounds__(PS_T, 2)
k_persistent(const PInst *__restrict__ insts, const PSeg *__restrict__ segs, int nsegs, int total, unsigned *head,
             unsigned *done, unsigned *status, float *out, const float2 *__restrict__ ptw,
             const float2 *__restrict__ etw, unsigned long long wait_ns, int stall_inst, int smem_elems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LH_REQUIRE_SMEM(smem_elems, float2)   // the host sizes it for every tile of the plan's instances
    float2 *sm = reinterpret_cast<float2 *>(smem_raw);
    __shared__ int s_base, s_seg, s_ok;
    // the current item's instance entry: the tile functions read its geometry
    // from shared memory (a global-memory reference would be reloaded after
    // every barrier of the transforms)
    __shared__ __align__(16) PInst s_in;
    int s_in_inst = -1;   // instance held in s_in (every thread tracks it)
    // thread 0's bookkeeping: the segment of the current item (items are
    // claimed in increasing order, so the segment only moves forward), the
    // (instance, pass) whose dependency is known complete, and this CTA's
    // finished tiles not yet added to their counter (added whenever the
    // segment changes, before any item of a later pass can wait on them)
    int seg = 0, ok_seg = -1, pend_seg = -1;
    unsigned pend = 0;
    // thread 0 claims one chunk ahead: the atomic's round trip overlaps the
    // current chunk's tiles.  Progress still holds: a CTA's claimed-ahead
    // chunk lies after its current one, so the earliest unfinished item is
    // either being worked on or next for a CTA whose current items are done.
    int nxt = 0;
    if (threadIdx.x == 0) nxt = (int)atomicAdd(head, (unsigned)PS_CHUNK);
    auto flush = [&]() {
        if (pend) {
            __threadfence();   // the CTA's writes (ordered before by the barrier) before the count
            atomicAdd(&done[segs[pend_seg].inst * PS_PASSES + segs[pend_seg].pass], pend);
            pend = 0;
        }
    };
    for (;;) {
        if (threadIdx.x == 0) {
            int base = nxt;
            if (base < total) nxt = (int)atomicAdd(head, (unsigned)PS_CHUNK);
            if (base < total && *(volatile unsigned *)status != DEV_OK) base = total;   // a CTA gave up: stop
            s_base = base;
        }
        __syncthreads();
        const int base = s_base;
        if (base >= total) break;
        for (int k = 0; k < PS_CHUNK && base + k < total; ++k) {
            const int item = base + k;
            if (threadIdx.x == 0) {
                while (seg + 1 < nsegs && segs[seg + 1].start <= item) ++seg;
                if (pend && pend_seg != seg) flush();
                int ok = 1;
                const PSeg sg = segs[seg];
                if (sg.pass > 0 && ok_seg != seg) {
                    // the instance's previous pass complete (stall_inst: a test
                    // asks one more tile than exists, so that the wait runs out)
                    const unsigned need =
                        (unsigned)insts[sg.inst].ntiles[sg.pass - 1] + (sg.inst == stall_inst ? 1u : 0u);
                    ok = ps_wait(&done[sg.inst * PS_PASSES + sg.pass - 1], need, wait_ns) ? 1 : 0;
                    if (!ok) atomicCAS(status, (unsigned)DEV_OK, (unsigned)DEV_ETIMEOUT);
                    ok_seg = seg;
                    __threadfence();   // the producers' writes before this CTA's reads
                }
                s_seg = seg;
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) return;
            const PSeg sg = segs[s_seg];
            if (sg.inst != s_in_inst) {
                constexpr int W = (int)(sizeof(PInst) / sizeof(int));
                static_assert(sizeof(PInst) % sizeof(int) == 0, "whole words");
                const int *src = reinterpret_cast<const int *>(insts + sg.inst);
                int *dst = reinterpret_cast<int *>(&s_in);
                for (int w = threadIdx.x; w < W; w += PS_T) dst[w] = src[w];
                s_in_inst = sg.inst;
                __syncthreads();
            }
            const PInst &in = s_in;
            const int t = item - sg.start;
            switch (sg.pass) {
            // an item of an energy pass is PS_EG consecutive units (short
            // tiles; the per-item bookkeeping would not pay for itself)
            case 0:
#pragma unroll 1
                for (int u = 0; u < PS_EG; ++u)
                    ps_energy_fwd(in, ((long long)t * PS_EG + u) * (PS_EW / ET_WARPS), etw, sm);
                break;
            case 1: ps_fwd_y(in, t, ptw, sm); break;
            case 2: ps_product(in, t, ptw, sm); break;
            case 3: ps_inv_y(in, t, ptw, sm); break;
            default:
#pragma unroll 1
                for (int u = 0; u < PS_EG; ++u)
                    ps_energy_inv(in, ((long long)t * PS_EG + u) * (PS_EW / ET_WARPS), out, etw, sm);
                break;
            }
            __syncthreads();   // every thread's writes of the tile before thread 0 counts it
            if (threadIdx.x == 0) {
                pend_seg = s_seg;
                ++pend;
            }
        }
        if (threadIdx.x == 0) flush();
    }
    if (threadIdx.x == 0) flush();
}

cudaError_t launch_persistent(const void *insts, const void *segs, int nsegs, int total, unsigned *head,
                              unsigned *done, unsigned *status, float *out, const float2 *ptw, const float2 *etw,
                              unsigned long long wait_ns, int stall_inst, int smem_elems, int grid, cudaStream_t s)
{
    static const cudaError_t e = smem_attrs(k_persistent, ps_smem_bytes());
    if (e != cudaSuccess) return e;
    k_persistent<<<grid, PS_T, sizeof(float2) * smem_elems, s>>>((const PInst *)insts, (const PSeg *)segs, nsegs,
                                                                   total, head, done, status, out, ptw, etw, wait_ns,
                                                                   stall_inst, smem_elems);
    return cudaGetLastError();
}
// CTAs of the persistent grid: every SM filled to the kernel's occupancy at
// the plan's shared-memory size
int ps_grid(int num_sms, int smem_elems)
{
    int per = 0;
    if (smem_attrs(k_persistent, ps_smem_bytes()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent, PS_T, sizeof(float2) * smem_elems) !=
            cudaSuccess ||
        per < 1)
        per = 1;
    return num_sms * per;
}
size_t ps_inst_bytes() { return sizeof(PInst); }
size_t ps_seg_bytes() { return sizeof(PSeg); }
// Host-side build of one instance's entry (device pointers into the plan).
void ps_fill_inst(void *dst, const Geom &g, void *X, void *Y, const AxisTab *axis, const void *eps,
                  const InstState *st, const Band *band, long long out_off)
{
    PInst &p = *reinterpret_cast<PInst *>(dst);
    p.g = g;
    p.X = (float2 *)X;
    p.Y = (float2 *)Y;
    p.axis = axis;
    p.eps = (const float2 *)eps;
    p.st = st;
    p.band = band;
    p.out_off = out_off;
    ps_tiles(g, p.ntiles, p.gx);
}
void ps_fill_seg(void *dst, int inst, int pass, int start, int ntiles)
{
    PSeg &s = *reinterpret_cast<PSeg *>(dst);
    s.inst = inst;
    s.pass = pass;
    s.start = start;
    s.ntiles = ntiles;
}
int ps_pass_tiles(const Geom &g, int pass)
{
    int n[PS_PASSES], gx[PS_PASSES];
    ps_tiles(g, n, gx);
    return n[pass];
}

}  // namespace lh
