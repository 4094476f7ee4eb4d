// lindhard_imchi_noalloc: a forward call that allocates no memory.
//
// Some callers cannot allocate device memory at the time they need Im chi:
// code running inside a framework that owns the whole device memory pool,
// real-time or embedded hosts that forbid cudaMalloc after start-up, and
// callers that must not synchronise the device (cudaMalloc and cudaFree can).
// For them this entry point runs the same kernels as lindhard_imchi on one
// instance, with every intermediate placed in a fixed device array that is
// part of the loaded library instead of a plan's workspace.  The caller only
// passes the input (optional A) and output buffers.
//
// The array is a file-scope __device__ variable, so each GPU that loads the
// library holds LINDHARD_NOALLOC_SCRATCH_BYTES of memory until the process
// exits.  Host code cannot pass the variable's name to a kernel (on the host
// the name is a stand-in, not a device address): the device address comes from
// cudaGetSymbolAddress, looked up once per device on that device's first call.
// Every call uses the same array; calls that may run at the same time on the
// GPU (different streams, or different host threads) race on it.
#include <stdio.h>

#include <mutex>

#include "kernels.cuh"

namespace lh {
lindhard_status geom_from_grid(const lindhard_grid &gr, Geom &g, int &prec);
lindhard_status band_for_call(const Geom &g, const lindhard_band *b, bool generate, Band &o);
lindhard_status set_error(lindhard_status st, const char *msg);
cudaError_t launch_twiddles(int len, float2 *tw32, double2 *tw64, cudaStream_t s);
cudaError_t launch_setup(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                         InstState *st, double *acc, unsigned *bar, unsigned *status, double *mu_out, int G,
                         cudaStream_t s);
size_t mu_acc_doubles(int G);
size_t mu_barrier_words();
int mu_grid_size(int num_sms, int npts);
cudaError_t launch_solve_mu(const Geom &g, const Band &band, const AxisTab *axis, InstState *st, double *acc,
                            unsigned *bar, unsigned *status, double *mu_out, int G, cudaStream_t s);
cudaError_t launch_fwd_energy(const Geom &g, const Band &band, const Work<float> &w, const float *A_in,
                              cudaStream_t s);
cudaError_t launch_fwd_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_x_product(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_energy(const Geom &g, const Work<float> &w, float *out, cudaStream_t s, int variant);
}  // namespace lh

using namespace lh;

// The fixed scratch array (LINDHARD_NOALLOC_SCRATCH_BYTES, declared in lindhard.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LINDHARD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_scratch_addr[kMaxDevices];  // device address of the array, per device
int g_num_sms[kMaxDevices];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array for the current device (looked up on
// the first call on each device).
lindhard_status scratch_for_device(unsigned char **ptr, int *num_sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(LINDHARD_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return set_error(LINDHARD_EUNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return set_error(LINDHARD_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return set_error(LINDHARD_ECUDA, "multiprocessor count query failed");
        g_num_sms[dev] = sms;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *ptr = g_scratch_addr[dev];
    *num_sms = g_num_sms[dev];
    return LINDHARD_OK;
}

}  // namespace

extern "C" lindhard_status lindhard_imchi_noalloc(const lindhard_grid *grid, const lindhard_band *band,
                                                  const float *A_in, float *out, double *mu_out, void *stream)
{
    if (!grid || !out) return set_error(LINDHARD_EINVAL, "grid and out must be non-NULL");
    Geom g;
    int prec = 0;
    lindhard_status st = geom_from_grid(*grid, g, prec);
    if (st != LINDHARD_OK) return st;
    if (prec != LINDHARD_FP32) return set_error(LINDHARD_EINVAL, "lindhard_imchi_noalloc computes in FP32 only");
    Band b = {};
    st = band_for_call(g, band, A_in == nullptr, b);
    if (st != LINDHARD_OK) return st;
    unsigned char *base = nullptr;
    int num_sms = 0;
    st = scratch_for_device(&base, &num_sms);
    if (st != LINDHARD_OK) return st;

    // carve the fixed array exactly as a plan's workspace for this one grid
    const int tw_len = g.P > g.PE ? g.P : g.PE;
    const int G = mu_grid_size(num_sms, g.npz * g.npz);
    size_t X = (size_t)g.N * g.N * 2 * g.SP, X3 = (size_t)g.Q * g.xs3;
    size_t Y = (size_t)g.N * g.xs2, Y4 = (size_t)g.Q * g.Q * g.SP;
    size_t o = 0, off_X, off_Y, off_axis, off_eps, off_tw32, off_tw64, off_state, off_status, off_acc, off_bar;
    off_X = o; o = up256(o + (X > X3 ? X : X3) * sizeof(float2));
    off_Y = o; o = up256(o + (Y > Y4 ? Y : Y4) * sizeof(float2));
    off_axis = o; o = up256(o + (size_t)g.N * sizeof(AxisTab));
    off_eps = o; o = up256(o + (size_t)g.n_eps * sizeof(float2));
    off_tw32 = o; o = up256(o + (size_t)twiddle_entries() * sizeof(float2));
    off_tw64 = o; o = up256(o + (size_t)twiddle_entries() * sizeof(double2));
    off_state = o; o = up256(o + sizeof(InstState));
    off_status = o; o = up256(o + sizeof(unsigned));
    off_acc = o; o = up256(o + mu_acc_doubles(G) * sizeof(double));
    off_bar = o; o = up256(o + mu_barrier_words() * sizeof(unsigned));
    if (o > (size_t)LINDHARD_NOALLOC_SCRATCH_BYTES) {
        char msg[160];
        snprintf(msg, sizeof msg, "grid needs %zu bytes of scratch; lindhard_imchi_noalloc has %zu",
                 o, (size_t)LINDHARD_NOALLOC_SCRATCH_BYTES);
        return set_error(LINDHARD_EINVAL, msg);
    }

    Work<float> w;
    w.X = base + off_X;
    w.Y = base + off_Y;
    w.axis = (AxisTab *)(base + off_axis);
    w.eps = base + off_eps;
    w.tw = base + off_tw32;
    w.tw_len = tw_len;
    w.tc = nullptr;
    w.state = (InstState *)(base + off_state);
    w.status = (unsigned *)(base + off_status);
    w.mu_acc = (double *)(base + off_acc);
    w.barrier = (unsigned *)(base + off_bar);

    // The array keeps the previous call's contents: the status word and the
    // chemical-potential launches' arrival counter must start at zero;
    // everything else is written before it is read.
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.barrier, 0, mu_barrier_words() * sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_twiddles(tw_len, (float2 *)(base + off_tw32), (double2 *)(base + off_tw64), s);
    if (e == cudaSuccess && A_in == nullptr) {
        e = launch_setup(g, b, w.axis, (float2 *)w.eps, nullptr, w.state, w.mu_acc, w.barrier, w.status, mu_out, G, s);
        if (e == cudaSuccess)
            e = launch_solve_mu(g, b, w.axis, w.state, w.mu_acc, w.barrier, w.status, mu_out, G, s);
    }
    if (e == cudaSuccess) e = launch_fwd_energy(g, b, w, A_in, s);
    if (e == cudaSuccess) e = launch_fwd_y(g, w, s, 1);
    if (e == cudaSuccess) e = launch_x_product(g, w, s, 0);
    if (e == cudaSuccess) e = launch_inv_y(g, w, s, 1);
    if (e == cudaSuccess) e = launch_inv_energy(g, w, out, s, 0);
    if (e != cudaSuccess) return set_error(LINDHARD_ECUDA, cudaGetErrorString(e));
    return LINDHARD_OK;
}
