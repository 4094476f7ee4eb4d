// Host implementation of the C ABI declared in include/lindhard.h: grid
// validation, FFT length selection, workspace layout and the launch sequence
// of one forward call.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <fstream>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace lh {
// launchers (k_*.cu)
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
cudaError_t launch_fwd_energy(const Geom &g, const Band &band, const Work<double> &w, const double *A_in,
                              cudaStream_t s);
cudaError_t launch_fwd_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_fwd_y(const Geom &g, const Work<double> &w, cudaStream_t s, int variant);
cudaError_t launch_x_product(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
cudaError_t launch_x_product(const Geom &g, const Work<double> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_y(const Geom &g, const Work<float> &w, cudaStream_t s, int variant);
bool direct_supported(const Geom &g);
bool mu_solve_in_setup(const Geom &g);
cudaError_t launch_direct_stage(int stage, const Geom &g, const Band &band, const Work<float> &w,
                                const float *A_in, float *out, cudaStream_t s);
bool tc_supported(int P);
size_t kk_table_bytes(int nw);
cudaError_t launch_dmu_partials(int kind, double t, double tp, double tpp, double gamma, int npz, double mu,
                                double *part, int blocks, cudaStream_t s);
constexpr int kDmuBlocks = 128;
cudaError_t launch_kk_tables(int nw, void *tab, cudaStream_t s);
cudaError_t launch_kk_rpa(const Geom &g, const float *im, float *re, float2 *rpa, const void *tab, double v0,
                          int variant, unsigned *status, cudaStream_t s);
size_t tc_mats_bytes();
size_t pr_twiddle_bytes();
size_t et_twiddle_bytes();
cudaError_t launch_et_twiddles(float2 *out, cudaStream_t s);
cudaError_t launch_pr_twiddles(float2 *out, cudaStream_t s);
bool pr_fwd_applies(const Geom &g);
bool pr_inv_applies(const Geom &g);
bool et_inv_applies(const Geom &g);
// persistent batch launch (k_persist.cu)
bool ps_supported(const Geom &g);
size_t ps_inst_bytes();
size_t ps_seg_bytes();
int ps_grid(int num_sms, int smem_elems);
int ps_inst_smem_elems(const Geom &g);
int ps_pass_tiles(const Geom &g, int pass);
void ps_fill_inst(void *dst, const Geom &g, void *X, void *Y, const AxisTab *axis, const void *eps,
                  const InstState *st, const Band *band, long long out_off);
void ps_fill_seg(void *dst, int inst, int pass, int start, int ntiles);
cudaError_t launch_persistent(const void *insts, const void *segs, int nsegs, int total, unsigned *head,
                              unsigned *done, unsigned *status, float *out, const float2 *ptw, const float2 *etw,
                              unsigned long long wait_ns, int stall_inst, int smem_elems, int grid, cudaStream_t s);
cudaError_t launch_setup_band(const Geom &g, const Band &band, AxisTab *axis, float2 *eps32, double *eps64,
                              InstState *st, double *acc, unsigned *bar, unsigned *status, double *mu_out, int G,
                              Band *band_out, cudaStream_t s);
cudaError_t launch_tc_mats(void *buf, cudaStream_t s);
cudaError_t launch_inv_y(const Geom &g, const Work<double> &w, cudaStream_t s, int variant);
cudaError_t launch_inv_energy(const Geom &g, const Work<float> &w, float *out, cudaStream_t s, int variant);
cudaError_t launch_inv_energy(const Geom &g, const Work<double> &w, double *out, cudaStream_t s, int variant);
cudaError_t launch_w_energy(const Geom &g, const float *w, float2 *WU1, const float2 *tw, int tw_len,
                            cudaStream_t s);
cudaError_t launch_w_y(const Geom &g, const float2 *WU1, float2 *WU2, const float2 *tw, int tw_len, cudaStream_t s);
cudaError_t launch_bw_product(const Geom &g, float2 *U2, const float2 *WU2, const float2 *tw, int tw_len,
                              const float2 *ptw, cudaStream_t s);
cudaError_t launch_bw_inv_y(const Geom &g, const float2 *G3, float2 *G4, const float2 *tw, int tw_len,
                            cudaStream_t s);
cudaError_t launch_bw_inv_energy(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                                 const InstState *st, const float2 *G4, float *dA, double *partial,
                                 const float2 *tw, int tw_len, cudaStream_t s);
int bw_energy_blocks(const Geom &g);
cudaError_t launch_sum_rule(const Geom &g, const Band &band, const AxisTab *axis, const float2 *eps,
                            const InstState *st, const float *A_in, const float *out, double *D, double *sum_q,
                            double *dos_corr, cudaStream_t s);
cudaError_t launch_reduce_params(const double *partial, int nblocks, double *out, cudaStream_t s);
int bw_partial_extra_rows();
}  // namespace lh

using namespace lh;

static thread_local std::string g_last_error;

static lindhard_status fail(lindhard_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

static lindhard_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LINDHARD_ECUDA;
}

static const int kMinLen = 16, kMaxLen = 4096, kMaxLen64 = 256;

static bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

static long long next_len(long long x)
{
    long long L = kMinLen;
    while (L < x) L <<= 1;
    return L;
}
// Smallest momentum-axis FFT length >= x: a power of two, or for FP32 also
// 3 * 2^k (48..1536), which pads N to exactly N + Q/2 = 1.5 N when Q = N.
static long long next_len_p(long long x, int prec)
{
    long long L = next_len(x);
    if (prec != LINDHARD_FP64)
        for (long long L3 = 48; L3 <= 1536; L3 <<= 1)
            if (L3 >= x && L3 < L) L = L3;
    return L;
}

struct lindhard_plan {
    int batch = 0;
    std::vector<Geom> geoms;
    std::vector<int> precision;
    int device = 0, num_sms = 0, mu_G = 1;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    // Workspace of one instance (offsets into ws).  One slot shared by all
    // instances in sequential plans; one slot per instance in concurrent plans.
    struct Slot {
        size_t X = 0, Y = 0, Z = 0, partial = 0, axis = 0, eps32 = 0, eps64 = 0, state = 0, acc = 0, bar = 0;
    };
    std::vector<Slot> slots;
    size_t off_tw32 = 0, off_tw64 = 0, off_status = 0, off_tc = 0, off_dmu = 0, off_prtw = 0, off_etw = 0;
    std::vector<size_t> off_kk;   // Kramers-Kronig weight tables per instance (FP32 grids)
    int tw_len = 0;
    bool backward = false;       // LINDHARD_PLAN_BACKWARD
    // engine variants per instance, set by the autotuner
    // (LINDHARD_PLAN_AUTOTUNE): p_y passes 0 single-column, 1 paired-column,
    // 2 paired-column with 12 values per thread, 3, 4 and 5 the TMA-staged
    // persistent forms of 1, 2 and 0, 6 paired columns on double-width tiles;
    // product pass 0 default tile, 1 tile with
    // 12 values per thread, 2 and 3 their TMA-staged persistent forms, 4 the
    // default tile with one more CTA per SM, 5 the default tile twice as wide
    // (6-10: the pruned engine's forms, as lindhard_plan_variants lists them)
    std::vector<int> yvar_fwd, yvar_inv, xvar;
    // inverse energy pass: 0 default, 1 TMA-staged persistent form
    std::vector<int> evar;
    bool concurrent = false;     // LINDHARD_PLAN_CONCURRENT
    bool graph = false;          // LINDHARD_PLAN_GRAPH
    bool direct = false;         // LINDHARD_PLAN_ENERGY_DIRECT
    // LINDHARD_PLAN_PERSISTENT: per-instance entries, queue segments,
    // per-instance per-pass completion counters (+ the queue head) and the
    // calls' bands, in the workspace; the wait limit and the test stall
    bool persistent = false;
    size_t off_ps_inst = 0, off_ps_seg = 0, off_ps_cnt = 0, off_ps_band = 0;
    int ps_nsegs = 0, ps_total = 0, ps_grid = 0, ps_smem = 0;
    unsigned long long wait_ns = 1000000000ull;
    int stall_inst = -1;
    // concurrent execution: instances on plan-owned streams, forked from and
    // joined back into the caller's stream with events
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_of;   // stream index of each instance
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    // graph mode: the forward sequence captured once and replayed while the
    // call's pointers and band values are unchanged
    cudaStream_t origin = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool warmed = false;
    const void *key_A = nullptr;
    void *key_out = nullptr;
    double *key_mu = nullptr;
    std::vector<lindhard_band> key_bands;
    // per-pass event timing (lindhard_plan_profile; sequential plans): bit i
    // of the mask times pass slot i
    unsigned profile = 0;
    struct Timed { int slot; cudaEvent_t a, b; };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> pool;
    double pass_ms[LINDHARD_NUM_PASSES] = {0};
    long long pass_n[LINDHARD_NUM_PASSES] = {0};
};

static cudaEvent_t pool_event(lindhard_plan *p)
{
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Runs `launch` and, when profiling, brackets it with an event pair on s.
template <typename F>
static cudaError_t timed(lindhard_plan *p, int slot, cudaStream_t s, F &&launch)
{
    if (!(p->profile & (1u << slot))) return launch();
    cudaEvent_t a = pool_event(p), b = pool_event(p);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    p->pending.push_back({slot, a, b});
    return e;
}

static void drain_events(lindhard_plan *p)
{
    for (auto &t : p->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            p->pass_ms[t.slot] += ms;
            p->pass_n[t.slot] += 1;
        }
        p->pool.push_back(t.a);
        p->pool.push_back(t.b);
    }
    p->pending.clear();
}

// Bytes of one complex element for a precision.
static size_t cx_bytes(int prec) { return prec == LINDHARD_FP64 ? 16 : 8; }

static lindhard_status make_geom(const lindhard_grid &gr, Geom &g, int &prec)
{
    if (gr.quantity != LINDHARD_IMCHI && gr.quantity != LINDHARD_IMCHI_T && gr.quantity != LINDHARD_SQW)
        return fail(LINDHARD_EINVAL, "quantity must be LINDHARD_IMCHI, LINDHARD_IMCHI_T or LINDHARD_SQW");
    if (gr.zones < 1) return fail(LINDHARD_EINVAL, "zones must be >= 1");
    if (gr.pts_per_zone < 2 || gr.pts_per_zone % 2) return fail(LINDHARD_EINVAL, "pts_per_zone must be even and >= 2");
    if (gr.n_eps < 2) return fail(LINDHARD_EINVAL, "n_eps must be >= 2");
    if (!(gr.e_max > 0) || !isfinite(gr.e_max)) return fail(LINDHARD_EINVAL, "e_max must be finite and > 0");
    if (gr.precision != LINDHARD_FP32 && gr.precision != LINDHARD_FP64 && gr.precision != LINDHARD_SPLITBF16_TC)
        return fail(LINDHARD_EUNSUPPORTED, "precision must be LINDHARD_FP32, LINDHARD_SPLITBF16_TC or LINDHARD_FP64");
    long long N = (long long)gr.zones * gr.pts_per_zone;
    if (N > kMaxLen) return fail(LINDHARD_EUNSUPPORTED, "zones * pts_per_zone exceeds 4096");
    long long n_omega = gr.n_omega ? gr.n_omega : gr.n_eps / 2;
    if (n_omega < 1 || n_omega > gr.n_eps) return fail(LINDHARD_EINVAL, "n_omega must be in [1, n_eps]");
    long long Q = gr.q_extent ? gr.q_extent : N;
    if (Q < 2 || Q % 2) return fail(LINDHARD_EINVAL, "q_extent must be even and >= 2");
    bool periodic = gr.zones == 1;
    if (Q > (periodic ? N : 2 * N)) return fail(LINDHARD_EINVAL, "q_extent too large");
    long long P;
    if (periodic) {
        // the reduced zone is one period: the circular correlation is the exact one
        if (!is_pow2(N) || N < kMinLen)
            return fail(LINDHARD_EUNSUPPORTED, "reduced zone needs pts_per_zone a power of two >= 16");
        P = N;
    } else {
        // lags |s| <= Q/2 of a length-N sequence: no wrap-around when P >= N + Q/2
        P = next_len_p(N + Q / 2, gr.precision);
    }
    // energy: with the occupied/empty split every lag m in [0, PE) is alias-free
    // once PE >= n_eps (the occupied part sits below the empty part).  At
    // finite temperature both parts cover the whole window, lags run over
    // (-n_eps, n_eps), and the kept ones [0, n_omega) and their mirrors
    // (-n_omega, 0] stay clear of wrapped partners once PE >= n_eps + n_omega - 1.
    // (FP32 forms: lengths 3 * 2^k too, e.g. 384 instead of 512 for n_eps 256, n_omega 128)
    long long PE = gr.quantity == LINDHARD_IMCHI ? next_len(gr.n_eps) : next_len_p(gr.n_eps + n_omega - 1, gr.precision);
    long long maxlen = gr.precision == LINDHARD_FP64 ? kMaxLen64 : kMaxLen;
    if (P > maxlen || PE > maxlen) return fail(LINDHARD_EUNSUPPORTED, "FFT length beyond the compiled range");
    if (gr.precision == LINDHARD_SPLITBF16_TC && !tc_supported((int)P))
        return fail(LINDHARD_EUNSUPPORTED, "no tensor-core form for this momentum FFT length "
                                           "(128, 192, 256, 384, 512, 768, 1024, 1536)");
    g.N = (int)N;
    g.npz = gr.pts_per_zone;
    g.periodic = periodic;
    g.n_eps = gr.n_eps;
    g.J0 = gr.n_eps / 2;
    g.P = (int)P;
    g.PE = (int)PE;
    g.H = (int)(PE / 2 + 1);
    g.SP = (g.H + 7) / 8 * 8;
    // The p_x pass reads and writes rows one plane apart; plane sizes are
    // multiples of large powers of two (P 2SP 8 bytes = 33 * 2^18 at 2048 x 512),
    // which concentrates those accesses on few memory channels.  256 bytes of
    // padding per plane spread them.
    g.xs2 = (long long)P * 2 * g.SP + 32;
    g.xs3 = (long long)P * g.SP + 32;
    g.Q = (int)Q;
    g.n_omega = (int)n_omega;
    g.band_kind = 0;
    g.e_max = gr.e_max;
    g.de = 2.0 * gr.e_max / gr.n_eps;
    g.dp = 2.0 * M_PI / gr.pts_per_zone;
    g.scale = -(g.de / (2.0 * M_PI)) / ((double)g.npz * g.npz) / ((double)P * P * PE);
    g.quantity = gr.quantity;
    if (gr.quantity == LINDHARD_SQW) g.scale = -g.scale / M_PI;   // (c / pi) sum A A f (1 - f)
    prec = gr.precision;
    return LINDHARD_OK;
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }
extern "C" void lindhard_plan_destroy(lindhard_plan *p);

// ---------------------------------------------------------------------------
// Autotuner.  For every distinct momentum geometry of an FP32 plan it times the
// engine variants of the two p_y passes and of the product pass with CUDA events
// (on the plan's own workspace; the data are whatever the workspace holds, the
// timing does not depend on them) and keeps the faster.  Results are cached per
// process, and in the JSON file named by LINDHARD_TUNE_CACHE when that is set:
// one entry per line, {"<gpu>|P=..|N=..|PE=..|Q=..|fwd_y": variant, ...}
// (also |inv_y and |x_product; variants as for lindhard_plan::yvar_fwd and
// xvar).  Cached entries in range are used as they are (a cache file may pin
// a variant).  Entries read from a cache file stay with that file: when the
// variable names another file they are dropped (entries timed in the process
// are kept), and a save writes only the timed entries and those of its own
// file, so variants pinned in one file never leak into another.
template <typename Real>
static Work<Real> work_of(lindhard_plan *p, int i);

static std::mutex g_tune_mutex;
struct TuneEntry {
    int variant;
    std::string origin;   // the cache file it was read from; empty: timed here
};
static std::map<std::string, TuneEntry> g_tune;
static std::string g_tune_path;   // cache file last merged into g_tune

static void tune_load()
{
    const char *path = getenv("LINDHARD_TUNE_CACHE");
    if (!path || g_tune_path == path) return;
    g_tune_path = path;
    for (auto it = g_tune.begin(); it != g_tune.end();)   // another file's entries
        it = it->second.origin.empty() ? std::next(it) : g_tune.erase(it);
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        size_t a = line.find('"'), b = line.find('"', a + 1), c = line.find(':', b);
        if (a == std::string::npos || b == std::string::npos || c == std::string::npos) continue;
        g_tune[line.substr(a + 1, b - a - 1)] = TuneEntry{atoi(line.c_str() + c + 1), g_tune_path};
    }
}
static void tune_save()
{
    const char *path = getenv("LINDHARD_TUNE_CACHE");
    if (!path) return;
    std::vector<std::pair<std::string, int>> out;
    for (auto &kv : g_tune)
        if (kv.second.origin.empty() || kv.second.origin == path) out.emplace_back(kv.first, kv.second.variant);
    std::ofstream f(path);
    f << "{\n";
    for (size_t i = 0; i < out.size(); ++i)
        f << "  \"" << out[i].first << "\": " << out[i].second << (i + 1 < out.size() ? ",\n" : "\n");
    f << "}\n";
}

template <typename F>
static float time_launches(F &&launch, cudaEvent_t a, cudaEvent_t b)
{
    for (int i = 0; i < 2; ++i) launch();
    cudaEventRecord(a, 0);
    for (int i = 0; i < 5; ++i) launch();
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

static cudaError_t autotune(lindhard_plan *p)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const char *log_env = getenv("LINDHARD_TUNE_LOG");
    const bool log = log_env && *log_env && strcmp(log_env, "0") != 0;
    for (int i = 0; i < p->batch && e == cudaSuccess; ++i) {
        const Geom &g = p->geoms[i];
        if (p->precision[i] == LINDHARD_FP64 || g.P < 128) continue;
        std::ostringstream key;
        key << prop.name << "|P=" << g.P << "|N=" << g.N << "|PE=" << g.PE << "|Q=" << g.Q;
        const std::string kf = key.str() + "|fwd_y", ki = key.str() + "|inv_y", kx = key.str() + "|x_product",
                          ke = key.str() + "|inv_energy";
        const bool f1 = fft_has_family1(g.P);
        std::vector<int> vy = {0, 1, 3, 5}, vx = {0, 2, 4};
        if (g.P >= 384) {
            vx.push_back(5);
            vy.push_back(6);
        }
        if (f1) {
            vy.push_back(2);
            vy.push_back(4);
            vx.push_back(1);
            vx.push_back(3);
        }
        // the pruned engine (one-third padding): forward p_y and inverse p_y
        // separately (N and Q), the product pass needs both
        std::vector<int> vyf = vy, vyi = vy;
        if (pr_fwd_applies(g)) { vyf.push_back(8); vyf.push_back(9); }
        if (pr_inv_applies(g)) { vyi.push_back(8); vyi.push_back(9); }
        if (pr_fwd_applies(g) && pr_inv_applies(g)) { vx.push_back(6); vx.push_back(7); }
        if (g.P >= 384) {   // their TMA-staged persistent forms (11: two CTAs per SM)
            if (pr_fwd_applies(g)) { vyf.push_back(10); vyf.push_back(11); }
            if (pr_inv_applies(g)) { vyi.push_back(10); vyi.push_back(11); }
            if (pr_fwd_applies(g) && pr_inv_applies(g)) {
                vx.push_back(8);
                vx.push_back(9);    // software-pipelined persistent forms
                vx.push_back(10);
            }
        }
        Work<float> w = work_of<float>(p, i);
        // fastest of the variants of one pass (timed only when not cached)
        auto pick = [&](const std::string &k, const std::vector<int> &vs, auto launch) {
            if (!g_tune.count(k) || std::find(vs.begin(), vs.end(), g_tune[k].variant) == vs.end()) {
                int best = vs[0];
                float tbest = 0.f;
                bool any = false;
                for (size_t j = 0; j < vs.size(); ++j) {
                    if (launch(vs[j]) != cudaSuccess) {   // a variant that cannot run here
                        (void)cudaGetLastError();
                        continue;
                    }
                    float t = time_launches([&] { return launch(vs[j]); }, a, b);
                    if (log) fprintf(stderr, "lindhard tune %s variant %d: %.4f ms\n", k.c_str(), vs[j], t / 5);
                    if (!any || t < tbest) { best = vs[j]; tbest = t; any = true; }
                }
                g_tune[k] = TuneEntry{best, std::string()};
            }
            return g_tune[k].variant;
        };
        p->yvar_fwd[i] = pick(kf, vyf, [&](int v) { return launch_fwd_y(g, w, 0, v); });
        if (p->precision[i] != LINDHARD_SPLITBF16_TC)
            p->yvar_inv[i] = pick(ki, vyi, [&](int v) { return launch_inv_y(g, w, 0, v); });
        p->xvar[i] = pick(kx, vx, [&](int v) { return launch_x_product(g, w, 0, v); });
        // the inverse energy pass writes the caller's output: time it into the
        // workspace's X buffer (at least as large as the output)
        std::vector<int> ve = {0, 1};
        if (et_inv_applies(g)) ve.push_back(2);
        p->evar[i] = pick(ke, ve, [&](int v) { return launch_inv_energy(g, w, (float *)w.X, 0, v); });
        e = cudaGetLastError();
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    tune_save();
    return e == cudaSuccess ? cudaDeviceSynchronize() : e;
}

extern "C" lindhard_status lindhard_plan_create(const lindhard_grid *grids, int batch, unsigned flags,
                                                lindhard_plan **out)
{
    if (!grids || !out || batch < 1) return fail(LINDHARD_EINVAL, "grids/out must be non-NULL and batch >= 1");
    const unsigned known = LINDHARD_PLAN_BACKWARD | LINDHARD_PLAN_CONCURRENT | LINDHARD_PLAN_GRAPH |
                           LINDHARD_PLAN_AUTOTUNE | LINDHARD_PLAN_ENERGY_DIRECT | LINDHARD_PLAN_PERSISTENT;
    if (flags & ~known) return fail(LINDHARD_EINVAL, "unknown plan flags");
    *out = nullptr;
    lindhard_plan *p = new (std::nothrow) lindhard_plan;
    if (!p) return fail(LINDHARD_ENOMEM, "host allocation failed");
    p->batch = batch;
    p->geoms.resize(batch);
    p->precision.resize(batch);
    p->backward = (flags & LINDHARD_PLAN_BACKWARD) != 0;
    p->graph = (flags & LINDHARD_PLAN_GRAPH) != 0;
    p->persistent = (flags & LINDHARD_PLAN_PERSISTENT) != 0;
    p->concurrent = p->graph || p->persistent || (flags & LINDHARD_PLAN_CONCURRENT) != 0;
    p->direct = (flags & LINDHARD_PLAN_ENERGY_DIRECT) != 0;
    if (p->persistent && (p->backward || p->direct)) {
        delete p;
        return fail(LINDHARD_EUNSUPPORTED, "the persistent batch launch is forward only, in the 3D form "
                                           "(not with LINDHARD_PLAN_BACKWARD or LINDHARD_PLAN_ENERGY_DIRECT)");
    }
    if (p->direct && p->backward) {
        delete p;
        return fail(LINDHARD_EUNSUPPORTED, "the energy-direct form is forward only (no LINDHARD_PLAN_BACKWARD)");
    }
    int maxLen = kMinLen, maxNpts = 1;
    for (int i = 0; i < batch; ++i) {
        lindhard_status st = make_geom(grids[i], p->geoms[i], p->precision[i]);
        if (st != LINDHARD_OK) {
            delete p;
            return st;
        }
        if (p->backward && p->precision[i] != LINDHARD_FP32) {
            delete p;
            return fail(LINDHARD_EUNSUPPORTED, "the backward pass is built for LINDHARD_FP32 grids");
        }
        if (p->direct && (p->precision[i] != LINDHARD_FP32 || p->geoms[i].quantity != LINDHARD_IMCHI ||
                          !direct_supported(p->geoms[i]))) {
            delete p;
            return fail(LINDHARD_EUNSUPPORTED, "the energy-direct form takes LINDHARD_FP32, LINDHARD_IMCHI grids "
                                               "with n_eps <= 1024 and n_omega <= 512");
        }
        if (p->persistent && (p->precision[i] != LINDHARD_FP32 || !ps_supported(p->geoms[i]))) {
            delete p;
            return fail(LINDHARD_EUNSUPPORTED, "the persistent batch launch takes LINDHARD_FP32, LINDHARD_IMCHI "
                                               "grids with zones > 1, q_extent = N, N + N/2 in {192, 384, 768, "
                                               "1536} and an energy FFT of 128, 256 or 512 points");
        }
        maxLen = std::max(maxLen, std::max(p->geoms[i].P, p->geoms[i].PE));
        maxNpts = std::max(maxNpts, p->geoms[i].npz * p->geoms[i].npz);
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "device query");
    }
    p->mu_G = mu_grid_size(p->num_sms, maxNpts);
    p->tw_len = maxLen;

    // bytes of each workspace part for instance i
    struct Need { size_t X, Y, Z, partial, axis, eps32, eps64; };
    auto need_of = [&](int i) {
        const Geom &g = p->geoms[i];
        size_t cb = cx_bytes(p->precision[i]);
        Need n;
        n.X = std::max((size_t)g.N * g.N * 2 * g.SP, (size_t)g.Q * (size_t)g.xs3) * cb;
        n.Y = std::max((size_t)g.N * (size_t)g.xs2, (size_t)g.Q * g.Q * g.SP) * cb;
        if (p->direct) {
            // X: planes, then the momentum transforms Z, then [Q][P][SPo];
            // Y: [N][P][2 SPt], then the correlations C, then [Q][Q][SPo]
            const DirectGeom d = direct_geom(g);
            n.X = std::max({(size_t)g.N * g.N * 2 * d.t.SP, (size_t)g.P * (size_t)d.zs,
                            (size_t)g.Q * (size_t)d.o.xs3}) * cb;
            n.Y = std::max({(size_t)g.N * (size_t)d.t.xs2, (size_t)g.P * (size_t)d.cs,
                            (size_t)g.Q * g.Q * d.o.SP}) * cb;
        }
        n.Z = p->backward ? (size_t)g.Q * (size_t)g.xs3 * cb : 0;
        // the last pass's per-CTA sums, then the first reduction level's
        n.partial = p->backward ? (size_t)(bw_energy_blocks(g) + bw_partial_extra_rows()) * 5 * sizeof(double) : 0;
        n.axis = (size_t)g.N * sizeof(AxisTab);
        n.eps32 = (size_t)g.n_eps * sizeof(float2);
        n.eps64 = (size_t)g.n_eps * sizeof(double);
        return n;
    };
    size_t o = 0;
    p->off_tw32 = o; o = align_up(o + (size_t)twiddle_entries() * sizeof(float2));
    p->off_tw64 = o; o = align_up(o + (size_t)twiddle_entries() * sizeof(double2));
    p->off_status = o; o = align_up(o + sizeof(unsigned));
    p->off_prtw = o; o = align_up(o + pr_twiddle_bytes());   // pruned engine's per-stage twiddles
    p->off_etw = o; o = align_up(o + et_twiddle_bytes());     // energy pass's per-stage twiddles
    p->off_dmu = o; o = align_up(o + sizeof(double) * 5 * kDmuBlocks);
    // tensor-core DFT matrices of every supported length (plans with a
    // LINDHARD_SPLITBF16_TC grid only)
    if (std::count(p->precision.begin(), p->precision.end(), (int)LINDHARD_SPLITBF16_TC) > 0) {
        p->off_tc = o; o = align_up(o + tc_mats_bytes());
    }
    if (p->persistent) {
        p->off_ps_inst = o; o = align_up(o + ps_inst_bytes() * batch);
        p->off_ps_seg = o; o = align_up(o + ps_seg_bytes() * 5 * batch);
        p->off_ps_cnt = o; o = align_up(o + sizeof(unsigned) * (5 * batch + 1));
        p->off_ps_band = o; o = align_up(o + sizeof(Band) * batch);
    }
    p->off_kk.assign(batch, 0);
    for (int i = 0; i < batch; ++i)
        if (p->precision[i] != LINDHARD_FP64) {
            p->off_kk[i] = o; o = align_up(o + kk_table_bytes(p->geoms[i].n_omega));
        }
    auto place = [&](const Need &n) {
        lindhard_plan::Slot sl;
        sl.X = o; o = align_up(o + n.X);
        sl.Y = o; o = align_up(o + n.Y);
        sl.Z = o; o = align_up(o + n.Z);
        sl.partial = o; o = align_up(o + n.partial);
        sl.axis = o; o = align_up(o + n.axis);
        sl.eps32 = o; o = align_up(o + n.eps32);
        sl.eps64 = o; o = align_up(o + n.eps64);
        sl.state = o; o = align_up(o + sizeof(InstState));
        sl.acc = o; o = align_up(o + mu_acc_doubles(p->mu_G) * sizeof(double));
        sl.bar = o; o = align_up(o + mu_barrier_words() * sizeof(unsigned));
        return sl;
    };
    if (p->concurrent) {
        for (int i = 0; i < batch; ++i) p->slots.push_back(place(need_of(i)));
    } else {
        Need m = {0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < batch; ++i) {
            Need n = need_of(i);
            m.X = std::max(m.X, n.X); m.Y = std::max(m.Y, n.Y); m.Z = std::max(m.Z, n.Z);
            m.partial = std::max(m.partial, n.partial); m.axis = std::max(m.axis, n.axis);
            m.eps32 = std::max(m.eps32, n.eps32); m.eps64 = std::max(m.eps64, n.eps64);
        }
        p->slots.push_back(place(m));
    }
    p->ws_bytes = o;
    e = cudaMalloc(&p->ws, p->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return fail(LINDHARD_ENOMEM, std::string("workspace cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemset(p->ws + p->off_status, 0, sizeof(unsigned));
    for (auto &sl : p->slots)
        if (e == cudaSuccess) e = cudaMemset(p->ws + sl.bar, 0, mu_barrier_words() * sizeof(unsigned));
    if (e == cudaSuccess)
        e = launch_twiddles(p->tw_len, (float2 *)(p->ws + p->off_tw32), (double2 *)(p->ws + p->off_tw64), 0);
    if (e == cudaSuccess) e = launch_pr_twiddles((float2 *)(p->ws + p->off_prtw), 0);
    if (e == cudaSuccess) e = launch_et_twiddles((float2 *)(p->ws + p->off_etw), 0);
    if (e == cudaSuccess && p->off_tc) e = launch_tc_mats(p->ws + p->off_tc, 0);
    for (int i = 0; i < batch && e == cudaSuccess; ++i)
        if (p->off_kk[i]) e = launch_kk_tables(p->geoms[i].n_omega, p->ws + p->off_kk[i], 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && p->concurrent) {
        int ns = std::min(batch, 16);
        p->streams.resize(ns);
        p->join_ev.resize(ns);
        e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
        for (int k = 0; k < ns && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&p->streams[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join_ev[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess && p->graph) e = cudaStreamCreateWithFlags(&p->origin, cudaStreamNonBlocking);
        // instances to streams longest first, each to the stream with the
        // least work so far (work ~ transform points P^2 PE), so that the
        // streams end together instead of one long stream finishing alone
        std::vector<int> order(batch);
        std::vector<double> work(batch), load(ns, 0.0);
        for (int i = 0; i < batch; ++i) {
            order[i] = i;
            work[i] = (double)p->geoms[i].P * p->geoms[i].P * p->geoms[i].PE;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
        p->stream_of.assign(batch, 0);
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            p->stream_of[i] = k;
            load[k] += work[i];
        }
    }
    p->yvar_fwd.assign(batch, 1);
    p->yvar_inv.assign(batch, 1);
    for (int i = 0; i < batch; ++i)
        if (p->precision[i] == LINDHARD_SPLITBF16_TC) p->yvar_inv[i] = 7;   // tensor-core inverse p_y pass
    p->xvar.assign(batch, 0);
    p->evar.assign(batch, 0);
    if (e == cudaSuccess && (flags & LINDHARD_PLAN_AUTOTUNE) && !p->direct) e = autotune(p);
    if (e == cudaSuccess && p->persistent) {
        // the instances' entries and the queue: every tile of pass 0 of every
        // instance, then pass 1, ... (each dependency lies earlier in the queue)
        std::vector<unsigned char> hi(ps_inst_bytes() * batch), hs(ps_seg_bytes() * 5 * batch);
        long long o_off = 0;
        for (int i = 0; i < batch; ++i) {
            Work<float> w = work_of<float>(p, i);
            ps_fill_inst(hi.data() + ps_inst_bytes() * i, p->geoms[i], w.X, w.Y, w.axis, w.eps, w.state,
                         (const Band *)(p->ws + p->off_ps_band) + i, o_off);
            o_off += (long long)p->geoms[i].Q * p->geoms[i].Q * p->geoms[i].n_omega;
        }
        int start = 0, k = 0;
        for (int pass = 0; pass < 5; ++pass)
            for (int i = 0; i < batch; ++i) {
                const int n = ps_pass_tiles(p->geoms[i], pass);
                ps_fill_seg(hs.data() + ps_seg_bytes() * k++, i, pass, start, n);
                start += n;
            }
        p->ps_nsegs = k;
        p->ps_total = start;
        for (int i = 0; i < batch; ++i) p->ps_smem = std::max(p->ps_smem, ps_inst_smem_elems(p->geoms[i]));
        p->ps_grid = ps_grid(p->num_sms, p->ps_smem);
        e = cudaMemcpy(p->ws + p->off_ps_inst, hi.data(), hi.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->ws + p->off_ps_seg, hs.data(), hs.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        lindhard_plan_destroy(p);
        return cuda_fail(e, "plan set-up");
    }
    *out = p;
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_sizes(const lindhard_plan *p, int index, lindhard_sizes *out)
{
    if (!p || !out || index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "bad plan/index/out");
    const Geom &g = p->geoms[index];
    long long cb = (long long)cx_bytes(p->precision[index]);
    long long rb = cb / 2;
    out->N = g.N;
    out->n_eps = g.n_eps;
    out->n_omega = g.n_omega;
    out->q_extent = g.Q;
    out->fft_p = g.P;
    out->fft_e = g.PE;
    out->out_elems = (long long)g.Q * g.Q * g.n_omega;
    out->a_elems = (long long)g.N * g.N * g.n_eps;
    // each intermediate written once and read once; only its non-redundant
    // (valid) entries count
    long long W1 = (long long)g.N * g.N * 2 * g.H;
    long long W2 = (long long)g.N * g.P * 2 * g.H;
    long long W3 = (long long)g.Q * g.P * g.H;
    long long W4 = (long long)g.Q * g.Q * g.H;
    out->hbm_bytes_forward = 2 * (W1 + W2 + W3 + W4) * cb + out->out_elems * rb;
    // set-up (tables + multisection pass 0), multisection pass 1, Halley step, 5 FFT passes;
    // zones of at most 98 points solve mu inside the set-up launch
    out->kernels_forward = mu_solve_in_setup(g) ? 6 : 8;
    // persistent plans: the instance's set-up launches (the batch's passes
    // are one further launch of the plan)
    if (p->persistent) out->kernels_forward = mu_solve_in_setup(g) ? 1 : 3;
    if (p->direct) {
        // planes, p_y, p_x, correlation, k_x inverse, k_y inverse, output; the
        // same write-once read-once count over the direct form's intermediates
        const DirectGeom d = direct_geom(g);
        const long long T = d.T, n = g.n_omega;
        out->hbm_bytes_forward = 2 * ((long long)g.N * g.N * T + (long long)g.N * g.P * T + (long long)g.P * g.P * T +
                                      (long long)g.P * g.P * n + (long long)g.Q * g.P * n + (long long)g.Q * g.Q * n) * cb +
                                 out->out_elems * rb;
        out->kernels_forward = mu_solve_in_setup(g) ? 8 : 10;
    }
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_workspace_bytes(const lindhard_plan *p, size_t *out)
{
    if (!p || !out) return fail(LINDHARD_EINVAL, "bad plan/out");
    *out = p->ws_bytes;
    return LINDHARD_OK;
}

// The temperature fields of a band (all that a caller-supplied A needs).
static lindhard_status band_temperature(const lindhard_band *b, Band &o)
{
    if (!(b->kT >= 0) || !isfinite(b->kT)) return fail(LINDHARD_EINVAL, "kT must be finite and >= 0");
    o.kT = b->kT;
    o.x_step64 = 0.0;
    o.x_step = 0.0f;
    return LINDHARD_OK;
}

// kT against the grid's quantity, and e_j / kT = (2 j + 1 - n_eps) x_step.
static lindhard_status band_for_geom(const Geom &g, Band &o)
{
    if (g.quantity == LINDHARD_IMCHI && o.kT != 0.0)
        return fail(LINDHARD_EINVAL, "kT must be 0 for LINDHARD_IMCHI grids (use LINDHARD_IMCHI_T or LINDHARD_SQW)");
    if (g.quantity != LINDHARD_IMCHI && !(o.kT > 0))
        return fail(LINDHARD_EINVAL, "LINDHARD_IMCHI_T and LINDHARD_SQW grids need kT > 0");
    if (o.kT > 0) {
        // capped so that the centre cell of an odd grid (2j + 1 = n_eps) keeps
        // x = 0 * step = 0 (f = 1/2) for any kT; every other cell saturates to
        // f = 0 or 1 long before the cap
        o.x_step64 = std::min(0.5 * g.de / o.kT, 1e30);
        o.x_step = (float)o.x_step64;
    }
    return LINDHARD_OK;
}

static lindhard_status make_band(const lindhard_band *b, Band &o)
{
    if (!b) return fail(LINDHARD_EINVAL, "bands must be non-NULL when A is generated");
    if (b->reserved != 0) return fail(LINDHARD_EINVAL, "band.reserved must be 0");
    if (b->band_kind != 0 && b->band_kind != 1) return fail(LINDHARD_EINVAL, "band_kind must be 0 or 1");
    if (!(b->gamma > 0) || !isfinite(b->gamma)) return fail(LINDHARD_EINVAL, "gamma must be finite and > 0");
    if (!(b->ff_a >= 0) || !isfinite(b->ff_a)) return fail(LINDHARD_EINVAL, "ff_a must be finite and >= 0");
    if (!isfinite(b->t) || !isfinite(b->tp) || !isfinite(b->tpp))
        return fail(LINDHARD_EINVAL, "hoppings must be finite");
    o.t = b->t;
    o.tp = b->tp;
    o.tpp = b->tpp;
    o.mu = b->mu;
    o.filling = b->filling;
    o.gamma = b->gamma;
    o.ff_a = b->ff_a;
    o.band_kind = b->band_kind;
    o.solve_mu = isnan(b->filling) ? 0 : 1;
    auto pair = [](double x, float *out) {
        out[0] = (float)x;
        out[1] = (float)(x - (double)out[0]);
    };
    pair(-2.0 * b->t, o.k1);
    pair(-4.0 * b->tp, o.k2);
    pair(-2.0 * b->tpp, o.k3);
    o.gam_pi = (float)(b->gamma / M_PI);
    o.gam2 = (float)(b->gamma * b->gamma);
    lindhard_status st = band_temperature(b, o);
    if (st != LINDHARD_OK) return st;
    if (o.solve_mu) {
        if (!(b->filling > 0 && b->filling < 2)) return fail(LINDHARD_EINVAL, "filling must be in (0, 2) or NaN");
    } else if (!isfinite(b->mu)) {
        return fail(LINDHARD_EINVAL, "mu must be finite when filling is NaN");
    }
    return LINDHARD_OK;
}

template <typename Real>
static Work<Real> work_of(lindhard_plan *p, int i)
{
    const lindhard_plan::Slot &sl = p->slots[p->concurrent ? i : 0];
    Work<Real> w;
    w.X = p->ws + sl.X;
    w.Y = p->ws + sl.Y;
    w.axis = (AxisTab *)(p->ws + sl.axis);
    w.eps = sizeof(Real) == 4 ? (void *)(p->ws + sl.eps32) : (void *)(p->ws + sl.eps64);
    w.tw = sizeof(Real) == 4 ? (const void *)(p->ws + p->off_tw32) : (const void *)(p->ws + p->off_tw64);
    w.tw_len = p->tw_len;
    w.tc = p->off_tc ? (const void *)(p->ws + p->off_tc) : nullptr;
    w.ptw = sizeof(Real) == 4 ? (const void *)(p->ws + p->off_prtw) : nullptr;
    w.etw = sizeof(Real) == 4 ? (const void *)(p->ws + p->off_etw) : nullptr;
    w.state = (InstState *)(p->ws + sl.state);
    w.status = (unsigned *)(p->ws + p->off_status);
    w.mu_acc = (double *)(p->ws + sl.acc);
    w.barrier = (unsigned *)(p->ws + sl.bar);
    return w;
}

// Stream that runs instance i: the caller's stream, or in concurrent plans
// one of the plan's streams (forked from `s` by fork_begin).
static cudaStream_t inst_stream(lindhard_plan *p, int i, cudaStream_t s)
{
    return p->concurrent ? p->streams[p->stream_of[i]] : s;
}
static cudaError_t fork_begin(lindhard_plan *p, cudaStream_t s)
{
    if (!p->concurrent) return cudaSuccess;
    cudaError_t e = cudaEventRecord(p->fork_ev, s);
    for (size_t k = 0; k < p->streams.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->streams[k], p->fork_ev, 0);
    return e;
}
static cudaError_t fork_end(lindhard_plan *p, cudaStream_t s)
{
    if (!p->concurrent) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < p->streams.size() && e == cudaSuccess; ++k) {
        e = cudaEventRecord(p->join_ev[k], p->streams[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join_ev[k], 0);
    }
    return e;
}

// The band of one instance for a call: every field when A is generated; with
// a caller-supplied A only the temperature, and only for finite-temperature
// grids.
static lindhard_status band_of_instance(const Geom &g, const lindhard_band *b, bool generate, Band &o)
{
    lindhard_status st = LINDHARD_OK;
    o = Band{};
    if (generate) {
        st = make_band(b, o);
        if (st == LINDHARD_OK && o.band_kind == 1 && g.periodic)
            st = fail(LINDHARD_EINVAL, "free electrons need zones > 1 (the band is not periodic)");
    } else if (g.quantity != LINDHARD_IMCHI) {
        if (!b) return fail(LINDHARD_EINVAL, "finite-temperature grids need bands (kT) with a caller-supplied A");
        st = band_temperature(b, o);
    }
    return st == LINDHARD_OK ? band_for_geom(g, o) : st;
}

static lindhard_status bands_of(lindhard_plan *p, const lindhard_band *bands, bool generate, std::vector<Band> &bs)
{
    for (int i = 0; i < p->batch; ++i) {
        lindhard_status st = band_of_instance(p->geoms[i], bands ? bands + i : nullptr, generate, bs[i]);
        if (st != LINDHARD_OK) return st;
    }
    return LINDHARD_OK;
}

// Enqueues the forward sequence of every instance (per-pass timing only in
// sequential plans).
// The persistent batch launch: each instance's set-up and chemical-potential
// launches on the plan's streams (which also store the call's band for the
// launch), then the completion counters cleared and the one launch of every
// instance's five passes.
static cudaError_t enqueue_persistent(lindhard_plan *p, const std::vector<Band> &bs, float *out, double *mu_out,
                                      cudaStream_t s0)
{
    cudaError_t e = fork_begin(p, s0);
    for (int i = 0; i < p->batch && e == cudaSuccess; ++i) {
        const Geom &g = p->geoms[i];
        cudaStream_t s = inst_stream(p, i, s0);
        Work<float> w = work_of<float>(p, i);
        e = launch_setup_band(g, bs[i], w.axis, (float2 *)w.eps, nullptr, w.state, w.mu_acc, w.barrier, w.status,
                              mu_out ? mu_out + i : nullptr, p->mu_G, (Band *)(p->ws + p->off_ps_band) + i, s);
        if (e == cudaSuccess)
            e = launch_solve_mu(g, bs[i], w.axis, w.state, w.mu_acc, w.barrier, w.status, mu_out ? mu_out + i : nullptr,
                                p->mu_G, s);
    }
    if (e == cudaSuccess) e = fork_end(p, s0);
    unsigned *cnt = (unsigned *)(p->ws + p->off_ps_cnt);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (5 * p->batch + 1), s0);
    if (e == cudaSuccess)
        e = launch_persistent(p->ws + p->off_ps_inst, p->ws + p->off_ps_seg, p->ps_nsegs, p->ps_total,
                              cnt + 5 * p->batch, cnt, (unsigned *)(p->ws + p->off_status), out,
                              (const float2 *)(p->ws + p->off_prtw), (const float2 *)(p->ws + p->off_etw), p->wait_ns,
                              p->stall_inst, p->ps_smem, p->ps_grid, s0);
    return e;
}

template <typename Real>
static cudaError_t enqueue_forward(lindhard_plan *p, const std::vector<Band> &bs, const Real *A_in, Real *out,
                                   double *mu_out, cudaStream_t s0)
{
    if constexpr (sizeof(Real) == 4)
        if (p->persistent && A_in == nullptr) return enqueue_persistent(p, bs, out, mu_out, s0);
    cudaError_t e = fork_begin(p, s0);
    size_t a_off = 0, o_off = 0;
    for (int i = 0; i < p->batch && e == cudaSuccess; ++i) {
        const Geom &g = p->geoms[i];
        const Band &b = bs[i];
        cudaStream_t s = inst_stream(p, i, s0);
        Work<Real> w = work_of<Real>(p, i);
        if (A_in == nullptr) {
            e = timed(p, 0, s, [&] {
                return launch_setup(g, b, w.axis, sizeof(Real) == 4 ? (float2 *)w.eps : nullptr,
                                    sizeof(Real) == 8 ? (double *)w.eps : nullptr, w.state, w.mu_acc, w.barrier,
                                    w.status, mu_out ? mu_out + i : nullptr, p->mu_G, s);
            });
            if (e == cudaSuccess)
                e = timed(p, 1, s, [&] {
                    return launch_solve_mu(g, b, w.axis, w.state, w.mu_acc, w.barrier, w.status,
                                           mu_out ? mu_out + i : nullptr, p->mu_G, s);
                });
        }
        const Real *a_i = A_in ? A_in + a_off : nullptr;
        Real *o_i = out + o_off;
        if constexpr (sizeof(Real) == 4) {
            if (p->direct) {
                // planes, p_y, p_x + energy correlation + k_x inverse, k_y inverse, output
                for (int k = 0; k < 5 && e == cudaSuccess; ++k)
                    e = timed(p, 2 + k, s, [&] { return launch_direct_stage(k, g, b, w, a_i, o_i, s); });
                a_off += (size_t)g.N * g.N * g.n_eps;
                o_off += (size_t)g.Q * g.Q * g.n_omega;
                continue;
            }
        }
        if (e == cudaSuccess) e = timed(p, 2, s, [&] { return launch_fwd_energy(g, b, w, a_i, s); });
        if (e == cudaSuccess) e = timed(p, 3, s, [&] { return launch_fwd_y(g, w, s, p->yvar_fwd[i]); });
        if (e == cudaSuccess) e = timed(p, 4, s, [&] { return launch_x_product(g, w, s, p->xvar[i]); });
        if (e == cudaSuccess) e = timed(p, 5, s, [&] { return launch_inv_y(g, w, s, p->yvar_inv[i]); });
        if (e == cudaSuccess) e = timed(p, 6, s, [&] { return launch_inv_energy(g, w, o_i, s, p->evar[i]); });
        a_off += (size_t)g.N * g.N * g.n_eps;
        o_off += (size_t)g.Q * g.Q * g.n_omega;
    }
    if (e == cudaSuccess) e = fork_end(p, s0);
    return e;
}

template <typename Real>
static lindhard_status forward_impl(lindhard_plan *p, const lindhard_band *bands, const Real *A_in, Real *out,
                                    double *mu_out, void *stream, int want_prec)
{
    if (!p || !out) return fail(LINDHARD_EINVAL, "plan and out must be non-NULL");
    for (int i = 0; i < p->batch; ++i)
        if ((p->precision[i] == LINDHARD_FP64) != (want_prec == LINDHARD_FP64))
            return fail(LINDHARD_EINVAL, "plan precision does not match the entry point");
    std::vector<Band> bs(p->batch);
    {
        lindhard_status st = bands_of(p, bands, A_in == nullptr, bs);
        if (st != LINDHARD_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->graph) {
        cudaError_t e = enqueue_forward<Real>(p, bs, A_in, out, mu_out, s);
        return e == cudaSuccess ? LINDHARD_OK : cuda_fail(e, "forward launch");
    }
    // Graph mode.  The captured graph holds the call's pointers and band
    // values; a call that differs in any of them captures again and updates
    // the executable graph in place.
    bool same = p->exec && p->key_A == (const void *)A_in && p->key_out == (void *)out && p->key_mu == mu_out;
    bool reads_bands = A_in == nullptr;
    for (int i = 0; i < p->batch; ++i) reads_bands = reads_bands || p->geoms[i].quantity != LINDHARD_IMCHI;
    if (same && reads_bands) {
        same = p->key_bands.size() == (size_t)p->batch;
        for (int i = 0; i < p->batch && same; ++i) same = memcmp(&p->key_bands[i], &bands[i], sizeof(lindhard_band)) == 0;
    }
    cudaError_t e = cudaSuccess;
    if (!same) {
        if (!p->warmed) {
            // one eager run outside capture: first launches of each kernel set
            // their shared-memory attributes, which is not a stream operation
            e = enqueue_forward<Real>(p, bs, A_in, out, mu_out, s);
            if (e != cudaSuccess) return cuda_fail(e, "forward launch");
            p->warmed = true;
        }
        const unsigned prof = p->profile;
        p->profile = 0;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(p->origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_forward<Real>(p, bs, A_in, out, mu_out, p->origin);
            e = cudaStreamEndCapture(p->origin, &graph);
            if (e == cudaSuccess) e = e2;
        }
        p->profile = prof;
        if (e == cudaSuccess) {
            cudaGraphExecUpdateResultInfo info;
            if (!p->exec || cudaGraphExecUpdate(p->exec, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                if (p->exec) cudaGraphExecDestroy(p->exec);
                p->exec = nullptr;
                e = cudaGraphInstantiate(&p->exec, graph, 0);
            }
        }
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->exec = nullptr;
            return cuda_fail(e, "graph capture");
        }
        p->key_A = A_in;
        p->key_out = out;
        p->key_mu = mu_out;
        p->key_bands.assign(bands ? bands : nullptr, bands ? bands + p->batch : nullptr);
        if (!bands) p->key_bands.clear();
    }
    e = cudaGraphLaunch(p->exec, s);
    return e == cudaSuccess ? LINDHARD_OK : cuda_fail(e, "graph launch");
}

extern "C" lindhard_status lindhard_imchi(lindhard_plan *p, const lindhard_band *bands, const float *A_in,
                                          float *out, double *mu_out, void *stream)
{
    return forward_impl<float>(p, bands, A_in, out, mu_out, stream, LINDHARD_FP32);
}

extern "C" lindhard_status lindhard_imchi_f64(lindhard_plan *p, const lindhard_band *bands, const double *A_in,
                                              double *out, double *mu_out, void *stream)
{
    return forward_impl<double>(p, bands, A_in, out, mu_out, stream, LINDHARD_FP64);
}

extern "C" lindhard_status lindhard_imchi_backward(lindhard_plan *p, const lindhard_band *bands, const float *A_in,
                                                   const float *w, float *dA, double *dparams, void *stream)
{
    if (!p || !w) return fail(LINDHARD_EINVAL, "plan and w must be non-NULL");
    if (!p->backward) return fail(LINDHARD_EINVAL, "create the plan with LINDHARD_PLAN_BACKWARD");
    if (!dA && !dparams) return fail(LINDHARD_EINVAL, "nothing to compute: dA and dparams are both NULL");
    if (dparams && A_in) return fail(LINDHARD_EINVAL, "dparams needs the generated A (A_in must be NULL)");
    std::vector<Band> bs(p->batch);
    {
        lindhard_status st = bands_of(p, bands, A_in == nullptr, bs);
        if (st != LINDHARD_OK) return st;
    }
    cudaStream_t s0 = (cudaStream_t)stream;
    size_t a_off = 0, o_off = 0;
    cudaError_t ef = fork_begin(p, s0);
    if (ef != cudaSuccess) return cuda_fail(ef, "backward launch");
    for (int i = 0; i < p->batch; ++i) {
        const Geom &g = p->geoms[i];
        const Band &b = bs[i];
        cudaStream_t s = inst_stream(p, i, s0);
        Work<float> wk = work_of<float>(p, i);
        const lindhard_plan::Slot &sl = p->slots[p->concurrent ? i : 0];
        float2 *X = (float2 *)wk.X, *Y = (float2 *)wk.Y, *Z = (float2 *)(p->ws + sl.Z);
        const float2 *tw = (const float2 *)wk.tw;
        double *partial = (double *)(p->ws + sl.partial);
        cudaError_t e = cudaSuccess;
        if (A_in == nullptr) {
            e = launch_setup(g, b, wk.axis, (float2 *)wk.eps, nullptr, wk.state, wk.mu_acc, wk.barrier, wk.status,
                             nullptr, p->mu_G, s);
            if (e == cudaSuccess)
                e = launch_solve_mu(g, b, wk.axis, wk.state, wk.mu_acc, wk.barrier, wk.status, nullptr, p->mu_G, s);
        }
        if (e == cudaSuccess) e = launch_fwd_energy(g, b, wk, A_in ? A_in + a_off : nullptr, s);   // X = U1
        if (e == cudaSuccess) e = launch_fwd_y(g, wk, s, p->yvar_fwd[i]);                           // Y = U2
        if (e == cudaSuccess) e = launch_w_energy(g, w + o_off, X, tw, p->tw_len, s);                // X = WU1
        if (e == cudaSuccess) e = launch_w_y(g, X, Z, tw, p->tw_len, s);                             // Z = WU2
        if (e == cudaSuccess) e = launch_bw_product(g, Y, Z, tw, p->tw_len, (const float2 *)wk.ptw, s);              // Y = G3
        if (e == cudaSuccess) e = launch_bw_inv_y(g, Y, X, tw, p->tw_len, s);                        // X = G4
        if (e == cudaSuccess)
            e = launch_bw_inv_energy(g, b, wk.axis, (const float2 *)wk.eps, wk.state, X, dA ? dA + a_off : nullptr,
                                     dparams ? partial : nullptr, tw, p->tw_len, s);
        if (e == cudaSuccess && dparams) e = launch_reduce_params(partial, bw_energy_blocks(g), dparams + 5 * i, s);
        if (e != cudaSuccess) return cuda_fail(e, "backward launch");
        a_off += (size_t)g.N * g.N * g.n_eps;
        o_off += (size_t)g.Q * g.Q * g.n_omega;
    }
    ef = fork_end(p, s0);
    return ef == cudaSuccess ? LINDHARD_OK : cuda_fail(ef, "backward launch");
}

extern "C" lindhard_status lindhard_sum_rule(lindhard_plan *p, int index, const lindhard_band *band,
                                             const float *A_in, const float *out, double *sum_q, double *dos_corr,
                                             void *stream)
{
    if (!p || !out || !sum_q || !dos_corr) return fail(LINDHARD_EINVAL, "plan, out, sum_q, dos_corr must be non-NULL");
    if (index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "index out of range");
    if (p->precision[index] == LINDHARD_FP64) return fail(LINDHARD_EINVAL, "the sum rule reads FP32 outputs");
    const Geom &g = p->geoms[index];
    if (g.Q != (g.periodic ? g.N : 2 * g.N))
        return fail(LINDHARD_EINVAL, "the sum rule needs every lag: q_extent = N (one zone) or 2N (several)");
    Band b = {};
    {
        lindhard_status st = band_of_instance(g, band, A_in == nullptr, b);
        if (st != LINDHARD_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Work<float> w = work_of<float>(p, index);
    // D(e) lives in the instance's X buffer (at least n_eps doubles)
    double *D = (double *)w.X;
    cudaError_t e = cudaSuccess;
    if (A_in == nullptr) {
        e = launch_setup(g, b, w.axis, (float2 *)w.eps, nullptr, w.state, w.mu_acc, w.barrier, w.status, nullptr,
                         p->mu_G, s);
        if (e == cudaSuccess)
            e = launch_solve_mu(g, b, w.axis, w.state, w.mu_acc, w.barrier, w.status, nullptr, p->mu_G, s);
    }
    if (e == cudaSuccess)
        e = launch_sum_rule(g, b, w.axis, (const float2 *)w.eps, w.state, A_in, out, D, sum_q, dos_corr, s);
    return e == cudaSuccess ? LINDHARD_OK : cuda_fail(e, "sum-rule launch");
}

extern "C" lindhard_status lindhard_dmu_dparams(lindhard_plan *p, int index, const lindhard_band *band, double mu,
                                                double *out, void *stream)
{
    if (!p || !band || !out) return fail(LINDHARD_EINVAL, "plan, band and out must be non-NULL");
    if (index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "index out of range");
    if (!isfinite(mu) || !(band->gamma > 0) || !isfinite(band->gamma) || !isfinite(band->t) || !isfinite(band->tp) ||
        !isfinite(band->tpp) || (band->band_kind != 0 && band->band_kind != 1))
        return fail(LINDHARD_EINVAL, "band parameters and mu must be finite, gamma > 0, band_kind 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    double *part = (double *)(p->ws + p->off_dmu);
    cudaError_t e = launch_dmu_partials(band->band_kind, band->t, band->tp, band->tpp, band->gamma,
                                        p->geoms[index].npz, mu, part, kDmuBlocks, s);
    double h[5 * kDmuBlocks];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, part, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "dmu reduction");
    double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < kDmuBlocks; ++b)
        for (int r = 0; r < 5; ++r) sum[r] += h[b * 5 + r];
    if (!(sum[0] > 0)) return fail(LINDHARD_EINVAL, "dn/dmu vanishes at this mu");
    for (int r = 0; r < 4; ++r) out[r] = -sum[r + 1] / sum[0];
    return LINDHARD_OK;
}

// Envelope of -Im chi along the [100] cut q = (q_x, 0) at transfer index m
// (Sec. 4, Fig. 5: its decay with q fitted by 1 / (1 + (q/k0)^2)).  The cut
// (Q values, stride Q n_omega floats in the output) is read with one strided
// copy; the zone maxima and the one-parameter least-squares fit are host work
// on Q values: for each reciprocal-lattice zone n >= 0 along the cut (lag
// offsets [n npz - npz/2, n npz + npz/2) from Q/2) that the lag window holds
// whole, the first largest -Im chi
// and its q; normalised by the largest of them; k0 minimises the squared
// residuals over the points with q > 0 (golden-section search over ln k0 in
// [ln dp, ln (Q dp)], 200 steps).
extern "C" lindhard_status lindhard_envelope_k0(lindhard_plan *p, int index, const float *imchi, int m, double *k0,
                                                double *q_out, double *y_out, int max_points, int *npoints,
                                                void *stream)
{
    if (!p || !imchi || !k0) return fail(LINDHARD_EINVAL, "plan, imchi and k0 must be non-NULL");
    if (index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "index out of range");
    if (p->precision[index] == LINDHARD_FP64) return fail(LINDHARD_EINVAL, "the envelope reads FP32 outputs");
    const Geom &g = p->geoms[index];
    if (g.quantity == LINDHARD_SQW) return fail(LINDHARD_EINVAL, "the envelope reads Im chi (not S(q, w))");
    if (m < 0 || m >= g.n_omega) return fail(LINDHARD_EINVAL, "transfer index out of range");
    if ((q_out || y_out) && max_points < 1) return fail(LINDHARD_EINVAL, "max_points must be >= 1");
    const int Q = g.Q, npz = g.npz;
    std::vector<float> cut(Q);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpy2DAsync(cut.data(), sizeof(float), imchi + (size_t)(Q / 2) * g.n_omega + m,
                                      sizeof(float) * (size_t)Q * g.n_omega, sizeof(float), Q,
                                      cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cut copy");
    const double dp = 2.0 * M_PI / npz;
    std::vector<double> qs, ys;
    for (int n = 0;; ++n) {
        const int lo = Q / 2 + n * npz - npz / 2, hi = lo + npz;
        if (lo < 0 || hi > Q) break;   // only zones the lag window holds whole
        int best = lo;
        for (int l = lo + 1; l < hi; ++l)
            if (-(double)cut[l] > -(double)cut[best]) best = l;
        qs.push_back((best - Q / 2) * dp);
        ys.push_back(-(double)cut[best]);
    }
    double ymax = 0.0;
    for (double y : ys) ymax = std::max(ymax, y);
    if (qs.empty() || !(ymax > 0)) return fail(LINDHARD_EINVAL, "-Im chi has no positive zone maximum on the cut");
    for (double &y : ys) y /= ymax;
    auto cost = [&](double lk) {
        const double k = exp(lk);
        double c = 0.0;
        for (size_t i = 0; i < qs.size(); ++i)
            if (qs[i] > 0) {
                const double r = ys[i] - 1.0 / (1.0 + (qs[i] / k) * (qs[i] / k));
                c += r * r;
            }
        return c;
    };
    double a = log(dp), b = log(Q * dp);
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double c = b - gr * (b - a), d = a + gr * (b - a), fc = cost(c), fd = cost(d);
    for (int it = 0; it < 200; ++it) {
        if (fc <= fd) {
            b = d; d = c; fd = fc;
            c = b - gr * (b - a);
            fc = cost(c);
        } else {
            a = c; c = d; fc = fd;
            d = a + gr * (b - a);
            fd = cost(d);
        }
    }
    *k0 = exp(0.5 * (a + b));
    const int np = (int)qs.size();
    if (npoints) *npoints = np;
    for (int i = 0; i < std::min(np, max_points); ++i) {
        if (q_out) q_out[i] = qs[i];
        if (y_out) y_out[i] = ys[i];
    }
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_kk_rpa(lindhard_plan *p, int index, const float *imchi, float *re_out,
                                           float *rpa_out, double v0, int variant, void *stream)
{
    if (!p || !imchi || !re_out) return fail(LINDHARD_EINVAL, "plan, imchi and re_out must be non-NULL");
    if (index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "index out of range");
    if (p->precision[index] == LINDHARD_FP64) return fail(LINDHARD_EINVAL, "the Kramers-Kronig pass reads FP32 outputs");
    if (variant != 0 && variant != 1) return fail(LINDHARD_EINVAL, "variant must be 0 (tensor cores) or 1 (FP32 SIMT)");
    if (!isfinite(v0)) return fail(LINDHARD_EINVAL, "v0 must be finite");
    const Geom &g = p->geoms[index];
    if (g.quantity == LINDHARD_SQW) return fail(LINDHARD_EINVAL, "the Kramers-Kronig pass reads Im chi (not S(q, w))");
    if (g.n_omega > (variant == 0 ? 256 : 1536))
        return fail(LINDHARD_EUNSUPPORTED, variant == 0 ? "the tensor-core form takes n_omega <= 256"
                                                        : "the SIMT form takes n_omega <= 1536");
    if (rpa_out && (reinterpret_cast<uintptr_t>(rpa_out) & 7u))
        return fail(LINDHARD_EINVAL, "rpa_out must be 8-byte aligned");
    cudaError_t e = launch_kk_rpa(g, imchi, re_out, reinterpret_cast<float2 *>(rpa_out), p->ws + p->off_kk[index], v0,
                                  variant, (unsigned *)(p->ws + p->off_status), (cudaStream_t)stream);
    return e == cudaSuccess ? LINDHARD_OK : cuda_fail(e, "Kramers-Kronig launch");
}

extern "C" lindhard_status lindhard_plan_profile_passes(lindhard_plan *p, unsigned mask)
{
    if (!p) return fail(LINDHARD_EINVAL, "plan must be non-NULL");
    mask &= (1u << LINDHARD_NUM_PASSES) - 1;
    if (mask && p->concurrent) return fail(LINDHARD_EUNSUPPORTED, "per-pass timing needs a sequential plan");
    drain_events(p);
    for (int i = 0; i < LINDHARD_NUM_PASSES; ++i) { p->pass_ms[i] = 0; p->pass_n[i] = 0; }
    p->profile = mask;
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_profile(lindhard_plan *p, int enable)
{
    return lindhard_plan_profile_passes(p, enable ? (1u << LINDHARD_NUM_PASSES) - 1 : 0u);
}

extern "C" lindhard_status lindhard_plan_pass_times(lindhard_plan *p, double *ms, long long *launches)
{
    if (!p || !ms || !launches) return fail(LINDHARD_EINVAL, "plan/ms/launches must be non-NULL");
    drain_events(p);
    for (int i = 0; i < LINDHARD_NUM_PASSES; ++i) { ms[i] = p->pass_ms[i]; launches[i] = p->pass_n[i]; }
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_set_wait_limit(lindhard_plan *p, unsigned long long wait_ns,
                                                        int stall_instance)
{
    if (!p) return fail(LINDHARD_EINVAL, "plan must be non-NULL");
    if (!p->persistent) return fail(LINDHARD_EINVAL, "the wait limit belongs to LINDHARD_PLAN_PERSISTENT plans");
    if (stall_instance < -1 || stall_instance >= p->batch) return fail(LINDHARD_EINVAL, "stall_instance out of range");
    p->wait_ns = wait_ns ? wait_ns : 1000000000ull;
    p->stall_inst = stall_instance;
    p->key_out = nullptr;   // a graph plan records again with the new values
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_variants(const lindhard_plan *p, int index, int *out)
{
    if (!p || !out) return fail(LINDHARD_EINVAL, "plan and out must be non-NULL");
    if (index < 0 || index >= p->batch) return fail(LINDHARD_EINVAL, "index out of range");
    out[0] = p->yvar_fwd[index];
    out[1] = p->yvar_inv[index];
    out[2] = p->xvar[index];
    out[3] = p->evar[index];
    return LINDHARD_OK;
}

extern "C" lindhard_status lindhard_plan_status(lindhard_plan *p, void *stream)
{
    if (!p) return fail(LINDHARD_EINVAL, "plan must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned h = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, p->ws + p->off_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->ws + p->off_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (h == DEV_ENOCONV) return fail(LINDHARD_ENOCONV, "no chemical potential for the filling");
    if (h == DEV_ETIMEOUT) return fail(LINDHARD_ETIMEOUT, "a bounded device wait timed out");
    return LINDHARD_OK;
}

extern "C" void lindhard_plan_destroy(lindhard_plan *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    drain_events(p);
    for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (cudaStream_t st : p->streams) if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : p->join_ev) if (ev) cudaEventDestroy(ev);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->origin) cudaStreamDestroy(p->origin);
    if (p->ws) cudaFree(p->ws);
    delete p;
}

extern "C" const char *lindhard_last_error(void) { return g_last_error.c_str(); }

// Helpers shared with other host translation units of the library.
namespace lh {
lindhard_status geom_from_grid(const lindhard_grid &gr, Geom &g, int &prec) { return make_geom(gr, g, prec); }
lindhard_status band_for_call(const Geom &g, const lindhard_band *b, bool generate, Band &o)
{
    return band_of_instance(g, b, generate, o);
}
lindhard_status set_error(lindhard_status st, const char *msg) { return fail(st, msg); }
}  // namespace lh
