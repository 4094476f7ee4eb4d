/*
 * lindhard.h -- C ABI of the GB300 FFT Lindhard susceptibility library.
 *
 * Computes, on one GPU, the Lindhard approximation of Wang et al.
 * ("Lindhard and RPA susceptibility computations in extended momentum space
 * in electron doped cuprates"):
 *
 *   Sec. 2, Eq. 9:  Im chi(q, w) = - Int_{-w}^{0} de/(2 pi) Int d^2p/(2 pi)^2
 *                                     A(p, e) A(p + q, e + w)
 *
 * in two dimensions (Sec. 3: k_z dispersion neglected), with the spectral
 * function of Sec. 2, Eqs. 4-5,
 *
 *   A(p, e) = |M(p)|^2 gamma / (pi [(e - xi_p)^2 + gamma^2]),
 *
 * and obtains it as the paper's method does (Sec. 3: the momentum
 * convolution replaced by products of Fourier transforms): a forward FFT of
 * the occupied and empty parts of A, their conjugate product, and an inverse
 * FFT.  The FFT also runs along the energy axis, so the whole (p, e)
 * correlation is one 3D transform.
 *
 * Grid conventions (shared by every entry point):
 *   lattice constant 1, zone width 2 pi; N = zones * pts_per_zone points per
 *   axis at p_i = (i - N/2) dp, dp = 2 pi / pts_per_zone, i in [0, N);
 *   n_eps cell-centred energies e_j = -e_max + (j + 1/2) de, de = 2 e_max / n_eps;
 *   the T = 0 occupation split (Sec. 3; Appendix A, Eq. A3): A at e_j < 0 is
 *   occupied, A at e_j >= 0 is empty (with odd n_eps, e = 0 is empty);
 *   outputs at w_m = m de, m in [0, n_omega), and q_l = (l - Q/2) dp,
 *   l in [0, Q), Q = q_extent, for both axes;
 *   measure d^2p/(2 pi)^2 -> 1/pts_per_zone^2 per grid point;
 *   zones == 1: reduced zone, p + q wraps (the band is periodic);
 *   zones  > 1: extended zone, A = 0 outside the grid.
 *
 * Memory: every pointer argument named "device" must point to memory of the
 * current CUDA device, owned by the caller, not aliased by any other argument.
 * Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 * stream) and is asynchronous: the call returns once the work is enqueued.
 * Host-side argument errors are returned before anything is enqueued.
 * Errors found on the device (no chemical potential for the filling) are
 * recorded in the plan and returned by lindhard_plan_status(), which
 * synchronises the stream.
 * A plan is not thread-safe: use one plan per stream.
 */
#ifndef LINDHARD_H
#define LINDHARD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LINDHARD_OK = 0,
    LINDHARD_EINVAL = 1,        /* an argument is out of range or NULL       */
    LINDHARD_ENOMEM = 2,        /* device or host allocation failed          */
    LINDHARD_ECUDA = 3,         /* a CUDA runtime call failed                */
    LINDHARD_ETIMEOUT = 4,      /* a bounded device wait (TMA copy or tensor-core
                                   products, 1 s) gave up; reported by
                                   lindhard_plan_status                       */
    LINDHARD_ENOCONV = 5,       /* no chemical potential for the filling     */
    LINDHARD_EUNSUPPORTED = 6   /* grid size or precision not built          */
} lindhard_status;

typedef enum {
    LINDHARD_FP32 = 0,          /* FP32 SIMT FFT, FP32 intermediates          */
    LINDHARD_SPLITBF16_TC = 1,  /* as LINDHARD_FP32, but the inverse p_y pass
                                   runs its two DFT stages (P = R1 R2) as
                                   matrix products on the tensor cores: BF16
                                   hi + lo operands, three products
                                   (hi.hi + lo.hi + hi.lo), FP32 accumulation.
                                   Momentum FFT lengths 128, 192, 256, 384,
                                   512, 768, 1024, 1536; forward only (plans
                                   with LINDHARD_PLAN_BACKWARD reject it)    */
    LINDHARD_FP64 = 2           /* FP64 everywhere; FFT lengths <= 256 only   */
} lindhard_precision;

/* What a grid's output holds (lindhard_grid.quantity).  With kT > 0 the
 * Fermi function f(e) = 1 / (exp(e / kT) + 1) of the grid energy (measured
 * from mu) replaces the T = 0 split: the occupied part is A f, the empty part
 * A (1 - f) (Appendix A, Eq. A1, whose occupation difference f(e) - f(e + w)
 * reduces to the window [-w, 0] of Eq. A3 at T = 0). */
typedef enum {
    LINDHARD_IMCHI = 0,         /* Im chi(q, w) at T = 0 (Eq. 9); band.kT = 0  */
    LINDHARD_IMCHI_T = 1,       /* Im chi_T(q, w) = -c sum_{p,j} A(p, e_j)
                                   A(p + q, e_{j+m}) [f(e_j) - f(e_{j+m})],
                                   c = (de / 2 pi) / pts_per_zone^2; band.kT > 0 */
    LINDHARD_SQW = 2            /* dynamical structure factor (Sec. 2, Eq. 1):
                                   S(q, w) = -(1/pi) Im chi_T(q, w) / (1 - exp(-w/kT)),
                                   computed as (c / pi) sum A(p, e_j) A(p + q, e_{j+m})
                                   f(e_j) [1 - f(e_{j+m})], the same quantity
                                   with its w -> 0 limit at m = 0; >= 0; band.kT > 0 */
} lindhard_quantity;

/* One instance's physics, eV, lattice constant 1 (Sec. 2 Eqs. 4-5, Sec. 3). */
typedef struct {
    double t, tp, tpp;  /* tight-binding hoppings: xi_p = -2t (cos px + cos py)
                           - 4t' cos px cos py - 2t'' (cos 2px + cos 2py) - mu */
    double mu;          /* chemical potential; used as given iff filling is NaN */
    double filling;     /* electrons per site incl. spin (rigid band, Sec. 3);
                           mu is then solved in FP64 so that
                           (2/npz^2) sum_k [1/2 - atan(xi_k/gamma)/pi] = filling
                           over the first-zone grid                        */
    double gamma;       /* Lorentzian half-width (Eq. 5), > 0                 */
    double ff_a;        /* |M(p)|^2 = exp(-|p|^2 ff_a^2 / 8); 0 => |M|^2 = 1   */
    int band_kind;      /* 0 tight binding; 1 free electrons, xi = |p|^2/2 - mu */
    int reserved;       /* must be 0                                          */
    double kT;          /* temperature, eV: 0 for LINDHARD_IMCHI grids, finite
                           and > 0 for LINDHARD_IMCHI_T and LINDHARD_SQW.  The
                           filling fixes mu by the T = 0 count above (the
                           thermal shift of mu is not applied; give mu with
                           filling = NaN to set it).  With a caller-supplied A
                           only kT is read.                                   */
} lindhard_band;

/* One instance's grid. */
typedef struct {
    int zones;          /* Brillouin zones per axis, >= 1                     */
    int pts_per_zone;   /* points per zone per axis, even, >= 2               */
    int n_eps;          /* energies on [-e_max, e_max], >= 2                  */
    double e_max;       /* energy half-window, eV, > 0                        */
    int n_omega;        /* energy transfers w_m = m de kept; 0 => n_eps / 2   */
    int q_extent;       /* lags kept per axis, even; 0 => N; <= 2N (zones > 1),
                           <= N (zones == 1)                                 */
    int precision;      /* lindhard_precision                                 */
    int quantity;       /* lindhard_quantity; LINDHARD_IMCHI_T and LINDHARD_SQW
                           pad the energy FFT to PE >= n_eps + n_omega - 1
                           (the occupied and empty parts overlap in energy)  */
} lindhard_grid;

typedef struct lindhard_plan lindhard_plan;

/* Sizes the library derives for one grid (for callers sizing buffers). */
typedef struct {
    long long N;            /* momentum points per axis                       */
    long long n_eps;        /* energies                                       */
    long long n_omega;      /* energy transfers kept                          */
    long long q_extent;     /* lags kept per axis                             */
    long long fft_p;        /* FFT length along each momentum axis            */
    long long fft_e;        /* FFT length along the energy axis               */
    long long out_elems;    /* q_extent^2 * n_omega                           */
    long long a_elems;      /* N^2 * n_eps (layout of A_in and dA)           */
    long long hbm_bytes_forward;  /* algorithmic HBM bytes of one forward call */
    long long kernels_forward;    /* kernel launches of one forward call with A generated and mu
                                     solved: with more than 98 points per zone one more when
                                     gamma < 0.02 eV (a third multisection pass); with at most 98
                                     the whole solve runs in the set-up launch (two fewer); with
                                     a caller-supplied A only the FFT passes; in a
                                     LINDHARD_PLAN_PERSISTENT plan the instance's set-up launches
                                     only (the batch adds one persistent launch)               */
} lindhard_sizes;

/* Plan flag: also allocate the buffers of lindhard_imchi_backward (one more
 * intermediate of Q x P x (PE/2 + 1) complex values and the per-CTA gradient
 * partial sums). */
#define LINDHARD_PLAN_BACKWARD 1u
/* Plan flag: one workspace per instance, and the instances of a call run as
 * independent branches on the plan's own streams (forked from and joined back
 * into the caller's stream), so small instances share the GPU. */
#define LINDHARD_PLAN_CONCURRENT 2u
/* Plan flag (implies LINDHARD_PLAN_CONCURRENT): lindhard_imchi records its
 * whole launch sequence for all instances once into a CUDA graph and replays
 * it; a call whose A_in, out, mu_out or band values differ from the recorded
 * ones records again (and updates the executable graph in place).  The first
 * call also runs the sequence once directly. */
#define LINDHARD_PLAN_GRAPH 4u
/* Plan flag: at creation, time the available engine variants of the passes
 * along p_y, of the product pass and of the inverse energy pass for each FP32
 * grid of the plan (CUDA events, a few launches each) and use the fastest;
 * results are cached per process and, when the environment variable
 * LINDHARD_TUNE_CACHE names a file, in that JSON file.  With the environment
 * variable LINDHARD_TUNE_LOG set (and not "0") every timed variant's mean
 * launch time is printed to stderr. */
#define LINDHARD_PLAN_AUTOTUNE 8u
/* Plan flag: compute Im chi in the paper's own arrangement (Sec. 3) instead of
 * the 3D transform: a 2D FFT over momentum for every energy plane (the
 * occupied plane e_t and the empty plane e_{J0+t} packed into one complex
 * transform), the energy sum of Eq. 9 done directly for every momentum
 * frequency k, C(k, w_m) = sum_j conj(a^_j(k)) b^_{j+m}(k) (FP32 fused
 * multiply-adds), and a 2D inverse FFT for every transfer.  Same outputs as
 * the 3D form up to rounding; kept to compare the two.  LINDHARD_FP32,
 * LINDHARD_IMCHI grids with n_eps <= 1024 and n_omega <= 512 only; forward
 * only (not with LINDHARD_PLAN_BACKWARD); LINDHARD_PLAN_AUTOTUNE tunes
 * nothing in this form.  Otherwise LINDHARD_EUNSUPPORTED. */
#define LINDHARD_PLAN_ENERGY_DIRECT 16u
/* Plan flag: run the five transform passes of every instance of the batch as
 * one persistent launch (a batch scheduler): the CTAs claim (instance, pass,
 * tile) items from a device queue ordered pass by pass, and an item waits,
 * with a bounded wait, until its instance's previous pass has completed (a
 * counter per instance and pass), so the passes of different instances
 * overlap and no pass ends in a launch tail.  The chemical-potential solves
 * and tables run first as ordinary launches, on the plan's streams.  Implies
 * LINDHARD_PLAN_CONCURRENT (one workspace per instance); combines with
 * LINDHARD_PLAN_GRAPH.  Every grid must be LINDHARD_FP32, LINDHARD_IMCHI,
 * zones > 1, q_extent = N with N + N/2 in {192, 384, 768, 1536} (the momentum
 * padding exactly one third) and an energy FFT of 128, 256 or 512 points;
 * otherwise LINDHARD_EUNSUPPORTED.  Not with LINDHARD_PLAN_BACKWARD or
 * LINDHARD_PLAN_ENERGY_DIRECT.  A call with a caller-supplied A runs the
 * instances as ordinary launches instead.  A wait that runs out (the limit
 * of lindhard_plan_set_wait_limit, 1 s by default) records LINDHARD_ETIMEOUT
 * for lindhard_plan_status, and every CTA stops. */
#define LINDHARD_PLAN_PERSISTENT 32u

/* Builds a plan for `batch` instances with the given grids (host array).
 * Validates the grids, picks FFT lengths (the smallest supported length that
 * keeps the circular correlation free of wrap-around: >= N + Q/2 per momentum
 * axis in the extended zone, N in the reduced zone, >= n_eps in energy), and
 * allocates the device workspace and twiddle tables on the current device.
 * Without LINDHARD_PLAN_CONCURRENT instances are computed one after another
 * and share one workspace sized for the largest.  flags: any of
 * LINDHARD_PLAN_BACKWARD, LINDHARD_PLAN_CONCURRENT, LINDHARD_PLAN_GRAPH,
 * LINDHARD_PLAN_AUTOTUNE, LINDHARD_PLAN_ENERGY_DIRECT, LINDHARD_PLAN_PERSISTENT.
 * On success *out receives the plan. */
lindhard_status lindhard_plan_create(const lindhard_grid *grids, int batch,
                                     unsigned flags, lindhard_plan **out);

/* Sizes for instance `index` of the plan. */
lindhard_status lindhard_plan_sizes(const lindhard_plan *plan, int index,
                                    lindhard_sizes *out);

/* Bytes of device workspace the plan owns. */
lindhard_status lindhard_plan_workspace_bytes(const lindhard_plan *plan,
                                              size_t *out);

/* Forward: Im chi(q_l, w_m) for every instance (Eq. 9), or the finite-
 * temperature quantity its grid names (lindhard_quantity).
 *   bands : host [batch]; read before return.
 *   A_in  : device, optional.  NULL => A is generated from bands (Eqs. 4-5).
 *           Otherwise the batch-concatenated caller A(p_i, e_j), float32,
 *           layout [N][N][n_eps] per instance (e fastest), and bands are
 *           ignored (may be NULL) unless a grid is LINDHARD_IMCHI_T or
 *           LINDHARD_SQW: then bands[i].kT is read.
 *   out   : device, float32, batch-concatenated, layout [Q][Q][n_omega] per
 *           instance (w fastest).
 * Every grid of the plan must use LINDHARD_FP32 (see lindhard_imchi_f64).
 *   mu_out: device, optional, double [batch]: the chemical potential used.
 * Returns before the work completes (stream-ordered). */
lindhard_status lindhard_imchi(lindhard_plan *plan, const lindhard_band *bands,
                               const float *A_in, float *out, double *mu_out,
                               void *stream);

/* As lindhard_imchi, for plans whose grids all use LINDHARD_FP64: A_in is
 * double [N][N][n_eps] per instance and out is double [Q][Q][n_omega]. */
lindhard_status lindhard_imchi_f64(lindhard_plan *plan, const lindhard_band *bands,
                                   const double *A_in, double *out, double *mu_out,
                                   void *stream);

/* Adjoint of lindhard_imchi for L = sum_{l,m} w[l_x][l_y][m] Im chi(q_l, w_m).
 * Eq. 9 is bilinear in the occupied part a and empty part b of A, so
 *   dL/dA(p, e_j) = -c sum_{s,m} w(s, m) b(p + s, e_{j+m})   (e_j < 0)
 *   dL/dA(p, e_j) = -c sum_{s,m} w(s, m) a(p - s, e_{j-m})   (e_j >= 0)
 * with c = de/(2 pi)/npz^2; both are correlations with w and are computed by
 * FFT like the forward call.  The plan must be created with
 * LINDHARD_PLAN_BACKWARD and FP32 grids.
 *   w       : device, float32, layout of `out` of lindhard_imchi.
 *   A_in    : as in lindhard_imchi (NULL => A generated from bands).
 *   dA      : device, optional, float32, layout of A_in: dL/dA(p_i, e_j).
 *   dparams : device, optional, double [batch][5]:
 *             dL/d(t, t', t'', mu, gamma) by the chain rule through Eqs. 4-5
 *             (A_in must be NULL), mu held fixed (a partial derivative even
 *             when mu was solved from the filling).
 * At least one of dA and dparams must be non-NULL.
 * Finite-temperature grids (Appendix A, Eq. A1; Eq. 1): L sums w times the
 * grid's quantity (Im chi_T or S(q, w)); with a = A f, b = A (1 - f) on every
 * cell and C(q, w) = sum a(p, e) b(p + q, e + w), Im chi_T = -c [C(q, w) -
 * C(-q, -w)] and S = (c/pi) C(q, w), so
 *   dL/dA(p, e_j) = kappa [f_j sum_{s,m} w'(s, m) b(p + s, e_{j+m})
 *                          + (1 - f_j) sum_{s,m} w'(s, m) a(p - s, e_{j-m})]
 * with kappa = -c, w'(s, m) = w(s, m) - w(-s, -m) (Im chi_T) or kappa = c/pi,
 * w' = w (S); bands must then be given (their kT) also with A_in. */
lindhard_status lindhard_imchi_backward(lindhard_plan *plan,
                                        const lindhard_band *bands,
                                        const float *A_in, const float *w,
                                        float *dA, double *dparams, void *stream);

/* Per-pass timing (sequential plans only).  With enable != 0 the plan
 * records a CUDA event pair on the call's stream around each of its kernel
 * launches (profiling); enable = 0 stops recording.  Either call clears the
 * accumulated times. */
lindhard_status lindhard_plan_profile(lindhard_plan *plan, int enable);

/* The same for a subset of the passes: bit i of `mask` times pass slot i
 * (see LINDHARD_NUM_PASSES below), so that timing one kernel perturbs the
 * others as little as possible; mask = 0 stops recording. */
lindhard_status lindhard_plan_profile_passes(lindhard_plan *plan, unsigned mask);

/* Kernels of one forward call, in launch order (the slots of
 * lindhard_plan_pass_times). */
#define LINDHARD_NUM_PASSES 7
/* 0 tables, 1 mu solve, 2 energy forward (generation + FFT), 3 p_y forward,
 * 4 p_x forward + product + p_x inverse, 5 p_y inverse, 6 energy inverse.   */

/* Waits for the recorded events and returns, per slot, the summed device time
 * in milliseconds (ms[LINDHARD_NUM_PASSES]) and the number of launches timed
 * (launches[LINDHARD_NUM_PASSES]) since profiling was enabled. */
lindhard_status lindhard_plan_pass_times(lindhard_plan *plan, double *ms, long long *launches);

/* FP64 sum-rule check of a computed output (Sec. 4's sum over q of Im chi,
 * Fig. 2(b), which counts electron-hole transitions): summing Eq. 9 over every
 * lag factorises into the energy correlation of the occupied and empty
 * densities of states,
 *   sum_q Im chi(q, w_m) = -c sum_j D_a(e_j) D_b(e_{j+m}),  D(e) = sum_p A(p, e).
 * For instance `index` of the plan, whose grid must keep every lag
 * (q_extent = N with one zone, 2N with several):
 *   out      : device, float32, that instance's output of lindhard_imchi.
 *   band / A_in : as in lindhard_imchi for that instance (A regenerated).
 *   sum_q    : device, double [n_omega]: left side, reduced from out in FP64.
 *   dos_corr : device, double [n_omega]: right side, from A in FP64.
 * Uses the plan's workspace (do not overlap with a call of the same plan).
 * Finite-temperature grids: the same exchange of sums with a = A f and
 * b = A (1 - f) gives dos_corr = -c sum_j D(e_j) D(e_{j+m}) [f(e_j) - f(e_{j+m})]
 * (LINDHARD_IMCHI_T) and (c/pi) sum_j D(e_j) D(e_{j+m}) f(e_j) [1 - f(e_{j+m})]
 * (LINDHARD_SQW), D(e) = sum_p A(p, e); band.kT is read. */
lindhard_status lindhard_sum_rule(lindhard_plan *plan, int index, const lindhard_band *band,
                                  const float *A_in, const float *out, double *sum_q, double *dos_corr,
                                  void *stream);

/* dmu/d(t, t', t'', gamma) at fixed filling, at chemical potential mu (e.g.
 * the value lindhard_imchi returned in mu_out): the rigid-band count of
 * lindhard_band.filling, n(mu) = (2/npz^2) sum_k [1/2 - atan(xi_k/gamma)/pi]
 * over the first-zone grid, is held fixed, so by the implicit function theorem
 * dmu/dtheta = -(dn/dtheta)/(dn/dmu) (Sec. 3 places mu to hold the filling).
 * With the partial derivatives at fixed mu from lindhard_imchi_backward, the
 * gradient at fixed filling is dL/dtheta + dL/dmu dmu/dtheta.  Uses t, tp,
 * tpp, gamma and band_kind of `band` and the instance's npz; FP64 reductions
 * on the device, summed on the host in a fixed order.  out: host double[4].
 * Synchronises `stream`. */
lindhard_status lindhard_dmu_dparams(lindhard_plan *plan, int index, const lindhard_band *band, double mu,
                                     double *out, void *stream);

/* Envelope of -Im chi along the [100] cut q = (q_x, 0) at transfer index m,
 * fitted by the Lorentzian shape 1 / (1 + (q/k0)^2) (Sec. 4, Fig. 5: the
 * decay of -Im chi with the momentum transfer).  For every reciprocal-lattice
 * zone n >= 0 along the cut (lag offsets [n npz - npz/2, n npz + npz/2) from
 * l_x = Q/2, with l_y = Q/2) that the lag window holds whole, the largest
 * -Im chi and its q form one point; the
 * points are normalised by the largest of them and k0 minimises the squared
 * residuals over the points with q > 0 (golden-section search over ln k0 in
 * [ln dp, ln (Q dp)]).  k0 in units of 1/a (lattice constant a = 1).
 * imchi: device, the instance's [Q][Q][n_omega] block.  k0: host double.
 * q_out, y_out: host double[max_points] for the points, or NULL; npoints: host
 * int (the number of points), or NULL.  Im chi grids (LINDHARD_IMCHI,
 * LINDHARD_IMCHI_T) only.  Synchronises `stream`. */
lindhard_status lindhard_envelope_k0(lindhard_plan *plan, int index, const float *imchi, int m, double *k0,
                                     double *q_out, double *y_out, int max_points, int *npoints, void *stream);

/* Real part of chi by the Kramers-Kronig relation and the RPA susceptibility
 * (Sec. 4): for instance `index`,
 *   Re chi(q, w_m) = sum_k W(m, k) Im chi(q, w_k),
 *   W(m, k) = (4/pi) k / (k^2 - m^2) for k >= 1 with k - m odd, else 0
 * (the principal value by Maclaurin's rule on the transfer grid, Im chi odd
 * in w, zero beyond the n_omega computed transfers), and
 *   chi_RPA = chi / (1 - V_q chi),  chi = Re chi + i Im chi,  V_q = v0 / |q|^2,
 * q = ((l_x - Q/2) dp, (l_y - Q/2) dp), v0 in eV (lattice constant 1); at
 * q = 0 chi_RPA is 0 (its limit), unless v0 = 0 (then chi_RPA = chi).
 * imchi: device, the instance's [Q][Q][n_omega] block as lindhard_imchi wrote
 * it.  re_out: device [Q][Q][n_omega].  rpa_out: device [Q][Q][n_omega][2]
 * (re, im; 8-byte aligned), or NULL.  variant 0: the far field |k - m| >= 8
 * on the tensor cores (BF16 hi/lo, three products, FP32 accumulation) and the
 * near band in FP32, n_omega <= 256; variant 1: FP32 SIMT throughout,
 * n_omega <= 1536 (otherwise LINDHARD_EUNSUPPORTED).  Plans whose grid is
 * LINDHARD_FP64 are rejected (LINDHARD_EINVAL), and so are LINDHARD_SQW
 * grids (the relation reads Im chi; LINDHARD_IMCHI_T is accepted).  Enqueued
 * on `stream`; no synchronisation. */
lindhard_status lindhard_kk_rpa(lindhard_plan *plan, int index, const float *imchi, float *re_out,
                                float *rpa_out, double v0, int variant, void *stream);

/* Limit of the bounded waits of the persistent batch launch
 * (LINDHARD_PLAN_PERSISTENT), in nanoseconds of the GPU's global timer
 * (default 1e9; 0 restores the default).  stall_instance >= 0 makes that
 * instance's wait for its first pass unsatisfiable (it asks one more tile
 * than the pass has), so that a test can make a wait run out on purpose: the
 * call then ends early, its output is not valid, and lindhard_plan_status
 * returns LINDHARD_ETIMEOUT; -1 for normal operation.  The plan's later
 * calls use the values set last.  EINVAL for a plan without the flag. */
lindhard_status lindhard_plan_set_wait_limit(lindhard_plan *plan, unsigned long long wait_ns, int stall_instance);

/* Engine variants the plan runs for instance `index` (set by
 * LINDHARD_PLAN_AUTOTUNE, else the defaults): out[0], out[1] = forward and
 * inverse passes along p_y (0 single-column engine, 1 paired columns,
 * 2 paired columns with 12 values per thread, 3, 4 and 5 the TMA-staged
 * persistent forms of 1, 2 and 0, 6 paired columns on double-width tiles,
 * 7 the tensor-core inverse, 8 and 9 the pruned engine on 8 and 4 column
 * pairs: a radix-24 stage at the padded end, for a padding of exactly one
 * third, N = 2P/3 forward and Q = 2P/3 inverse; 10 its TMA-staged
 * persistent form, 11 the same with two CTAs per SM, P >= 384);
 * out[2] = the p_x product pass (0 default
 * tile, 1 tile with 12 values per thread, 2 and 3 their TMA-staged forms,
 * 4 the default tile with one more CTA per SM, 5 the default tile twice as
 * wide, 6 and 7 the pruned engine on 8 and 4 columns, N = Q = 2P/3, 8 its
 * TMA-staged persistent form, 9 its software-pipelined persistent form
 * (the next tile's inputs loaded during the inverse transform, half through
 * registers, half through shared memory), 10 the same with the twiddle
 * tables in shared memory, P >= 384);
 * out[3] = the inverse energy
 * pass (0 default, 1 TMA-staged persistent form, 2 one warp per pair of
 * output lines, energy FFT lengths 128, 256, 512, 384 and 768).
 * out: host, int[4]. */
lindhard_status lindhard_plan_variants(const lindhard_plan *plan, int index, int *out);

/* Synchronises `stream` and returns the first device-side error recorded by
 * the plan since the last call (LINDHARD_OK if none), then clears it. */
lindhard_status lindhard_plan_status(lindhard_plan *plan, void *stream);

/* Releases the plan's device memory.  Synchronises the device first. */
void lindhard_plan_destroy(lindhard_plan *plan);

/* Bytes of the fixed device array used by lindhard_imchi_noalloc. */
#define LINDHARD_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Forward call that allocates nothing (the paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory when they need
 * Im chi -- inside a framework that owns the device memory pool, on hosts that
 * forbid allocation after start-up, or where cudaMalloc/cudaFree would
 * synchronise the device).  It computes exactly what lindhard_imchi computes
 * for one instance (`grid`, `band`, `A_in`, `out`, `mu_out` as there; FP32
 * only), with all intermediates in one fixed device array of
 * LINDHARD_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library
 * holds until the process exits.  Grids whose intermediates do not fit are
 * rejected with LINDHARD_EINVAL and a message giving the bytes needed (the
 * 32 x 32 x 48 reduced-zone grid needs about 1.5 MiB; 2 zones of 32 points
 * with 128 energies about 14 MiB).  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the array, so calls
 * that can overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Device-side failures (a filling with no chemical
 * potential) are not reported by this entry point; use a plan and
 * lindhard_plan_status() where that check is needed. */
lindhard_status lindhard_imchi_noalloc(const lindhard_grid *grid, const lindhard_band *band,
                                       const float *A_in, float *out, double *mu_out, void *stream);

/* Human-readable text of the last host-side error in this thread. */
const char *lindhard_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LINDHARD_H */
