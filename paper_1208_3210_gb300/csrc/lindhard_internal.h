// Internal types shared by the kernels and the host plan code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lindhard.h"

namespace lh {

// Geometry of one instance, derived on the host from lindhard_grid.
struct Geom {
    int N;          // momentum points per axis (zones * npz)
    int npz;        // points per zone per axis
    int periodic;   // 1: reduced zone, p + q wraps
    int n_eps;      // energies
    int J0;         // e_j < 0 (occupied) iff j < J0 (= n_eps / 2)
    int P;          // FFT length per momentum axis
    int PE;         // FFT length along energy
    int H;          // PE / 2 + 1 non-redundant energy frequencies
    int SP;         // row stride of half spectra (H rounded up to 8)
    long long xs2;  // stride between p_x planes of the [N][P][2 SP] buffers, P 2SP + pad
    long long xs3;  // stride between q_x planes of the [Q][P][SP] buffers, P SP + pad
    int Q;          // lags kept per momentum axis
    int n_omega;    // energy transfers kept
    int band_kind;  // 0 tight binding, 1 free electrons
    int quantity;   // lindhard_quantity: 0 Im chi (T = 0), 1 Im chi_T, 2 S(q, w)
    double e_max, de, dp;
    double scale;   // -(de / 2 pi) / npz^2 / (P * P * PE): Eq. 9 prefactor and FFT norm
                    // (for S(q, w): +(de / 2 pi) / npz^2 / pi / (P * P * PE))
};

// Layouts of the energy-direct form (the paper's own arrangement, Sec. 3: a 2D
// transform over momentum for every energy plane, the energy sum done directly
// for every momentum frequency).  The energy planes are packed in pairs,
// z_t = A(., e_t) + i A(., e_{J0 + t}), t < T = n_eps - J0 (occupied plane t,
// empty plane J0 + t), as the columns of the layouts the p_y passes read.
struct DirectGeom {
    Geom t;          // planes: [N][N][2 SPt] -> [N][P][2 SPt] (SP = H = SPt, xs2)
    Geom o;          // transfers: [Q][P][SPo] -> [Q][Q][SPo] (SP = SPo, H = n_omega, xs3)
    int T;           // plane pairs
    long long zs;    // plane stride of the momentum transforms Z [P][P][2 SPt]
    long long cs;    // plane stride of the correlations C [P][P][SPo]
};
inline DirectGeom direct_geom(const Geom &g)
{
    DirectGeom d;
    d.T = g.n_eps - g.J0;
    d.t = g;
    d.t.SP = d.t.H = ((d.T + 1) / 2 + 7) / 8 * 8;
    d.t.xs2 = (long long)g.P * 2 * d.t.SP + 32;
    d.o = g;
    d.o.SP = (g.n_omega + 7) / 8 * 8;
    d.o.H = g.n_omega;
    d.o.xs3 = (long long)g.P * d.o.SP + 32;
    d.zs = (long long)g.P * 2 * d.t.SP + 32;
    d.cs = (long long)g.P * d.o.SP + 32;
    return d;
}

// Per-call physics of one instance, passed by value to the kernels.
struct Band {
    double t, tp, tpp, mu, filling, gamma, ff_a;
    int band_kind;
    int solve_mu;   // 1: mu from filling
    // FP32 forms for the energy pass: -2t, -4t', -2t'' as unevaluated
    // (hi, lo) pairs, and gamma / pi
    float k1[2], k2[2], k3[2], gam_pi, gam2;
    // temperature (0: the T = 0 split); e_j / kT = (2 j + 1 - n_eps) x_step
    double kT, x_step64;
    float x_step;
};

// Device-side per-instance state written by the set-up kernels.
struct InstState {
    double mu;          // chemical potential used
    double last_step;   // size of the last Newton correction (convergence check)
    float mu_hi, mu_lo; // mu as an unevaluated FP32 pair
    float pad[2];
};

// mu into the state, with its FP32 (hi, lo) pair.
__host__ __device__ inline void set_mu(InstState *st, double mu)
{
    st->mu = mu;
    const float h = (float)mu;
    st->mu_hi = h;
    st->mu_lo = (float)(mu - (double)h);
}

// Status word codes recorded on the device.
enum { DEV_OK = 0, DEV_ENOCONV = 1, DEV_ETIMEOUT = 2 };

// Per-axis FP64 tables for one instance (N entries each).
struct AxisTab {
    double c1;   // cos(p_i)
    double c2;   // cos(2 p_i)
    double g;    // exp(-p_i^2 ff_a^2 / 8), so |M(p)|^2 = g(px) g(py)
    double p2;   // p_i^2
    // the same as unevaluated FP32 pairs hi + lo (hi = fl(x)), and g in FP32
    float c1h, c1l, c2h, c2l, p2h, p2l, gf, pad;
};

// Workspace of one instance (device pointers into the plan's allocation).
template <typename Real>
struct Work {
    void *X;               // half spectra: forward energy pass output, later x-product output
    void *Y;               // y pass output, later inverse-y output
    AxisTab *axis;         // [N]
    void *eps;             // energy table: float2 (hi, lo) or double, [n_eps]
    const void *tw;        // twiddle tables (see twiddles_for): float2 or double2
    int tw_len;            // longest transform length of the plan
    const void *tc;        // tensor-core DFT matrices (k_tc.cu), or null
    const void *ptw = nullptr;   // per-stage twiddle tables of the pruned engine (FP32), or null
    const void *etw = nullptr;   // per-stage twiddle tables of the lines-across-lanes energy pass, or null
    InstState *state;      // [1]
    unsigned *status;      // plan-wide device status word
    double *mu_acc;        // scratch for the chemical potential solve
    unsigned *barrier;     // arrival counter of the chemical-potential launches
};

}  // namespace lh
