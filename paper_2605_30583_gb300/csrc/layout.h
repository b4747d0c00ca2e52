// Memory layout of libgbba's single device workspace (Sec. V-A of arXiv 2605.30583:
// one allocation for the whole optimisation, every array a view into it).
//
// Parameter-space vectors (x, h, r, z, p, q, g, D) are FP32 (FP64 in the plain form)
// of length n_vec = pt_off + 12 n_quads, n_quads = ceil(n_pts / 4), with camera c at
// [9c, 9c+9) and internal point i at [pt_off + 3i, pt_off + 3i + 3); pt_off is a
// multiple of 4, so four consecutive points are three aligned float4.  Padding
// entries stay zero.  Internal point order is the
// locality order built at bind time; pt_user / pt_internal map between the two.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace gbba {

constexpr int TILE_PTS = 256;       // points per tile; an observation's tile slot fits 8 bits
constexpr int HIST_CAP = 1024;      // LM iterations recorded in the device history
constexpr int MAX_GRID = 4096;      // upper bound on blocks of any reduction kernel
constexpr int NPART = 4;            // doubles of partial sums per block
constexpr int NSLOT = 32;           // atomic accumulator slots per scalar sum
constexpr int SLOT_STRIDE = 16;     // doubles between slots (one 128-byte line)
constexpr int MAX_PBLOCKS = 1024;   // CTAs of the persistent PCG kernel
// Exchange area of the persistent PCG kernels: three rotating slot sets of NSLOT
// slots, each slot XCH_NV sums (doubles), cleared before every launch.
constexpr int XCH_NV = 4;
constexpr int PSLOT_TOTAL = 3 * NSLOT * SLOT_STRIDE;
static_assert(XCH_NV <= SLOT_STRIDE, "a slot holds every sum of one exchange");
// Camera accumulator sets of the one-exchange kernel (rotating over iterations).
constexpr int CA_SETS = 3;
// A camera run of a tile this long or longer is walked in camera-uniform warp steps.
constexpr int LONG_RUN = 16;

// Camera record (floats), written once per parameter change (FP64 math, FP32 store).
enum : int { CP_R = 0, CP_T = 9, CP_F = 12, CP_K1 = 13, CP_K2 = 14, CP_PAD = 15,
             CP_JL = 16, CP_STRIDE = 32 };
// Camera low-order record (floats): the rounding errors of R, t, f, k1, k2 at the
// offsets CP_R .. CP_K2 of the camera record, for double-float residuals.
enum : int { CLO_STRIDE = 16 };
// Camera direction record (floats): phi = J_l(w) d_w (3), d_t (3), d_intr (3), pad.
enum : int { CD_PHI = 0, CD_T = 3, CD_I = 6, CD_STRIDE = 12 };
// Camera matvec accumulator (floats): sum (R X) x u (3), sum u (3), intrinsic part (3), pad.
enum : int { CA_STRIDE = 12 };
// Camera gradient accumulator (doubles): g = J_c^T r (9), pad (3).
enum : int { CL_G = 0, CL_STRIDE = 12 };
// Camera block accumulator (floats): upper triangle of J_c^T J_c row by row (45), pad (3).
enum : int { CH_STRIDE = 48 };
// Point linearisation record (floats): upper triangle xx, xy, xz, yy, yz, zz.
enum : int { PH_STRIDE = 6 };
// Inverse preconditioner blocks: full 9x9 per camera (floats), packed 3x3 per point.
enum : int { MC_STRIDE = 81, MP_STRIDE = 6 };

// Index of (i, j), i <= j, in a row-major upper triangle of an n x n matrix.
__host__ __device__ constexpr int tri_index(int n, int i, int j) {
    return i * n - (i * (i - 1)) / 2 + (j - i);
}

struct DevOptions {
    int32_t max_lm, max_pcg;
    double tol, mu0, min_diag, max_diag, max_mu, eps;
    int32_t retract;   // 1: rotations updated by retraction R <- Exp(d) R (J w.r.t. d)
    int32_t loss;      // robust loss: 0 squared, 1 Huber, 2 Cauchy
    double loss_scale;
    int64_t wait_ns;   // limit on each grid-wide wait of the persistent PCG kernels
    int32_t res_df;    // mixed form: residuals in double-float arithmetic (else FP32)
};

// Layout-compatible with ba_iter_stat of the public header.
struct IterRec {
    double cost, cost_new, mu, rho, model_decrease;
    int32_t pcg_iters, accepted;
    int64_t t_ns;
};

enum : int { TK_LIN = 0, TK_COST, TK_PRE, TK_DIR, TK_MV, TK_UPD, TK_CAND, TK_MISC, TK_FAC, TK_FACEV, TK_RES,
             TK_COUNT = 16 };

struct DevState {
    DevOptions opt;
    double mu, nu, F, F_new, F0, rho, L, gh, jh2;
    double rz, rr0, rr, alpha, beta, pDp, jp2, cost_out;
    // pose factors: 1/2 sum |r_f|^2 at the linearisation point and at the candidate,
    // and |J_f h|^2 (written by the factor kernels, added by the observation kernels)
    double fac_cost, fac_cost_new, fac_jh2;
    // mixed form: 1/2 sum rho(|r|^2) of the observations at the candidate (k_residual)
    double F_res;
    // Per-iteration sums, spread over NSLOT slots (block b adds into slot b % NSLOT,
    // one 128-byte line each) so concurrent atomics do not queue on one address.
    double acc_mv[NSLOT * SLOT_STRIDE];   // k = 0: |J p|^2, k = 1: p^T D p
    double acc_up[NSLOT * SLOT_STRIDE];   // k = 0: r^T z,   k = 1: |r|^2
    int32_t lm_iter, lm_active, accepted, relin, n_accepted, status;
    int32_t pcg_iter, pcg_active, pcg_total, pad0;
    int64_t t_start, t_end;
    uint32_t tickets[TK_COUNT];
    unsigned long long bar_count;   // arrivals at the grid barriers of the persistent PCG kernel
    int32_t bar_err, pad1;
    IterRec hist[HIST_CAP];
};

// Device views of one bound problem.  Built on the host from the workspace base.
template <typename T>
struct Views {
    int32_t n_cams, n_pts, n_tiles, n_quads;
    int64_t n_obs;
    int64_t pt_off, n_vec;
    int64_t pc_stride;           // floats between the two camera-direction buffers
    // observations, tile-major and camera-sorted inside each tile
    const uint32_t* obs_key;     // cam << 8 | tile slot
    const T* obs_uv;             // [n_obs][2]
    const uint32_t* obs_user;    // caller's observation index
    const uint32_t* tile_off;    // [n_tiles + 1]
    const uint32_t* pt_user;     // internal -> caller point index
    const uint32_t* pt_internal; // caller -> internal point index
    const uint32_t* obs_pm;      // point-major order: positions (in the order above) of each
    const uint32_t* pt_obs_off;  //   internal point's observations, offsets [n_pts + 1]
    // long runs: inside a tile the camera runs of at least LONG_RUN observations come
    // first; long_run[3 e + 0, 1, 2] = start (absolute position), length and camera of long
    // run e, tile t's long runs are e in [long_off[t], long_off[t + 1]), and its short runs
    // occupy [short_start[t], tile_off[t + 1])
    const uint32_t* long_off;       // [n_tiles + 1]
    const uint32_t* long_run;       // [3 * long runs]
    const uint32_t* short_start;    // [n_tiles]
    // vectors of length n_vec
    T *x, *x_new, *h, *r, *z, *p, *q, *g, *D;
    T* s;             // A p of the one-reduction PCG recurrences (separate-kernel form)
    // Mixed form: the parameters' FP64 master copy (x, x_new above are its FP32
    // roundings, which every FP32 kernel reads).  Steps are applied to the master copy,
    // so a step smaller than an FP32 ulp of a parameter still accumulates, and each
    // evaluation rounds afresh: the rounding then enters F and F' alike instead of
    // adding a one-sided cost to every candidate.  nullptr in the plain form.
    double *xm, *xm_new;
    // Mixed form: low-order camera records (CLO_STRIDE floats, at x and at x') and the
    // observations' residuals in solver order ([n_obs][2], k_residual), which the
    // linearisation reads.  nullptr in the plain form.
    float *cam_lo, *cam_lo_new;
    float* rbuf;
    // camera records
    float *cam_pre, *cam_pre_new, *cam_dir, *cam_acc;
    float* pc;        // camera part of the PCG direction, double-buffered [2][pc_stride]
    double* cam_lin;
    float* cam_H;
    double *cam64, *cam64_new, *cam_H64;   // plain FP64 form: camera records and J_c^T J_c
    T* pt_H;          // [4 n_quads][6]
    T* Minv_c;        // [n_cams][81]
    T* Minv_p;        // [4 n_quads][6]
    T* jac;           // plain form only: stored Jacobian [n_obs][2][12]
    T* res;           // plain form only: stored residuals [n_obs][2]
    float* obs_w;     // IRLS weights of the robust loss, solver observation order [n_obs]
    // pose factors (relative pose of two cameras), n_fac of them
    int32_t n_fac;
    const uint32_t* fac_cam;   // [n_fac][2]: cameras a, b
    const double* fac_meas;    // [n_fac][6]: rotation vector and translation of the measurement
    const double* fac_sqrt;    // [n_fac][6]: square root of the diagonal information
    float* fac_J;              // [n_fac][6][12]: Jacobian over (phi_a, t_a, phi_b, t_b), scaled
    DevState* st;
    double* partials; // [MAX_GRID][NPART]
    void* staging;    // user-layout parameter staging (FP64, 9 n_cams + 3 n_pts)
};

}  // namespace gbba
