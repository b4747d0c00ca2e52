// Memory layout of libgbba's single device workspace (Sec. V-A of arXiv 2605.30583:
// one allocation for the whole optimisation, every array a view into it).
//
// Parameter-space vectors (x, h, r, z, p, q, g, D) are FP32 (FP64 in the plain form)
// of length n_vec = pt_off + round_up(3 n_pts, 4), with camera c at [9c, 9c+9) and
// internal point i at [pt_off + 3i, pt_off + 3i + 3).  Internal point order is the
// locality order built at bind time; pt_user / pt_internal map between the two.
#pragma once

#include <stddef.h>
#include <stdint.h>

namespace gbba {

constexpr int TILE_PTS = 128;       // points per tile; an observation's tile slot fits 8 bits
constexpr int HIST_CAP = 1024;      // LM iterations recorded in the device history
constexpr int MAX_GRID = 4096;      // upper bound on blocks of any reduction kernel
constexpr int NPART = 4;            // doubles of partial sums per block

// Camera record (floats), written once per parameter change (FP64 math, FP32 store).
enum : int { CP_R = 0, CP_T = 9, CP_F = 12, CP_K1 = 13, CP_K2 = 14, CP_PAD = 15,
             CP_JL = 16, CP_STRIDE = 32 };
// Camera direction record (floats): phi = J_l(w) d_w (3), d_t (3), d_intr (3), pad.
enum : int { CD_PHI = 0, CD_T = 3, CD_I = 6, CD_STRIDE = 12 };
// Camera matvec accumulator (floats): sum (R X) x u (3), sum u (3), intrinsic part (3), pad.
enum : int { CA_STRIDE = 12 };
// Camera linearisation accumulator (doubles): g = J_c^T r (9), upper triangle of
// J_c^T J_c row by row (45), pad (2).
enum : int { CL_G = 0, CL_H = 9, CL_STRIDE = 56 };
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
};

// Layout-compatible with ba_iter_stat of the public header.
struct IterRec {
    double cost, cost_new, mu, rho, model_decrease;
    int32_t pcg_iters, accepted;
    int64_t t_ns;
};

enum : int { TK_LIN = 0, TK_COST, TK_PRE, TK_DIR, TK_MV, TK_UPD, TK_CAND, TK_MISC, TK_COUNT = 16 };

struct DevState {
    DevOptions opt;
    double mu, nu, F, F_new, F0, rho, L, gh, jh2;
    double rz, rr0, rr, alpha, beta, pDp, jp2, cost_out;
    int32_t lm_iter, lm_active, accepted, relin, n_accepted, status;
    int32_t pcg_iter, pcg_active, pcg_total, pad0;
    int64_t t_start, t_end;
    uint32_t tickets[TK_COUNT];
    IterRec hist[HIST_CAP];
};

// Device views of one bound problem.  Built on the host from the workspace base.
template <typename T>
struct Views {
    int32_t n_cams, n_pts, n_tiles;
    int64_t n_obs;
    int64_t pt_off, n_vec;
    // observations, tile-major and camera-sorted inside each tile
    const uint32_t* obs_key;     // cam << 8 | tile slot
    const T* obs_uv;             // [n_obs][2]
    const uint32_t* obs_user;    // caller's observation index
    const uint32_t* tile_off;    // [n_tiles + 1]
    const uint32_t* pt_user;     // internal -> caller point index
    const uint32_t* pt_internal; // caller -> internal point index
    // vectors of length n_vec
    T *x, *x_new, *h, *r, *z, *p, *q, *g, *D;
    // camera records
    float *cam_pre, *cam_pre_new, *cam_dir, *cam_acc;
    double* cam_lin;
    T* pt_H;          // [n_pts][6]
    T* Minv_c;        // [n_cams][81]
    T* Minv_p;        // [n_pts][6]
    T* jac;           // plain form only: stored Jacobian [n_obs][2][12]
    T* res;           // plain form only: stored residuals [n_obs][2]
    DevState* st;
    double* partials; // [MAX_GRID][NPART]
    void* staging;    // user-layout parameter staging (FP64, 9 n_cams + 3 n_pts)
};

}  // namespace gbba
