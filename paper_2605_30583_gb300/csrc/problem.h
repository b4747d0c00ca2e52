// Host-side problem object of libgbba (internal).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "gbba.h"
#include "kernels.h"
#include "layout.h"

namespace gbba {

void set_error(const char* fmt, ...);
ba_status cuda_status(cudaError_t e, const char* what);

#define GBBA_CUDA(call)                                                    \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::gbba::cuda_status(e_, #call);      \
    } while (0)

// Offsets (bytes) of every array inside the workspace.
struct Layout {
    size_t state, partials, obs_key, obs_uv, obs_user, tile_off, pt_user, pt_internal, obs_pm, pt_obs_off;
    size_t vec[10];                      // x, x_new, h, r, z, p, q, g, D, s
    size_t blk_tile, blk_cam_off, blk_cams, pslots;
    size_t long_off, long_run, short_start;
    size_t xm, xm_new;                   // mixed form: FP64 master parameters (0 in the plain form)
    size_t cam_lo, cam_lo_new, rbuf;     // mixed form: low-order camera records, residuals
    size_t cam_pre, cam_pre_new, cam_dir, cam_acc, pc, cam_lin, cam_H, cam64, cam64_new, cam_H64, pt_H, Minv_c, Minv_p, jac, res, obs_w,
        staging;
    size_t fac_cam, fac_meas, fac_sqrt, fac_J;
    size_t s_cam_idx, s_pt_idx, s_pixels, s_pt_key, s_tile_cnt, s_keys, s_vals, sort_cap;
    size_t total;
};

struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace gbba

namespace gbba {
// Allocator whose resize leaves new elements uninitialised (the observation copies are
// filled by parallel copies right after).
template <typename T>
struct NoInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind {
        using other = NoInitAlloc<U>;
    };
    NoInitAlloc() = default;
    template <typename U>
    NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
    template <typename U>
    void construct(U* ptr) noexcept {
        ::new (static_cast<void*>(ptr)) U;
    }
    template <typename U, typename... A>
    void construct(U* ptr, A&&... a) {
        ::new (static_cast<void*>(ptr)) U(std::forward<A>(a)...);
    }
};
}  // namespace gbba

struct ba_problem {
    int32_t n_cams = 0, n_pts = 0, n_tiles = 0;
    int64_t n_obs = 0;
    int32_t precision = BA_PREC_MIXED;
    std::vector<uint32_t, gbba::NoInitAlloc<uint32_t>> cam_idx, pt_idx;
    std::vector<double, gbba::NoInitAlloc<double>> pixels;
    // pose factors (set before the workspace is bound)
    int32_t n_fac = 0;
    std::vector<uint32_t> fac_cam;   // [n_fac][2]
    std::vector<double> fac_meas;    // [n_fac][6]
    std::vector<double> fac_sqrt;    // [n_fac][6]
    int64_t pt_off = 0, n_vec = 0;
    gbba::Layout lay{};
    // bound state
    bool bound = false;
    bool linearized = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
    gbba::Views<float> vf{};
    gbba::Views<double> vd{};
    gbba::LaunchCfg L{};
    gbba::GraphCache graph{};            // conditional-loop graph (any options)
    gbba::GraphCache graph_unrolled{};   // fixed predicated sequence for (unrolled_lm, unrolled_pcg)
    int32_t unrolled_lm = -1, unrolled_pcg = -1;
    int device = 0;
    // persistent PCG plan (mixed precision, problems whose tiles fit in shared memory)
    bool persistent = false;        // the plan fits, in at least one form
    bool fits_one = false, fits_two = false;   // ... in the one-exchange / two-exchange form
    bool use_persistent = false;    // the plan is used by the current solve sequences
    bool use_schur = false;
    bool use_cg = false;            // the current solve sequences use the one-reduction PCG rounds         // the current solve sequences use the Schur-complement PCG
    int p_grid = 0, p_smem_one = 0, p_smem_two = 0;
    int p_form = 0;                 // form of the current solve sequences (gbba::PCG_*)
    uint32_t* blk_tile = nullptr;   // device, [p_grid + 1]
    uint32_t* blk_cam_off = nullptr;   // device, [p_grid + 1]: per-CTA camera list offsets
    uint32_t* blk_cams = nullptr;      // device, the lists (inside the ordering region of the workspace)
    double* pslots = nullptr;       // device, [PSLOT_TOTAL]

};

namespace gbba {
Layout compute_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, int32_t precision, int32_t n_fac = 0);
template <typename T>
Views<T> make_views(ba_problem* p);
}  // namespace gbba
