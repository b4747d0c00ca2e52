// Host-side problem object of libgbba (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
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
    size_t state, partials, obs_key, obs_uv, obs_user, tile_off, pt_user, pt_internal;
    size_t vec[9];                       // x, x_new, h, r, z, p, q, g, D
    size_t cam_pre, cam_pre_new, cam_dir, cam_acc, cam_lin, pt_H, Minv_c, Minv_p, jac, res, staging;
    size_t s_cam_idx, s_pt_idx, s_pixels, s_pt_key, s_tile_cnt, s_keys, s_vals, sort_cap;
    size_t total;
};

struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace gbba

struct ba_problem {
    int32_t n_cams = 0, n_pts = 0, n_tiles = 0;
    int64_t n_obs = 0;
    int32_t precision = BA_PREC_MIXED;
    std::vector<uint32_t> cam_idx, pt_idx;
    std::vector<double> pixels;
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
    gbba::GraphCache graph{};
    int device = 0;
};

namespace gbba {
Layout compute_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, int32_t precision);
template <typename T>
Views<T> make_views(ba_problem* p);
}  // namespace gbba
