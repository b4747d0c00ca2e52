// Host-side declarations of libgbba's kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace gbba {

typedef unsigned long long CondHandle;   // cudaGraphConditionalHandle

constexpr int LIN_TB = 128;   // threads per tile CTA, linearisation
constexpr int MV_TB = 128;    // threads per tile CTA, normal operator
constexpr int EV_TB = 256;    // threads per tile CTA, candidate evaluation
constexpr int PCG_TB = 512;   // threads per CTA of the persistent PCG kernel

// Raises a kernel's dynamic shared-memory limit to at least `bytes` and never lowers
// it: the limit is per function, shared by every problem in the process, so a later
// problem with smaller tiles must not break launches of an earlier one.
inline cudaError_t ensure_dynamic_smem(const void* func, int bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, func);
    if (e != cudaSuccess) return e;
    if (a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

struct LaunchCfg {
    int item_block = 256;
    int item_grid = 1024;   // cap on blocks of per-node kernels
    int lin_grid = 1024;    // cap on blocks of tile kernels
    int mv_grid = 1024;
    int ev_grid = 1024;
    int res_grid = 1024;    // residual pass (residual.cu)
    // tile kernels (tile_kernels.cu: long runs in camera-uniform warp steps); a grid of 0
    // selects the per-thread-chunk kernel of kernels_mixed.cu instead
    int tn_grid = 0;   // normal operator, one CTA per tile
    int tl_grid = 0;   // linearisation
    int te_grid = 0;   // candidate evaluation
    // the largest tile's long runs, short-run observations and long-run observations
    // (the compact observation table the tile kernels stage)
    int tk_run_cap = 0, tk_short_cap = 0, tk_long_cap = 0;
    int tn_smem = 0, tl_smem = 0, te_smem = 0;   // their dynamic shared memory (staged observations)
    // no camera observes a point twice (checked at bind): the operator's warps add their
    // point sums into private copies with plain adds
    int tn_plain_q = 0;
};

// residual pass of the mixed form (residual.cu): r at x (at_candidate 0) or at x' (1),
// and the cost into st->F_res (squared: the squared loss whatever the options, as
// ba_evaluate reports it)
void launch_residual(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int at_candidate, int squared = 0);
int occupancy_blocks_residual();

// mixed precision (kernels_mixed.cu)
void launch_camera_precompute(const Views<float>& v, const LaunchCfg& L, cudaStream_t s);
void launch_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode,
                      float* res_out, float* jac_out, CondHandle lm_cond, int use_cond);
void launch_precond(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use,
                    double* pslots);
void launch_matvec(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                   const float* zs, int use_beta);
void launch_update(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use,
                   int cameras_only = 0);
// tile kernels (tile_kernels.cu): launch shapes, then the launches
void plan_tile_kernels(LaunchCfg& L, int n_tiles, int sms, int max_long_obs, int max_short_obs, int max_long_runs);
void launch_tile_normal(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                        const float* zs, int use_beta);
void launch_tile_eval(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle lm_cond, int use_cond);
// One round of the separate-kernel PCG with the one-reduction recurrences: the cameras'
// update and direction records, the pose factors' operator, then the tiles (update fused
// into the staging, operator, reduction and stop decision in the last CTA).
void launch_cg_round(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate, CondHandle c,
                     int use);
void launch_tile_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode, float* res_out,
                           float* jac_out, CondHandle lm_cond, int use_cond);
// Schur-complement PCG (kernels_mixed.cu): mode 0 right-hand side, 1 operator, 2 back-substitution
void launch_schur(const Views<float>& v, cudaStream_t s, int mode, const int32_t* gate);
void launch_schur_start(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use);
// pose factors (pose_factor.cu); no-ops without factors
void launch_factor_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode);
void launch_factor_eval(const Views<float>& v, const LaunchCfg& L, cudaStream_t s);
void launch_factor_matvec(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                          const float* zs, int use_beta);
void launch_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s);
void launch_eval_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use);
void launch_commit(const Views<float>& v, const LaunchCfg& L, cudaStream_t s);
void launch_init_state(DevState* st, cudaStream_t s);
void launch_finish_state(DevState* st, cudaStream_t s);
void launch_pack(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const void* cams,
                 const void* pts, int dtype);
void launch_unpack(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const double* src, void* cams,
                   void* pts, int dtype);
void launch_set_direction(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const float* src);
void launch_normal_out(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, float* out);
// persistent PCG (pcg_persistent.cu)
// Two forms, numbered like ba_options.pcg_kernel: PCG_TWO_EXCHANGE (0) runs the
// textbook recurrences with two grid-wide exchanges per iteration; PCG_ONE_EXCHANGE
// (2) rearranges them so that one exchange per iteration carries both inner products.
enum : int { PCG_TWO_EXCHANGE = 0, PCG_ONE_EXCHANGE = 2 };
// Entries of blk_cams: camera id, bit 31 set in the one list that owns the camera.
constexpr uint32_t BLK_CAM_OWNER = 0x80000000u;
int persistent_max_smem();
// Self-test of the FP64 reciprocal of the block inversions: y[i] = rcp64(x[i]).
void launch_selftest_rcp64(const double* x, double* y, int64_t n, cudaStream_t s);
// Self-test of the bounded grid wait (16 bytes of device scratch).
cudaError_t launch_selftest_wait(void* scratch, int grid, long long timeout_ns, cudaStream_t s);
cudaError_t persistent_prepare(int form, int smem_bytes, int* blocks_per_sm);
cudaError_t launch_pcg_persistent(const Views<float>& v, const uint32_t* blk_tile, const uint32_t* blk_cam_off,
                                  const uint32_t* blk_cams, double* pslots, int grid, int smem_bytes, int form,
                                  cudaStream_t s);
// Dynamic shared memory of the one-exchange kernel for a CTA with `no` observations,
// `np` points and `ncb` listed cameras, in the order the kernel carves it.
__host__ __device__ inline size_t pcg1_smem_bytes(size_t no, size_t np, size_t ncb) {
    const size_t n3p = (3 * np + 3) & ~(size_t)3;
    size_t b = (4 * no + 15) & ~(size_t)15;          // observation keys
    b += 32 * np;                                     // (X, D_0) and (u, D_1) as float4
    b += 4 * ((np + 3) & ~(size_t)3);                 // D_2
    b += 4 * 5 * n3p;                                 // p, s, r, h, q
    b += 4 * ((6 * np + 3) & ~(size_t)3);             // M^-1 blocks
    b += 4 * ((ncb + 3) & ~(size_t)3);                // camera ids
    b += 4 * ((((ncb + 31) >> 5) + 3) & ~(size_t)3);  // owner bits
    b += 4 * (16 + 12 + 5 * 9) * ncb;                 // records, directions, u p s r h
    return b;
}
int occupancy_blocks_linearize();
int occupancy_blocks_matvec();
int occupancy_blocks_eval();

// plain FP64 form (kernels_fp64.cu)
void launch64_camera_precompute(const Views<double>& v, const LaunchCfg& L, cudaStream_t s);
void launch64_linearize(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, int mode, double* r, double* J,
                        CondHandle c, int use);
void launch64_precond(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use);
void launch64_direction(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const double* zs, int use_beta,
                        const int32_t* gate);
void launch64_matvec(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate);
void launch64_update(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use);
void launch64_candidate(const Views<double>& v, const LaunchCfg& L, cudaStream_t s);
void launch64_eval_candidate(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use);
void launch64_commit(const Views<double>& v, const LaunchCfg& L, cudaStream_t s);
void launch64_pack(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts,
                   int dtype);
void launch64_unpack(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, void* cams, void* pts, int dtype);
void launch64_set_vec(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const double* src, double* dst);
void launch64_get_vec(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const double* src, double* dst);

// autograd (cost and its adjoint at caller parameters; x' and the candidate camera
// records serve as scratch, the problem's parameters are left untouched)
void launch_cost_grad(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts,
                      int dtype, int want_grad, double* cost_dev);
void launch_grad_out(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const double* grad_out, void* gc,
                     void* gp, int dtype);
void launch64_cost_grad(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts,
                        int dtype, int want_grad, double* cost_dev);
void launch64_grad_out(const Views<double>& v, const LaunchCfg& L, cudaStream_t s, const double* grad_out, void* gc,
                       void* gp, int dtype);

// ordering (order.cu).  All buffers are device memory inside the workspace.
struct OrderBuffers {
    const uint32_t* cam_idx;   // [n_obs] uploaded
    const uint32_t* pt_idx;    // [n_obs]
    const double* pixels;      // [n_obs][2]
    uint32_t* pt_key;          // [n_pts] scratch
    uint32_t* tile_cnt;        // [n_tiles + 1] scratch
    uint64_t* keys;            // [pow2(max(n_obs, n_pts))] scratch
    uint32_t* vals;            // [pow2(...)] scratch
    size_t sort_cap;
};
template <typename T>
void build_order(const Views<T>& v, const OrderBuffers& b, cudaStream_t s);
// Sets *flag (device, zeroed by the caller) when two neighbouring keys of the ordered
// observation table are equal: a camera that observes a point twice (or, rarely, the
// same camera and slot on both sides of a tile boundary; a false alarm only costs the
// operator its plain point sums).  order.cu.
void flag_repeated_keys(const uint32_t* obs_key, int64_t n_obs, uint32_t* flag, cudaStream_t s);
// Ascending sort of (key, value) pairs, n a power of two >= 2 (order.cu).
void sort_pairs(uint64_t* keys, uint32_t* vals, size_t n, cudaStream_t s);


}  // namespace gbba
