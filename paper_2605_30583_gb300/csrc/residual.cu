// Residual pass of the mixed-precision form: r = f s p - u of every observation (the
// Snavely reprojection factor of Sec. VI-A), written to v.rbuf in solver order, and the
// cost 1/2 sum rho(|r|^2) into st->F_res: every cost of the mixed form (F at the start
// of a solve, F' of a candidate, the evaluation's cost) comes from this one sum.
//
// Precision.  Everything else in the mixed form is FP32 with FP64 reductions, but the
// residual is a difference of ~500 px terms that cancel to ~1 px, so FP32 leaves it with
// an error of ~1e-4 px that depends on the parameters' last bits.  On problems with flat
// directions (points seen along nearly parallel rays) LM walks along them into places
// where those errors happen to lower the FP32 cost, and stops at parameters whose true
// cost is higher than the plain FP64 solver's optimum.  With res_df (the default) the
// residual is computed in double-float arithmetic (df.cuh) from the FP64 master
// parameters (points) and the double-float camera records, and only then rounded to
// FP32: the cost LM sees is then the true cost to ~1e-7 px per residual.  The Jacobian,
// the normal operator and PCG stay FP32.
//
// One CTA per tile (grid-stride): the tile's points are staged in shared memory, then
// the threads walk the tile's observations in order (coalesced keys, pixels and
// results); consecutive observations share their camera, whose records come through L1.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace gbba {
namespace {

constexpr int RS_TB = 256;

template <int TB>
__global__ void __launch_bounds__(TB) k_residual(Views<float> v, int at_candidate, int squared) {
    DevState* st = v.st;
    // a candidate is only evaluated while LM runs (the decision kernel reads F' then)
    if (at_candidate && st->lm_active == 0) return;
    __shared__ float4 sXh[TILE_PTS], sXl[TILE_PTS];   // the tile's points, double-float
    const double* xm = at_candidate ? v.xm_new : v.xm;
    const float* rec = at_candidate ? v.cam_pre_new : v.cam_pre;
    const float* lor = at_candidate ? v.cam_lo_new : v.cam_lo;
    const float eps = (float)st->opt.eps;
    const int loss = squared ? 0 : st->opt.loss;
    const float lscale = (float)st->opt.loss_scale;
    const bool dfp = st->opt.res_df != 0;
    // the cost: Kahan pair of the high parts of |r|^2 (double-float |r|^2 before any
    // rounding, so F resolves steps far below an FP32 ulp of the residuals) and the sum
    // of their low parts
    float cs = 0.0f, cc = 0.0f, cl = 0.0f;
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        for (int i = threadIdx.x; i < npt; i += TB) {
            const DF a = df_from_double(xm[base + 3 * i]), b = df_from_double(xm[base + 3 * i + 1]),
                     c = df_from_double(xm[base + 3 * i + 2]);
            sXh[i] = make_float4(a.hi, b.hi, c.hi, 0.0f);
            sXl[i] = make_float4(a.lo, b.lo, c.lo, 0.0f);
        }
        __syncthreads();
        for (uint32_t j = lo + threadIdx.x; j < hi; j += TB) {
            const uint32_t key = __ldg(v.obs_key + j);
            const uint32_t c = key >> 8, slot = key & 0xffu;
            const float2 uv = __ldg(reinterpret_cast<const float2*>(v.obs_uv) + j);
            const float4 xh = sXh[slot];
            float r0, r1;
            DF s2 = {0.0f, 0.0f};
            if (dfp) {
                const float4 xl = sXl[slot];
                const CamDF cam = load_cam_df(rec + (size_t)c * CP_STRIDE, lor + (size_t)c * CLO_STRIDE);
                const DF X[3] = {{xh.x, xl.x}, {xh.y, xl.y}, {xh.z, xl.z}};
                DF d0, d1;
                residual_df(cam, X, eps, uv.x, uv.y, d0, d1);
                r0 = df_to_float(d0);
                r1 = df_to_float(d1);
                s2 = df_add(df_mul(d0, d0), df_mul(d1, d1));
            } else {
                const Cam cam = load_cam(rec + (size_t)c * CP_STRIDE);
                project_residual(cam, xh.x, xh.y, xh.z, eps, uv.x, uv.y, r0, r1);
                s2.hi = fmaf(r0, r0, r1 * r1);
            }
            reinterpret_cast<float2*>(v.rbuf)[j] = make_float2(r0, r1);
            if (loss) {   // robust loss: rho of the FP32-rounded |r|^2
                kahan_add(cs, cc, loss_rho(df_to_float(s2), loss, lscale));
            } else {
                kahan_add(cs, cc, s2.hi);
                cl += s2.lo;
            }
        }
        __syncthreads();   // the next tile's staging overwrites the points
    }
    double in[1] = {(double)cs - (double)cc + (double)cl}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_RES], out) && threadIdx.x == 0) st->F_res = 0.5 * out[0];
}

}  // namespace

void launch_residual(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int at_candidate, int squared) {
    const int grid = std::max(1, std::min({v.n_tiles, L.res_grid, MAX_GRID}));
    k_residual<RS_TB><<<grid, RS_TB, 0, s>>>(v, at_candidate, squared);
}

int occupancy_blocks_residual() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_residual<RS_TB>, RS_TB, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, n);
}

}  // namespace gbba
