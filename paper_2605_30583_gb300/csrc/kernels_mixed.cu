// Mixed-precision LM + PCGNR kernels (FP32 bulk arithmetic, FP64 sums, FP64
// block inversions).  Sec. V of arXiv 2605.30583: Levenberg-Marquardt, no Schur
// complement, PCGNR on the full damped normal equations, block-Jacobi
// preconditioner with one block per node; Sec. VI-A: the reprojection factor.
//
// The Jacobian is never stored.  Every product with J or J^T recomputes the 2x12
// Jacobian of an observation from the camera record (R, t, f, k1, k2, J_l) and the
// point: on this hardware the ~100 FP32 operations per observation cost less than
// streaming 96 bytes of stored Jacobian per observation from HBM.
//
// Work decomposition: a tile is TILE_PTS consecutive points (locality order) and all
// their observations, sorted by camera inside the tile.  One CTA handles a tile;
// each thread takes a contiguous chunk of the tile's observations, keeps the camera
// sums of the current camera run in registers, and at the end of its chunk a
// warp-segmented reduction combines lanes of the same camera before one atomic per
// camera run (the role of the Shared Add accessor of Sec. IV-A).  Point sums go to
// shared memory (the tile owns its points) and are written once per tile.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"
#include "mixed_common.cuh"

namespace gbba {


// ------------------------------------------------------------------ K0 --------
// Camera records from the current parameters (their FP64 master copy); zeroes the
// linearisation sums.
__global__ void k_camera_precompute(Views<float> v) {
    for (int c = 32 * (int)blockIdx.x + (int)threadIdx.x; threadIdx.x < 32 && c < v.n_cams; c += 32 * (int)gridDim.x) {
        double p[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k] = v.xm[9 * (size_t)c + k];
        camera_record(p, v.cam_pre + (size_t)c * CP_STRIDE, v.st->opt.retract != 0, v.cam_lo + (size_t)c * CLO_STRIDE);
        double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
#pragma unroll
        for (int k = 0; k < CL_STRIDE; ++k) cl[k] = 0.0;
        float* ch = v.cam_H + (size_t)c * CH_STRIDE;
#pragma unroll
        for (int k = 0; k < CH_STRIDE; ++k) ch[k] = 0.0f;
    }
}

// ------------------------------------------------------------------ K1 --------
// Linearisation (fused score + Jacobian products, Sec. V-A): cost F = 1/2 |r|^2,
// g = J^T r and the diagonal blocks J_c^T J_c, J_p^T J_p.  Two passes per tile:
//   camera pass: the tile's camera-sorted observations, camera sums in registers,
//     one set of atomics per camera run (g in FP64, J_c^T J_c in FP32 float4 atomics);
//   point pass: one thread per point over its observations (point-major index), point
//     sums in registers, no atomics; it also sums the cost.
// `mode`: 0 = first linearisation of a solve (initialises the LM state), 1 =
// relinearisation after an accepted step (gated by st->relin), 2 = evaluation only
// (optional r and J output in the caller's observation order).
constexpr int LIN_ACC = 9 + CH_STRIDE;   // g (9) + J_c^T J_c upper triangle padded to 48

__device__ __forceinline__ void flush_lin(const Views<float>& v, uint32_t c, float (&a)[LIN_ACC]) {
    double* g = v.cam_lin + (size_t)c * CL_STRIDE;
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(g + k, (double)a[k]);
    float4* h = reinterpret_cast<float4*>(v.cam_H + (size_t)c * CH_STRIDE);
#pragma unroll
    for (int k = 0; k < CH_STRIDE / 4; ++k)
        atomicAdd(h + k, make_float4(a[9 + 4 * k], a[10 + 4 * k], a[11 + 4 * k], a[12 + 4 * k]));
#pragma unroll
    for (int k = 0; k < LIN_ACC; ++k) a[k] = 0.0f;
}

// Six CTAs per SM (80 registers, some spilled to L1): the medium workload's 782 tiles then
// run in one wave instead of 1.3 waves of four CTAs per SM (126 -> 109 us).
template <int TB>
__global__ void __launch_bounds__(TB, 6) k_linearize(Views<float> v, int mode, float* res_out, float* jac_out,
                                                  CondHandle lm_cond, int use_cond) {
    if (mode == 1 && v.st->relin == 0) return;
    __shared__ float4 sx[TILE_PTS];
    __shared__ float sg[3 * TILE_PTS], sh[6 * TILE_PTS];   // the tile's points: J_p^T r, J_p^T J_p
    const float eps = (float)v.st->opt.eps;
    // robust loss (evaluation, mode 2, is always the squared loss)
    const int loss = mode == 2 ? 0 : v.st->opt.loss;
    const float lscale = (float)v.st->opt.loss_scale;
    float cost = 0.0f, costc = 0.0f;   // Kahan pair
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        __syncthreads();
        for (int i = threadIdx.x; i < npt; i += TB) {
            sx[i] = make_float4(v.x[base + 3 * i], v.x[base + 3 * i + 1], v.x[base + 3 * i + 2], 0.0f);
#pragma unroll
            for (int q = 0; q < 3; ++q) sg[3 * i + q] = 0.0f;
#pragma unroll
            for (int q = 0; q < 6; ++q) sh[6 * i + q] = 0.0f;
        }
        __syncthreads();
        // one pass over the tile's camera-sorted observations: camera sums in registers
        // (one flush per camera run), the tile's point sums in shared memory
        {
            const uint32_t n = hi - lo;
            const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
            const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
            uint32_t cur = NO_CAM;
            float acc[LIN_ACC];
#pragma unroll
            for (int k = 0; k < LIN_ACC; ++k) acc[k] = 0.0f;
            Cam cam;
            float JL[9];
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    if (cur != NO_CAM) flush_lin(v, cur, acc);
                    cur = c;
                    cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
#pragma unroll
                    for (int k = 0; k < 9; ++k) JL[k] = __ldg(v.cam_pre + (size_t)c * CP_STRIDE + CP_JL + k);
                }
                const float4 X = sx[slot];
                const Geo g = project_geo(cam, X.x, X.y, X.z, eps);
                float r0 = __ldg(v.rbuf + 2 * (size_t)j), r1 = __ldg(v.rbuf + 2 * (size_t)j + 1);   // k_residual
                // camera Jacobian rows: [J_w | J_t | J_intr], J_w[:,k] = A (J_l[:,k] x RX)
                float j0[9], j1[9];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float w0 = JL[k], w1 = JL[3 + k], w2 = JL[6 + k];
                    const float c0 = fmaf(w1, g.RX[2], -w2 * g.RX[1]);
                    const float c1 = fmaf(w2, g.RX[0], -w0 * g.RX[2]);
                    const float c2 = fmaf(w0, g.RX[1], -w1 * g.RX[0]);
                    j0[k] = fmaf(g.A[0], c0, fmaf(g.A[1], c1, g.A[2] * c2));
                    j1[k] = fmaf(g.A[3], c0, fmaf(g.A[4], c1, g.A[5] * c2));
                    j0[3 + k] = g.A[k];
                    j1[3 + k] = g.A[3 + k];
                }
                const float fn2 = cam.f * g.n2;
                j0[6] = g.s * g.p[0]; j0[7] = fn2 * g.p[0]; j0[8] = fn2 * g.n2 * g.p[0];
                j1[6] = g.s * g.p[1]; j1[7] = fn2 * g.p[1]; j1[8] = fn2 * g.n2 * g.p[1];
                float jx0[3], jx1[3];   // point Jacobian rows J_X = A R
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    jx0[q] = fmaf(g.A[0], cam.R[q], fmaf(g.A[1], cam.R[3 + q], g.A[2] * cam.R[6 + q]));
                    jx1[q] = fmaf(g.A[3], cam.R[q], fmaf(g.A[4], cam.R[3 + q], g.A[5] * cam.R[6 + q]));
                }
                if (mode == 2) {   // evaluation output: the unweighted residual and Jacobian
                    const uint32_t o = v.obs_user[j];
                    if (res_out) { res_out[2 * (size_t)o] = r0; res_out[2 * (size_t)o + 1] = r1; }
                    if (jac_out) {
                        float* Jo = jac_out + 24 * (size_t)o;
#pragma unroll
                        for (int k = 0; k < 9; ++k) { Jo[k] = j0[k]; Jo[12 + k] = j1[k]; }
#pragma unroll
                        for (int q = 0; q < 3; ++q) { Jo[9 + q] = jx0[q]; Jo[21 + q] = jx1[q]; }
                    }
                }
                const float s2 = fmaf(r0, r0, r1 * r1);
                if (loss) {   // IRLS weight w = rho'(|r|^2): rows scaled by sqrt(w)
                    const float w = loss_weight(s2, loss, lscale);
                    if (mode != 2) v.obs_w[j] = w;
                    kahan_add(cost, costc, loss_rho(s2, loss, lscale));
                    const float sw = sqrtf(w);
                    r0 *= sw;
                    r1 *= sw;
#pragma unroll
                    for (int k = 0; k < 9; ++k) { j0[k] *= sw; j1[k] *= sw; }
#pragma unroll
                    for (int q = 0; q < 3; ++q) { jx0[q] *= sw; jx1[q] *= sw; }
                } else {
                    kahan_add(cost, costc, s2);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) acc[CL_G + i] = fmaf(j0[i], r0, fmaf(j1[i], r1, acc[CL_G + i]));
#pragma unroll
                for (int i = 0; i < 9; ++i)
#pragma unroll
                    for (int k = i; k < 9; ++k) {
                        const int t = 9 + tri_index(9, i, k);
                        acc[t] = fmaf(j0[i], j0[k], fmaf(j1[i], j1[k], acc[t]));
                    }
                float* gq = sg + 3 * slot;
                float* hq = sh + 6 * slot;
#pragma unroll
                for (int q = 0; q < 3; ++q) atomicAdd(gq + q, fmaf(jx0[q], r0, jx1[q] * r1));
#pragma unroll
                for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
                    for (int b2 = a2; b2 < 3; ++b2)
                        atomicAdd(hq + tri_index(3, a2, b2), fmaf(jx0[a2], jx0[b2], jx1[a2] * jx1[b2]));
            }
            // camera sums: combine lanes of the same camera, one set of atomics per run
            const bool head = seg_reduce<LIN_ACC>(cur, acc);
            if (head && cur != NO_CAM) flush_lin(v, cur, acc);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < npt; i += TB) {
#pragma unroll
            for (int q = 0; q < 3; ++q) v.g[base + 3 * i + q] = sg[3 * i + q];
#pragma unroll
            for (int q = 0; q < PH_STRIDE; ++q) v.pt_H[(size_t)(pt0 + i) * PH_STRIDE + q] = sh[6 * i + q];
        }
    }
    double in[1] = {(double)cost - (double)costc}, out[1];
    if (grid_reduce<1>(in, v.partials, &v.st->tickets[TK_LIN], out) && threadIdx.x == 0) {
        DevState* st = v.st;
        // the cost is the residual pass's (k_residual, at these parameters); pose factors:
        // k_factor_linearize.  After an accepted step the LM decision has already set F.
        (void)out;
        const double F = st->F_res + (v.n_fac > 0 ? st->fac_cost : 0.0);
        st->cost_out = F;
        if (mode == 0) {
            st->F = F;
            st->F0 = F;
            const bool ok = isfinite(F);
            if (!ok) st->status = 4;
            st->lm_active = (ok && F > 0.0 && st->opt.max_lm > 0) ? 1 : 0;
            if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
        }
    }
}

// ------------------------------------------------------------------ K3 --------
// Block-Jacobi preconditioner (Sec. V: one block per node) of J^T J + mu D, inverted
// by FP64 Cholesky, and the start of PCGNR: h = 0, r = -g, z = M^-1 r, p = 0.
// Camera c of an item kernel runs in lane c % 32 of warp 0 of block (c / 32) % gridDim:
// 32 cameras share every warp instruction (the FP64 pipe takes whole warps, so a warp
// with one busy lane costs as much as a full one) and the cameras spread over the SMs.
// The other warps of the block skip the loop.
#define FOR_CAMERAS(c, v) \
    for (int c = 32 * (int)blockIdx.x + (int)threadIdx.x; threadIdx.x < 32 && c < (v).n_cams; \
         c += 32 * (int)gridDim.x)
#define FOR_POINTS(i, v) \
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (v).n_pts; i += gridDim.x * blockDim.x)

// Blocks [0, cam_blocks) invert the camera blocks (a warp per camera); the others
// invert the point blocks (a thread per point), so the long FP64 camera eliminations run
// beside the point work instead of before it in the same warps.
__global__ void k_precond(Views<float> v, CondHandle pcg_cond, int use_cond, double* pslots, int cam_blocks) {
    DevState* st = v.st;
    if (pslots != nullptr && blockIdx.x == 0) {   // state of the persistent PCG kernel
        for (int i = threadIdx.x; i < PSLOT_TOTAL; i += blockDim.x) pslots[i] = 0.0;
        if (threadIdx.x == 0) {
            st->bar_count = 0ull;
            st->bar_err = 0;
        }
    }
    if (st->lm_active == 0) {
        // the PCG loop that follows must see a cleared flag
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(pcg_cond, 0u);
        return;
    }
    const double mu = st->mu, lo = st->opt.min_diag, hi = st->opt.max_diag;
    double rz = 0.0, rr = 0.0;
    const int lane = threadIdx.x & 31;
    const int warps = cam_blocks * (blockDim.x >> 5);
    const bool cam_role = (int)blockIdx.x < cam_blocks;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cam_role && c < v.n_cams; c += warps) {
        const double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
        double col[9];
        const int j = lane < 18 ? lane : 17;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (j < 9) {
                const int lo_i = i < j ? i : j, hi_i = i < j ? j : i;
                double h = (double)v.cam_H[(size_t)c * CH_STRIDE + tri_index(9, lo_i, hi_i)];
                if (i == j) h += mu * fmin(fmax(h, lo), hi);
                col[i] = h;
            } else {
                col[i] = (i == j - 9) ? 1.0 : 0.0;
            }
        }
        // diagonal of J^T J for D and for the fallback, before elimination
        const double hdiag = (lane < 9) ? (double)v.cam_H[(size_t)c * CH_STRIDE + tri_index(9, lane, lane)] : 0.0;
        const bool ok = warp_block_inverse9(col, lane);
        float* Mo = v.Minv_c + (size_t)c * MC_STRIDE;
        if (lane >= 9 && lane < 18) {
            const int jj = lane - 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) Mo[i * 9 + jj] = (float)col[i];
        }
        if (!ok && lane < 9) {   // not SPD in FP64: inverse diagonal
            const double dd = hdiag + mu * fmin(fmax(hdiag, lo), hi);
#pragma unroll
            for (int i = 0; i < 9; ++i) Mo[i * 9 + lane] = (i == lane && dd > 0.0) ? (float)(1.0 / dd) : 0.0f;
        }
        __syncwarp();
        if (lane < 9) {
            const size_t e = 9 * (size_t)c + lane;
            v.D[e] = (float)fmin(fmax(hdiag, lo), hi);
            const float ri = (float)(-cl[CL_G + lane]);
            // z_i = sum_k M[i][k] r_k
            float z = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) z = fmaf(Mo[lane * 9 + k], (float)(-cl[CL_G + k]), z);
            v.r[e] = ri;
            v.z[e] = z;
            v.p[e] = 0.0f;
            v.s[e] = 0.0f;
            v.h[e] = 0.0f;
            v.pc[e] = 0.0f;
            v.pc[v.pc_stride + e] = 0.0f;
            rz += (double)ri * (double)z;
            rr += (double)ri * (double)ri;
        }
        if (lane < CA_STRIDE) {
            v.cam_acc[(size_t)c * CA_STRIDE + lane] = 0.0f;
            if (pslots != nullptr)   // the persistent kernel rotates over all the sets
                for (int set = 1; set < CA_SETS; ++set)
                    v.cam_acc[((size_t)set * v.n_cams + c) * CA_STRIDE + lane] = 0.0f;
        }
    }
    const int pt_stride = ((int)gridDim.x - cam_blocks) * blockDim.x;
    for (int i = ((int)blockIdx.x - cam_blocks) * blockDim.x + threadIdx.x; !cam_role && i < v.n_pts; i += pt_stride) {
        const float* H = v.pt_H + (size_t)i * PH_STRIDE;
        const size_t e = v.pt_off + 3 * (size_t)i;
        double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
        const double d0 = fmin(fmax(a00, lo), hi), d1 = fmin(fmax(a11, lo), hi), d2 = fmin(fmax(a22, lo), hi);
        a00 += mu * d0; a11 += mu * d1; a22 += mu * d2;
        // inverse of the SPD 3x3 block by its adjugate: M = adj(A) / det(A)
        double m[6];
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        if (det > 0.0 && isfinite(det) && a00 > 0.0 && c22 > 0.0) {
            const double id = rcp64(det);
            m[0] = c00 * id; m[1] = c01 * id; m[2] = c02 * id;
            m[3] = c11 * id; m[4] = c12 * id; m[5] = c22 * id;
        } else {   // not SPD in FP64: inverse diagonal
            m[0] = a00 > 0 ? 1.0 / a00 : 0.0; m[1] = 0.0; m[2] = 0.0;
            m[3] = a11 > 0 ? 1.0 / a11 : 0.0; m[4] = 0.0;
            m[5] = a22 > 0 ? 1.0 / a22 : 0.0;
        }
        float* Mo = v.Minv_p + (size_t)i * MP_STRIDE;
        for (int k = 0; k < 6; ++k) Mo[k] = (float)m[k];
        v.D[e] = (float)d0; v.D[e + 1] = (float)d1; v.D[e + 2] = (float)d2;
        const float r0 = -v.g[e], r1 = -v.g[e + 1], r2 = -v.g[e + 2];
        const float z0 = fmaf(Mo[0], r0, fmaf(Mo[1], r1, Mo[2] * r2));
        const float z1 = fmaf(Mo[1], r0, fmaf(Mo[3], r1, Mo[4] * r2));
        const float z2 = fmaf(Mo[2], r0, fmaf(Mo[4], r1, Mo[5] * r2));
        v.r[e] = r0; v.r[e + 1] = r1; v.r[e + 2] = r2;
        v.z[e] = z0; v.z[e + 1] = z1; v.z[e + 2] = z2;
        v.p[e] = 0.0f; v.p[e + 1] = 0.0f; v.p[e + 2] = 0.0f;
        v.s[e] = 0.0f; v.s[e + 1] = 0.0f; v.s[e + 2] = 0.0f;
        v.h[e] = 0.0f; v.h[e + 1] = 0.0f; v.h[e + 2] = 0.0f;
        rz += (double)(r0 * z0 + r1 * z1 + r2 * z2);
        rr += (double)(r0 * r0 + r1 * r1 + r2 * r2);
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_PRE], out) && threadIdx.x == 0) {
        st->rz = out[0];
        st->rr0 = out[1];
        st->rr = out[1];
        st->beta = 0.0;
        st->alpha = 0.0;
        st->pcg_iter = 0;
        for (int k = 0; k < NSLOT * SLOT_STRIDE; ++k) st->acc_mv[k] = st->acc_up[k] = 0.0;
        // a non-finite r^T z means a non-finite gradient or block (a Jacobian that
        // overflowed, e.g. a point at a camera centre): a numeric failure, not a stall
        if (!isfinite(out[0]) || !isfinite(out[1])) st->status = 4;
        st->pcg_active = (out[1] > 0.0 && isfinite(out[0]) && st->opt.max_pcg > 0) ? 1 : 0;
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ K4 --------
// Camera part of one PCG direction step, before k_matvec: p_c = zs_c + beta p_prev_c
// for every camera (double-buffered: pc[parity] holds p_prev, pc[parity ^ 1] receives
// p), its direction record (phi = J_l p_w, p_t, p_intr) into cam_dir, and the camera
// part of p^T D p into st->acc_mv.  One thread per camera entry; the three rotation
// rows of phi recompute the camera's p_w themselves.
__global__ void k_cam_direction(Views<float> v, const int32_t* gate, const float* zs, int use_beta) {
    if (gated_off(gate)) return;
    __shared__ double red[32];
    DevState* st = v.st;
    const int par = st->pcg_iter & 1;
    const float beta = use_beta ? (float)st->beta : 0.0f;
    const float* pc_old = v.pc + (size_t)par * v.pc_stride;
    float* pc_new = v.pc + (size_t)(par ^ 1) * v.pc_stride;
    float pdp = 0.0f, pdpc = 0.0f;   // Kahan pair
    const int n = 9 * v.n_cams;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int c = e / 9, k = e - 9 * c;
        auto p_of = [&](int i) {
            const size_t x = 9 * (size_t)c + i;
            return beta != 0.0f ? fmaf(beta, pc_old[x], zs[x]) : zs[x];
        };
        const float pk = p_of(k);
        pc_new[e] = pk;
        kahan_add(pdp, pdpc, v.D[e] * pk * pk);
        float d = pk;
        if (k < 3) {
            const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL + 3 * k;
            d = fmaf(__ldg(JL), p_of(0), fmaf(__ldg(JL + 1), p_of(1), __ldg(JL + 2) * p_of(2)));
        }
        v.cam_dir[(size_t)c * CD_STRIDE + k] = d;   // CD_PHI = 0, CD_T = 3, CD_I = 6
    }
    const double bp = block_sum((double)pdp - (double)pdpc, red);
    if (threadIdx.x == 0) slot_add(st->acc_mv, 1, bp);
}

// One PCG direction step fused with the damped normal operator, after k_cam_direction:
//   p = zs + beta p_prev for the points (zs = z during PCG; beta = 0 applies to a given p)
//   q = J^T J p + mu D p                 (points; cameras are finished in K5)
//   |J p|^2 and the points' p^T D p are added to st->acc_mv.
// Each tile's keys, points and point directions are staged in shared memory; a camera
// switch loads the camera's record and direction record.

template <int TB>
__global__ void __launch_bounds__(TB, 8) k_matvec(Views<float> v, const int32_t* gate, const float* zs, int use_beta) {
    if (gated_off(gate)) return;
    __shared__ float sx[3 * TILE_PTS], sd[3 * TILE_PTS], sq[3 * TILE_PTS];
    __shared__ double red[32];
    DevState* st = v.st;
    const float beta = use_beta ? (float)st->beta : 0.0f;
    const float mu = (float)st->mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;
    // Kahan pairs; the camera part of p^T D p comes from k_cam_direction
    float pdp = 0.0f, jp2 = 0.0f, pdpc = 0.0f, jp2c = 0.0f;
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        for (int i = threadIdx.x; i < 3 * npt; i += TB) {
            const float pn = beta != 0.0f ? fmaf(beta, v.p[base + i], zs[base + i]) : zs[base + i];
            v.p[base + i] = pn;
            sd[i] = pn;
            sx[i] = v.x[base + i];
            sq[i] = 0.0f;
            kahan_add(pdp, pdpc, v.D[base + i] * pn * pn);
        }
        __syncthreads();
        const uint32_t n = hi - lo;
        const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
        const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
        uint32_t cur = NO_CAM;
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
        Cam cam;
        float dir[9];
        uint32_t j = a;
        while (j < b) {
            const uint32_t key = __ldg(v.obs_key + j);
            const uint32_t c = key >> 8, slot = key & 0xffu;
            if (c != cur) {
                if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                cur = c;
                cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);   // from k_cam_direction
            }
            if (weighted) {   // robust loss: per-observation IRLS weights
                kahan_add(jp2, jp2c, obs_normal<true>(cam, dir, sx + 3 * slot, sd + 3 * slot, eps, acc,
                                                      sq + 3 * slot, __ldg(v.obs_w + j)));
                j += 1;
                continue;
            }
            if (j + 1 < b) {
                const uint32_t key1 = __ldg(v.obs_key + j + 1);
                if ((key1 >> 8) == c) {
                    // two observations of the same camera: independent chains interleave
                    const uint32_t slot1 = key1 & 0xffu;
                    const float a0 = obs_normal(cam, dir, sx + 3 * slot, sd + 3 * slot, eps, acc, sq + 3 * slot);
                    const float a1 = obs_normal(cam, dir, sx + 3 * slot1, sd + 3 * slot1, eps, acc, sq + 3 * slot1);
                    kahan_add(jp2, jp2c, a0);
                    kahan_add(jp2, jp2c, a1);
                    j += 2;
                    continue;
                }
            }
            kahan_add(jp2, jp2c, obs_normal(cam, dir, sx + 3 * slot, sd + 3 * slot, eps, acc, sq + 3 * slot));
            j += 1;
        }
        const bool head = seg_reduce<9>(cur, acc);
        if (head && cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * npt; i += TB) v.q[base + i] = fmaf(mu, v.D[base + i] * sd[i], sq[i]);
        __syncthreads();
    }
    const double bj = block_sum((double)jp2 - (double)jp2c, red);
    const double bp = block_sum((double)pdp - (double)pdpc, red);
    if (threadIdx.x == 0) {
        slot_add(st->acc_mv, 0, bj);
        slot_add(st->acc_mv, 1, bp);
    }
}

// ------------------------------------------------------------------ K5 --------
// alpha = r^T z / (|J p|^2 + mu p^T D p); h += alpha p; r -= alpha q; z = M^-1 r; the
// sums r^T z and |r|^2 go to st->acc_up.  Cameras first finish
// q = (J_l^T sum RX x u, sum u, intrinsic part) + mu D p from the K4 accumulators.
// Points run four at a time with float4 accesses.  Never gated: its last block
// decides whether PCG continues, sets the loop flag and clears the accumulators.
__global__ void k_update(Views<float> v, CondHandle pcg_cond, int use_cond, int cameras_only) {
    DevState* st = v.st;
    __shared__ double red[32];
    __shared__ double sh_mv[2];
    __shared__ bool is_last;
    const int active = st->pcg_active;
    float rz = 0.0f, rr = 0.0f, rzc = 0.0f, rrc = 0.0f;   // Kahan pairs
    double alpha_d = 0.0;
    bool bad = false;
    if (active) {
        if (threadIdx.x < 32) {
            const double a0 = slot_sum_warp(st->acc_mv, 0), a1 = slot_sum_warp(st->acc_mv, 1);
            if (threadIdx.x == 0) { sh_mv[0] = a0; sh_mv[1] = a1; }
        }
        __syncthreads();
        const double denom = sh_mv[0] + st->mu * sh_mv[1];
        bad = !(denom > 0.0) || !isfinite(denom);
        alpha_d = bad ? 0.0 : st->rz / denom;
    }
    if (active && !bad) {
        const float alpha = (float)alpha_d;
        const float mu = (float)st->mu;
        const float* pcur = v.pc + (size_t)((st->pcg_iter & 1) ^ 1) * v.pc_stride;
        FOR_CAMERAS(c, v) {
            const size_t e = 9 * (size_t)c;
            float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
            const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
            float q[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) q[k] = fmaf(JL[k], ca[0], fmaf(JL[3 + k], ca[1], JL[6 + k] * ca[2]));
#pragma unroll
            for (int k = 3; k < 9; ++k) q[k] = ca[k];
#pragma unroll
            for (int k = 0; k < CA_STRIDE; ++k) ca[k] = 0.0f;
            float rn[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float pk = pcur[e + k];
                const float qk = fmaf(mu, v.D[e + k] * pk, q[k]);
                v.p[e + k] = pk;
                v.h[e + k] = fmaf(alpha, pk, v.h[e + k]);
                rn[k] = fmaf(-alpha, qk, v.r[e + k]);
                v.r[e + k] = rn[k];
            }
            const float* M = v.Minv_c + (size_t)c * MC_STRIDE;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float z = 0.0f;
#pragma unroll
                for (int k = 0; k < 9; ++k) z = fmaf(M[9 * i + k], rn[k], z);
                v.z[e + i] = z;
                kahan_add(rz, rzc, rn[i] * z);
                kahan_add(rr, rrc, rn[i] * rn[i]);
            }
        }
        for (int qd = blockIdx.x * blockDim.x + threadIdx.x; !cameras_only && qd < v.n_quads;
             qd += gridDim.x * blockDim.x) {
            const size_t e = v.pt_off + 12 * (size_t)qd;
            float4* p4 = reinterpret_cast<float4*>(v.p + e);
            float4* h4 = reinterpret_cast<float4*>(v.h + e);
            float4* r4 = reinterpret_cast<float4*>(v.r + e);
            const float4* q4 = reinterpret_cast<const float4*>(v.q + e);
            float4* z4 = reinterpret_cast<float4*>(v.z + e);
            const float4* m4 = reinterpret_cast<const float4*>(v.Minv_p + 24 * (size_t)qd);
            float P[12], H[12], R[12], Q[12], M[24];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 a = p4[k], b = h4[k], c = r4[k], d = q4[k];
                P[4 * k] = a.x; P[4 * k + 1] = a.y; P[4 * k + 2] = a.z; P[4 * k + 3] = a.w;
                H[4 * k] = b.x; H[4 * k + 1] = b.y; H[4 * k + 2] = b.z; H[4 * k + 3] = b.w;
                R[4 * k] = c.x; R[4 * k + 1] = c.y; R[4 * k + 2] = c.z; R[4 * k + 3] = c.w;
                Q[4 * k] = d.x; Q[4 * k + 1] = d.y; Q[4 * k + 2] = d.z; Q[4 * k + 3] = d.w;
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float4 a = __ldg(m4 + k);
                M[4 * k] = a.x; M[4 * k + 1] = a.y; M[4 * k + 2] = a.z; M[4 * k + 3] = a.w;
            }
            float Z[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                H[k] = fmaf(alpha, P[k], H[k]);
                R[k] = fmaf(-alpha, Q[k], R[k]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float* m = M + 6 * j;
                const float* rj = R + 3 * j;
                Z[3 * j + 0] = fmaf(m[0], rj[0], fmaf(m[1], rj[1], m[2] * rj[2]));
                Z[3 * j + 1] = fmaf(m[1], rj[0], fmaf(m[3], rj[1], m[4] * rj[2]));
                Z[3 * j + 2] = fmaf(m[2], rj[0], fmaf(m[4], rj[1], m[5] * rj[2]));
            }
#pragma unroll
            for (int k = 0; k < 12; k += 3) {
                kahan_add(rz, rzc, fmaf(R[k], Z[k], fmaf(R[k + 1], Z[k + 1], R[k + 2] * Z[k + 2])));
                kahan_add(rr, rrc, fmaf(R[k], R[k], fmaf(R[k + 1], R[k + 1], R[k + 2] * R[k + 2])));
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                h4[k] = make_float4(H[4 * k], H[4 * k + 1], H[4 * k + 2], H[4 * k + 3]);
                r4[k] = make_float4(R[4 * k], R[4 * k + 1], R[4 * k + 2], R[4 * k + 3]);
                z4[k] = make_float4(Z[4 * k], Z[4 * k + 1], Z[4 * k + 2], Z[4 * k + 3]);
            }
        }
    }
    const double brz = block_sum((double)rz - (double)rzc, red);
    const double brr = block_sum((double)rr - (double)rrc, red);
    if (threadIdx.x == 0) {
        if (active && !bad) {
            slot_add(st->acc_up, 0, brz);
            slot_add(st->acc_up, 1, brr);
        }
        __threadfence();
        const unsigned int t = atomicAdd(&st->tickets[TK_UPD], 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    const double rzn = slot_sum_warp(st->acc_up, 0), rrn = slot_sum_warp(st->acc_up, 1);
    // the whole warp clears the slots; lane 0 takes the decisions
    for (int k = threadIdx.x; k < NSLOT * SLOT_STRIDE; k += 32) st->acc_mv[k] = st->acc_up[k] = 0.0;
    if (threadIdx.x != 0) return;
    if (active) {
        if (bad) {
            st->pcg_active = 0;
            if (!isfinite(sh_mv[0]) || !isfinite(sh_mv[1])) st->status = 4;
        } else {
            st->alpha = alpha_d;
            st->jp2 = sh_mv[0];
            st->pDp = sh_mv[1];
            st->pcg_iter += 1;
            st->pcg_total += 1;
            st->rr = rrn;
            const double tol = st->opt.tol;
            if (!isfinite(rzn) || !isfinite(rrn)) {
                st->status = 4;
                st->pcg_active = 0;
            } else if (rrn <= tol * tol * st->rr0 || st->pcg_iter >= st->opt.max_pcg) {
                st->pcg_active = 0;
            } else {
                st->beta = rzn / st->rz;
                st->rz = rzn;
            }
        }
    }
    st->tickets[TK_UPD] = 0u;
    if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
}

// ------------------------------------------------------------------ K7 --------
// Candidate x' = x + h, g^T h, camera records at x', and the camera direction
// records of h at x (for |J h|^2).
__global__ void k_candidate(Views<float> v) {
    DevState* st = v.st;
    // the one-reduction PCG leaves its last round's camera sums behind
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.n_cams * CA_STRIDE; i += gridDim.x * blockDim.x)
        v.cam_acc[i] = 0.0f;
    if (st->lm_active == 0) return;
    const bool retract = st->opt.retract != 0;
    double gh = 0.0;
    FOR_CAMERAS(c, v) {
        {
            const size_t e = 9 * (size_t)c;
            const double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
            // the step applied to the FP64 master copy; the FP32 copy is its rounding
            double xn[9];
            float hc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                hc[k] = v.h[e + k];
                xn[k] = v.xm[e + k] + (double)hc[k];
                gh += cl[CL_G + k] * (double)hc[k];
            }
            if (retract) {   // R' = Exp(h_w) R(w)
                const double w[3] = {v.xm[e], v.xm[e + 1], v.xm[e + 2]};
                const double hw[3] = {hc[0], hc[1], hc[2]};
                compose_rotvec(hw, w, xn);
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                v.xm_new[e + k] = xn[k];
                v.x_new[e + k] = (float)xn[k];
            }
            camera_record(xn, v.cam_pre_new + (size_t)c * CP_STRIDE, retract, v.cam_lo_new + (size_t)c * CLO_STRIDE);
            const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
            float* d = v.cam_dir + (size_t)c * CD_STRIDE;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                d[CD_PHI + i] = fmaf(JL[3 * i], hc[0], fmaf(JL[3 * i + 1], hc[1], JL[3 * i + 2] * hc[2]));
#pragma unroll
            for (int k = 0; k < 6; ++k) d[CD_T + k] = hc[3 + k];
        }
    }
    // points four at a time (a quad's twelve entries as 16-byte accesses; the padding
    // entries of the last quad are zero and stay zero)
    for (int qd = blockIdx.x * blockDim.x + threadIdx.x; qd < v.n_quads; qd += gridDim.x * blockDim.x) {
        const size_t e = v.pt_off + 12 * (size_t)qd;
        const float4* h4 = reinterpret_cast<const float4*>(v.h + e);
        const float4* g4 = reinterpret_cast<const float4*>(v.g + e);
        const double2* m2 = reinterpret_cast<const double2*>(v.xm + e);
        float H[12], G[12];
        double X[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 a = h4[k], b = g4[k];
            H[4 * k] = a.x; H[4 * k + 1] = a.y; H[4 * k + 2] = a.z; H[4 * k + 3] = a.w;
            G[4 * k] = b.x; G[4 * k + 1] = b.y; G[4 * k + 2] = b.z; G[4 * k + 3] = b.w;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 a = m2[k];
            X[2 * k] = a.x;
            X[2 * k + 1] = a.y;
        }
        float sgh = 0.0f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            X[k] += (double)H[k];
            sgh = fmaf(G[k], H[k], sgh);
        }
        double2* n2 = reinterpret_cast<double2*>(v.xm_new + e);
        float4* x4 = reinterpret_cast<float4*>(v.x_new + e);
#pragma unroll
        for (int k = 0; k < 6; ++k) n2[k] = make_double2(X[2 * k], X[2 * k + 1]);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            x4[k] = make_float4((float)X[4 * k], (float)X[4 * k + 1], (float)X[4 * k + 2], (float)X[4 * k + 3]);
        gh += (double)sgh;
    }
    double in[1] = {gh}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_CAND], out) && threadIdx.x == 0) st->gh = out[0];
}

// ------------------------------------------------------------------ K2 --------
// Candidate evaluation: F' = 1/2 |r(x')|^2 and |J(x) h|^2; the last block applies
// the LM rule of Sec. V (Madsen's quality-based damping): rho = (F - F') / L with
// L = -g^T h - 1/2 |J h|^2; accept iff rho > 0; mu <- mu max(1/3, 1 - (2 rho - 1)^3),
// nu <- 2 on acceptance, mu <- mu nu, nu <- 2 nu on rejection.  Never gated: its
// last block sets the LM loop flag.
template <int TB>
__global__ void __launch_bounds__(TB) k_eval_candidate(Views<float> v, CondHandle lm_cond, int use_cond) {
    DevState* st = v.st;
    const int active = st->lm_active;
    const float eps = (float)st->opt.eps;
    const int loss = st->opt.loss;
    double jh2 = 0.0;
    if (active) {
        for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
            const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
            const int pt0 = tile * TILE_PTS;
            const uint32_t n = hi - lo;
            const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
            const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
            uint32_t cur = NO_CAM;
            Cam co;
            float dir[9];
            float jc = 0.0f, jcc = 0.0f;   // Kahan pair
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    cur = c;
                    co = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                    load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
                }
                const size_t xi = v.pt_off + 3 * (size_t)(pt0 + slot);
                const Geo g = project_geo(co, v.x[xi], v.x[xi + 1], v.x[xi + 2], eps);
                float t0, t1;
                jdir(g, co, dir, v.h[xi], v.h[xi + 1], v.h[xi + 2], t0, t1);
                // |J h|^2 weighted at x (F' comes from k_residual)
                kahan_add(jc, jcc, (loss ? __ldg(v.obs_w + j) : 1.0f) * fmaf(t0, t0, t1 * t1));
            }
            jh2 += (double)jc - (double)jcc;
        }
    }
    double in[1] = {jh2}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_COST], out) && threadIdx.x == 0) {
        // pose factors: k_factor_eval ran just before
        const bool fac = v.n_fac > 0;
        lm_decide(st, active, st->F_res + (fac ? st->fac_cost_new : 0.0), out[0] + (fac ? st->fac_jh2 : 0.0));
        if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ K8 --------
// Commit an accepted step: x = x' (FP64 master and FP32 copies), camera records =
// those of x', and clear the
// camera linearisation sums for the relinearisation that follows.
__global__ void k_commit(Views<float> v) {
    if (v.st->accepted == 0) return;
    // flat, coalesced 16-byte copies: x <- x' over the whole parameter vector (cameras,
    // their zero padding, point quads), camera records <- the candidate's, and the
    // camera linearisation sums cleared for the next linearisation
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
    const float4* xs = reinterpret_cast<const float4*>(v.x_new);
    float4* xd = reinterpret_cast<float4*>(v.x);
    for (size_t i = tid; i < (size_t)v.n_vec / 4; i += nth) xd[i] = xs[i];
    const double2* ms = reinterpret_cast<const double2*>(v.xm_new);
    double2* md = reinterpret_cast<double2*>(v.xm);
    for (size_t i = tid; i < (size_t)v.n_vec / 2; i += nth) md[i] = ms[i];
    const float4* cs = reinterpret_cast<const float4*>(v.cam_pre_new);
    float4* cd = reinterpret_cast<float4*>(v.cam_pre);
    for (size_t i = tid; i < (size_t)v.n_cams * (CP_STRIDE / 4); i += nth) cd[i] = cs[i];
    const float4* ls = reinterpret_cast<const float4*>(v.cam_lo_new);
    float4* ld = reinterpret_cast<float4*>(v.cam_lo);
    for (size_t i = tid; i < (size_t)v.n_cams * (CLO_STRIDE / 4); i += nth) ld[i] = ls[i];
    for (size_t i = tid; i < (size_t)v.n_cams * CL_STRIDE; i += nth) v.cam_lin[i] = 0.0;
    float4* ch = reinterpret_cast<float4*>(v.cam_H);
    for (size_t i = tid; i < (size_t)v.n_cams * (CH_STRIDE / 4); i += nth) ch[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// ------------------------------------------------------------ Schur complement ---
// PCG on the camera Schur complement (the alternative Sec. V sets aside):
// S = H'cc - Hcp H'pp^-1 Hpc with H' = J^T W J + mu D (W the robust-loss weights, all
// ones for the squared loss).  A tile holds every observation of its points, so the
// point elimination is local to one tile CTA: pass 1 sums y_p = J_p^T W J_c d over the
// tile (shared memory), z_p = H'pp^-1 y_p per point, pass 2 sums the camera parts
// J_c^T W (J_c d - J_p z).  The camera PCG vectors use the camera segments of r z p h
// and k_update in its cameras-only form.

enum : int { SCHUR_RHS = 0, SCHUR_MV = 1, SCHUR_BACK = 2 };

// t = J_c d for a camera direction record d (no point part)
__device__ __forceinline__ void jc_apply(const GeoLite& g, const Cam& c, const float (&dir)[9], float& t0, float& t1) {
    const float dP0 = fmaf(dir[1], g.RX[2], -dir[2] * g.RX[1]) + dir[CD_T + 0];
    const float dP1 = fmaf(dir[2], g.RX[0], -dir[0] * g.RX[2]) + dir[CD_T + 1];
    const float dP2 = fmaf(dir[0], g.RX[1], -dir[1] * g.RX[0]) + dir[CD_T + 2];
    apply_A(g, dP0, dP1, dP2, t0, t1);
    const float fn2 = c.f * g.n2;
    const float ci = fmaf(g.s, dir[CD_I + 0], fmaf(fn2, dir[CD_I + 1], fn2 * g.n2 * dir[CD_I + 2]));
    t0 = fmaf(ci, g.p[0], t0);
    t1 = fmaf(ci, g.p[1], t1);
}

// t = J_p z = A R z
__device__ __forceinline__ void jp_apply(const GeoLite& g, const Cam& c, const float* z, float& t0, float& t1) {
    const float d0 = fmaf(c.R[0], z[0], fmaf(c.R[1], z[1], c.R[2] * z[2]));
    const float d1 = fmaf(c.R[3], z[0], fmaf(c.R[4], z[1], c.R[5] * z[2]));
    const float d2 = fmaf(c.R[6], z[0], fmaf(c.R[7], z[1], c.R[8] * z[2]));
    apply_A(g, d0, d1, d2, t0, t1);
}

// y += J_p^T t = R^T A^T t (shared-memory atomics)
__device__ __forceinline__ void jp_adjoint(const GeoLite& g, const Cam& c, float t0, float t1, float* y) {
    float u0, u1, u2;
    apply_At(g, t0, t1, u0, u1, u2);
    atomicAdd(y + 0, fmaf(c.R[0], u0, fmaf(c.R[3], u1, c.R[6] * u2)));
    atomicAdd(y + 1, fmaf(c.R[1], u0, fmaf(c.R[4], u1, c.R[7] * u2)));
    atomicAdd(y + 2, fmaf(c.R[2], u0, fmaf(c.R[5], u1, c.R[8] * u2)));
}

// acc += J_c^T t, its rotation part w.r.t. phi (k_update and k_schur_start apply J_l^T)
__device__ __forceinline__ void jc_adjoint(const GeoLite& g, const Cam& c, float t0, float t1, float (&acc)[9]) {
    float u0, u1, u2;
    apply_At(g, t0, t1, u0, u1, u2);
    acc[0] += fmaf(g.RX[1], u2, -g.RX[2] * u1);
    acc[1] += fmaf(g.RX[2], u0, -g.RX[0] * u2);
    acc[2] += fmaf(g.RX[0], u1, -g.RX[1] * u0);
    acc[3] += u0;
    acc[4] += u1;
    acc[5] += u2;
    const float pt = fmaf(g.p[0], t0, g.p[1] * t1);
    const float fn2 = c.f * g.n2;
    acc[6] = fmaf(g.s, pt, acc[6]);
    acc[7] = fmaf(fn2, pt, acc[7]);
    acc[8] = fmaf(fn2 * g.n2, pt, acc[8]);
}

// MODE SCHUR_RHS:  camera sums of J_c^T W J_p (H'pp^-1 g_p)      -> cam_acc
//      SCHUR_MV:   camera sums of J_c^T W (J_c p - J_p z)         -> cam_acc, and the
//                  slot sums sum w |J_c p|^2 - sum y^T z, p_c^T D_c p_c (alpha's denominator)
//      SCHUR_BACK: h_p = H'pp^-1 (-g_p - J_p^T W J_c h_c)
template <int TB, int MODE>
__global__ void __launch_bounds__(TB) k_schur(Views<float> v, const int32_t* gate) {
    if (gated_off(gate)) return;
    __shared__ float sx[3 * TILE_PTS], sy[3 * TILE_PTS];
    __shared__ double red[32];
    DevState* st = v.st;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;
    const int par = st->pcg_iter & 1;
    const float beta = MODE == SCHUR_MV ? (float)st->beta : 0.0f;
    const float* pc_old = v.pc + (size_t)par * v.pc_stride;
    float* pc_new = v.pc + (size_t)(par ^ 1) * v.pc_stride;
    const float* dsrc = MODE == SCHUR_MV ? v.z : v.h;   // camera direction source (with beta, pc_old)
    float tt = 0.0f, yz = 0.0f, pdp = 0.0f;
    if (MODE == SCHUR_MV)   // camera part of p owned by this CTA
        for (int c = blockIdx.x; c < v.n_cams; c += gridDim.x)
            if (threadIdx.x < 9) {
                const size_t e = 9 * (size_t)c + threadIdx.x;
                const float pk = beta != 0.0f ? fmaf(beta, pc_old[e], v.z[e]) : v.z[e];
                pc_new[e] = pk;
                pdp = fmaf(v.D[e] * pk, pk, pdp);
            }
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        for (int i = threadIdx.x; i < 3 * npt; i += TB) {
            sx[i] = v.x[base + i];
            sy[i] = 0.0f;
        }
        if (MODE == SCHUR_RHS)   // z_p = H'pp^-1 g_p
            for (int i = threadIdx.x; i < npt; i += TB) {
                const float* m = v.Minv_p + 6 * (size_t)(pt0 + i);
                const float g0 = v.g[base + 3 * i], g1 = v.g[base + 3 * i + 1], g2 = v.g[base + 3 * i + 2];
                sy[3 * i] = fmaf(m[0], g0, fmaf(m[1], g1, m[2] * g2));
                sy[3 * i + 1] = fmaf(m[1], g0, fmaf(m[3], g1, m[4] * g2));
                sy[3 * i + 2] = fmaf(m[2], g0, fmaf(m[4], g1, m[5] * g2));
            }
        __syncthreads();
        const uint32_t n = hi - lo;
        const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
        const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
        if (MODE != SCHUR_RHS) {
            // pass 1: y_p = sum J_p^T W J_c d
            uint32_t cur = NO_CAM;
            Cam cam;
            float dir[9];
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    cur = c;
                    cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                    camera_dir(v, c, dsrc, pc_old, beta, dir);
                }
                const GeoLite g = project_lite(cam, sx[3 * slot], sx[3 * slot + 1], sx[3 * slot + 2], eps);
                float t0, t1;
                jc_apply(g, cam, dir, t0, t1);
                const float w = weighted ? __ldg(v.obs_w + j) : 1.0f;
                tt = fmaf(w, fmaf(t0, t0, t1 * t1), tt);
                jp_adjoint(g, cam, w * t0, w * t1, sy + 3 * slot);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < npt; i += TB) {
                const float* m = v.Minv_p + 6 * (size_t)(pt0 + i);
                const float y0 = sy[3 * i], y1 = sy[3 * i + 1], y2 = sy[3 * i + 2];
                if (MODE == SCHUR_MV) {   // z_p = H'pp^-1 y_p
                    const float z0 = fmaf(m[0], y0, fmaf(m[1], y1, m[2] * y2));
                    const float z1 = fmaf(m[1], y0, fmaf(m[3], y1, m[4] * y2));
                    const float z2 = fmaf(m[2], y0, fmaf(m[4], y1, m[5] * y2));
                    yz = fmaf(y0, z0, fmaf(y1, z1, fmaf(y2, z2, yz)));
                    sy[3 * i] = z0;
                    sy[3 * i + 1] = z1;
                    sy[3 * i + 2] = z2;
                } else {                  // h_p = H'pp^-1 (-g_p - y_p)
                    const float b0 = -v.g[base + 3 * i] - y0, b1 = -v.g[base + 3 * i + 1] - y1;
                    const float b2 = -v.g[base + 3 * i + 2] - y2;
                    v.h[base + 3 * i] = fmaf(m[0], b0, fmaf(m[1], b1, m[2] * b2));
                    v.h[base + 3 * i + 1] = fmaf(m[1], b0, fmaf(m[3], b1, m[4] * b2));
                    v.h[base + 3 * i + 2] = fmaf(m[2], b0, fmaf(m[4], b1, m[5] * b2));
                }
            }
            __syncthreads();
        }
        if (MODE != SCHUR_BACK) {
            // pass 2: camera sums of J_c^T W s, s = J_c d - J_p z (operator) or J_p z (RHS)
            uint32_t cur = NO_CAM;
            float acc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
            Cam cam;
            float dir[9];
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                    cur = c;
                    cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                    if (MODE == SCHUR_MV) camera_dir(v, c, dsrc, pc_old, beta, dir);
                }
                const GeoLite g = project_lite(cam, sx[3 * slot], sx[3 * slot + 1], sx[3 * slot + 2], eps);
                float s0, s1;
                jp_apply(g, cam, sy + 3 * slot, s0, s1);
                if (MODE == SCHUR_MV) {
                    float t0, t1;
                    jc_apply(g, cam, dir, t0, t1);
                    s0 = t0 - s0;
                    s1 = t1 - s1;
                }
                const float w = weighted ? __ldg(v.obs_w + j) : 1.0f;
                jc_adjoint(g, cam, w * s0, w * s1, acc);
            }
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
        }
        __syncthreads();
    }
    if (MODE == SCHUR_MV) {
        const double bj = block_sum((double)tt - (double)yz, red);
        const double bp = block_sum((double)pdp, red);
        if (threadIdx.x == 0) {
            slot_add(st->acc_mv, 0, bj);
            slot_add(st->acc_mv, 1, bp);
        }
    }
}

// Start of the reduced PCG: r_c = -g_c + (camera sums of the right-hand-side pass),
// z = M_c^-1 r (the camera blocks of H'), p = h_c = 0; scalars as k_precond sets them.
__global__ void k_schur_start(Views<float> v, CondHandle pcg_cond, int use_cond) {
    DevState* st = v.st;
    if (st->lm_active == 0) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(pcg_cond, 0u);
        return;
    }
    double rz = 0.0, rr = 0.0;
    FOR_CAMERAS(c, v) {
        const size_t e = 9 * (size_t)c;
        float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
        const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
        const double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
        float q[9], rn[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) q[k] = fmaf(JL[k], ca[0], fmaf(JL[3 + k], ca[1], JL[6 + k] * ca[2]));
#pragma unroll
        for (int k = 3; k < 9; ++k) q[k] = ca[k];
#pragma unroll
        for (int k = 0; k < CA_STRIDE; ++k) ca[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            rn[k] = (float)(-cl[CL_G + k]) + q[k];
            v.r[e + k] = rn[k];
            v.p[e + k] = 0.0f;
            v.h[e + k] = 0.0f;
        }
        const float* M = v.Minv_c + (size_t)c * MC_STRIDE;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float z = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) z = fmaf(M[9 * i + k], rn[k], z);
            v.z[e + i] = z;
            rz += (double)rn[i] * (double)z;
            rr += (double)rn[i] * (double)rn[i];
        }
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_PRE], out) && threadIdx.x == 0) {
        st->rz = out[0];
        st->rr0 = out[1];
        st->rr = out[1];
        st->beta = 0.0;
        st->pcg_iter = 0;
        for (int k = 0; k < NSLOT * SLOT_STRIDE; ++k) st->acc_mv[k] = st->acc_up[k] = 0.0;
        // a non-finite r^T z means a non-finite gradient or block (a Jacobian that
        // overflowed, e.g. a point at a camera centre): a numeric failure, not a stall
        if (!isfinite(out[0]) || !isfinite(out[1])) st->status = 4;
        st->pcg_active = (out[1] > 0.0 && isfinite(out[0]) && st->opt.max_pcg > 0) ? 1 : 0;
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------- state / misc ---

__global__ void k_init_state(DevState* st) {
    st->mu = st->opt.mu0;
    st->nu = 2.0;
    st->lm_iter = 0;
    st->lm_active = 0;
    st->accepted = 0;
    st->relin = 0;
    st->n_accepted = 0;
    st->status = 0;
    st->pcg_iter = 0;
    st->pcg_active = 0;
    st->pcg_total = 0;
    st->t_start = global_ns();
    st->t_end = st->t_start;
}

__global__ void k_finish_state(DevState* st) { st->t_end = global_ns(); }

// Parameters between the caller layout (cams [n][9], pts [n][3], float or double)
// and the internal vector layout: set writes the FP64 master copy and its FP32
// rounding, get reads the master copy.
template <typename S>
__global__ void k_pack(Views<float> v, const S* cams, const S* pts) {
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            for (int k = 0; k < 9; ++k) {
                const double a = (double)cams[9 * (size_t)it + k];
                v.xm[9 * (size_t)it + k] = a;
                v.x[9 * (size_t)it + k] = (float)a;
            }
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) {
                const double a = (double)pts[3 * (size_t)u + k];
                v.xm[e + k] = a;
                v.x[e + k] = (float)a;
            }
        }
    }
}

template <typename S>
__global__ void k_unpack(Views<float> v, const double* src, S* cams, S* pts) {
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            for (int k = 0; k < 9; ++k) cams[9 * (size_t)it + k] = (S)src[9 * (size_t)it + k];
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) pts[3 * (size_t)u + k] = (S)src[e + k];
        }
    }
}

// out (caller layout) of the damped normal operator: cameras finish J_l^T and mu D p
// from the K4 accumulators, points copy q.
template <typename S>
__global__ void k_normal_out(Views<float> v, S* out) {
    const float mu = (float)v.st->mu;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const size_t e = 9 * (size_t)it;
            float* ca = v.cam_acc + (size_t)it * CA_STRIDE;
            const float* JL = v.cam_pre + (size_t)it * CP_STRIDE + CP_JL;
            for (int k = 0; k < 9; ++k) {
                float q = k < 3 ? fmaf(JL[k], ca[0], fmaf(JL[3 + k], ca[1], JL[6 + k] * ca[2])) : ca[k];
                out[e + k] = (S)fmaf(mu, v.D[e + k] * v.p[e + k], q);
            }
            for (int k = 0; k < CA_STRIDE; ++k) ca[k] = 0.0f;
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) out[9 * (size_t)v.n_cams + 3 * (size_t)u + k] = (S)v.q[e + k];
        }
    }
}

// p (internal layout) from a caller-layout vector.
template <typename S>
__global__ void k_set_direction(Views<float> v, const S* src) {
    FOR_CAMERAS(c, v) {
        for (int k = 0; k < 9; ++k) v.p[9 * (size_t)c + k] = (float)src[9 * (size_t)c + k];
    }
    FOR_POINTS(u, v) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) v.p[e + k] = (float)src[9 * (size_t)v.n_cams + 3 * (size_t)u + k];
    }
}

// ------------------------------------------------------------------ launchers --

namespace {
inline int grid_items(const LaunchCfg& L, int items) {
    int g = (items + L.item_block - 1) / L.item_block;
    return g < 1 ? 1 : (g > L.item_grid ? L.item_grid : g);
}
inline int grid_tiles(int cap, int n_tiles) { return n_tiles < 1 ? 1 : (n_tiles > cap ? cap : n_tiles); }
// Blocks for a camera-only kernel: one warp of 32 cameras per block (FOR_CAMERAS).
inline int grid_cams(const LaunchCfg& L, int n_cams) {
    const int g = (n_cams + 31) / 32;
    return g < 1 ? 1 : (g > L.item_grid ? L.item_grid : g);
}
}  // namespace

void launch_camera_precompute(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_camera_precompute<<<grid_cams(L, v.n_cams), 32, 0, s>>>(v);
}
void launch_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode,
                      float* res_out, float* jac_out, CondHandle lm_cond, int use_cond) {
    launch_factor_linearize(v, L, s, mode);   // its cost is added by the linearisation
    if (L.tl_grid > 0)   // tiles with their camera tables in shared memory
        launch_tile_linearize(v, L, s, mode, res_out, jac_out, lm_cond, use_cond);
    else
        k_linearize<LIN_TB><<<grid_tiles(L.lin_grid, v.n_tiles), LIN_TB, 0, s>>>(v, mode, res_out, jac_out,
                                                                                 lm_cond, use_cond);
}
void launch_precond(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use,
                    double* pslots) {
    // camera blocks: a warp per camera; point blocks: a thread per point
    const int wpb = L.item_block / 32;
    const int cam_blocks = std::max(1, std::min((v.n_cams + wpb - 1) / wpb, L.item_grid / 2));
    const int pt_blocks = std::max(1, std::min(grid_items(L, v.n_pts), L.item_grid - cam_blocks));
    k_precond<<<cam_blocks + pt_blocks, L.item_block, 0, s>>>(v, c, use, pslots, cam_blocks);
}
void launch_matvec(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                   const float* zs, int use_beta) {
    // one thread per camera entry, no more blocks than that needs (each adds one slot sum)
    const int cd_grid = std::max(1, std::min(L.item_grid, (9 * v.n_cams + L.item_block - 1) / L.item_block));
    k_cam_direction<<<cd_grid, L.item_block, 0, s>>>(v, gate, zs, use_beta);
    if (L.tn_grid > 0)   // tiles with their camera tables in shared memory
        launch_tile_normal(v, L, s, gate, zs, use_beta);
    else
        k_matvec<MV_TB><<<v.n_tiles > 0 ? v.n_tiles : 1, MV_TB, 0, s>>>(v, gate, zs, use_beta);
    launch_factor_matvec(v, L, s, gate, zs, use_beta);   // pose factors, if any
}
void launch_schur(const Views<float>& v, cudaStream_t s, int mode, const int32_t* gate) {
    const int grid = v.n_tiles > 0 ? v.n_tiles : 1;
    if (mode == SCHUR_RHS) k_schur<MV_TB, SCHUR_RHS><<<grid, MV_TB, 0, s>>>(v, gate);
    else if (mode == SCHUR_MV) k_schur<MV_TB, SCHUR_MV><<<grid, MV_TB, 0, s>>>(v, gate);
    else k_schur<MV_TB, SCHUR_BACK><<<grid, MV_TB, 0, s>>>(v, gate);
}
void launch_schur_start(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k_schur_start<<<grid_cams(L, v.n_cams), L.item_block, 0, s>>>(v, c, use);
}
void launch_update(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use,
                   int cameras_only) {
    k_update<<<cameras_only ? std::max(grid_cams(L, v.n_cams), 1) : std::max(grid_items(L, v.n_quads), grid_cams(L, v.n_cams)),
               L.item_block, 0, s>>>(v, c, use, cameras_only);
}
void launch_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_candidate<<<std::max(grid_items(L, v.n_quads), grid_cams(L, v.n_cams)), L.item_block, 0, s>>>(v);
}
void launch_eval_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    launch_factor_eval(v, L, s);
    if (L.te_grid > 0)   // tiles with their camera tables in shared memory
        launch_tile_eval(v, L, s, c, use);
    else
        k_eval_candidate<EV_TB><<<grid_tiles(L.ev_grid, v.n_tiles), EV_TB, 0, s>>>(v, c, use);
}
void launch_commit(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_commit<<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v);
}
void launch_init_state(DevState* st, cudaStream_t s) { k_init_state<<<1, 1, 0, s>>>(st); }
void launch_finish_state(DevState* st, cudaStream_t s) { k_finish_state<<<1, 1, 0, s>>>(st); }

void launch_pack(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const void* cams,
                 const void* pts, int dtype) {
    const int g = grid_items(L, v.n_cams + v.n_pts);
    if (dtype == 1) k_pack<double><<<g, L.item_block, 0, s>>>(v, (const double*)cams, (const double*)pts);
    else k_pack<float><<<g, L.item_block, 0, s>>>(v, (const float*)cams, (const float*)pts);
}
void launch_unpack(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const double* src, void* cams,
                   void* pts, int dtype) {
    const int g = grid_items(L, v.n_cams + v.n_pts);
    if (dtype == 1) k_unpack<double><<<g, L.item_block, 0, s>>>(v, src, (double*)cams, (double*)pts);
    else k_unpack<float><<<g, L.item_block, 0, s>>>(v, src, (float*)cams, (float*)pts);
}
void launch_set_direction(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const float* src) {
    k_set_direction<float><<<std::max(grid_items(L, v.n_pts), grid_cams(L, v.n_cams)), L.item_block, 0, s>>>(v, src);
}
void launch_normal_out(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, float* out) {
    k_normal_out<float><<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v, out);
}

int occupancy_blocks_linearize() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_linearize<LIN_TB>, LIN_TB, 0);
    return n;
}
int occupancy_blocks_matvec() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_matvec<MV_TB>, MV_TB, 0);
    return n;
}
int occupancy_blocks_eval() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_eval_candidate<EV_TB>, EV_TB, 0);
    return n;
}

}  // namespace gbba

// ------------------------------------------------------------- autograd ------
namespace gbba {

// Parameters in caller layout -> internal layout at `dst` (x' is used as scratch so
// the problem's own parameters stay untouched).
template <typename S>
__global__ void k_pack_to(Views<float> v, const S* cams, const S* pts, float* dst) {
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            for (int k = 0; k < 9; ++k) dst[9 * (size_t)it + k] = (float)cams[9 * (size_t)it + k];
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) dst[e + k] = (float)pts[3 * (size_t)u + k];
        }
    }
}

__global__ void k_camera_records_from(Views<float> v, const float* src, float* dst) {
    FOR_CAMERAS(c, v) {
        double p[9];
        for (int k = 0; k < 9; ++k) p[k] = (double)src[9 * (size_t)c + k];
        camera_record(p, dst + (size_t)c * CP_STRIDE);
        for (int k = 0; k < CL_STRIDE; ++k) v.cam_lin[(size_t)c * CL_STRIDE + k] = 0.0;
    }
}

// Cost F = 1/2 |r|^2 at (xs, camera records crec) and, if want_grad, its adjoint
// J^T r: camera part into cam_lin (FP64 atomics once per camera run), point part into
// g (internal layout).  Camera pass over the tile's camera-sorted observations, point
// pass per point over its observations (which also sums the cost).
template <int TB>
__global__ void __launch_bounds__(TB) k_cost_grad(Views<float> v, const float* __restrict__ xs,
                                                  const float* __restrict__ crec, int want_grad, double* cost_dev) {
    __shared__ float4 sx[TILE_PTS];
    const float eps = (float)v.st->opt.eps;
    float cost = 0.0f;
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        __syncthreads();
        for (int i = threadIdx.x; i < npt; i += TB)
            sx[i] = make_float4(xs[base + 3 * i], xs[base + 3 * i + 1], xs[base + 3 * i + 2], 0.0f);
        __syncthreads();
        if (want_grad) {
            const uint32_t n = hi - lo;
            const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
            const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
            uint32_t cur = NO_CAM;
            float acc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
            Cam cam;
            float JL[9];
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    if (cur != NO_CAM) {
#pragma unroll
                        for (int k = 0; k < 9; ++k) {
                            atomicAdd(v.cam_lin + (size_t)cur * CL_STRIDE + k, (double)acc[k]);
                            acc[k] = 0.0f;
                        }
                    }
                    cur = c;
                    cam = load_cam(crec + (size_t)c * CP_STRIDE);
#pragma unroll
                    for (int k = 0; k < 9; ++k) JL[k] = __ldg(crec + (size_t)c * CP_STRIDE + CP_JL + k);
                }
                const float4 X = sx[slot];
                const Geo g = project_geo(cam, X.x, X.y, X.z, eps);
                const float fs = cam.f * g.s;
                const float r0 = fmaf(fs, g.p[0], -__ldg(v.obs_uv + 2 * (size_t)j));
                const float r1 = fmaf(fs, g.p[1], -__ldg(v.obs_uv + 2 * (size_t)j + 1));
                // J_c^T r: rotation part J_l^T (RX x u) with u = A^T r, then u, then intrinsics
                const float u0 = fmaf(g.A[0], r0, g.A[3] * r1);
                const float u1 = fmaf(g.A[1], r0, g.A[4] * r1);
                const float u2 = fmaf(g.A[2], r0, g.A[5] * r1);
                const float w0 = fmaf(g.RX[1], u2, -g.RX[2] * u1);
                const float w1 = fmaf(g.RX[2], u0, -g.RX[0] * u2);
                const float w2 = fmaf(g.RX[0], u1, -g.RX[1] * u0);
#pragma unroll
                for (int k = 0; k < 3; ++k) acc[k] = fmaf(JL[k], w0, fmaf(JL[3 + k], w1, fmaf(JL[6 + k], w2, acc[k])));
                acc[3] += u0;
                acc[4] += u1;
                acc[5] += u2;
                const float pr = fmaf(g.p[0], r0, g.p[1] * r1);
                const float fn2 = cam.f * g.n2;
                acc[6] = fmaf(g.s, pr, acc[6]);
                acc[7] = fmaf(fn2, pr, acc[7]);
                acc[8] = fmaf(fn2 * g.n2, pr, acc[8]);
            }
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM) {
#pragma unroll
                for (int k = 0; k < 9; ++k) atomicAdd(v.cam_lin + (size_t)cur * CL_STRIDE + k, (double)acc[k]);
            }
        }
        for (int i = threadIdx.x; i < npt; i += TB) {
            const int ip = pt0 + i;
            const float4 X = sx[i];
            float gp0 = 0.0f, gp1 = 0.0f, gp2 = 0.0f;
            const uint32_t k0 = __ldg(v.pt_obs_off + ip), k1 = __ldg(v.pt_obs_off + ip + 1);
            for (uint32_t k = k0; k < k1; ++k) {
                const uint32_t j = __ldg(v.obs_pm + k);
                const uint32_t c = __ldg(v.obs_key + j) >> 8;
                const Cam cam = load_cam(crec + (size_t)c * CP_STRIDE);
                const Geo g = project_geo(cam, X.x, X.y, X.z, eps);
                const float fs = cam.f * g.s;
                const float r0 = fmaf(fs, g.p[0], -__ldg(v.obs_uv + 2 * (size_t)j));
                const float r1 = fmaf(fs, g.p[1], -__ldg(v.obs_uv + 2 * (size_t)j + 1));
                cost = fmaf(r0, r0, fmaf(r1, r1, cost));
                if (want_grad) {   // J_X^T r = R^T A^T r
                    const float u0 = fmaf(g.A[0], r0, g.A[3] * r1);
                    const float u1 = fmaf(g.A[1], r0, g.A[4] * r1);
                    const float u2 = fmaf(g.A[2], r0, g.A[5] * r1);
                    gp0 += fmaf(cam.R[0], u0, fmaf(cam.R[3], u1, cam.R[6] * u2));
                    gp1 += fmaf(cam.R[1], u0, fmaf(cam.R[4], u1, cam.R[7] * u2));
                    gp2 += fmaf(cam.R[2], u0, fmaf(cam.R[5], u1, cam.R[8] * u2));
                }
            }
            if (want_grad) {
                v.g[base + 3 * i] = gp0;
                v.g[base + 3 * i + 1] = gp1;
                v.g[base + 3 * i + 2] = gp2;
            }
        }
    }
    double in[1] = {(double)cost}, out[1];
    if (grid_reduce<1>(in, v.partials, &v.st->tickets[TK_MISC], out) && threadIdx.x == 0) {
        v.st->cost_out = 0.5 * out[0];
        if (cost_dev) *cost_dev = 0.5 * out[0];
    }
}

// grad_cams = grad_out * g_c, grad_pts = grad_out * g_p, caller layout.
template <typename S>
__global__ void k_grad_out(Views<float> v, const double* __restrict__ grad_out, S* gc, S* gp) {
    const double s = *grad_out;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n_cams; c += gridDim.x * blockDim.x)
        for (int k = 0; k < 9; ++k) gc[9 * (size_t)c + k] = (S)(s * v.cam_lin[(size_t)c * CL_STRIDE + k]);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < v.n_pts; u += gridDim.x * blockDim.x) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) gp[3 * (size_t)u + k] = (S)(s * (double)v.g[e + k]);
    }
}

void launch_cost_grad(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts,
                      int dtype, int want_grad, double* cost_dev) {
    const int gi = std::max(1, std::min((v.n_cams + v.n_pts + 255) / 256, L.item_grid));
    if (dtype == 1) k_pack_to<double><<<gi, 256, 0, s>>>(v, (const double*)cams, (const double*)pts, v.x_new);
    else k_pack_to<float><<<gi, 256, 0, s>>>(v, (const float*)cams, (const float*)pts, v.x_new);
    k_camera_records_from<<<grid_cams(L, v.n_cams), 32, 0, s>>>(v, v.x_new, v.cam_pre_new);
    const int gt = std::max(1, std::min(v.n_tiles, L.lin_grid));
    k_cost_grad<LIN_TB><<<gt, LIN_TB, 0, s>>>(v, v.x_new, v.cam_pre_new, want_grad, cost_dev);
}

void launch_grad_out(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const double* grad_out, void* gc,
                     void* gp, int dtype) {
    const int g = std::max(1, std::min((std::max(v.n_cams, v.n_pts) + 255) / 256, L.item_grid));
    if (dtype == 1) k_grad_out<double><<<g, 256, 0, s>>>(v, grad_out, (double*)gc, (double*)gp);
    else k_grad_out<float><<<g, 256, 0, s>>>(v, grad_out, (float*)gc, (float*)gp);
}

}  // namespace gbba
