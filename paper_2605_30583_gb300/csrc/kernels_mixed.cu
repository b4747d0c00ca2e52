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

#include "device_common.cuh"
#include "kernels.h"

namespace gbba {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t NO_CAM = 0xffffffffu;

// Warp-segmented suffix sum: lanes with equal `key` in consecutive positions form a
// segment; afterwards the first lane of each segment holds the segment's sum.
template <int V>
__device__ __forceinline__ bool seg_reduce(uint32_t key, float (&acc)[V]) {
    const int lane = threadIdx.x & 31;
    const uint32_t prev = __shfl_up_sync(FULL, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const uint32_t hm = __ballot_sync(FULL, head);
    const uint32_t after = hm & ~((2u << lane) - 1u);
    const int end = after ? (__ffs(after) - 1) : 32;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const float o = __shfl_down_sync(FULL, acc[k], d);
            if (lane + d < end) acc[k] += o;
        }
    }
    return head;
}

__device__ __forceinline__ void flush_matvec(float* __restrict__ dst, float (&a)[9]) {
    atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a[0], a[1], a[2], a[3]));
    atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(a[4], a[5], a[6], a[7]));
    atomicAdd(dst + 8, a[8]);
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = 0.0f;
}

__device__ __forceinline__ void load_dir(const float* __restrict__ rec, float (&d)[9]) {
    const float4* r4 = reinterpret_cast<const float4*>(rec);
    const float4 a = __ldg(r4), b = __ldg(r4 + 1), c = __ldg(r4 + 2);
    d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
    d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w; d[8] = c.x;
}

// t = J d for one observation: J d = A (phi x RX + d_t + R d_X) + c_i p with
// phi = J_l d_w (precomputed per camera) and c_i = s d_f + f n2 d_k1 + f n2^2 d_k2.
__device__ __forceinline__ void jdir(const Geo& g, const Cam& c, const float (&dir)[9],
                                     float dX0, float dX1, float dX2, float& t0, float& t1) {
    const float* phi = dir + CD_PHI;
    float dP0 = fmaf(phi[1], g.RX[2], -phi[2] * g.RX[1]) + dir[CD_T + 0];
    float dP1 = fmaf(phi[2], g.RX[0], -phi[0] * g.RX[2]) + dir[CD_T + 1];
    float dP2 = fmaf(phi[0], g.RX[1], -phi[1] * g.RX[0]) + dir[CD_T + 2];
    dP0 = fmaf(c.R[0], dX0, fmaf(c.R[1], dX1, fmaf(c.R[2], dX2, dP0)));
    dP1 = fmaf(c.R[3], dX0, fmaf(c.R[4], dX1, fmaf(c.R[5], dX2, dP1)));
    dP2 = fmaf(c.R[6], dX0, fmaf(c.R[7], dX1, fmaf(c.R[8], dX2, dP2)));
    const float fn2 = c.f * g.n2;
    const float ci = fmaf(g.s, dir[CD_I + 0], fmaf(fn2, dir[CD_I + 1], fn2 * g.n2 * dir[CD_I + 2]));
    t0 = fmaf(g.A[0], dP0, fmaf(g.A[1], dP1, fmaf(g.A[2], dP2, ci * g.p[0])));
    t1 = fmaf(g.A[3], dP0, fmaf(g.A[4], dP1, fmaf(g.A[5], dP2, ci * g.p[1])));
}

__device__ __forceinline__ bool gated_off(const int32_t* gate) { return gate != nullptr && *gate == 0; }

}  // namespace

// ------------------------------------------------------------------ K0 --------
// Camera records from the current parameters; zeroes the linearisation sums.
__global__ void k_camera_precompute(Views<float> v) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.n_cams; c += gridDim.x * blockDim.x) {
        double p[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k] = (double)v.x[9 * (size_t)c + k];
        camera_record(p, v.cam_pre + (size_t)c * CP_STRIDE);
        double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
#pragma unroll 8
        for (int k = 0; k < CL_STRIDE; ++k) cl[k] = 0.0;
    }
}

// ------------------------------------------------------------------ K1 --------
// Linearisation (fused score + Jacobian products, Sec. V-A): cost F = 1/2 |r|^2,
// g = J^T r and the diagonal blocks J_c^T J_c, J_p^T J_p.  `mode`: 0 = first
// linearisation of a solve (initialises the LM state), 1 = relinearisation after an
// accepted step (gated by st->relin), 2 = evaluation only (optional r and J output in
// the caller's observation order).
template <int TB>
__global__ void __launch_bounds__(TB) k_linearize(Views<float> v, int mode, float* res_out,
                                                  float* jac_out, CondHandle lm_cond, int use_cond) {
    if (mode == 1 && v.st->relin == 0) return;
    __shared__ float sp[TILE_PTS * 9];   // per point: g (3), H upper triangle (6)
    const float eps = (float)v.st->opt.eps;
    double cost = 0.0;
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        for (int i = threadIdx.x; i < TILE_PTS * 9; i += TB) sp[i] = 0.0f;
        __syncthreads();
        const uint32_t n = hi - lo;
        const uint32_t chunk = (n + TB - 1) / TB;
        const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
        uint32_t cur = NO_CAM;
        float acc[54];
#pragma unroll
        for (int k = 0; k < 54; ++k) acc[k] = 0.0f;
        Cam cam;
        float JL[9];
        float costc = 0.0f;
        for (uint32_t j = a; j < b; ++j) {
            const uint32_t key = v.obs_key[j];
            const uint32_t c = key >> 8, slot = key & 0xffu;
            if (c != cur) {
                if (cur != NO_CAM) {
                    double* dst = v.cam_lin + (size_t)cur * CL_STRIDE;
#pragma unroll
                    for (int k = 0; k < 54; ++k) {
                        atomicAdd(dst + k, (double)acc[k]);
                        acc[k] = 0.0f;
                    }
                }
                cur = c;
                cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
#pragma unroll
                for (int k = 0; k < 9; ++k) JL[k] = __ldg(v.cam_pre + (size_t)c * CP_STRIDE + CP_JL + k);
            }
            const size_t xi = v.pt_off + 3 * (size_t)(pt0 + slot);
            const float X0 = v.x[xi], X1 = v.x[xi + 1], X2 = v.x[xi + 2];
            const Geo g = project_geo(cam, X0, X1, X2, eps);
            const float fs = cam.f * g.s;
            const float r0 = fmaf(fs, g.p[0], -v.obs_uv[2 * (size_t)j]);
            const float r1 = fmaf(fs, g.p[1], -v.obs_uv[2 * (size_t)j + 1]);
            costc = fmaf(r0, r0, fmaf(r1, r1, costc));
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
            // point Jacobian J_X = A R
            float jx0[3], jx1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                jx0[k] = fmaf(g.A[0], cam.R[k], fmaf(g.A[1], cam.R[3 + k], g.A[2] * cam.R[6 + k]));
                jx1[k] = fmaf(g.A[3], cam.R[k], fmaf(g.A[4], cam.R[3 + k], g.A[5] * cam.R[6 + k]));
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) acc[CL_G + i] = fmaf(j0[i], r0, fmaf(j1[i], r1, acc[CL_G + i]));
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int k = i; k < 9; ++k) {
                    const int t = CL_H + tri_index(9, i, k);
                    acc[t] = fmaf(j0[i], j0[k], fmaf(j1[i], j1[k], acc[t]));
                }
            float* ps = sp + 9 * slot;
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(ps + i, fmaf(jx0[i], r0, jx1[i] * r1));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = i; k < 3; ++k)
                    atomicAdd(ps + 3 + tri_index(3, i, k), fmaf(jx0[i], jx0[k], jx1[i] * jx1[k]));
            if (mode == 2) {
                const uint32_t o = v.obs_user[j];
                if (res_out) { res_out[2 * (size_t)o] = r0; res_out[2 * (size_t)o + 1] = r1; }
                if (jac_out) {
                    float* J = jac_out + 24 * (size_t)o;
#pragma unroll
                    for (int k = 0; k < 9; ++k) { J[k] = j0[k]; J[12 + k] = j1[k]; }
#pragma unroll
                    for (int k = 0; k < 3; ++k) { J[9 + k] = jx0[k]; J[21 + k] = jx1[k]; }
                }
            }
        }
        // camera sums: combine lanes of the same camera, one set of atomics per run
        const bool head = seg_reduce<54>(cur, acc);
        if (head && cur != NO_CAM) {
            double* dst = v.cam_lin + (size_t)cur * CL_STRIDE;
#pragma unroll
            for (int k = 0; k < 54; ++k) atomicAdd(dst + k, (double)acc[k]);
        }
        cost += (double)costc;
        __syncthreads();
        for (int i = threadIdx.x; i < npt * 3; i += TB) {
            const int s = i / 3, k = i % 3;
            v.g[v.pt_off + 3 * (size_t)pt0 + i] = sp[9 * s + k];
        }
        for (int i = threadIdx.x; i < npt * PH_STRIDE; i += TB) {
            const int s = i / PH_STRIDE, k = i % PH_STRIDE;
            v.pt_H[(size_t)(pt0 + s) * PH_STRIDE + k] = sp[9 * s + 3 + k];
        }
        __syncthreads();
    }
    double in[1] = {cost}, out[1];
    if (grid_reduce<1>(in, v.partials, &v.st->tickets[TK_LIN], out) && threadIdx.x == 0) {
        DevState* st = v.st;
        const double F = 0.5 * out[0];
        st->cost_out = F;
        if (mode == 0) {
            st->F = F;
            st->F0 = F;
            const bool ok = isfinite(F);
            if (!ok) st->status = 4;
            st->lm_active = (ok && F > 0.0 && st->opt.max_lm > 0) ? 1 : 0;
            if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
        } else if (mode == 1) {
            st->F = F;
        }
    }
}

// ------------------------------------------------------------------ K3 --------
// Block-Jacobi preconditioner (Sec. V: one block per node) of J^T J + mu D, inverted
// by FP64 Cholesky, and the start of PCGNR: h = 0, r = -g, z = M^-1 r, p = 0.
__device__ void chol_inverse(double* A, int n, double* Minv, bool& ok) {
    // A: n x n full, row-major, overwritten by L.  Minv = L^-T L^-1.
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) { ok = false; return; }
        const double d = sqrt(s);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / d;
        }
    }
    // L^-1 (lower) into Minv's storage first, column by column
    double Li[81];
    for (int i = 0; i < n * n; ++i) Li[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        Li[j * n + j] = 1.0 / A[j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double t = 0.0;
            for (int k = j; k < i; ++k) t -= A[i * n + k] * Li[k * n + j];
            Li[i * n + j] = t / A[i * n + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double t = 0.0;
            for (int k = (i > j ? i : j); k < n; ++k) t += Li[k * n + i] * Li[k * n + j];
            Minv[i * n + j] = t;
        }
}

__global__ void k_precond(Views<float> v, CondHandle pcg_cond, int use_cond) {
    DevState* st = v.st;
    if (st->lm_active == 0) {
        // the PCG loop that follows must see a cleared flag
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(pcg_cond, 0u);
        return;
    }
    const double mu = st->mu, lo = st->opt.min_diag, hi = st->opt.max_diag;
    double rz = 0.0, rr = 0.0;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const int c = it;
            const double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
            double A[81], M[81];
            double Dd[9];
            for (int i = 0; i < 9; ++i)
                for (int j = i; j < 9; ++j) {
                    const double h = cl[CL_H + tri_index(9, i, j)];
                    A[i * 9 + j] = h;
                    A[j * 9 + i] = h;
                }
            for (int i = 0; i < 9; ++i) {
                Dd[i] = fmin(fmax(A[i * 9 + i], lo), hi);
                A[i * 9 + i] += mu * Dd[i];
            }
            double diag[9];
            for (int i = 0; i < 9; ++i) diag[i] = A[i * 9 + i];
            bool ok = true;
            chol_inverse(A, 9, M, ok);
            if (!ok) {   // not SPD in FP64: fall back to the inverse diagonal
                for (int i = 0; i < 81; ++i) M[i] = 0.0;
                for (int i = 0; i < 9; ++i) M[i * 9 + i] = diag[i] > 0.0 ? 1.0 / diag[i] : 0.0;
            }
            float* Mo = v.Minv_c + (size_t)c * MC_STRIDE;
            for (int i = 0; i < 81; ++i) Mo[i] = (float)M[i];
            float rf[9];
            for (int i = 0; i < 9; ++i) {
                v.D[9 * (size_t)c + i] = (float)Dd[i];
                rf[i] = (float)(-cl[CL_G + i]);
            }
            for (int i = 0; i < 9; ++i) {
                float z = 0.0f;
                for (int k = 0; k < 9; ++k) z = fmaf(Mo[i * 9 + k], rf[k], z);
                const size_t e = 9 * (size_t)c + i;
                v.r[e] = rf[i];
                v.z[e] = z;
                v.p[e] = 0.0f;
                v.h[e] = 0.0f;
                rz += (double)rf[i] * (double)z;
                rr += (double)rf[i] * (double)rf[i];
            }
            float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
            for (int k = 0; k < CA_STRIDE; ++k) ca[k] = 0.0f;
        } else {
            const int i = it - v.n_cams;
            const float* H = v.pt_H + (size_t)i * PH_STRIDE;
            const size_t e = v.pt_off + 3 * (size_t)i;
            double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
            const double d0 = fmin(fmax(a00, lo), hi), d1 = fmin(fmax(a11, lo), hi), d2 = fmin(fmax(a22, lo), hi);
            a00 += mu * d0; a11 += mu * d1; a22 += mu * d2;
            // Cholesky of the 3x3 block and its inverse M = L^-T L^-1
            double m[6];
            const double l00s = a00;
            bool ok = l00s > 0.0;
            double l00 = 0, l10 = 0, l20 = 0, l11 = 0, l21 = 0, l22 = 0;
            if (ok) {
                l00 = sqrt(l00s);
                l10 = a01 / l00;
                l20 = a02 / l00;
                const double s11 = a11 - l10 * l10;
                ok = s11 > 0.0;
                if (ok) {
                    l11 = sqrt(s11);
                    l21 = (a12 - l20 * l10) / l11;
                    const double s22 = a22 - l20 * l20 - l21 * l21;
                    ok = s22 > 0.0;
                    if (ok) l22 = sqrt(s22);
                }
            }
            if (ok) {
                const double i00 = 1.0 / l00, i11 = 1.0 / l11, i22 = 1.0 / l22;
                const double i10 = -l10 * i00 * i11;
                const double i21 = -l21 * i11 * i22;
                const double i20 = -(l20 * i00 + l21 * i10) * i22;
                m[0] = i00 * i00 + i10 * i10 + i20 * i20;
                m[1] = i10 * i11 + i20 * i21;
                m[2] = i20 * i22;
                m[3] = i11 * i11 + i21 * i21;
                m[4] = i21 * i22;
                m[5] = i22 * i22;
            } else {
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
            v.h[e] = 0.0f; v.h[e + 1] = 0.0f; v.h[e + 2] = 0.0f;
            rz += (double)(r0 * z0 + r1 * z1 + r2 * z2);
            rr += (double)(r0 * r0 + r1 * r1 + r2 * r2);
        }
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_PRE], out) && threadIdx.x == 0) {
        st->rz = out[0];
        st->rr0 = out[1];
        st->rr = out[1];
        st->beta = 0.0;
        st->pcg_iter = 0;
        st->pcg_active = (out[1] > 0.0 && isfinite(out[0]) && st->opt.max_pcg > 0) ? 1 : 0;
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ K6 --------
// PCG direction p = z + beta p; camera direction records phi = J_l p_w; p^T D p.
__global__ void k_direction(Views<float> v) {
    DevState* st = v.st;
    if (st->pcg_active == 0) return;
    const float beta = (float)st->beta;
    double pdp = 0.0;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const size_t e = 9 * (size_t)it;
            float pc[9];
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                pc[k] = fmaf(beta, v.p[e + k], v.z[e + k]);
                v.p[e + k] = pc[k];
                s = fmaf(v.D[e + k] * pc[k], pc[k], s);
            }
            pdp += (double)s;
            const float* JL = v.cam_pre + (size_t)it * CP_STRIDE + CP_JL;
            float* d = v.cam_dir + (size_t)it * CD_STRIDE;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                d[CD_PHI + i] = fmaf(JL[3 * i], pc[0], fmaf(JL[3 * i + 1], pc[1], JL[3 * i + 2] * pc[2]));
#pragma unroll
            for (int k = 0; k < 6; ++k) d[CD_T + k] = pc[3 + k];
        } else {
            const size_t e = v.pt_off + 3 * (size_t)(it - v.n_cams);
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float pk = fmaf(beta, v.p[e + k], v.z[e + k]);
                v.p[e + k] = pk;
                s = fmaf(v.D[e + k] * pk, pk, s);
            }
            pdp += (double)s;
        }
    }
    double in[1] = {pdp}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_DIR], out) && threadIdx.x == 0) st->pDp = out[0];
}

// ------------------------------------------------------------------ K4 --------
// Damped normal operator q = J^T J p + mu D p (points; cameras finish in K5) and
// |J p|^2.  The last block forms alpha = r^T z / (|J p|^2 + mu p^T D p).
// gate: pointer to the flag that enables the kernel (null = always run).
template <int TB>
__global__ void __launch_bounds__(TB) k_matvec(Views<float> v, const int32_t* gate) {
    if (gated_off(gate)) return;
    __shared__ float qp[TILE_PTS * 3];
    DevState* st = v.st;
    const float mu = (float)st->mu;
    const float eps = (float)st->opt.eps;
    double jp2 = 0.0;
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
        const int pt0 = tile * TILE_PTS;
        const int npt = min(TILE_PTS, v.n_pts - pt0);
        for (int i = threadIdx.x; i < TILE_PTS * 3; i += TB) qp[i] = 0.0f;
        __syncthreads();
        const uint32_t n = hi - lo;
        const uint32_t chunk = (n + TB - 1) / TB;
        const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
        uint32_t cur = NO_CAM;
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
        Cam cam;
        float dir[9];
        float jp2c = 0.0f;
        for (uint32_t j = a; j < b; ++j) {
            const uint32_t key = __ldg(v.obs_key + j);
            const uint32_t c = key >> 8, slot = key & 0xffu;
            if (c != cur) {
                if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                cur = c;
                cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
            }
            const size_t xi = v.pt_off + 3 * (size_t)(pt0 + slot);
            const float X0 = __ldg(v.x + xi), X1 = __ldg(v.x + xi + 1), X2 = __ldg(v.x + xi + 2);
            const float dX0 = v.p[xi], dX1 = v.p[xi + 1], dX2 = v.p[xi + 2];
            const Geo g = project_geo(cam, X0, X1, X2, eps);
            float t0, t1;
            jdir(g, cam, dir, dX0, dX1, dX2, t0, t1);
            jp2c = fmaf(t0, t0, fmaf(t1, t1, jp2c));
            // adjoint: u = A^T t; camera gets (RX x u, u, intrinsic part), point gets R^T u
            const float u0 = fmaf(g.A[0], t0, g.A[3] * t1);
            const float u1 = fmaf(g.A[1], t0, g.A[4] * t1);
            const float u2 = fmaf(g.A[2], t0, g.A[5] * t1);
            acc[0] += fmaf(g.RX[1], u2, -g.RX[2] * u1);
            acc[1] += fmaf(g.RX[2], u0, -g.RX[0] * u2);
            acc[2] += fmaf(g.RX[0], u1, -g.RX[1] * u0);
            acc[3] += u0;
            acc[4] += u1;
            acc[5] += u2;
            const float pt = fmaf(g.p[0], t0, g.p[1] * t1);
            const float fn2 = cam.f * g.n2;
            acc[6] = fmaf(g.s, pt, acc[6]);
            acc[7] = fmaf(fn2, pt, acc[7]);
            acc[8] = fmaf(fn2 * g.n2, pt, acc[8]);
            float* qs = qp + 3 * slot;
            atomicAdd(qs + 0, fmaf(cam.R[0], u0, fmaf(cam.R[3], u1, cam.R[6] * u2)));
            atomicAdd(qs + 1, fmaf(cam.R[1], u0, fmaf(cam.R[4], u1, cam.R[7] * u2)));
            atomicAdd(qs + 2, fmaf(cam.R[2], u0, fmaf(cam.R[5], u1, cam.R[8] * u2)));
        }
        const bool head = seg_reduce<9>(cur, acc);
        if (head && cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
        jp2 += (double)jp2c;
        __syncthreads();
        const size_t base = v.pt_off + 3 * (size_t)pt0;
        for (int i = threadIdx.x; i < npt * 3; i += TB)
            v.q[base + i] = fmaf(mu * v.D[base + i], v.p[base + i], qp[i]);
        __syncthreads();
    }
    double in[1] = {jp2}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_MV], out) && threadIdx.x == 0) {
        st->jp2 = out[0];
        const double denom = out[0] + st->mu * st->pDp;
        if (denom > 0.0 && isfinite(denom)) {
            st->alpha = st->rz / denom;
        } else {
            st->alpha = 0.0;
            if (st->pcg_active) {
                st->pcg_active = 0;
                if (!isfinite(denom)) st->status = 4;
            }
        }
    }
}

// ------------------------------------------------------------------ K5 --------
// h += alpha p; r -= alpha q; z = M^-1 r; r^T z and |r|^2.  Cameras first finish
// q = J_l^T (sum RX x u), sum u, intrinsic part + mu D p from the K4 accumulators.
// Never gated: its last block decides whether PCG continues and sets the loop flag.
__global__ void k_update(Views<float> v, CondHandle pcg_cond, int use_cond) {
    DevState* st = v.st;
    const int active = st->pcg_active;
    double rz = 0.0, rr = 0.0;
    if (active) {
        const float alpha = (float)st->alpha;
        const float mu = (float)st->mu;
        const int items = v.n_cams + v.n_pts;
        for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
            if (it < v.n_cams) {
                const int c = it;
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
                    const float pk = v.p[e + k];
                    const float qk = fmaf(mu * v.D[e + k], pk, q[k]);
                    v.h[e + k] = fmaf(alpha, pk, v.h[e + k]);
                    rn[k] = fmaf(-alpha, qk, v.r[e + k]);
                    v.r[e + k] = rn[k];
                }
                const float* M = v.Minv_c + (size_t)c * MC_STRIDE;
                float s_rz = 0.0f, s_rr = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float z = 0.0f;
#pragma unroll
                    for (int k = 0; k < 9; ++k) z = fmaf(M[9 * i + k], rn[k], z);
                    v.z[e + i] = z;
                    s_rz = fmaf(rn[i], z, s_rz);
                    s_rr = fmaf(rn[i], rn[i], s_rr);
                }
                rz += (double)s_rz;
                rr += (double)s_rr;
            } else {
                const int i = it - v.n_cams;
                const size_t e = v.pt_off + 3 * (size_t)i;
                float rn[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float pk = v.p[e + k];
                    v.h[e + k] = fmaf(alpha, pk, v.h[e + k]);
                    rn[k] = fmaf(-alpha, v.q[e + k], v.r[e + k]);
                    v.r[e + k] = rn[k];
                }
                const float* M = v.Minv_p + (size_t)i * MP_STRIDE;
                const float z0 = fmaf(M[0], rn[0], fmaf(M[1], rn[1], M[2] * rn[2]));
                const float z1 = fmaf(M[1], rn[0], fmaf(M[3], rn[1], M[4] * rn[2]));
                const float z2 = fmaf(M[2], rn[0], fmaf(M[4], rn[1], M[5] * rn[2]));
                v.z[e] = z0; v.z[e + 1] = z1; v.z[e + 2] = z2;
                rz += (double)fmaf(rn[0], z0, fmaf(rn[1], z1, rn[2] * z2));
                rr += (double)fmaf(rn[0], rn[0], fmaf(rn[1], rn[1], rn[2] * rn[2]));
            }
        }
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_UPD], out) && threadIdx.x == 0) {
        if (active) {
            st->pcg_iter += 1;
            st->pcg_total += 1;
            st->rr = out[1];
            const double tol = st->opt.tol;
            const bool converged = out[1] <= tol * tol * st->rr0;
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                st->status = 4;
                st->pcg_active = 0;
            } else if (converged || st->pcg_iter >= st->opt.max_pcg) {
                st->pcg_active = 0;
            } else {
                st->beta = out[0] / st->rz;
                st->rz = out[0];
            }
        }
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ K7 --------
// Candidate x' = x + h, g^T h, camera records at x', and the camera direction
// records of h at x (for |J h|^2).
__global__ void k_candidate(Views<float> v) {
    DevState* st = v.st;
    if (st->lm_active == 0) return;
    double gh = 0.0;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const int c = it;
            const size_t e = 9 * (size_t)c;
            const double* cl = v.cam_lin + (size_t)c * CL_STRIDE;
            double xn[9];
            float hc[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                hc[k] = v.h[e + k];
                const float xk = v.x[e + k] + hc[k];
                v.x_new[e + k] = xk;
                xn[k] = (double)xk;
                gh += cl[CL_G + k] * (double)hc[k];
            }
            camera_record(xn, v.cam_pre_new + (size_t)c * CP_STRIDE);
            const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
            float* d = v.cam_dir + (size_t)c * CD_STRIDE;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                d[CD_PHI + i] = fmaf(JL[3 * i], hc[0], fmaf(JL[3 * i + 1], hc[1], JL[3 * i + 2] * hc[2]));
#pragma unroll
            for (int k = 0; k < 6; ++k) d[CD_T + k] = hc[3 + k];
        } else {
            const size_t e = v.pt_off + 3 * (size_t)(it - v.n_cams);
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float hk = v.h[e + k];
                v.x_new[e + k] = v.x[e + k] + hk;
                s = fmaf(v.g[e + k], hk, s);
            }
            gh += (double)s;
        }
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
    double fnew = 0.0, jh2 = 0.0;
    if (active) {
        for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
            const uint32_t lo = v.tile_off[tile], hi = v.tile_off[tile + 1];
            const int pt0 = tile * TILE_PTS;
            const uint32_t n = hi - lo;
            const uint32_t chunk = (n + TB - 1) / TB;
            const uint32_t a = min(lo + threadIdx.x * chunk, hi), b = min(a + chunk, hi);
            uint32_t cur = NO_CAM;
            Cam cn, co;
            float dir[9];
            float fc = 0.0f, jc = 0.0f;
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = __ldg(v.obs_key + j);
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    cur = c;
                    cn = load_cam(v.cam_pre_new + (size_t)c * CP_STRIDE);
                    co = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                    load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
                }
                const size_t xi = v.pt_off + 3 * (size_t)(pt0 + slot);
                float r0, r1;
                project_residual(cn, v.x_new[xi], v.x_new[xi + 1], v.x_new[xi + 2], eps,
                                 v.obs_uv[2 * (size_t)j], v.obs_uv[2 * (size_t)j + 1], r0, r1);
                fc = fmaf(r0, r0, fmaf(r1, r1, fc));
                const Geo g = project_geo(co, v.x[xi], v.x[xi + 1], v.x[xi + 2], eps);
                float t0, t1;
                jdir(g, co, dir, v.h[xi], v.h[xi + 1], v.h[xi + 2], t0, t1);
                jc = fmaf(t0, t0, fmaf(t1, t1, jc));
            }
            fnew += (double)fc;
            jh2 += (double)jc;
        }
    }
    double in[2] = {fnew, jh2}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_COST], out) && threadIdx.x == 0) {
        if (active) {
            const double Fn = 0.5 * out[0];
            const double L = -st->gh - 0.5 * out[1];
            const double rho = (L > 0.0) ? (st->F - Fn) / L : -1.0;
            const bool acc = isfinite(Fn) && L > 0.0 && rho > 0.0;
            const int itn = st->lm_iter;
            if (itn < HIST_CAP) {
                IterRec& h = st->hist[itn];
                h.cost = st->F;
                h.cost_new = Fn;
                h.mu = st->mu;
                h.rho = rho;
                h.model_decrease = L;
                h.pcg_iters = st->pcg_iter;
                h.accepted = acc ? 1 : 0;
                h.t_ns = global_ns() - st->t_start;
            }
            st->F_new = Fn;
            st->rho = rho;
            st->L = L;
            st->jh2 = out[1];
            st->lm_iter = itn + 1;
            if (acc) {
                const double t = 2.0 * rho - 1.0;
                st->mu = st->mu * fmax(1.0 / 3.0, 1.0 - t * t * t);
                st->nu = 2.0;
                st->F = Fn;
                st->n_accepted += 1;
            } else {
                st->mu = st->mu * st->nu;
                st->nu = 2.0 * st->nu;
            }
            st->accepted = acc ? 1 : 0;
            const bool more = st->lm_iter < st->opt.max_lm && st->mu <= st->opt.max_mu &&
                              st->F > 0.0 && st->status == 0;
            st->lm_active = more ? 1 : 0;
            st->relin = (acc && more) ? 1 : 0;
        } else {
            st->accepted = 0;
            st->relin = 0;
        }
        if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ K8 --------
// Commit an accepted step: x = x', camera records = those of x', and clear the
// camera linearisation sums for the relinearisation that follows.
__global__ void k_commit(Views<float> v) {
    if (v.st->accepted == 0) return;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const size_t e = 9 * (size_t)it;
#pragma unroll
            for (int k = 0; k < 9; ++k) v.x[e + k] = v.x_new[e + k];
            const float4* s = reinterpret_cast<const float4*>(v.cam_pre_new + (size_t)it * CP_STRIDE);
            float4* d = reinterpret_cast<float4*>(v.cam_pre + (size_t)it * CP_STRIDE);
#pragma unroll
            for (int k = 0; k < CP_STRIDE / 4; ++k) d[k] = s[k];
            double* cl = v.cam_lin + (size_t)it * CL_STRIDE;
#pragma unroll 8
            for (int k = 0; k < CL_STRIDE; ++k) cl[k] = 0.0;
        } else {
            const size_t e = v.pt_off + 3 * (size_t)(it - v.n_cams);
#pragma unroll
            for (int k = 0; k < 3; ++k) v.x[e + k] = v.x_new[e + k];
        }
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
// and the internal vector layout.
template <typename S>
__global__ void k_pack(Views<float> v, const S* cams, const S* pts) {
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            for (int k = 0; k < 9; ++k) v.x[9 * (size_t)it + k] = (float)cams[9 * (size_t)it + k];
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) v.x[e + k] = (float)pts[3 * (size_t)u + k];
        }
    }
}

template <typename S>
__global__ void k_unpack(Views<float> v, const float* src, S* cams, S* pts) {
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
                out[e + k] = (S)fmaf(mu * v.D[e + k], v.p[e + k], q);
            }
            for (int k = 0; k < CA_STRIDE; ++k) ca[k] = 0.0f;
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) out[9 * (size_t)v.n_cams + 3 * (size_t)u + k] = (S)v.q[e + k];
        }
    }
}

// p from a caller-layout vector; camera direction records and p^T D p.
template <typename S>
__global__ void k_set_direction(Views<float> v, const S* src) {
    double pdp = 0.0;
    const int items = v.n_cams + v.n_pts;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        if (it < v.n_cams) {
            const size_t e = 9 * (size_t)it;
            float pc[9];
            for (int k = 0; k < 9; ++k) {
                pc[k] = (float)src[e + k];
                v.p[e + k] = pc[k];
                pdp += (double)v.D[e + k] * pc[k] * pc[k];
            }
            const float* JL = v.cam_pre + (size_t)it * CP_STRIDE + CP_JL;
            float* d = v.cam_dir + (size_t)it * CD_STRIDE;
            for (int i = 0; i < 3; ++i)
                d[CD_PHI + i] = fmaf(JL[3 * i], pc[0], fmaf(JL[3 * i + 1], pc[1], JL[3 * i + 2] * pc[2]));
            for (int k = 0; k < 6; ++k) d[CD_T + k] = pc[3 + k];
        } else {
            const int u = it - v.n_cams;
            const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
            for (int k = 0; k < 3; ++k) {
                const float pk = (float)src[9 * (size_t)v.n_cams + 3 * (size_t)u + k];
                v.p[e + k] = pk;
                pdp += (double)v.D[e + k] * pk * pk;
            }
        }
    }
    double in[1] = {pdp}, out[1];
    if (grid_reduce<1>(in, v.partials, &v.st->tickets[TK_DIR], out) && threadIdx.x == 0) v.st->pDp = out[0];
}

// ------------------------------------------------------------------ launchers --

namespace {
inline int grid_items(const LaunchCfg& L, int items) {
    int g = (items + L.item_block - 1) / L.item_block;
    return g < 1 ? 1 : (g > L.item_grid ? L.item_grid : g);
}
inline int grid_tiles(int cap, int n_tiles) { return n_tiles < 1 ? 1 : (n_tiles > cap ? cap : n_tiles); }
}  // namespace

void launch_camera_precompute(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_camera_precompute<<<grid_items(L, v.n_cams), L.item_block, 0, s>>>(v);
}
void launch_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode,
                      float* res_out, float* jac_out, CondHandle lm_cond, int use_cond) {
    k_linearize<LIN_TB><<<grid_tiles(L.lin_grid, v.n_tiles), LIN_TB, 0, s>>>(v, mode, res_out, jac_out,
                                                                             lm_cond, use_cond);
}
void launch_precond(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k_precond<<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v, c, use);
}
void launch_direction(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_direction<<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v);
}
void launch_matvec(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate) {
    k_matvec<MV_TB><<<grid_tiles(L.mv_grid, v.n_tiles), MV_TB, 0, s>>>(v, gate);
}
void launch_update(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k_update<<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v, c, use);
}
void launch_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s) {
    k_candidate<<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v);
}
void launch_eval_candidate(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
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
void launch_unpack(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const float* src, void* cams,
                   void* pts, int dtype) {
    const int g = grid_items(L, v.n_cams + v.n_pts);
    if (dtype == 1) k_unpack<double><<<g, L.item_block, 0, s>>>(v, src, (double*)cams, (double*)pts);
    else k_unpack<float><<<g, L.item_block, 0, s>>>(v, src, (float*)cams, (float*)pts);
}
void launch_set_direction(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const float* src) {
    k_set_direction<float><<<grid_items(L, v.n_cams + v.n_pts), L.item_block, 0, s>>>(v, src);
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
