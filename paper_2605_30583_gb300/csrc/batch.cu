// Batched LM + PCGNR: many independent small bundle-adjustment problems solved by one
// persistent kernel.  Each CTA takes whole problems from a device work queue (largest
// first) and runs the complete solve of Sec. V for that problem at block scope --
// linearisation, block-Jacobi preconditioner, PCGNR, candidate step and LM decision --
// with block barriers only, so no CTA ever waits on another.  The arithmetic is the
// one of the single-problem mixed-precision path: FP32 residuals, Jacobian products
// and vectors; FP64 block inversions, PCG dot products and cost sums.
//
// Per problem the observations are sorted by camera, and within a camera's run by
// point from a camera-dependent starting point; a point-major index
// serves the passes that need all observations of one point.  During PCG the CTA keeps
// the problem's camera records, camera direction records, camera accumulators and the
// point part of the product q = (J^T J) p in shared memory.
//
// Schedules (threads per CTA, resident CTAs per SM) are picked by a timing autotuner
// whose choices are cached per process, keyed by the GPU's name and the batch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "gbba.h"
#include "kernels.h"
#include "mixed_common.cuh"
#include "problem.h"

namespace gbba {

struct BatchStats {
    double initial_cost, final_cost;
    int32_t lm_iters, accepted, pcg_iters, status;
};

struct BatchView {
    int32_t n_problems;
    int32_t cam_cap;            // cameras per problem that the shared-memory tables hold
    int32_t pt_cap;             // points per problem that the shared-memory tables hold
    const int32_t* order;       // problems, largest first
    const int32_t* cam_off;     // [P + 1] global camera offsets
    const int32_t* pt_off;      // [P + 1] global point offsets
    const int64_t* obs_off;     // [P + 1]
    const int64_t* vec_off;     // [P + 1] offsets of each problem's [9 nc | 3 np] vector block
    const uint32_t* obs_key;    // local camera << 16 | local point, sorted per problem by camera
    const float* obs_uv;        // [n_obs][2]
    const uint32_t* pm_pos;     // point-major: global positions of each point's observations
    const uint32_t* pt_obs_off; // [total points + 1] offsets into pm_pos
    float *x, *x_new, *h, *r, *z, *p, *g, *D;
    float *cam_pre, *cam_pre_new;   // [total cams][CP_STRIDE]
    double* cam_g;                  // [total cams][CL_STRIDE]
    float* cam_H;                   // [total cams][CH_STRIDE]
    float* Minv_c;                  // [total cams][81]
    float *pt_H, *Minv_p;           // [total points][6]
    BatchStats* stats;              // [P]
    unsigned int* queue;            // work counter
    DevOptions opt;
};

namespace {

constexpr int SCAM = 16, SDIR = 12, SACC = 12;   // shared floats per camera

// Camera record of the problem's own writes: plain (coherent) loads, since records
// are rewritten inside the kernel.
__device__ __forceinline__ Cam cam_plain(const float* rec) {
    const float4* r4 = reinterpret_cast<const float4*>(rec);
    const float4 a = r4[0], b = r4[1], c = r4[2], d = r4[3];
    Cam m;
    m.R[0] = a.x; m.R[1] = a.y; m.R[2] = a.z; m.R[3] = a.w;
    m.R[4] = b.x; m.R[5] = b.y; m.R[6] = b.z; m.R[7] = b.w;
    m.R[8] = c.x; m.t[0] = c.y; m.t[1] = c.z; m.t[2] = c.w;
    m.f = d.x; m.k1 = d.y; m.k2 = d.z;
    return m;
}

// Block-wide sums broadcast to every thread: two FP32 values (FP32 within a warp, FP64
// across warps) or two FP64 values.
__device__ __forceinline__ void bsum2(float a, float b, double* sh, double& ra, double& rb) {
    block_sum2(a, b, sh, ra, rb);
    if (threadIdx.x == 0) { sh[62] = ra; sh[63] = rb; }
    __syncthreads();
    ra = sh[62];
    rb = sh[63];
    __syncthreads();
}

__device__ __forceinline__ void bsum2d(double a, double b, double* sh, double& ra, double& rb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[w] = a; sh[nw + w] = b; }
    __syncthreads();
    ra = rb = 0.0;
    for (int i = 0; i < nw; ++i) { ra += sh[i]; rb += sh[nw + i]; }
    __syncthreads();
}

struct Prob {
    int nc, np;
    int64_t no;
    int c0, p0;          // global camera / point offsets
    int64_t o0, v0;      // global observation offset, vector offset
};

__device__ __forceinline__ Prob load_prob(const BatchView& b, int q) {
    Prob P;
    P.c0 = b.cam_off[q];
    P.nc = b.cam_off[q + 1] - P.c0;
    P.p0 = b.pt_off[q];
    P.np = b.pt_off[q + 1] - P.p0;
    P.o0 = b.obs_off[q];
    P.no = b.obs_off[q + 1] - P.o0;
    P.v0 = b.vec_off[q];
    return P;
}

// Camera records (rotation, J_l, ...) of the problem's cameras from the parameters in
// `xs`; optionally clears the camera linearisation sums.
__device__ void b_camera_records(const BatchView& b, const Prob& P, const float* xs, float* rec, bool clear) {
    for (int c = threadIdx.x; c < P.nc; c += blockDim.x) {
        double pr[9];
        for (int k = 0; k < 9; ++k) pr[k] = (double)xs[P.v0 + 9 * c + k];
        camera_record(pr, rec + (size_t)(P.c0 + c) * CP_STRIDE, b.opt.retract != 0);
        if (clear) {
            for (int k = 0; k < CL_STRIDE; ++k) b.cam_g[(size_t)(P.c0 + c) * CL_STRIDE + k] = 0.0;
            for (int k = 0; k < CH_STRIDE; ++k) b.cam_H[(size_t)(P.c0 + c) * CH_STRIDE + k] = 0.0f;
        }
    }
}

constexpr int BLIN = 9 + CH_STRIDE;   // g_c (9) and the upper triangle of J_c^T J_c (45, padded to 48)

__device__ __forceinline__ void b_flush_lin(const BatchView& b, int gc, float (&a)[BLIN]) {
    double* g = b.cam_g + (size_t)gc * CL_STRIDE;
    for (int k = 0; k < 9; ++k) atomicAdd(g + k, (double)a[k]);
    float4* h = reinterpret_cast<float4*>(b.cam_H + (size_t)gc * CH_STRIDE);
    for (int k = 0; k < CH_STRIDE / 4; ++k)
        atomicAdd(h + k, make_float4(a[9 + 4 * k], a[10 + 4 * k], a[11 + 4 * k], a[12 + 4 * k]));
    for (int k = 0; k < BLIN; ++k) a[k] = 0.0f;
}

// Linearisation of one problem (Sec. V): camera pass over the camera-sorted
// observations accumulates g_c = J_c^T r and J_c^T J_c; point pass over the point-major
// index computes g_p = J_p^T r, J_p^T J_p and the cost.  Returns F = 1/2 |r|^2 in every
// thread.
__device__ double b_linearize(const BatchView& b, const Prob& P, float eps, double* sh) {
    {
        const int64_t chunk = odd_chunk<int64_t>(P.no, (int64_t)blockDim.x);
        const int64_t a = min(P.o0 + (int64_t)threadIdx.x * chunk, P.o0 + P.no), e = min(a + chunk, P.o0 + P.no);
        uint32_t cur = NO_CAM;
        float acc[BLIN];
        for (int k = 0; k < BLIN; ++k) acc[k] = 0.0f;
        Cam cam;
        float JL[9];
        for (int64_t j = a; j < e; ++j) {
            const uint32_t key = b.obs_key[j];
            const uint32_t c = key >> 16, lp = key & 0xffffu;
            if (c != cur) {
                if (cur != NO_CAM) b_flush_lin(b, P.c0 + cur, acc);
                cur = c;
                const float* rec = b.cam_pre + (size_t)(P.c0 + c) * CP_STRIDE;
                cam = cam_plain(rec);
                for (int k = 0; k < 9; ++k) JL[k] = rec[CP_JL + k];
            }
            const float* X = b.x + P.v0 + 9 * P.nc + 3 * lp;
            const Geo g = project_geo(cam, X[0], X[1], X[2], eps);
            const float fs = cam.f * g.s;
            const float r0 = fmaf(fs, g.p[0], -b.obs_uv[2 * j]);
            const float r1 = fmaf(fs, g.p[1], -b.obs_uv[2 * j + 1]);
            // J_c rows: rotation through J_l (phi = J_l d_w), translation A, intrinsics
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
#pragma unroll
            for (int i = 0; i < 9; ++i) acc[i] = fmaf(j0[i], r0, fmaf(j1[i], r1, acc[i]));
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int k = i; k < 9; ++k) {
                    const int t = 9 + tri_index(9, i, k);
                    acc[t] = fmaf(j0[i], j0[k], fmaf(j1[i], j1[k], acc[t]));
                }
        }
        const bool head = seg_reduce<BLIN>(cur, acc);
        if (head && cur != NO_CAM) b_flush_lin(b, P.c0 + cur, acc);
    }
    double cost = 0.0;
    for (int i = threadIdx.x; i < P.np; i += blockDim.x) {
        const int gp = P.p0 + i;
        const float* X = b.x + P.v0 + 9 * P.nc + 3 * i;
        const float X0 = X[0], X1 = X[1], X2 = X[2];
        float gq[3] = {0, 0, 0}, hq[6] = {0, 0, 0, 0, 0, 0};
        for (uint32_t k = b.pt_obs_off[gp]; k < b.pt_obs_off[gp + 1]; ++k) {
            const uint32_t j = b.pm_pos[k];
            const uint32_t c = b.obs_key[j] >> 16;
            const Cam cam = cam_plain(b.cam_pre + (size_t)(P.c0 + c) * CP_STRIDE);
            const Geo g = project_geo(cam, X0, X1, X2, eps);
            const float fs = cam.f * g.s;
            const float r0 = fmaf(fs, g.p[0], -b.obs_uv[2 * (size_t)j]);
            const float r1 = fmaf(fs, g.p[1], -b.obs_uv[2 * (size_t)j + 1]);
            cost += (double)fmaf(r0, r0, r1 * r1);
            float jx0[3], jx1[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                jx0[q] = fmaf(g.A[0], cam.R[q], fmaf(g.A[1], cam.R[3 + q], g.A[2] * cam.R[6 + q]));
                jx1[q] = fmaf(g.A[3], cam.R[q], fmaf(g.A[4], cam.R[3 + q], g.A[5] * cam.R[6 + q]));
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) gq[q] = fmaf(jx0[q], r0, fmaf(jx1[q], r1, gq[q]));
#pragma unroll
            for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
                for (int b2 = a2; b2 < 3; ++b2) {
                    const int t = tri_index(3, a2, b2);
                    hq[t] = fmaf(jx0[a2], jx0[b2], fmaf(jx1[a2], jx1[b2], hq[t]));
                }
        }
        for (int q = 0; q < 3; ++q) b.g[P.v0 + 9 * P.nc + 3 * i + q] = gq[q];
        for (int q = 0; q < 6; ++q) b.pt_H[(size_t)gp * 6 + q] = hq[q];
    }
    double F, unused;
    bsum2d(cost, 0.0, sh, F, unused);   // its barriers also publish the camera sums
    return 0.5 * F;
}

// Block-Jacobi preconditioner of J^T J + mu D (FP64 inversions, stored FP32) and the
// PCG start r = -g, z = M^-1 r, p = h = 0.  Returns r^T z and |r|^2.
__device__ void b_precond(const BatchView& b, const Prob& P, double mu, double* sh, double& rz, double& rr) {
    const DevOptions& o = b.opt;
    float* Dv = b.D + P.v0;
    float* r = b.r + P.v0;
    float* z = b.z + P.v0;
    float* pv = b.p + P.v0;
    float* h = b.h + P.v0;
    const float* gv = b.g + P.v0;
    float lrz = 0.0f, lrr = 0.0f;
    const int lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < P.nc; c += blockDim.x >> 5) {   // one warp per camera
        const float* Hc = b.cam_H + (size_t)(P.c0 + c) * CH_STRIDE;
        const int j = lane < 18 ? lane : 17;
        double col[9];
        for (int i = 0; i < 9; ++i) {
            if (j < 9) {
                double hv = Hc[tri_index(9, i < j ? i : j, i < j ? j : i)];
                if (i == j) hv += mu * fmin(fmax(hv, o.min_diag), o.max_diag);
                col[i] = hv;
            } else {
                col[i] = (i == j - 9) ? 1.0 : 0.0;
            }
        }
        const double hd = lane < 9 ? (double)Hc[tri_index(9, lane, lane)] : 0.0;
        const bool ok = warp_block_inverse9(col, lane);
        float* Mo = b.Minv_c + (size_t)(P.c0 + c) * 81;
        if (lane >= 9 && lane < 18)
            for (int i = 0; i < 9; ++i) Mo[i * 9 + (lane - 9)] = (float)col[i];
        if (!ok && lane < 9) {   // not SPD in FP64: inverse diagonal
            const double dd = hd + mu * fmin(fmax(hd, o.min_diag), o.max_diag);
            for (int i = 0; i < 9; ++i) Mo[i * 9 + lane] = (i == lane && dd > 0.0) ? (float)(1.0 / dd) : 0.0f;
        }
        __syncwarp();
        if (lane < 9) {
            const int e = 9 * c + lane;
            Dv[e] = (float)fmin(fmax(hd, o.min_diag), o.max_diag);
            const double* gc = b.cam_g + (size_t)(P.c0 + c) * CL_STRIDE;
            const float ri = (float)(-gc[lane]);
            float zz = 0.0f;
            for (int k = 0; k < 9; ++k) zz = fmaf(Mo[lane * 9 + k], (float)(-gc[k]), zz);
            r[e] = ri; z[e] = zz; pv[e] = 0.0f; h[e] = 0.0f;
            lrz = fmaf(ri, zz, lrz);
            lrr = fmaf(ri, ri, lrr);
        }
        __syncwarp();
    }
    for (int i = threadIdx.x; i < P.np; i += blockDim.x) {
        const float* Hp = b.pt_H + (size_t)(P.p0 + i) * 6;
        const int e = 9 * P.nc + 3 * i;
        double a00 = Hp[0], a01 = Hp[1], a02 = Hp[2], a11 = Hp[3], a12 = Hp[4], a22 = Hp[5];
        const double d0 = fmin(fmax(a00, o.min_diag), o.max_diag), d1 = fmin(fmax(a11, o.min_diag), o.max_diag),
                     d2 = fmin(fmax(a22, o.min_diag), o.max_diag);
        a00 += mu * d0; a11 += mu * d1; a22 += mu * d2;
        // inverse of the SPD 3x3 block by its adjugate
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        double m[6];
        if (det > 0.0 && isfinite(det) && a00 > 0.0 && c22 > 0.0) {
            const double id = rcp64(det);
            m[0] = c00 * id; m[1] = c01 * id; m[2] = c02 * id; m[3] = c11 * id; m[4] = c12 * id; m[5] = c22 * id;
        } else {
            m[0] = a00 > 0 ? 1.0 / a00 : 0.0; m[1] = 0.0; m[2] = 0.0;
            m[3] = a11 > 0 ? 1.0 / a11 : 0.0; m[4] = 0.0; m[5] = a22 > 0 ? 1.0 / a22 : 0.0;
        }
        float Mo[6];
        for (int k = 0; k < 6; ++k) Mo[k] = (float)m[k];
        float* Mg = b.Minv_p + (size_t)(P.p0 + i) * 6;
        for (int k = 0; k < 6; ++k) Mg[k] = Mo[k];
        Dv[e] = (float)d0; Dv[e + 1] = (float)d1; Dv[e + 2] = (float)d2;
        const float r0 = -gv[e], r1 = -gv[e + 1], r2 = -gv[e + 2];
        const float z0 = fmaf(Mo[0], r0, fmaf(Mo[1], r1, Mo[2] * r2));
        const float z1 = fmaf(Mo[1], r0, fmaf(Mo[3], r1, Mo[4] * r2));
        const float z2 = fmaf(Mo[2], r0, fmaf(Mo[4], r1, Mo[5] * r2));
        r[e] = r0; r[e + 1] = r1; r[e + 2] = r2;
        z[e] = z0; z[e + 1] = z1; z[e + 2] = z2;
        pv[e] = pv[e + 1] = pv[e + 2] = 0.0f;
        h[e] = h[e + 1] = h[e + 2] = 0.0f;
        lrz = fmaf(r0, z0, fmaf(r1, z1, fmaf(r2, z2, lrz)));
        lrr = fmaf(r0, r0, fmaf(r1, r1, fmaf(r2, r2, lrr)));
    }
    bsum2(lrz, lrr, sh, rz, rr);
}

// Shared-memory tables of the CTA's current problem.
struct Shm {
    float *cam, *dir, *acc;                // per camera: records (16), direction records (12), sums (12)
    float *rc, *zc, *hc, *pc, *dc, *jl;    // per camera, 9 each: camera block of r z h p D, and J_l
    float *q, *x, *p;                      // per point, 3 each (x and p only with staged points)
};

// PCGNR on (J^T J + mu D) h = -g from h = 0 (Sec. V): p = z + beta p;
// alpha = r^T z / (|J p|^2 + mu p^T D p); h += alpha p; r -= alpha (J^T J p + mu D p);
// z = M^-1 r; stop when |r| <= tol |r0| or after max_pcg iterations.  J p and J^T (J p)
// are recomputed per observation from the camera records in shared memory.  Returns
// the iteration count; sets status 4 on a non-finite quantity.
//
// The camera block of every PCG vector lives in shared memory; with SP (staged points)
// so do the points' parameters X and the point part of p, and the per-observation
// gathers of the product never leave the SM.  The loops over points issue all their
// loads before any store (several elements per thread) so that global-memory latency
// overlaps; camera work goes to the last threads, which hold the fewest points.
//
// mu is folded into every product with D before it is summed or applied: once the cost
// reaches the FP32 noise floor, rejected steps drive mu to 1e20 and beyond, where p
// scales like 1/mu and D p^2 alone would underflow FP32 while mu D p^2 stays O(r z).
template <int TB, bool SP>
__device__ int b_pcg(const BatchView& b, const Prob& P, double mu, double rz, double rr0, const Shm& S, double* sh,
                     int& status) {
    const DevOptions& o = b.opt;
    const float eps = (float)o.eps;
    const int tid = threadIdx.x;
    const int nc9 = 9 * P.nc, n3 = 3 * P.np;
    if (!(rr0 > 0.0) || !(rz > 0.0) || !isfinite(rz) || o.max_pcg <= 0) return 0;
    const float* __restrict__ xg = b.x + P.v0 + nc9;
    float* __restrict__ hg = b.h + P.v0;
    float* __restrict__ rg = b.r + P.v0 + nc9;
    float* __restrict__ zg = b.z + P.v0 + nc9;
    const float* __restrict__ Dg = b.D + P.v0 + nc9;
    const float* __restrict__ Mp = b.Minv_p + (size_t)P.p0 * 6;
    const float* __restrict__ Mc = b.Minv_c + (size_t)P.c0 * 81;
    const uint32_t* __restrict__ keys = b.obs_key;
    const float muf = (float)mu;
    for (int i = tid; i < nc9; i += TB) {
        S.rc[i] = b.r[P.v0 + i];
        S.zc[i] = b.z[P.v0 + i];
        S.dc[i] = b.D[P.v0 + i];
        S.hc[i] = 0.0f;
        S.pc[i] = 0.0f;
        S.jl[i] = b.cam_pre[(size_t)(P.c0 + i / 9) * CP_STRIDE + CP_JL + i % 9];
    }
    if (SP)
        for (int e = tid; e < n3; e += TB) {
            S.x[e] = xg[e];
            S.p[e] = 0.0f;
        }
    const float* Xp = SP ? S.x : xg;            // point parameters
    float* Pp = SP ? S.p : b.p + P.v0 + nc9;    // point part of the direction (zero after the preconditioner)
    __syncthreads();
    const double tol2 = o.tol * o.tol;
    int k = 0;
    double beta = 0.0;
    for (;;) {
        // ---- direction p = z + beta p, camera direction records, mu p^T D p
        float pdp = 0.0f;
        const float bf = (float)beta;
        for (int c = TB - 1 - tid; c < P.nc; c += TB) {
            float pc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                pc[q] = fmaf(bf, S.pc[9 * c + q], S.zc[9 * c + q]);
                S.pc[9 * c + q] = pc[q];
                pdp = fmaf(muf * (S.dc[9 * c + q] * pc[q]), pc[q], pdp);
            }
            const float* JL = S.jl + 9 * c;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                S.dir[SDIR * c + i] = fmaf(JL[3 * i], pc[0], fmaf(JL[3 * i + 1], pc[1], JL[3 * i + 2] * pc[2]));
#pragma unroll
            for (int q = 3; q < 9; ++q) S.dir[SDIR * c + q] = pc[q];
#pragma unroll
            for (int q = 0; q < SACC; ++q) S.acc[SACC * c + q] = 0.0f;
        }
        for (int e0 = tid; e0 < n3; e0 += 4 * TB) {
            float zv[4], dv[4], pv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * TB;
                const bool in = e < n3;
                zv[u] = in ? zg[e] : 0.0f;
                dv[u] = in ? Dg[e] : 0.0f;
                pv[u] = in ? Pp[e] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * TB;
                if (e < n3) {
                    const float pk = fmaf(bf, pv[u], zv[u]);
                    Pp[e] = pk;
                    pdp = fmaf(muf * (dv[u] * pk), pk, pdp);
                    S.q[e] = 0.0f;
                }
            }
        }
        __syncthreads();
        // ---- q = J^T J p: each thread a contiguous run of camera-sorted observations
        // (so a thread changes camera rarely and its flushes are staggered against the
        // other lanes'), keys fetched one group of four ahead
        float jp2 = 0.0f;
        {
            const int64_t chunk = odd_chunk<int64_t>(P.no, (int64_t)TB);
            const int64_t a = min(P.o0 + (int64_t)tid * chunk, P.o0 + P.no), e = min(a + chunk, P.o0 + P.no);
            uint32_t cur = NO_CAM;
            float acc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
            Cam cam;
            float dir[9];
            uint32_t kn[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) kn[u] = (a + u < e) ? keys[a + u] : NO_CAM;
            for (int64_t j = a; j < e; j += 4) {
                uint32_t kc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    kc[u] = kn[u];
                    kn[u] = (j + 4 + u < e) ? keys[j + 4 + u] : NO_CAM;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kc[u] == NO_CAM) continue;
                    const uint32_t c = kc[u] >> 16, lp = kc[u] & 0xffffu;
                    if (c != cur) {
                        if (cur != NO_CAM) {
#pragma unroll
                            for (int q = 0; q < 9; ++q) {
                                atomicAdd(S.acc + SACC * cur + q, acc[q]);
                                acc[q] = 0.0f;
                            }
                        }
                        cur = c;
                        const float4* r4 = reinterpret_cast<const float4*>(S.cam + SCAM * c);
                        const float4 c0 = r4[0], c1 = r4[1], c2 = r4[2], c3 = r4[3];
                        cam.R[0] = c0.x; cam.R[1] = c0.y; cam.R[2] = c0.z; cam.R[3] = c0.w;
                        cam.R[4] = c1.x; cam.R[5] = c1.y; cam.R[6] = c1.z; cam.R[7] = c1.w;
                        cam.R[8] = c2.x; cam.t[0] = c2.y; cam.t[1] = c2.z; cam.t[2] = c2.w;
                        cam.f = c3.x; cam.k1 = c3.y; cam.k2 = c3.z;
#pragma unroll
                        for (int q = 0; q < 9; ++q) dir[q] = S.dir[SDIR * c + q];
                    }
                    jp2 += obs_normal(cam, dir, Xp + 3 * lp, Pp + 3 * lp, eps, acc, S.q + 3 * lp);
                }
            }
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM)
#pragma unroll
                for (int q = 0; q < 9; ++q) atomicAdd(S.acc + SACC * cur + q, acc[q]);
        }
        double sj, sp;
        bsum2(jp2, pdp, sh, sj, sp);   // barriers publish S.acc / S.q
        const double denom = sj + sp;
        if (!(denom > 0.0) || !isfinite(denom)) {
            if (!isfinite(denom)) status = 4;
            break;
        }
        // ---- h += alpha p, r -= alpha (q + mu D p), z = M^-1 r
        const float af = (float)(rz / denom);
        float lrz = 0.0f, lrr = 0.0f;
        for (int c = TB - 1 - tid; c < P.nc; c += TB) {
            const float* JL = S.jl + 9 * c;
            const float* ca = S.acc + SACC * c;
            float qv[9], rn[9], M[81];
#pragma unroll
            for (int t = 0; t < 81; ++t) M[t] = Mc[81 * c + t];
#pragma unroll
            for (int q = 0; q < 3; ++q) qv[q] = fmaf(JL[q], ca[0], fmaf(JL[3 + q], ca[1], JL[6 + q] * ca[2]));
#pragma unroll
            for (int q = 3; q < 9; ++q) qv[q] = ca[q];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const int e = 9 * c + q;
                const float pk = S.pc[e];
                S.hc[e] = fmaf(af, pk, S.hc[e]);
                rn[q] = fmaf(-af, fmaf(muf, S.dc[e] * pk, qv[q]), S.rc[e]);
                S.rc[e] = rn[q];
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float zz = 0.0f;
#pragma unroll
                for (int q = 0; q < 9; ++q) zz = fmaf(M[9 * i + q], rn[q], zz);
                S.zc[9 * c + i] = zz;
                lrz = fmaf(rn[i], zz, lrz);
                lrr = fmaf(rn[i], rn[i], lrr);
            }
        }
        for (int i0 = tid; i0 < P.np; i0 += 2 * TB) {
            float pk[2][3], hk[2][3], dk[2][3], rk[2][3], qk[2][3], m[2][6];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + u * TB;
                const bool in = i < P.np;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    pk[u][q] = in ? Pp[3 * i + q] : 0.0f;
                    hk[u][q] = in ? hg[nc9 + 3 * i + q] : 0.0f;
                    dk[u][q] = in ? Dg[3 * i + q] : 0.0f;
                    rk[u][q] = in ? rg[3 * i + q] : 0.0f;
                    qk[u][q] = in ? S.q[3 * i + q] : 0.0f;
                }
#pragma unroll
                for (int t = 0; t < 6; ++t) m[u][t] = in ? Mp[6 * i + t] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = i0 + u * TB;
                if (i < P.np) {
                    float rn[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        hg[nc9 + 3 * i + q] = fmaf(af, pk[u][q], hk[u][q]);
                        rn[q] = fmaf(-af, fmaf(muf, dk[u][q] * pk[u][q], qk[u][q]), rk[u][q]);
                        rg[3 * i + q] = rn[q];
                    }
                    const float* mm = m[u];
                    const float z0 = fmaf(mm[0], rn[0], fmaf(mm[1], rn[1], mm[2] * rn[2]));
                    const float z1 = fmaf(mm[1], rn[0], fmaf(mm[3], rn[1], mm[4] * rn[2]));
                    const float z2 = fmaf(mm[2], rn[0], fmaf(mm[4], rn[1], mm[5] * rn[2]));
                    zg[3 * i] = z0;
                    zg[3 * i + 1] = z1;
                    zg[3 * i + 2] = z2;
                    lrz = fmaf(rn[0], z0, fmaf(rn[1], z1, fmaf(rn[2], z2, lrz)));
                    lrr = fmaf(rn[0], rn[0], fmaf(rn[1], rn[1], fmaf(rn[2], rn[2], lrr)));
                }
            }
        }
        double rzn, rrn;
        bsum2(lrz, lrr, sh, rzn, rrn);
        ++k;
        if (!isfinite(rzn) || !isfinite(rrn)) {
            status = 4;
            break;
        }
        if (rrn <= tol2 * rr0 || k >= o.max_pcg || !(rzn > 0.0)) break;
        beta = rzn / rz;
        rz = rzn;
    }
    // camera block of h back to the global vector for the candidate step
    for (int i = tid; i < nc9; i += TB) hg[i] = S.hc[i];
    __syncthreads();
    return k;
}

// Candidate x' = x + h and its evaluation: F(x') (camera records of x' in cam_pre_new),
// |J(x) h|^2 (camera records of x in shared memory) and g^T h, all FP64 sums.
template <int TB>
__device__ void b_candidate(const BatchView& b, const Prob& P, const float* sCam, float* sDir, double* sh,
                            double& Fn, double& jh2, double& gh) {
    const float eps = (float)b.opt.eps;
    const int tid = threadIdx.x, n = 9 * P.nc + 3 * P.np;
    const float* x = b.x + P.v0;
    float* xn = b.x_new + P.v0;
    const float* h = b.h + P.v0;
    const float* gv = b.g + P.v0;
    double lgh = 0.0;
    for (int e = tid; e < n; e += TB) {
        xn[e] = x[e] + h[e];
        const double ge = e < 9 * P.nc ? b.cam_g[(size_t)(P.c0 + e / 9) * CL_STRIDE + e % 9] : (double)gv[e];
        lgh += ge * (double)h[e];
    }
    __syncthreads();
    if (b.opt.retract) {   // rotations: R' = Exp(h_w) R(w)
        for (int c = tid; c < P.nc; c += TB) {
            const double w[3] = {x[9 * c], x[9 * c + 1], x[9 * c + 2]};
            const double hw[3] = {h[9 * c], h[9 * c + 1], h[9 * c + 2]};
            double wn[3];
            compose_rotvec(hw, w, wn);
            for (int k = 0; k < 3; ++k) xn[9 * c + k] = (float)wn[k];
        }
        __syncthreads();
    }
    b_camera_records(b, P, b.x_new, b.cam_pre_new, false);
    for (int c = tid; c < P.nc; c += TB) {   // direction records of h at x
        const float* JL = b.cam_pre + (size_t)(P.c0 + c) * CP_STRIDE + CP_JL;
        const float* hc = h + 9 * c;
        for (int i = 0; i < 3; ++i)
            sDir[SDIR * c + i] = fmaf(JL[3 * i], hc[0], fmaf(JL[3 * i + 1], hc[1], JL[3 * i + 2] * hc[2]));
        for (int q = 3; q < 9; ++q) sDir[SDIR * c + q] = hc[q];
    }
    __syncthreads();
    double lf = 0.0, ljh = 0.0;
    for (int64_t j = P.o0 + tid; j < P.o0 + P.no; j += TB) {
        const uint32_t key = b.obs_key[j];
        const uint32_t c = key >> 16, lp = key & 0xffffu;
        const int e3 = 9 * P.nc + 3 * lp;
        const Cam cn = cam_plain(b.cam_pre_new + (size_t)(P.c0 + c) * CP_STRIDE);
        float r0, r1;
        project_residual(cn, xn[e3], xn[e3 + 1], xn[e3 + 2], eps, b.obs_uv[2 * j], b.obs_uv[2 * j + 1], r0, r1);
        lf += (double)fmaf(r0, r0, r1 * r1);
        const float4* r4 = reinterpret_cast<const float4*>(sCam + SCAM * c);
        const float4 c0 = r4[0], c1 = r4[1], c2 = r4[2], c3 = r4[3];
        Cam co;
        co.R[0] = c0.x; co.R[1] = c0.y; co.R[2] = c0.z; co.R[3] = c0.w;
        co.R[4] = c1.x; co.R[5] = c1.y; co.R[6] = c1.z; co.R[7] = c1.w;
        co.R[8] = c2.x; co.t[0] = c2.y; co.t[1] = c2.z; co.t[2] = c2.w;
        co.f = c3.x; co.k1 = c3.y; co.k2 = c3.z;
        const float* d = sDir + SDIR * c;
        const GeoLite g = project_lite(co, x[e3], x[e3 + 1], x[e3 + 2], eps);
        // J h = A (phi x RX + h_t + R h_X) + c_i p
        float dP0 = fmaf(d[1], g.RX[2], -d[2] * g.RX[1]) + d[3];
        float dP1 = fmaf(d[2], g.RX[0], -d[0] * g.RX[2]) + d[4];
        float dP2 = fmaf(d[0], g.RX[1], -d[1] * g.RX[0]) + d[5];
        const float* hx = h + e3;
        dP0 = fmaf(co.R[0], hx[0], fmaf(co.R[1], hx[1], fmaf(co.R[2], hx[2], dP0)));
        dP1 = fmaf(co.R[3], hx[0], fmaf(co.R[4], hx[1], fmaf(co.R[5], hx[2], dP1)));
        dP2 = fmaf(co.R[6], hx[0], fmaf(co.R[7], hx[1], fmaf(co.R[8], hx[2], dP2)));
        const float fn2 = co.f * g.n2;
        const float ci = fmaf(g.s, d[6], fmaf(fn2, d[7], fn2 * g.n2 * d[8]));
        float t0, t1;
        apply_A(g, dP0, dP1, dP2, t0, t1);
        t0 = fmaf(ci, g.p[0], t0);
        t1 = fmaf(ci, g.p[1], t1);
        ljh += (double)fmaf(t0, t0, t1 * t1);
    }
    double fs;
    bsum2d(lf, ljh, sh, fs, jh2);
    double unused;
    bsum2d(lgh, 0.0, sh, gh, unused);
    Fn = 0.5 * fs;
}

}  // namespace

// MINB = resident CTAs per SM the register allocation must allow (a register cap of
// 65536 / (TB * MINB)); the linearisation may then spill a little, the PCG loop not.
// SP: point parameters and directions staged in shared memory during PCG.
template <int TB, int MINB, bool SP>
__global__ void __launch_bounds__(TB, MINB) k_batch_solve(BatchView b) {
    extern __shared__ __align__(16) unsigned char smem[];
    Shm S;
    S.cam = reinterpret_cast<float*>(smem);
    S.dir = S.cam + SCAM * b.cam_cap;
    S.acc = S.dir + SDIR * b.cam_cap;
    S.rc = S.acc + SACC * b.cam_cap;
    S.zc = S.rc + 9 * b.cam_cap;
    S.hc = S.zc + 9 * b.cam_cap;
    S.pc = S.hc + 9 * b.cam_cap;
    S.dc = S.pc + 9 * b.cam_cap;
    S.jl = S.dc + 9 * b.cam_cap;
    S.q = S.jl + 9 * b.cam_cap;
    S.x = S.q + 3 * b.pt_cap;
    S.p = S.x + 3 * b.pt_cap;
    float* sCam = S.cam;
    float* sDir = S.dir;
    __shared__ double sh[64];
    __shared__ int s_q;
    const DevOptions& o = b.opt;
    const float eps = (float)o.eps;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_q = (int)atomicAdd(b.queue, 1u);
        __syncthreads();
        const int slot = s_q;
        __syncthreads();
        if (slot >= b.n_problems) break;
        const int q = b.order[slot];
        const Prob P = load_prob(b, q);
        const int n = 9 * P.nc + 3 * P.np;
        b_camera_records(b, P, b.x, b.cam_pre, true);
        __syncthreads();
        double F = b_linearize(b, P, eps, sh);
        const double F0 = F;
        double mu = o.mu0, nu = 2.0;
        int it = 0, n_acc = 0, pcg_total = 0, status = isfinite(F) ? 0 : 4;
        bool active = status == 0 && F > 0.0 && o.max_lm > 0;
        while (active) {
            double rz, rr0;
            b_precond(b, P, mu, sh, rz, rr0);
            for (int i = tid; i < SCAM * P.nc; i += TB)   // camera records of x for the products
                sCam[i] = b.cam_pre[(size_t)(P.c0 + i / SCAM) * CP_STRIDE + i % SCAM];
            __syncthreads();
            pcg_total += b_pcg<TB, SP>(b, P, mu, rz, rr0, S, sh, status);
            double Fn, jh2, gh;
            b_candidate<TB>(b, P, sCam, sDir, sh, Fn, jh2, gh);
            // LM decision (Madsen): the same rule as the single-problem solver
            const double L = -gh - 0.5 * jh2;
            const double rho = L > 0.0 ? (F - Fn) / L : -1.0;
            const bool acc = isfinite(Fn) && L > 0.0 && rho > 0.0;
            ++it;
            if (acc) {
                const double t = 2.0 * rho - 1.0;
                mu *= fmax(1.0 / 3.0, 1.0 - t * t * t);
                nu = 2.0;
                F = Fn;
                ++n_acc;
            } else {
                mu *= nu;
                nu *= 2.0;
            }
            active = it < o.max_lm && mu <= o.max_mu && F > 0.0 && status == 0;
            if (acc) {   // every thread took the same decision from the same sums
                float* x = b.x + P.v0;
                const float* xn = b.x_new + P.v0;
                for (int e = tid; e < n; e += TB) x[e] = xn[e];
                if (active) {
                    __syncthreads();
                    b_camera_records(b, P, b.x, b.cam_pre, true);
                    __syncthreads();
                    F = b_linearize(b, P, eps, sh);
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            BatchStats s;
            s.initial_cost = F0;
            s.final_cost = F;
            s.lm_iters = it;
            s.accepted = n_acc;
            s.pcg_iters = pcg_total;
            s.status = status;
            b.stats[q] = s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ ordering -----

// Key of every observation for the camera-major order: (problem, camera, rotated
// point).  Within a camera's run the points start from a camera-dependent offset, so
// threads walking different cameras' runs in step touch different points.
constexpr uint32_t PT_ROTATION = 89;

__device__ __forceinline__ uint32_t rot_pt(uint32_t pt, uint32_t cam, uint32_t np) {
    return (uint32_t)((pt + (uint64_t)PT_ROTATION * cam) % np);
}

__device__ __forceinline__ uint32_t unrot_pt(uint32_t rpt, uint32_t cam, uint32_t np) {
    return (uint32_t)((rpt + np - ((uint64_t)PT_ROTATION * cam) % np) % np);
}

__global__ void k_batch_keys(const uint32_t* cam_loc, const uint32_t* pt_loc, const int32_t* obs_prob,
                             const int32_t* pt_off, int64_t n_obs, size_t sort_n, uint64_t* keys, uint32_t* vals) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < sort_n; o += (size_t)gridDim.x * blockDim.x) {
        if (o < (size_t)n_obs) {
            const int32_t q = obs_prob[o];
            const uint32_t np = (uint32_t)(pt_off[q + 1] - pt_off[q]);
            keys[o] = ((uint64_t)q << 40) | ((uint64_t)cam_loc[o] << 16) | (uint64_t)rot_pt(pt_loc[o], cam_loc[o], np);
            vals[o] = (uint32_t)o;
        } else {
            keys[o] = ~0ull;
            vals[o] = 0xffffffffu;
        }
    }
}

__global__ void k_batch_gather(const uint64_t* keys, const uint32_t* vals, const double* pixels, const int32_t* pt_off,
                               int64_t n_obs, uint32_t* obs_key, float* obs_uv) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_obs; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[j];
        const uint32_t o = vals[j];
        const int32_t q = (int32_t)(k >> 40);
        const uint32_t np = (uint32_t)(pt_off[q + 1] - pt_off[q]);
        const uint32_t cam = (uint32_t)((k >> 16) & 0xffffu);
        obs_key[j] = (cam << 16) | unrot_pt((uint32_t)(k & 0xffffu), cam, np);   // local camera << 16 | local point
        obs_uv[2 * j] = (float)pixels[2 * (size_t)o];
        obs_uv[2 * j + 1] = (float)pixels[2 * (size_t)o + 1];
    }
}

// Point-major keys: (global point, position in the camera-major order).
__global__ void k_batch_pm_keys(const uint32_t* vals, const uint32_t* pt_loc, const int32_t* obs_prob,
                                const int32_t* pt_off, int64_t n_obs, size_t sort_n, uint64_t* keys) {
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < sort_n; j += (size_t)gridDim.x * blockDim.x) {
        if (j < (size_t)n_obs) {
            const uint32_t o = vals[j];
            const uint64_t gp = (uint64_t)(pt_off[obs_prob[o]] + (int32_t)pt_loc[o]);
            keys[j] = (gp << 32) | (uint64_t)j;
        } else {
            keys[j] = ~0ull;
        }
    }
}

__global__ void k_batch_pm_finish(const uint64_t* keys, int64_t n_obs, int total_pts, uint32_t* pm_pos,
                                  uint32_t* pt_obs_off) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_obs; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[k];
        pm_pos[k] = (uint32_t)(key & 0xffffffffu);
        const uint32_t gp = (uint32_t)(key >> 32);
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != gp) pt_obs_off[gp] = (uint32_t)k;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) pt_obs_off[total_pts] = (uint32_t)n_obs;
}

// Host FP64 AoS parameters (staged on the device) <-> the per-problem FP32 vectors.
__global__ void k_batch_pack(BatchView b, const int32_t* cam_prob, const int32_t* pt_prob, int total_cams,
                             int total_pts, double* cams, double* pts, int to_device) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_cams + total_pts; i += gridDim.x * blockDim.x) {
        if (i < total_cams) {
            const int q = cam_prob[i];
            const int64_t e = b.vec_off[q] + 9 * (int64_t)(i - b.cam_off[q]);
            for (int k = 0; k < 9; ++k) {
                if (to_device) b.x[e + k] = (float)cams[9 * (size_t)i + k];
                else cams[9 * (size_t)i + k] = (double)b.x[e + k];
            }
        } else {
            const int u = i - total_cams;
            const int q = pt_prob[u];
            const int64_t e = b.vec_off[q] + 9 * (int64_t)(b.cam_off[q + 1] - b.cam_off[q]) + 3 * (int64_t)(u - b.pt_off[q]);
            for (int k = 0; k < 3; ++k) {
                if (to_device) b.x[e + k] = (float)pts[3 * (size_t)u + k];
                else pts[3 * (size_t)u + k] = (double)b.x[e + k];
            }
        }
    }
}

}  // namespace gbba

// ------------------------------------------------------------------ host ----------

using namespace gbba;

struct ba_batch {
    int32_t P = 0, total_cams = 0, total_pts = 0, max_nc = 0, max_np = 0;
    int64_t n_obs = 0, n_vec = 0;
    std::vector<int32_t> cam_off, pt_off, order, cam_prob, pt_prob, obs_prob;
    std::vector<int64_t> obs_off, vec_off;
    std::vector<uint32_t> cam_idx, pt_idx;
    std::vector<double> pixels;
    size_t total = 0;
    size_t o_order, o_cam_off, o_pt_off, o_obs_off, o_vec_off, o_cam_prob, o_pt_prob, o_obs_prob, o_key, o_uv, o_pm,
        o_pto, o_vec[9], o_cpre, o_cpre_new, o_cg, o_cH, o_Mc, o_pH, o_Mp, o_stats, o_queue, o_stage;
    size_t o_s_cam, o_s_pt, o_s_px, o_s_keys, o_s_vals, sort_cap;
    char* ws = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;
    BatchView view{};
    int tb = 256, cps = 0, grid = 0;   // threads per CTA, CTAs per SM (0 = occupancy limit), CTAs
    bool sp = false;                   // points staged in shared memory
    size_t smem = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    DevOptions graph_opt{};
    int graph_tb = 0, graph_cps = -1, graph_grid = 0;
    bool graph_sp = false;
};

namespace {

inline size_t al(size_t x) { return (x + 255) / 256 * 256; }

void batch_layout(ba_batch* B) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = al(o);
        o = r + bytes;
        return r;
    };
    const size_t P = (size_t)B->P, nc = (size_t)B->total_cams, np = (size_t)B->total_pts, no = (size_t)B->n_obs;
    B->o_order = take(4 * P);
    B->o_cam_off = take(4 * (P + 1));
    B->o_pt_off = take(4 * (P + 1));
    B->o_obs_off = take(8 * (P + 1));
    B->o_vec_off = take(8 * (P + 1));
    B->o_cam_prob = take(4 * nc);
    B->o_pt_prob = take(4 * np);
    B->o_obs_prob = take(4 * no);
    B->o_key = take(4 * no);
    B->o_uv = take(8 * no);
    B->o_pm = take(4 * no);
    B->o_pto = take(4 * (np + 1));
    for (auto& v : B->o_vec) v = take(4 * (size_t)B->n_vec);   // x x_new h r z p g D, x snapshot
    B->o_cpre = take(4 * CP_STRIDE * nc);
    B->o_cpre_new = take(4 * CP_STRIDE * nc);
    B->o_cg = take(8 * CL_STRIDE * nc);
    B->o_cH = take(4 * CH_STRIDE * nc);
    B->o_Mc = take(4 * 81 * nc);
    B->o_pH = take(4 * 6 * np);
    B->o_Mp = take(4 * 6 * np);
    B->o_stats = take(sizeof(BatchStats) * P);
    B->o_queue = take(256);
    B->o_stage = take(8 * (9 * nc + 3 * np));
    // ordering scratch, used only while binding: overlaps the solver vectors
    size_t s = B->o_vec[0];
    auto take_s = [&](size_t bytes) {
        const size_t r = al(s);
        s = r + bytes;
        return r;
    };
    size_t cap = 2;
    while (cap < no) cap <<= 1;
    B->sort_cap = cap;
    B->o_s_cam = take_s(4 * no);
    B->o_s_pt = take_s(4 * no);
    B->o_s_px = take_s(16 * no);
    B->o_s_keys = take_s(8 * cap);
    B->o_s_vals = take_s(4 * cap);
    B->total = al(std::max(o, s));
}

// Dynamic shared memory of one CTA: per camera of the largest problem its record,
// direction record, sums, camera block of r z h p D and J_l; per point q, and with
// staged points also X and p.
size_t batch_smem_bytes(const ba_batch* B, bool sp) {
    return 4 * (size_t)(SCAM + SDIR + SACC + 6 * 9) * B->max_nc + 4 * (sp ? 9 : 3) * (size_t)B->max_np;
}

typedef void (*BatchKernel)(BatchView);

// Compiled variants.  Global-memory points: 128 threads (register cap for 3 CTAs per
// SM), 256 threads with the whole register file for one CTA or capped for two, 512
// threads.  Staged points: 256 threads (one or two CTAs per SM) and 512 threads.
BatchKernel batch_kernel(int tb, int cps, bool sp) {
    if (sp) {
        if (tb == 512) return k_batch_solve<512, 1, true>;
        return cps == 1 ? k_batch_solve<256, 1, true> : k_batch_solve<256, 2, true>;
    }
    if (tb == 128) return k_batch_solve<128, 3, false>;
    if (tb == 512) return k_batch_solve<512, 1, false>;
    return cps == 1 ? k_batch_solve<256, 1, false> : k_batch_solve<256, 2, false>;
}

bool schedule_valid(int tb, bool sp) { return sp ? (tb == 256 || tb == 512) : (tb == 128 || tb == 256 || tb == 512); }

bool smem_fits(const ba_batch* B, bool sp) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return batch_smem_bytes(B, sp) + 1024 <= (size_t)optin;   // 1 KiB for the static shared arrays
}

cudaError_t batch_occupancy(const ba_batch* B, int tb, int cps, bool sp, int* sms, int* bps) {
    const size_t smem = batch_smem_bytes(B, sp);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    const BatchKernel k = batch_kernel(tb, cps, sp);
    if (e == cudaSuccess) e = ensure_dynamic_smem((const void*)k, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, tb, smem);
    return e;
}

cudaError_t batch_configure(ba_batch* B, int tb, int cps, bool sp) {
    int sms = 0, bps = 0;
    cudaError_t e = batch_occupancy(B, tb, cps, sp, &sms, &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = cps > 0 ? std::min(cps, bps) : bps;
    B->tb = tb;
    B->cps = cps;
    B->sp = sp;
    B->smem = batch_smem_bytes(B, sp);
    B->grid = std::max(1, std::min(B->P, sms * per_sm));
    return cudaSuccess;
}

void batch_enqueue(ba_batch* B, cudaStream_t s) {
    cudaMemsetAsync(B->view.queue, 0, sizeof(unsigned int), s);
    batch_kernel(B->tb, B->cps, B->sp)<<<B->grid, B->tb, B->smem, s>>>(B->view);
}

DevOptions dev_options(const ba_options* o) {
    DevOptions d{};
    d.max_lm = o->max_lm_iters;
    d.max_pcg = o->max_pcg_iters;
    d.tol = o->pcg_rel_tol;
    d.mu0 = 1.0 / o->initial_trust_region;
    d.min_diag = o->min_diag;
    d.max_diag = o->max_diag;
    d.max_mu = std::min(o->max_mu, 1e16);   // FP32 PCG vectors ~ g / (mu D): squares underflow past ~1e19
    d.eps = o->eps_depth;
    d.retract = o->rotation_update;
    return d;
}

bool options_ok(const ba_options* o) {
    return o && o->max_lm_iters >= 0 && o->max_pcg_iters >= 0 && o->initial_trust_region > 0 && o->min_diag > 0 &&
           o->max_diag >= o->min_diag && o->pcg_rel_tol >= 0 && o->eps_depth >= 0 && o->max_mu > 0 &&
           (o->rotation_update == 0 || o->rotation_update == 1) && o->loss == 0 && o->solver == 0;
}

// Launch of the solve: a captured graph (queue reset + persistent kernel), rebuilt
// when the options or the schedule change since both are baked into the launch.
ba_status batch_launch(ba_batch* B, const DevOptions& d, int use_graph) {
    B->view.opt = d;
    if (!use_graph) {
        batch_enqueue(B, B->stream);
        GBBA_CUDA(cudaGetLastError());
        return BA_OK;
    }
    const bool same = B->exec && B->graph_tb == B->tb && B->graph_cps == B->cps && B->graph_sp == B->sp &&
                      B->graph_grid == B->grid &&
                      memcmp(&B->graph_opt, &d, sizeof(d)) == 0;
    if (!same) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
        cudaStream_t cs;
        GBBA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            batch_enqueue(B, cs);
            e = cudaStreamEndCapture(cs, &B->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_status(e, "batch graph");
        B->graph_opt = d;
        B->graph_tb = B->tb;
        B->graph_cps = B->cps;
        B->graph_sp = B->sp;
        B->graph_grid = B->grid;
    }
    GBBA_CUDA(cudaGraphLaunch(B->exec, B->stream));
    return BA_OK;
}

struct TunedSchedule {
    int tb, cps;
    bool sp;
};
std::mutex g_tune_mutex;
std::map<std::string, TunedSchedule> g_tune_cache;

std::string tune_key(const ba_batch* B, const DevOptions& d) {
    int dev = 0;
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|P=%d|obs=%lld|cams=%d|pts=%d|maxc=%d|maxp=%d|lm=%d|pcg=%d|tol=%g", prop.name,
                  B->P, (long long)B->n_obs, B->total_cams, B->total_pts, B->max_nc, B->max_np, d.max_lm, d.max_pcg,
                  d.tol);
    return buf;
}

}  // namespace

extern "C" {

ba_status ba_batch_create(int32_t n_problems, const int32_t* cam_off, const int32_t* pt_off, const int64_t* obs_off,
                          const uint32_t* cam_idx, const uint32_t* pt_idx, const double* pixels, ba_batch** out) {
    if (!out) {
        set_error("ba_batch_create: out is null");
        return BA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n_problems < 1 || !cam_off || !pt_off || !obs_off || !cam_idx || !pt_idx || !pixels) {
        set_error("ba_batch_create: need n_problems >= 1 and non-null arrays");
        return BA_ERR_INVALID_ARG;
    }
    if (cam_off[0] != 0 || pt_off[0] != 0 || obs_off[0] != 0) {
        set_error("ba_batch_create: offset arrays must start at 0");
        return BA_ERR_INVALID_ARG;
    }
    for (int q = 0; q < n_problems; ++q) {
        const int nc = cam_off[q + 1] - cam_off[q], np = pt_off[q + 1] - pt_off[q];
        const int64_t no = obs_off[q + 1] - obs_off[q];
        if (nc < 1 || nc > BA_BATCH_MAX_CAMS || np < 1 || np > BA_BATCH_MAX_PTS || no < 1) {
            set_error("ba_batch_create: problem %d has %d cameras, %d points, %lld observations (limits: 1..%d "
                      "cameras, 1..%d points, >= 1 observation)", q, nc, np, (long long)no, BA_BATCH_MAX_CAMS,
                      BA_BATCH_MAX_PTS);
            return BA_ERR_INVALID_ARG;
        }
    }
    const int64_t n_obs = obs_off[n_problems];
    const int64_t total_pts = pt_off[n_problems];
    if (n_obs >= (int64_t)0x7fffffffLL || total_pts >= (int64_t)0x7fffffffLL) {
        set_error("ba_batch_create: too many observations or points in total");
        return BA_ERR_INVALID_ARG;
    }
    ba_batch* B = new (std::nothrow) ba_batch();
    if (!B) {
        set_error("ba_batch_create: out of host memory");
        return BA_ERR_INVALID_ARG;
    }
    B->P = n_problems;
    B->cam_off.assign(cam_off, cam_off + n_problems + 1);
    B->pt_off.assign(pt_off, pt_off + n_problems + 1);
    B->obs_off.assign(obs_off, obs_off + n_problems + 1);
    B->total_cams = cam_off[n_problems];
    B->total_pts = pt_off[n_problems];
    B->n_obs = n_obs;
    B->cam_idx.assign(cam_idx, cam_idx + n_obs);
    B->pt_idx.assign(pt_idx, pt_idx + n_obs);
    B->pixels.assign(pixels, pixels + 2 * n_obs);
    B->vec_off.resize(n_problems + 1);
    B->vec_off[0] = 0;
    B->obs_prob.resize(n_obs);
    B->cam_prob.resize(B->total_cams);
    B->pt_prob.resize(B->total_pts);
    std::vector<uint32_t> deg;
    for (int q = 0; q < n_problems; ++q) {
        const int nc = cam_off[q + 1] - cam_off[q], np = pt_off[q + 1] - pt_off[q];
        B->max_nc = std::max(B->max_nc, nc);
        B->max_np = std::max(B->max_np, np);
        B->vec_off[q + 1] = B->vec_off[q] + 9 * nc + 3 * np;
        for (int c = cam_off[q]; c < cam_off[q + 1]; ++c) B->cam_prob[c] = q;
        for (int u = pt_off[q]; u < pt_off[q + 1]; ++u) B->pt_prob[u] = q;
        deg.assign(np, 0);
        for (int64_t o = obs_off[q]; o < obs_off[q + 1]; ++o) {
            B->obs_prob[o] = q;
            if (cam_idx[o] >= (uint32_t)nc || pt_idx[o] >= (uint32_t)np) {
                set_error("ba_batch_create: observation %lld of problem %d has a local index out of range",
                          (long long)o, q);
                delete B;
                return BA_ERR_INVALID_ARG;
            }
            deg[pt_idx[o]] += 1;
        }
        for (int u = 0; u < np; ++u)
            if (deg[u] < 2) {
                set_error("ba_batch_create: point %d of problem %d is observed fewer than twice", u, q);
                delete B;
                return BA_ERR_INVALID_ARG;
            }
    }
    B->n_vec = B->vec_off[n_problems];
    // largest problems first: the work queue then ends on short problems
    B->order.resize(n_problems);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b2) {
        return (obs_off[a + 1] - obs_off[a]) > (obs_off[b2 + 1] - obs_off[b2]);
    });
    batch_layout(B);
    *out = B;
    return BA_OK;
}

void ba_batch_destroy(ba_batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    delete B;
}

ba_status ba_batch_workspace_size(const ba_batch* B, size_t* bytes) {
    if (!B || !bytes) {
        set_error("ba_batch_workspace_size: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    *bytes = B->total;
    return BA_OK;
}

ba_status ba_batch_bind_workspace(ba_batch* B, void* ws, size_t bytes, void* stream) {
    if (!B || !ws) {
        set_error("ba_batch_bind_workspace: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    if (((uintptr_t)ws & 255u) != 0) {
        set_error("ba_batch_bind_workspace: workspace must be 256-byte aligned");
        return BA_ERR_INVALID_ARG;
    }
    if (bytes < B->total) {
        set_error("ba_batch_bind_workspace: workspace has %zu bytes, needs %zu", bytes, B->total);
        return BA_ERR_WORKSPACE_TOO_SMALL;
    }
    if (!smem_fits(B, false)) {
        set_error("ba_batch_bind_workspace: the largest problem needs %zu bytes of shared memory, more than one CTA "
                  "may use", batch_smem_bytes(B, false));
        return BA_ERR_INVALID_ARG;
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->bound = false;
    B->ws = (char*)ws;
    B->stream = (cudaStream_t)stream;
    char* w = B->ws;
    cudaStream_t s = B->stream;
    auto up = [&](size_t off, const void* src, size_t n) {
        return cudaMemcpyAsync(w + off, src, n, cudaMemcpyHostToDevice, s);
    };
    GBBA_CUDA(up(B->o_order, B->order.data(), 4 * B->order.size()));
    GBBA_CUDA(up(B->o_cam_off, B->cam_off.data(), 4 * B->cam_off.size()));
    GBBA_CUDA(up(B->o_pt_off, B->pt_off.data(), 4 * B->pt_off.size()));
    GBBA_CUDA(up(B->o_obs_off, B->obs_off.data(), 8 * B->obs_off.size()));
    GBBA_CUDA(up(B->o_vec_off, B->vec_off.data(), 8 * B->vec_off.size()));
    GBBA_CUDA(up(B->o_cam_prob, B->cam_prob.data(), 4 * B->cam_prob.size()));
    GBBA_CUDA(up(B->o_pt_prob, B->pt_prob.data(), 4 * B->pt_prob.size()));
    GBBA_CUDA(up(B->o_obs_prob, B->obs_prob.data(), 4 * B->obs_prob.size()));
    GBBA_CUDA(up(B->o_s_cam, B->cam_idx.data(), 4 * B->cam_idx.size()));
    GBBA_CUDA(up(B->o_s_pt, B->pt_idx.data(), 4 * B->pt_idx.size()));
    GBBA_CUDA(up(B->o_s_px, B->pixels.data(), 8 * B->pixels.size()));
    // (problem, camera, rotated point) order, then the point-major index, sorted on the device
    uint64_t* keys = (uint64_t*)(w + B->o_s_keys);
    uint32_t* vals = (uint32_t*)(w + B->o_s_vals);
    const int TB = 256;
    const int gb = (int)std::min<size_t>(8192, (B->sort_cap + TB - 1) / TB);
    k_batch_keys<<<gb, TB, 0, s>>>((const uint32_t*)(w + B->o_s_cam), (const uint32_t*)(w + B->o_s_pt),
                                   (const int32_t*)(w + B->o_obs_prob), (const int32_t*)(w + B->o_pt_off), B->n_obs,
                                   B->sort_cap, keys, vals);
    sort_pairs(keys, vals, B->sort_cap, s);
    k_batch_gather<<<gb, TB, 0, s>>>(keys, vals, (const double*)(w + B->o_s_px), (const int32_t*)(w + B->o_pt_off),
                                     B->n_obs, (uint32_t*)(w + B->o_key), (float*)(w + B->o_uv));
    k_batch_pm_keys<<<gb, TB, 0, s>>>(vals, (const uint32_t*)(w + B->o_s_pt), (const int32_t*)(w + B->o_obs_prob),
                                      (const int32_t*)(w + B->o_pt_off), B->n_obs, B->sort_cap, keys);
    sort_pairs(keys, vals, B->sort_cap, s);
    k_batch_pm_finish<<<gb, TB, 0, s>>>(keys, B->n_obs, B->total_pts, (uint32_t*)(w + B->o_pm),
                                        (uint32_t*)(w + B->o_pto));
    GBBA_CUDA(cudaGetLastError());
    const size_t vb = B->o_vec[0];
    GBBA_CUDA(cudaMemsetAsync(w + vb, 0, B->o_stats + sizeof(BatchStats) * B->P - vb, s));
    GBBA_CUDA(cudaStreamSynchronize(s));
    BatchView& v = B->view;
    v.n_problems = B->P;
    v.cam_cap = B->max_nc;
    v.pt_cap = B->max_np;
    v.order = (const int32_t*)(w + B->o_order);
    v.cam_off = (const int32_t*)(w + B->o_cam_off);
    v.pt_off = (const int32_t*)(w + B->o_pt_off);
    v.obs_off = (const int64_t*)(w + B->o_obs_off);
    v.vec_off = (const int64_t*)(w + B->o_vec_off);
    v.obs_key = (const uint32_t*)(w + B->o_key);
    v.obs_uv = (const float*)(w + B->o_uv);
    v.pm_pos = (const uint32_t*)(w + B->o_pm);
    v.pt_obs_off = (const uint32_t*)(w + B->o_pto);
    float** vecs[8] = {&v.x, &v.x_new, &v.h, &v.r, &v.z, &v.p, &v.g, &v.D};
    for (int i = 0; i < 8; ++i) *vecs[i] = (float*)(w + B->o_vec[i]);
    v.cam_pre = (float*)(w + B->o_cpre);
    v.cam_pre_new = (float*)(w + B->o_cpre_new);
    v.cam_g = (double*)(w + B->o_cg);
    v.cam_H = (float*)(w + B->o_cH);
    v.Minv_c = (float*)(w + B->o_Mc);
    v.pt_H = (float*)(w + B->o_pH);
    v.Minv_p = (float*)(w + B->o_Mp);
    v.stats = (BatchStats*)(w + B->o_stats);
    v.queue = (unsigned int*)(w + B->o_queue);
    // default schedule: staged points with 512 threads when they fit, else 256 threads
    if (smem_fits(B, true)) {
        GBBA_CUDA(batch_configure(B, 512, 0, true));
    } else {
        GBBA_CUDA(batch_configure(B, 256, 0, false));
    }
    B->bound = true;
    return BA_OK;
}

static ba_status batch_params(ba_batch* B, double* cams, double* pts, int to_device) {
    if (!B || !B->bound) {
        set_error("batch: no workspace bound");
        return BA_ERR_STATE;
    }
    if (!cams || !pts) {
        set_error("batch: null parameter array");
        return BA_ERR_INVALID_ARG;
    }
    char* w = B->ws;
    double* stg = (double*)(w + B->o_stage);
    const size_t nc9 = 9 * (size_t)B->total_cams, np3 = 3 * (size_t)B->total_pts;
    cudaStream_t s = B->stream;
    if (to_device) {
        GBBA_CUDA(cudaMemcpyAsync(stg, cams, 8 * nc9, cudaMemcpyHostToDevice, s));
        GBBA_CUDA(cudaMemcpyAsync(stg + nc9, pts, 8 * np3, cudaMemcpyHostToDevice, s));
    }
    const int items = B->total_cams + B->total_pts;
    k_batch_pack<<<std::max(1, std::min(8192, (items + 255) / 256)), 256, 0, s>>>(
        B->view, (const int32_t*)(w + B->o_cam_prob), (const int32_t*)(w + B->o_pt_prob), B->total_cams,
        B->total_pts, stg, stg + nc9, to_device);
    GBBA_CUDA(cudaGetLastError());
    if (!to_device) {
        GBBA_CUDA(cudaMemcpyAsync(cams, stg, 8 * nc9, cudaMemcpyDeviceToHost, s));
        GBBA_CUDA(cudaMemcpyAsync(pts, stg + nc9, 8 * np3, cudaMemcpyDeviceToHost, s));
    }
    GBBA_CUDA(cudaStreamSynchronize(s));   // the staging buffer is reused by the next call
    return BA_OK;
}

ba_status ba_batch_set_params(ba_batch* B, const double* cams, const double* pts) {
    return batch_params(B, const_cast<double*>(cams), const_cast<double*>(pts), 1);
}

ba_status ba_batch_get_params(ba_batch* B, double* cams, double* pts) { return batch_params(B, cams, pts, 0); }

static ba_status read_stats(ba_batch* B, std::vector<BatchStats>& hs) {
    hs.resize((size_t)B->P);
    GBBA_CUDA(cudaMemcpyAsync(hs.data(), B->view.stats, sizeof(BatchStats) * hs.size(), cudaMemcpyDeviceToHost,
                              B->stream));
    GBBA_CUDA(cudaStreamSynchronize(B->stream));
    return BA_OK;
}

ba_status ba_batch_solve(ba_batch* B, const ba_options* o, ba_stats* stats) {
    if (!B || !B->bound) {
        set_error("ba_batch_solve: no workspace bound");
        return BA_ERR_STATE;
    }
    if (o && (o->loss != 0 || o->solver != 0)) {
        set_error("ba_batch_solve: robust losses and the Schur-complement solver are not available in the batched mode");
        return BA_ERR_NOT_IMPLEMENTED;
    }
    if (!options_ok(o)) {
        set_error("ba_batch_solve: invalid options");
        return BA_ERR_INVALID_ARG;
    }
    ba_status st = batch_launch(B, dev_options(o), o->use_graph);
    if (st != BA_OK || !stats) return st;
    std::vector<BatchStats> hs;
    st = read_stats(B, hs);
    if (st != BA_OK) return st;
    for (int q = 0; q < B->P; ++q) {
        stats[q].initial_cost = hs[q].initial_cost;
        stats[q].final_cost = hs[q].final_cost;
        stats[q].lm_iters = hs[q].lm_iters;
        stats[q].accepted = hs[q].accepted;
        stats[q].pcg_iters_total = hs[q].pcg_iters;
        stats[q].status = hs[q].status;
        stats[q].solve_ns = 0;
    }
    return BA_OK;
}

ba_status ba_batch_get_costs(ba_batch* B, double* initial_costs, double* final_costs) {
    if (!B || !B->bound) {
        set_error("ba_batch_get_costs: no workspace bound");
        return BA_ERR_STATE;
    }
    std::vector<BatchStats> hs;
    ba_status st = read_stats(B, hs);
    if (st != BA_OK) return st;
    for (int q = 0; q < B->P; ++q) {
        if (initial_costs) initial_costs[q] = hs[q].initial_cost;
        if (final_costs) final_costs[q] = hs[q].final_cost;
    }
    return BA_OK;
}

ba_status ba_batch_set_schedule(ba_batch* B, int32_t threads, int32_t ctas_per_sm, int32_t flags) {
    if (!B || !B->bound) {
        set_error("ba_batch_set_schedule: no workspace bound");
        return BA_ERR_STATE;
    }
    const bool sp = (flags & BA_SCHED_STAGE_POINTS) != 0;
    if (!schedule_valid(threads, sp) || ctas_per_sm < 0 || (flags & ~BA_SCHED_STAGE_POINTS)) {
        set_error("ba_batch_set_schedule: threads must be 128, 256 or 512 (256 or 512 with staged points), "
                  "ctas_per_sm >= 0, flags a combination of BA_SCHED_*");
        return BA_ERR_INVALID_ARG;
    }
    if (sp && !smem_fits(B, true)) {
        set_error("ba_batch_set_schedule: staged points need %zu bytes of shared memory per CTA, more than allowed",
                  batch_smem_bytes(B, true));
        return BA_ERR_INVALID_ARG;
    }
    GBBA_CUDA(batch_configure(B, threads, ctas_per_sm, sp));
    return BA_OK;
}

ba_status ba_batch_get_schedule(const ba_batch* B, int32_t* threads, int32_t* ctas_per_sm, int32_t* flags,
                                int32_t* grid) {
    if (!B || !B->bound) {
        set_error("ba_batch_get_schedule: no workspace bound");
        return BA_ERR_STATE;
    }
    if (threads) *threads = B->tb;
    if (ctas_per_sm) *ctas_per_sm = B->cps;
    if (flags) *flags = B->sp ? BA_SCHED_STAGE_POINTS : 0;
    if (grid) *grid = B->grid;
    return BA_OK;
}

ba_status ba_batch_autotune(ba_batch* B, const ba_options* o, int32_t flags, ba_batch_trial* trials,
                            int32_t trial_cap, int32_t* n_trials) {
    if (!B || !B->bound) {
        set_error("ba_batch_autotune: no workspace bound");
        return BA_ERR_STATE;
    }
    if (!options_ok(o) || trial_cap < 0 || (trial_cap > 0 && !trials)) {
        set_error("ba_batch_autotune: invalid options or trial array");
        return BA_ERR_INVALID_ARG;
    }
    if (n_trials) *n_trials = 0;
    const DevOptions d = dev_options(o);
    const std::string key = tune_key(B, d);
    if (!(flags & BA_TUNE_IGNORE_CACHE)) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            GBBA_CUDA(batch_configure(B, it->second.tb, it->second.cps, it->second.sp));
            return BA_OK;
        }
    }
    // candidates: every compiled variant at each CTAs-per-SM count from 1 to its
    // occupancy limit, with and without staged points (where they fit)
    struct Cand {
        int tb, cps;
        bool sp;
    };
    std::vector<Cand> cand;
    const int variants[7][3] = {{128, 0, 0}, {256, 1, 0}, {256, 0, 0}, {512, 0, 0},
                                {256, 1, 1}, {256, 0, 1}, {512, 0, 1}};
    for (const auto& vr : variants) {
        const bool sp = vr[2] != 0;
        if (sp && !smem_fits(B, true)) continue;
        int sms = 0, bps = 0;
        GBBA_CUDA(batch_occupancy(B, vr[0], vr[1], sp, &sms, &bps));
        if (vr[1] == 1) {
            if (bps >= 1) cand.push_back({vr[0], 1, sp});
            continue;
        }
        for (int c = (vr[0] == 256 ? 2 : 1); c <= bps; ++c) cand.push_back({vr[0], c, sp});
    }
    if (cand.empty()) {
        set_error("ba_batch_autotune: no block size fits the shared-memory needs of this batch");
        return BA_ERR_INVALID_ARG;
    }
    // every trial solves from the same starting point: snapshot x, restore before each
    char* w = B->ws;
    float* x = B->view.x;
    float* x0 = (float*)(w + B->o_vec[8]);
    const size_t xb = 4 * (size_t)B->n_vec;
    GBBA_CUDA(cudaMemcpyAsync(x0, x, xb, cudaMemcpyDeviceToDevice, B->stream));
    cudaEvent_t e0, e1;
    GBBA_CUDA(cudaEventCreate(&e0));
    GBBA_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    int best_i = -1;
    ba_status st = BA_OK;
    for (size_t i = 0; i < cand.size() && st == BA_OK; ++i) {
        cudaError_t e = batch_configure(B, cand[i].tb, cand[i].cps, cand[i].sp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(x, x0, xb, cudaMemcpyDeviceToDevice, B->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, B->stream);
        if (e != cudaSuccess) {
            st = cuda_status(e, "autotune");
            break;
        }
        st = batch_launch(B, d, 0);
        if (st != BA_OK) break;
        e = cudaEventRecord(e1, B->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = cuda_status(e, "autotune");
            break;
        }
        if ((int32_t)i < trial_cap) {
            trials[i].threads = cand[i].tb;
            trials[i].ctas_per_sm = cand[i].cps;
            trials[i].flags = cand[i].sp ? BA_SCHED_STAGE_POINTS : 0;
            trials[i].grid = B->grid;
            trials[i].ms = ms;
        }
        if (n_trials) *n_trials = (int32_t)std::min<size_t>(i + 1, (size_t)trial_cap);
        if (best_i < 0 || ms < best) {
            best = ms;
            best_i = (int)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaMemcpyAsync(x, x0, xb, cudaMemcpyDeviceToDevice, B->stream);
    if (st != BA_OK) return st;
    GBBA_CUDA(e);
    GBBA_CUDA(cudaStreamSynchronize(B->stream));
    GBBA_CUDA(batch_configure(B, cand[best_i].tb, cand[best_i].cps, cand[best_i].sp));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = TunedSchedule{cand[best_i].tb, cand[best_i].cps, cand[best_i].sp};
    }
    return BA_OK;
}

}  // extern "C"
