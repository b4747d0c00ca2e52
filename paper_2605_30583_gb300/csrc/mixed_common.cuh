// Per-observation building blocks of the mixed-precision normal operator, shared by
// the multi-kernel path and the persistent PCG kernel.
#pragma once

#include "device_common.cuh"

namespace gbba {

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

// Warp sum of N per-lane values by recursive halving: at each of the five levels the two
// lanes of a pair (lane, lane ^ o) split the values they still carry, each keeping one
// half and adding the partner's copy of it (about 4 N + 10 instructions, where a
// butterfly of every value takes 10 N).  Every lane ends with split_sum_slots(N) values;
// the first `returned` of them are complete sums, v[k] of value idx + k, and together
// the lanes hold each of the N sums exactly once.
__host__ __device__ constexpr int split_sum_slots(int n) {
    return ((((((n + 1) / 2 + 1) / 2 + 1) / 2 + 1) / 2) + 1) / 2;
}

template <int N>
__device__ __forceinline__ int warp_split_sum(float (&v)[N], int lane, int& idx) {
    int m = N;    // values every lane carries (the same in all lanes)
    int rc = N;   // of which real (the rest pad the upper halves of odd splits)
    idx = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int h = (m + 1) / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < (N + 1) / 2; ++k) {
            if (k < h) {
                const float hi = (k + h < m) ? v[k + h] : 0.0f;
                const float send = up ? v[k] : hi;
                const float keep = up ? hi : v[k];
                v[k] = keep + __shfl_xor_sync(FULL, send, o);
            }
        }
        if (up) {
            idx += h;
            rc = rc > h ? rc - h : 0;
        } else {
            rc = rc < h ? rc : h;
        }
        m = h;
    }
    return rc;
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

// Observations per thread when a CTA of `threads` threads splits `n` of them into
// contiguous chunks, rounded up to an odd count.  A camera's run covers consecutive
// tile slots, so lanes inside one run sit `chunk` slots apart: an odd stride sends
// their float4 point loads to distinct bank groups and their three-float point
// accumulations to distinct banks, where an even one (16 is the worst) serialises
// up to 16 of them.
template <typename T>
__host__ __device__ __forceinline__ T odd_chunk(T n, T threads) {
    return ((n + threads - 1) / threads) | (T)1;
}

__device__ __forceinline__ bool gated_off(const int32_t* gate) { return gate != nullptr && *gate == 0; }


// Camera direction record of camera c for p_c = zs_c + beta p_prev_c: phi = J_l p_w,
// then p_t and the intrinsic part.  zs and p_prev may change between launches or
// grid-wide phases, so they are read through L2 (never stale in L1).
__device__ __forceinline__ void camera_dir(const Views<float>& v, uint32_t c, const float* __restrict__ zs,
                                           const float* __restrict__ pc_old, float beta, float (&dir)[9]) {
    float pcv[9];
    const size_t e = 9 * (size_t)c;
#pragma unroll
    for (int k = 0; k < 9; ++k) pcv[k] = beta != 0.0f ? fmaf(beta, __ldcg(pc_old + e + k), __ldcg(zs + e + k)) : __ldcg(zs + e + k);
    const float4* j4 = reinterpret_cast<const float4*>(v.cam_pre + (size_t)c * CP_STRIDE + CP_JL);
    const float4 a = __ldg(j4), b = __ldg(j4 + 1), cc = __ldg(j4 + 2);
    const float JL[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, cc.x};
#pragma unroll
    for (int i = 0; i < 3; ++i) dir[CD_PHI + i] = fmaf(JL[3 * i], pcv[0], fmaf(JL[3 * i + 1], pcv[1], JL[3 * i + 2] * pcv[2]));
#pragma unroll
    for (int k = 3; k < 9; ++k) dir[k] = pcv[k];
}

// Contribution of one observation to the normal operator: t = J d (returns |t|^2),
// camera sums (RX x u, u, intrinsic part) into acc, point part R^T u into qs (shared).
// WEIGHTED: the robust loss's IRLS weight w scales the observation's rows of J^T J
// (u = A^T (w t), returns w |t|^2).  PLAIN_Q: qs belongs to the calling warp alone and
// no other lane of it touches the same point in this step, so plain adds replace the
// shared-memory atomics.
template <bool WEIGHTED = false, bool PLAIN_Q = false>
__device__ __forceinline__ float obs_normal(const Cam& cam, const float (&dir)[9], const float* xs,
                                            const float* ds, float eps, float (&acc)[9], float* qs,
                                            float w = 1.0f) {
    const GeoLite g = project_lite(cam, xs[0], xs[1], xs[2], eps);
    // J d = A (phi x RX + d_t + R d_X) + c_i p
    float dP0 = fmaf(dir[1], g.RX[2], -dir[2] * g.RX[1]) + dir[CD_T + 0];
    float dP1 = fmaf(dir[2], g.RX[0], -dir[0] * g.RX[2]) + dir[CD_T + 1];
    float dP2 = fmaf(dir[0], g.RX[1], -dir[1] * g.RX[0]) + dir[CD_T + 2];
    dP0 = fmaf(cam.R[0], ds[0], fmaf(cam.R[1], ds[1], fmaf(cam.R[2], ds[2], dP0)));
    dP1 = fmaf(cam.R[3], ds[0], fmaf(cam.R[4], ds[1], fmaf(cam.R[5], ds[2], dP1)));
    dP2 = fmaf(cam.R[6], ds[0], fmaf(cam.R[7], ds[1], fmaf(cam.R[8], ds[2], dP2)));
    const float fn2 = cam.f * g.n2;
    const float ci = fmaf(g.s, dir[CD_I + 0], fmaf(fn2, dir[CD_I + 1], fn2 * g.n2 * dir[CD_I + 2]));
    float t0, t1;
    apply_A(g, dP0, dP1, dP2, t0, t1);
    t0 = fmaf(ci, g.p[0], t0);
    t1 = fmaf(ci, g.p[1], t1);
    const float tt = fmaf(t0, t0, t1 * t1);
    if (WEIGHTED) {
        t0 *= w;
        t1 *= w;
    }
    // adjoint: u = A^T t
    float u0, u1, u2;
    apply_At(g, t0, t1, u0, u1, u2);
    acc[0] += fmaf(g.RX[1], u2, -g.RX[2] * u1);
    acc[1] += fmaf(g.RX[2], u0, -g.RX[0] * u2);
    acc[2] += fmaf(g.RX[0], u1, -g.RX[1] * u0);
    acc[3] += u0;
    acc[4] += u1;
    acc[5] += u2;
    const float pt = fmaf(g.p[0], t0, g.p[1] * t1);
    acc[6] = fmaf(g.s, pt, acc[6]);
    acc[7] = fmaf(fn2, pt, acc[7]);
    acc[8] = fmaf(fn2 * g.n2, pt, acc[8]);
    const float q0 = fmaf(cam.R[0], u0, fmaf(cam.R[3], u1, cam.R[6] * u2));
    const float q1 = fmaf(cam.R[1], u0, fmaf(cam.R[4], u1, cam.R[7] * u2));
    const float q2 = fmaf(cam.R[2], u0, fmaf(cam.R[5], u1, cam.R[8] * u2));
    if (PLAIN_Q) {
        qs[0] += q0;
        qs[1] += q1;
        qs[2] += q2;
    } else {
        atomicAdd(qs + 0, q0);
        atomicAdd(qs + 1, q1);
        atomicAdd(qs + 2, q2);
    }
    return WEIGHTED ? w * tt : tt;
}

// One pose factor in the normal operator: t = J_f (d_a; d_b) over the (phi, t) parts of
// the two cameras' direction records, J_f^T t added to their camera sums (phi part to
// entries 0-2, translation part to 3-5, as the observations' sums); returns |t|^2.
__device__ __forceinline__ float factor_normal(const float* __restrict__ Jf, const float* da, const float* db,
                                               float* acc_a, float* acc_b) {
    const float x[12] = {da[CD_PHI], da[CD_PHI + 1], da[CD_PHI + 2], da[CD_T], da[CD_T + 1], da[CD_T + 2],
                         db[CD_PHI], db[CD_PHI + 1], db[CD_PHI + 2], db[CD_T], db[CD_T + 1], db[CD_T + 2]};
    float t[6], tt = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float ti = 0.0f;
#pragma unroll
        for (int j = 0; j < 12; ++j) ti = fmaf(__ldg(Jf + 12 * i + j), x[j], ti);
        t[i] = ti;
        tt = fmaf(ti, ti, tt);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float ga = 0.0f, gb = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            ga = fmaf(__ldg(Jf + 12 * i + j), t[i], ga);
            gb = fmaf(__ldg(Jf + 12 * i + 6 + j), t[i], gb);
        }
        atomicAdd(acc_a + j, ga);
        atomicAdd(acc_b + j, gb);
    }
    return tt;
}

}  // namespace gbba
