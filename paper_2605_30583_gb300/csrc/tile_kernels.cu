// Tile kernels of the mixed-precision form: the damped normal operator of the
// separate-kernel PCG, the linearisation and the candidate evaluation.
//
// Work decomposition.  A tile is TILE_PTS consecutive points (locality order) and all
// their observations.  Inside a tile each camera's observations form one run, and the
// runs of at least LONG_RUN observations come first (order.cu); on the large workloads
// they hold most of the observations.  A CTA stages in shared memory, in one round
// trip, the tile's points, its compact observation table (a one-byte point slot per long-run
// observation, the key of each short-run observation) and its table
// of long runs {start, length, camera}; then
//   * its warps take the long runs in turn and walk each in camera-uniform steps of 32
//     consecutive observations: the camera sits in registers for the whole run, and the
//     run's camera sums stay in per-lane
//     registers until the run ends, when one recursive-halving warp reduction
//     (warp_split_sum) hands each lane complete sums to add to the global camera
//     accumulators;
//   * its threads split the short runs that follow into contiguous chunks; a thread
//     reads a camera through L1 when its chunk enters the camera's run and adds its
//     camera sums to the global accumulators when it leaves it.
// Point sums go into shared memory (the tile owns its points) and are written once per
// tile.  This is our counterpart of the paper's Shared Read / Shared Add accessors
// (Sec. IV-A).  In the operator each warp adds its long runs' point sums into a copy of
// its own with plain adds (the points of one run are distinct, so no two lanes of a step
// meet), and the copies are summed when the tile is written; a problem with repeated
// (camera, point) observations keeps one copy and shared-memory atomics.
//
// Per-thread sums that feed FP64 reductions (|J p|^2, p^T D p, the cost) are kept in
// FP32 with Kahan's compensated summation, summed inside each warp in compensated FP32
// pairs and across warps and CTAs in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"
#include "mixed_common.cuh"

namespace gbba {

namespace {

struct TileRange {
    uint32_t lo, hi, l0, nl, ss;   // observations [lo, hi), long runs [l0, l0 + nl), short tail from ss
    int pt0, npt;
    size_t base;                   // the tile's first point entry in parameter vectors
};

__device__ __forceinline__ TileRange tile_range(const Views<float>& v, int tile) {
    TileRange r;
    r.lo = v.tile_off[tile];
    r.hi = v.tile_off[tile + 1];
    r.l0 = v.long_off[tile];
    r.nl = v.long_off[tile + 1] - r.l0;
    r.ss = v.short_start[tile];
    r.pt0 = tile * TILE_PTS;
    r.npt = min(TILE_PTS, v.n_pts - r.pt0);
    r.base = v.pt_off + 3 * (size_t)r.pt0;
    return r;
}

// Compact staging of a tile's observation table: sRun[3 r + k] of long run l0 + r, the
// point slot (one byte) of each long-run observation (its camera is in the run's table
// entry), and the whole key of each short-run observation.  `Caps` sizes the three
// regions for the largest tile of each kind.
struct Caps {
    int run, shrt, lng;   // long runs, short-run observations, long-run observations
};

__host__ __device__ __forceinline__ size_t compact_bytes(const Caps& c) {
    return 12 * (size_t)c.run + 4 * (size_t)c.shrt + (size_t)c.lng;
}

template <int TB>
__device__ __forceinline__ void stage_compact(const Views<float>& v, const TileRange& T, const Caps& cap,
                                              unsigned char* dsm, uint32_t*& sRun, uint32_t*& sShort,
                                              uint8_t*& sSlot) {
    sRun = reinterpret_cast<uint32_t*>(dsm);
    sShort = sRun + 3 * cap.run;
    sSlot = reinterpret_cast<uint8_t*>(sShort + cap.shrt);
    const uint32_t nlo = T.ss - T.lo, n = T.hi - T.lo;
    for (uint32_t i = threadIdx.x; i < n; i += TB) {
        const uint32_t key = __ldg(v.obs_key + T.lo + i);
        if (i < nlo) sSlot[i] = (uint8_t)(key & 0xffu);
        else sShort[i - nlo] = key;
    }
    for (uint32_t i = threadIdx.x; i < 3 * T.nl; i += TB) sRun[i] = __ldg(v.long_run + 3 * (size_t)T.l0 + i);
}


// Block sums of compensated per-thread partials (Kahan pairs s - c): FP32 pairs inside
// each warp, FP64 across the warps; valid in thread 0.  `sh` holds 2 * (TB / 32) doubles.
template <int TB>
__device__ __forceinline__ void block_pair_sums(float sa, float ca, float sb, float cb, double* sh, double& ra,
                                                double& rb) {
    block_sum2c(sa, ca, sb, cb, sh, ra, rb);
}

// ------------------------------------------------------------------ normal operator ---
// q = J^T W J p + mu D p for the tile's points (written), camera parts J^T W J p into the
// camera accumulators (k_update adds mu D p and applies J_l^T), |J p|^2 and the points'
// p^T D p into the slot sums (the cameras' p^T D p comes from k_cam_direction).  The
// points' direction step p = zs + beta p_prev is fused into the staging.  One CTA per
// tile.

// Eight CTAs per SM (at most 64 registers per thread; with per-warp point sums a CTA
// holds ~20 KB of static shared memory plus its compact observation table).
// PLAIN_Q: every warp keeps its own copy of the tile's point sums, added to with plain
// shared-memory adds (valid when no camera observes a point twice; see the file head).
// Replacing the point-sum atomics of the long runs this way took the operator from 302
// to 289 us on the 28.8M-observation workload.
template <int TB, bool PLAIN_Q>
__global__ void __launch_bounds__(TB, 8) k_tile_normal(Views<float> v, const int32_t* gate, const float* zs,
                                                       int use_beta, Caps cap) {
    if (gated_off(gate)) return;
    constexpr int NQ = PLAIN_Q ? TB / 32 : 1;   // point-sum copies
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float4 sX4[TILE_PTS], sP4[TILE_PTS];
    __shared__ float sQ[NQ * 3 * TILE_PTS];
    __shared__ unsigned int s_next;
    __shared__ double red[2 * (TB / 32)];
    DevState* st = v.st;
    const float beta = use_beta ? (float)st->beta : 0.0f;
    const float mu = (float)st->mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;
    const int lane = threadIdx.x & 31;
    const TileRange T = tile_range(v, blockIdx.x);
    float jp_s = 0.0f, jp_c = 0.0f, pd_s = 0.0f, pd_c = 0.0f;
    {
        // every load before the stores of p (which may alias them)
        static_assert((3 * TILE_PTS) % TB == 0, "whole entry steps");
        constexpr int EPT = 3 * TILE_PTS / TB;
        const int ne = 3 * T.npt;
        float* sPf = reinterpret_cast<float*>(sP4);
        float* sXf = reinterpret_cast<float*>(sX4);
        float Z[EPT], P[EPT], Dd[EPT], X[EPT];
#pragma unroll
        for (int t = 0; t < EPT; ++t) {
            const int i = threadIdx.x + t * TB;
            if (i < ne) {
                Z[t] = zs[T.base + i];
                P[t] = beta != 0.0f ? v.p[T.base + i] : 0.0f;
                Dd[t] = v.D[T.base + i];
                X[t] = v.x[T.base + i];
            }
        }
#pragma unroll
        for (int t = 0; t < EPT; ++t) {
            const int i = threadIdx.x + t * TB;
            if (i < ne) {
                const float pn = beta != 0.0f ? fmaf(beta, P[t], Z[t]) : Z[t];
                v.p[T.base + i] = pn;
                const int slot = i / 3, k = i - 3 * slot;
                sPf[4 * slot + k] = pn;
                sXf[4 * slot + k] = X[t];
                sQ[i] = mu * (Dd[t] * pn);
                kahan_add(pd_s, pd_c, Dd[t] * pn * pn);
            }
        }
    }
    for (int i = threadIdx.x; i < (NQ - 1) * 3 * TILE_PTS; i += TB) sQ[3 * TILE_PTS + i] = 0.0f;
    float* const sQw = sQ + (PLAIN_Q ? (threadIdx.x >> 5) * 3 * TILE_PTS : 0);   // this warp's copy
    uint32_t *sRun, *sShort;
    uint8_t* sSlot;
    stage_compact<TB>(v, T, cap, dsm, sRun, sShort, sSlot);
    if (threadIdx.x == 0) s_next = 0u;
    __syncthreads();
    // long runs: camera-uniform steps of 32 observations
    for (;;) {
        unsigned int r = 0;
        if (lane == 0) r = atomicAdd(&s_next, 1u);
        r = __shfl_sync(FULL, r, 0);
        if (r >= T.nl) break;
        const uint32_t start = sRun[3 * r] - T.lo, len = sRun[3 * r + 1], c = sRun[3 * r + 2];
        const Cam cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
        float dir[9];
        load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
        uint32_t off = lane;
        for (; off < len; off += 32) {
            const uint32_t j = T.lo + start + off;
            const uint32_t slot = sSlot[start + off];
            const float4 xp = sX4[slot], pp = sP4[slot];
            const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
            const float tt = weighted ? obs_normal<true, PLAIN_Q>(cam, dir, xs, ds, eps, acc, sQw + 3 * slot,
                                                                 __ldg(v.obs_w + j))
                                      : obs_normal<false, PLAIN_Q>(cam, dir, xs, ds, eps, acc, sQw + 3 * slot);
            kahan_add(jp_s, jp_c, tt);
        }
        if (PLAIN_Q) __syncwarp();   // the warp's next run may meet the same points
        int idx;
        const int nv = warp_split_sum<9>(acc, lane, idx);
        if (nv > 0) atomicAdd(v.cam_acc + (size_t)c * CA_STRIDE + idx, acc[0]);
    }
    // short runs: one contiguous chunk per thread
    {
        const uint32_t n = T.hi - T.ss;
        const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
        const uint32_t a = T.ss + min(threadIdx.x * chunk, n), b = T.ss + min(threadIdx.x * chunk + chunk, n);
        uint32_t cur = NO_CAM;
        float acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
        Cam cam;
        float dir[9];
        for (uint32_t j = a; j < b; ++j) {
            const uint32_t key = sShort[j - T.ss];
            const uint32_t c = key >> 8, slot = key & 0xffu;
            if (c != cur) {
                if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                cur = c;
                cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
            }
            const float4 xp = sX4[slot], pp = sP4[slot];
            const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
            // lanes of a warp may meet one point here: atomics (into the warp's copy)
            const float tt = weighted ? obs_normal<true>(cam, dir, xs, ds, eps, acc, sQw + 3 * slot, __ldg(v.obs_w + j))
                                      : obs_normal(cam, dir, xs, ds, eps, acc, sQw + 3 * slot);
            kahan_add(jp_s, jp_c, tt);
        }
        if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * T.npt; i += TB) {
        float qi = sQ[i];
#pragma unroll
        for (int w = 1; w < NQ; ++w) qi += sQ[w * 3 * TILE_PTS + i];
        v.q[T.base + i] = qi;
    }
    double bj, bp;
    block_pair_sums<TB>(jp_s, jp_c, pd_s, pd_c, red, bj, bp);
    if (threadIdx.x == 0) {
        slot_add(st->acc_mv, 0, bj);
        slot_add(st->acc_mv, 1, bp);
    }
}

constexpr int TN_TB = 128;

// ------------------------------------------------------- one-reduction PCG rounds ---
// The separate-kernel PCG with its recurrences arranged as in the CG of Chronopoulos and
// Gear (J. Comput. Appl. Math. 25, 1989): with u = M^-1 r, w = A u and s = A p carried by
// s = w + beta s, both inner products gamma = r^T u and delta = u^T A u = |J u|^2 +
// mu u^T D u of a round come from one reduction, and each round applies the previous
// round's update before its operator:
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev),
//   p = u + beta p,  s = w + beta s,  h += alpha p,  r -= alpha s,  u = M^-1 r.
// Round k (st->pcg_iter = k) runs k_cg_cameras (the cameras' update k - 1 from the camera
// sums of round k - 1, then their direction records) and k_tile_cg (the points' update
// k - 1 fused into the tile staging, then w = A u); the last CTA of k_tile_cg takes the
// reduction, the stop test on |r_k| and alpha, beta.  Same iterates as the textbook
// recurrences in exact arithmetic; the updated residual drifts from the true one sooner
// in FP32.  Round 0 only stages u = z = M^-1 r_0 from the preconditioner.

// Slot-sum components of a round: |J u|^2, u^T D u, r^T u, |r|^2.
enum : int { CG_JU = 0, CG_UDU = 1, CG_RU = 2, CG_RR = 3 };

// Cameras of a k_cg_cameras block: one thread per camera entry (coalesced vectors),
// the 9x9 preconditioner rows and the direction record through shared memory.
constexpr int CGC_CAMS = 32;
constexpr int CGC_TB = 9 * CGC_CAMS;

__global__ void __launch_bounds__(CGC_TB) k_cg_cameras(Views<float> v, const int32_t* gate) {
    if (gated_off(gate)) return;
    __shared__ float sr[CGC_TB], su[CGC_TB];
    __shared__ double red[2 * (CGC_TB / 32)];
    DevState* st = v.st;
    const int k = st->pcg_iter;
    const float alpha = (float)st->alpha, beta = (float)st->beta, mu = (float)st->mu;
    const int i = threadIdx.x, cl = i / 9, kk = i - 9 * cl;
    const int c = blockIdx.x * CGC_CAMS + cl;
    const bool live = c < v.n_cams;
    const size_t e = 9 * (size_t)blockIdx.x * CGC_CAMS + i;
    float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
    const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
    float ri = 0.0f, d = 0.0f;
    if (live) {
        d = v.D[e];
        if (k > 0) {
            // w = J^T J u (from the camera sums) + mu D u, then update k - 1
            const float w = kk < 3 ? fmaf(JL[kk], ca[0], fmaf(JL[3 + kk], ca[1], JL[6 + kk] * ca[2])) : ca[kk];
            const float uo = v.z[e];
            const float pi = fmaf(beta, v.p[e], uo);
            const float si = fmaf(beta, v.s[e], fmaf(mu, d * uo, w));
            v.p[e] = pi;
            v.s[e] = si;
            v.h[e] = fmaf(alpha, pi, v.h[e]);
            ri = fmaf(-alpha, si, v.r[e]);
            v.r[e] = ri;
        } else {
            ri = v.r[e];
        }
    }
    sr[i] = ri;
    __syncthreads();   // every camera sum has been read
    float u = 0.0f;
    if (live) {
        if (k > 0) {
            ca[kk] = 0.0f;
            const float* M = v.Minv_c + (size_t)c * MC_STRIDE + 9 * kk;
#pragma unroll
            for (int q = 0; q < 9; ++q) u = fmaf(M[q], sr[9 * cl + q], u);
            v.z[e] = u;
        } else {
            u = v.z[e];
        }
    }
    su[i] = u;
    float gs = 0.0f, gc = 0.0f, rs = 0.0f, rc = 0.0f, us = 0.0f, uc = 0.0f;   // Kahan pairs
    kahan_add(gs, gc, ri * u);
    kahan_add(rs, rc, ri * ri);
    kahan_add(us, uc, d * u * u);
    __syncthreads();
    if (live) {   // direction record: phi = J_l u_w (3), u_t (3), u_intr (3)
        const float dv = kk < 3 ? fmaf(JL[3 * kk], su[9 * cl], fmaf(JL[3 * kk + 1], su[9 * cl + 1],
                                                                  JL[3 * kk + 2] * su[9 * cl + 2]))
                                : u;
        v.cam_dir[(size_t)c * CD_STRIDE + kk] = dv;
    }
    double bg, br, bu, dummy;
    block_sum2c(gs, gc, rs, rc, red, bg, br);
    block_sum2c(us, uc, 0.0f, 0.0f, red, bu, dummy);
    if (threadIdx.x == 0) {
        slot_add(st->acc_mv, CG_RU, bg);
        slot_add(st->acc_mv, CG_RR, br);
        slot_add(st->acc_mv, CG_UDU, bu);
    }
}

template <int TB>
__global__ void __launch_bounds__(TB, 6) k_tile_cg(Views<float> v, const int32_t* gate, Caps cap, CondHandle pcg_cond,
                                                int use_cond) {
    if (gated_off(gate)) return;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float4 sX4[TILE_PTS], sP4[TILE_PTS];      // X and u of the tile's points
    __shared__ float sQ[3 * TILE_PTS];
    __shared__ unsigned int s_next;
    __shared__ double red[2 * (TB / 32)];
    __shared__ bool is_last;
    DevState* st = v.st;
    const int k = st->pcg_iter;
    const float alpha = (float)st->alpha, beta = (float)st->beta, mu = (float)st->mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;
    const int lane = threadIdx.x & 31;
    const TileRange T = tile_range(v, blockIdx.x);
    float jp_s = 0.0f, jp_c = 0.0f, ud_s = 0.0f, ud_c = 0.0f;   // |J u|^2, u^T D u
    float ru_s = 0.0f, ru_c = 0.0f, rr_s = 0.0f, rr_c = 0.0f;   // r^T u, |r|^2
    // The points' update k - 1 and their u = M^-1 r, entry-parallel (coalesced): every
    // load first (the stores that follow may alias them, so loads issued after a store
    // would wait for it), then the update entry by entry with r into sQ; then u of each
    // entry from its point's three residual entries and row of M; then u and mu D u
    // into the staging arrays.
    static_assert((3 * TILE_PTS) % TB == 0, "whole entry steps");
    constexpr int EPT = 3 * TILE_PTS / TB;   // entries per thread
    const int ne = 3 * T.npt;
    float* sPf = reinterpret_cast<float*>(sP4);
    float* sXf = reinterpret_cast<float*>(sX4);
    float R[EPT], X[EPT], Dd[EPT], Z[EPT], Qw[EPT], P[EPT], S[EPT], H[EPT], M0[EPT], M1[EPT], M2[EPT];
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
        const int i = threadIdx.x + t * TB;
        if (i < ne) {
            const size_t e = T.base + i;
            R[t] = v.r[e];
            X[t] = v.x[e];
            Dd[t] = v.D[e];
            Z[t] = v.z[e];
            if (k > 0) {
                Qw[t] = v.q[e];   // w = A u of the previous round (mu D u included)
                P[t] = v.p[e];
                S[t] = v.s[e];
                H[t] = v.h[e];
                // row kk of the point's packed symmetric block (xx, xy, xz, yy, yz, zz)
                const int slot = i / 3, kk = i - 3 * slot;
                const float* m = v.Minv_p + (size_t)(T.pt0 + slot) * MP_STRIDE;
                M0[t] = __ldg(m + (kk == 0 ? 0 : (kk == 1 ? 1 : 2)));
                M1[t] = __ldg(m + (kk == 0 ? 1 : (kk == 1 ? 3 : 4)));
                M2[t] = __ldg(m + (kk == 0 ? 2 : (kk == 1 ? 4 : 5)));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
        const int i = threadIdx.x + t * TB;
        if (i < ne) {
            const size_t e = T.base + i;
            if (k > 0) {
                const float pi = fmaf(beta, P[t], Z[t]);
                const float si = fmaf(beta, S[t], Qw[t]);
                v.p[e] = pi;
                v.s[e] = si;
                v.h[e] = fmaf(alpha, pi, H[t]);
                R[t] = fmaf(-alpha, si, R[t]);
                v.r[e] = R[t];
            }
            sQ[i] = R[t];
            const int slot = i / 3;
            sXf[4 * slot + (i - 3 * slot)] = X[t];
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
        const int i = threadIdx.x + t * TB;
        if (i < ne) {
            const int slot = i / 3;
            if (k > 0) {
                Z[t] = fmaf(M0[t], sQ[3 * slot], fmaf(M1[t], sQ[3 * slot + 1], M2[t] * sQ[3 * slot + 2]));
                v.z[T.base + i] = Z[t];
            }
            kahan_add(ru_s, ru_c, R[t] * Z[t]);
            kahan_add(rr_s, rr_c, R[t] * R[t]);
            kahan_add(ud_s, ud_c, Dd[t] * Z[t] * Z[t]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
        const int i = threadIdx.x + t * TB;
        if (i < ne) {
            const int slot = i / 3;
            sPf[4 * slot + (i - 3 * slot)] = Z[t];
            sQ[i] = mu * (Dd[t] * Z[t]);
        }
    }
    uint32_t *sRun, *sShort;
    uint8_t* sSlot;
    stage_compact<TB>(v, T, cap, dsm, sRun, sShort, sSlot);
    if (threadIdx.x == 0) s_next = 0u;
    __syncthreads();
    // w = A u: long runs in camera-uniform steps, then the short tail by chunks
    for (;;) {
        unsigned int rr = 0;
        if (lane == 0) rr = atomicAdd(&s_next, 1u);
        rr = __shfl_sync(FULL, rr, 0);
        if (rr >= T.nl) break;
        const uint32_t start = sRun[3 * rr] - T.lo, len = sRun[3 * rr + 1], c = sRun[3 * rr + 2];
        const Cam cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
        float dir[9];
        load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
        float acc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
        for (uint32_t off = lane; off < len; off += 32) {
            const uint32_t j = T.lo + start + off;
            const uint32_t slot = sSlot[start + off];
            const float4 xp = sX4[slot], pp = sP4[slot];
            const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
            const float tt = weighted ? obs_normal<true>(cam, dir, xs, ds, eps, acc, sQ + 3 * slot, __ldg(v.obs_w + j))
                                      : obs_normal(cam, dir, xs, ds, eps, acc, sQ + 3 * slot);
            kahan_add(jp_s, jp_c, tt);
        }
        int idx;
        const int nv = warp_split_sum<9>(acc, lane, idx);
        if (nv > 0) atomicAdd(v.cam_acc + (size_t)c * CA_STRIDE + idx, acc[0]);
    }
    {
        const uint32_t n = T.hi - T.ss;
        const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
        const uint32_t a = T.ss + min(threadIdx.x * chunk, n), b = T.ss + min(threadIdx.x * chunk + chunk, n);
        uint32_t cur = NO_CAM;
        float acc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
        Cam cam;
        float dir[9];
        for (uint32_t j = a; j < b; ++j) {
            const uint32_t key = sShort[j - T.ss];
            const uint32_t c = key >> 8, slot = key & 0xffu;
            if (c != cur) {
                if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                cur = c;
                cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                load_dir(v.cam_dir + (size_t)c * CD_STRIDE, dir);
            }
            const float4 xp = sX4[slot], pp = sP4[slot];
            const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
            const float tt = weighted ? obs_normal<true>(cam, dir, xs, ds, eps, acc, sQ + 3 * slot, __ldg(v.obs_w + j))
                                      : obs_normal(cam, dir, xs, ds, eps, acc, sQ + 3 * slot);
            kahan_add(jp_s, jp_c, tt);
        }
        if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * T.npt; i += TB) v.q[T.base + i] = sQ[i];
    double b_jp, b_ud, b_ru, b_rr;
    block_sum2c(jp_s, jp_c, ud_s, ud_c, red, b_jp, b_ud);
    block_sum2c(ru_s, ru_c, rr_s, rr_c, red, b_ru, b_rr);
    if (threadIdx.x == 0) {
        slot_add(st->acc_mv, CG_JU, b_jp);
        slot_add(st->acc_mv, CG_UDU, b_ud);
        slot_add(st->acc_mv, CG_RU, b_ru);
        slot_add(st->acc_mv, CG_RR, b_rr);
        __threadfence();
        is_last = atomicAdd(&st->tickets[TK_UPD], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last || threadIdx.x >= 32) return;
    __threadfence();
    const double ju = slot_sum_warp(st->acc_mv, CG_JU), udu = slot_sum_warp(st->acc_mv, CG_UDU);
    const double gam = slot_sum_warp(st->acc_mv, CG_RU), rho = slot_sum_warp(st->acc_mv, CG_RR);
    for (int i = threadIdx.x; i < NSLOT * SLOT_STRIDE; i += 32) st->acc_mv[i] = 0.0;
    if (threadIdx.x != 0) return;
    st->tickets[TK_UPD] = 0u;
    if (k > 0) st->pcg_total += 1;   // this round applied update k - 1
    const double delta = ju + st->mu * udu;
    bool stop = false;
    if (!isfinite(gam) || !isfinite(rho) || !isfinite(delta)) {
        st->status = 4;
        stop = true;
    } else if (k > 0 && (rho <= st->opt.tol * st->opt.tol * st->rr0 || k >= st->opt.max_pcg)) {
        stop = true;
    }
    double a_new = 0.0, b_new = 0.0;
    if (!stop) {
        b_new = k > 0 ? gam / st->rz : 0.0;
        const double den = k > 0 ? delta - b_new * gam / st->alpha : delta;
        if (!(den > 0.0)) stop = true;
        else a_new = gam / den;
    }
    st->rr = rho;
    if (stop) {
        st->pcg_iter = k;
        st->pcg_active = 0;
    } else {
        st->alpha = a_new;
        st->beta = b_new;
        st->rz = gam;
        st->pcg_iter = k + 1;
    }
    if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
}

// ---------------------------------------------------------------- linearisation ---
// Linearisation (fused score + Jacobian products, Sec. V-A): cost F = 1/2 sum rho(|r|^2),
// g = J^T W r and the diagonal blocks J_c^T W J_c, J_p^T W J_p.  `mode` as k_linearize:
// 0 first linearisation of a solve, 1 relinearisation after an accepted step (gated by
// st->relin), 2 evaluation only (squared loss; optional r and J in the caller's order).
constexpr int TL_ACC = 9 + 45;   // per-lane camera sums: g, upper triangle of J_c^T J_c
constexpr int TL_TB = 128;

struct LinObs {
    float r0, r1, j0[9], j1[9], jx0[3], jx1[3];
};

// Jacobian rows of one observation (J_w[:,k] = A (J_l[:,k] x RX)) and its residual r
// (from k_residual).
__device__ __forceinline__ LinObs lin_obs(const Cam& cam, const float (&JL)[9], float4 X, float2 r, float eps) {
    LinObs o;
    const Geo g = project_geo(cam, X.x, X.y, X.z, eps);
    o.r0 = r.x;
    o.r1 = r.y;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float w0 = JL[k], w1 = JL[3 + k], w2 = JL[6 + k];
        const float c0 = fmaf(w1, g.RX[2], -w2 * g.RX[1]);
        const float c1 = fmaf(w2, g.RX[0], -w0 * g.RX[2]);
        const float c2 = fmaf(w0, g.RX[1], -w1 * g.RX[0]);
        o.j0[k] = fmaf(g.A[0], c0, fmaf(g.A[1], c1, g.A[2] * c2));
        o.j1[k] = fmaf(g.A[3], c0, fmaf(g.A[4], c1, g.A[5] * c2));
        o.j0[3 + k] = g.A[k];
        o.j1[3 + k] = g.A[3 + k];
    }
    const float fn2 = cam.f * g.n2;
    o.j0[6] = g.s * g.p[0]; o.j0[7] = fn2 * g.p[0]; o.j0[8] = fn2 * g.n2 * g.p[0];
    o.j1[6] = g.s * g.p[1]; o.j1[7] = fn2 * g.p[1]; o.j1[8] = fn2 * g.n2 * g.p[1];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        o.jx0[q] = fmaf(g.A[0], cam.R[q], fmaf(g.A[1], cam.R[3 + q], g.A[2] * cam.R[6 + q]));
        o.jx1[q] = fmaf(g.A[3], cam.R[q], fmaf(g.A[4], cam.R[3 + q], g.A[5] * cam.R[6 + q]));
    }
    return o;
}

// Everything one observation adds: evaluation outputs (mode 2), the IRLS weight, the cost,
// the camera sums (registers) and the point sums (shared memory).
template <bool PLAIN = false>
__device__ __forceinline__ void lin_accumulate(const Views<float>& v, LinObs& o, uint32_t j, uint32_t slot, int mode,
                                               int loss, float lscale, float* res_out, float* jac_out,
                                               float (&acc)[TL_ACC], float* sG, float* sH, float& cs, float& cc) {
    if (mode == 2) {   // evaluation output: the unweighted residual and Jacobian
        const uint32_t u = v.obs_user[j];
        if (res_out) { res_out[2 * (size_t)u] = o.r0; res_out[2 * (size_t)u + 1] = o.r1; }
        if (jac_out) {
            float* Jo = jac_out + 24 * (size_t)u;
#pragma unroll
            for (int k = 0; k < 9; ++k) { Jo[k] = o.j0[k]; Jo[12 + k] = o.j1[k]; }
#pragma unroll
            for (int q = 0; q < 3; ++q) { Jo[9 + q] = o.jx0[q]; Jo[21 + q] = o.jx1[q]; }
        }
    }
    const float s2 = fmaf(o.r0, o.r0, o.r1 * o.r1);
    if (loss) {   // IRLS weight w = rho'(|r|^2): rows scaled by sqrt(w)
        const float w = loss_weight(s2, loss, lscale);
        if (mode != 2) v.obs_w[j] = w;
        kahan_add(cs, cc, loss_rho(s2, loss, lscale));
        const float sw = sqrtf(w);
        o.r0 *= sw;
        o.r1 *= sw;
#pragma unroll
        for (int k = 0; k < 9; ++k) { o.j0[k] *= sw; o.j1[k] *= sw; }
#pragma unroll
        for (int q = 0; q < 3; ++q) { o.jx0[q] *= sw; o.jx1[q] *= sw; }
    } else {
        kahan_add(cs, cc, s2);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = fmaf(o.j0[i], o.r0, fmaf(o.j1[i], o.r1, acc[i]));
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int k = i; k < 9; ++k) {
            const int t = 9 + tri_index(9, i, k);
            acc[t] = fmaf(o.j0[i], o.j0[k], fmaf(o.j1[i], o.j1[k], acc[t]));
        }
    float* gq = sG + 3 * slot;
    float* hq = sH + 6 * slot;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float x = fmaf(o.jx0[q], o.r0, o.jx1[q] * o.r1);
        if (PLAIN) gq[q] += x;
        else atomicAdd(gq + q, x);
    }
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int b2 = a2; b2 < 3; ++b2) {
            const float x = fmaf(o.jx0[a2], o.jx0[b2], o.jx1[a2] * o.jx1[b2]);
            if (PLAIN) hq[tri_index(3, a2, b2)] += x;
            else atomicAdd(hq + tri_index(3, a2, b2), x);
        }
}

__device__ __forceinline__ void load_jl(const float* __restrict__ rec, float (&JL)[9]) {
    const float4* j4 = reinterpret_cast<const float4*>(rec + CP_JL);
    const float4 a = __ldg(j4), b = __ldg(j4 + 1), c = __ldg(j4 + 2);
    JL[0] = a.x; JL[1] = a.y; JL[2] = a.z; JL[3] = a.w;
    JL[4] = b.x; JL[5] = b.y; JL[6] = b.z; JL[7] = b.w; JL[8] = c.x;
}

// A thread's camera sums of one run into the global accumulators (g in FP64, the
// J_c^T J_c triangle as float4 atomics), then cleared.
__device__ __forceinline__ void flush_lin_global(const Views<float>& v, uint32_t c, float (&a)[TL_ACC]) {
    double* g = v.cam_lin + (size_t)c * CL_STRIDE;
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(g + k, (double)a[k]);
    float4* h = reinterpret_cast<float4*>(v.cam_H + (size_t)c * CH_STRIDE);
#pragma unroll
    for (int k = 0; k < 11; ++k)
        atomicAdd(h + k, make_float4(a[9 + 4 * k], a[10 + 4 * k], a[11 + 4 * k], a[12 + 4 * k]));
    atomicAdd(v.cam_H + (size_t)c * CH_STRIDE + 44, a[53]);
#pragma unroll
    for (int k = 0; k < TL_ACC; ++k) a[k] = 0.0f;
}

// PLAIN: every warp keeps its own copy of the tile's point sums, added to with plain
// shared-memory adds in its long runs (as in k_tile_normal).
template <int TB, bool PLAIN>
__global__ void __launch_bounds__(TB, 4) k_tile_linearize(Views<float> v, int mode, float* res_out, float* jac_out,
                                                       CondHandle lm_cond, int use_cond, Caps cap) {
    if (mode == 1 && v.st->relin == 0) return;
    constexpr int NQ = PLAIN ? TB / 32 : 1;   // point-sum copies
    extern __shared__ __align__(16) unsigned char dsm[];
    const float2* rbuf = reinterpret_cast<const float2*>(v.rbuf);   // residuals (k_residual)
    __shared__ float4 sX4[TILE_PTS];
    __shared__ float sG[NQ * 3 * TILE_PTS], sH[NQ * PH_STRIDE * TILE_PTS];   // J_p^T W r, J_p^T W J_p (upper)
    float* const sGw = sG + (PLAIN ? (threadIdx.x >> 5) * 3 * TILE_PTS : 0);
    float* const sHw = sH + (PLAIN ? (threadIdx.x >> 5) * PH_STRIDE * TILE_PTS : 0);
    __shared__ unsigned int s_next;
    const float eps = (float)v.st->opt.eps;
    // robust loss (evaluation, mode 2, is always the squared loss)
    const int loss = mode == 2 ? 0 : v.st->opt.loss;
    const float lscale = (float)v.st->opt.loss_scale;
    const int lane = threadIdx.x & 31;
    float cs = 0.0f, cc = 0.0f;   // compensated cost
    for (int tile = blockIdx.x; tile < v.n_tiles; tile += gridDim.x) {
        const TileRange T = tile_range(v, tile);
        for (int i = threadIdx.x; i < T.npt; i += TB)
            sX4[i] = make_float4(v.x[T.base + 3 * i], v.x[T.base + 3 * i + 1], v.x[T.base + 3 * i + 2], 0.0f);
        for (int i = threadIdx.x; i < NQ * 3 * TILE_PTS; i += TB) sG[i] = 0.0f;
        for (int i = threadIdx.x; i < NQ * PH_STRIDE * TILE_PTS; i += TB) sH[i] = 0.0f;
        uint32_t *sRun, *sShort;
        uint8_t* sSlot;
        stage_compact<TB>(v, T, cap, dsm, sRun, sShort, sSlot);
        if (threadIdx.x == 0) s_next = 0u;
        __syncthreads();
        // long runs: camera-uniform steps of 32 observations
        for (;;) {
            unsigned int r = 0;
            if (lane == 0) r = atomicAdd(&s_next, 1u);
            r = __shfl_sync(FULL, r, 0);
            if (r >= T.nl) break;
            const uint32_t start = sRun[3 * r] - T.lo, len = sRun[3 * r + 1], c = sRun[3 * r + 2];
            const float* rec = v.cam_pre + (size_t)c * CP_STRIDE;
            const Cam cam = load_cam(rec);
            float JL[9];
            load_jl(rec, JL);
            float acc[TL_ACC];
#pragma unroll
            for (int k = 0; k < TL_ACC; ++k) acc[k] = 0.0f;
            for (uint32_t off = lane; off < len; off += 32) {
                const uint32_t i = start + off, j = T.lo + i;
                const uint32_t slot = sSlot[i];
                LinObs o = lin_obs(cam, JL, sX4[slot], __ldg(rbuf + j), eps);
                lin_accumulate<PLAIN>(v, o, j, slot, mode, loss, lscale, res_out, jac_out, acc, sGw, sHw, cs, cc);
            }
            if (PLAIN) __syncwarp();   // the warp's next run may meet the same points
            int idx;
            const int nv = warp_split_sum<TL_ACC>(acc, lane, idx);
#pragma unroll
            for (int k = 0; k < split_sum_slots(TL_ACC); ++k) {
                const int i = idx + k;
                if (k < nv) {
                    if (i < 9) atomicAdd(v.cam_lin + (size_t)c * CL_STRIDE + CL_G + i, (double)acc[k]);
                    else atomicAdd(v.cam_H + (size_t)c * CH_STRIDE + (i - 9), acc[k]);
                }
            }
        }
        // short runs: one contiguous chunk per thread
        {
            const uint32_t n = T.hi - T.ss;
            const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
            const uint32_t a = T.ss + min(threadIdx.x * chunk, n), b = T.ss + min(threadIdx.x * chunk + chunk, n);
            uint32_t cur = NO_CAM;
            float acc[TL_ACC];
#pragma unroll
            for (int k = 0; k < TL_ACC; ++k) acc[k] = 0.0f;
            Cam cam;
            float JL[9];
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = sShort[j - T.ss];
                const uint32_t c = key >> 8, slot = key & 0xffu;
                if (c != cur) {
                    if (cur != NO_CAM) flush_lin_global(v, cur, acc);
                    cur = c;
                    cam = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
                    load_jl(v.cam_pre + (size_t)c * CP_STRIDE, JL);
                }
                LinObs o = lin_obs(cam, JL, sX4[slot], __ldg(rbuf + j), eps);
                lin_accumulate(v, o, j, slot, mode, loss, lscale, res_out, jac_out, acc, sGw, sHw, cs, cc);
            }
            if (cur != NO_CAM) flush_lin_global(v, cur, acc);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * T.npt; i += TB) {
            float gi = sG[i];
#pragma unroll
            for (int w = 1; w < NQ; ++w) gi += sG[w * 3 * TILE_PTS + i];
            v.g[T.base + i] = gi;
        }
        for (int i = threadIdx.x; i < PH_STRIDE * T.npt; i += TB) {
            float hi = sH[i];
#pragma unroll
            for (int w = 1; w < NQ; ++w) hi += sH[w * PH_STRIDE * TILE_PTS + i];
            v.pt_H[(size_t)T.pt0 * PH_STRIDE + i] = hi;
        }
        __syncthreads();   // the next tile's staging overwrites the shared sums
    }
    double in[1] = {(double)cs - (double)cc}, out[1];
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

// ------------------------------------------------------------ candidate evaluation ---
// |J(x) h|^2 (weighted at x); with F' = 1/2 sum rho(|r(x')|^2) from k_residual, the last
// block applies the LM rule of Sec. V (lm_decide).  Never gated: its last block sets the
// LM loop flag.
constexpr int TE_TB = 128;

struct EvalCam {
    Cam co;       // record at x
    float dir[9]; // direction record of h (k_candidate)
};

__device__ __forceinline__ EvalCam load_eval_cam(const Views<float>& v, uint32_t c) {
    EvalCam e;
    e.co = load_cam(v.cam_pre + (size_t)c * CP_STRIDE);
    const float4* d4 = reinterpret_cast<const float4*>(v.cam_dir + (size_t)c * CD_STRIDE);
    const float4 a = __ldcg(d4), b = __ldcg(d4 + 1), cc = __ldcg(d4 + 2);
    e.dir[0] = a.x; e.dir[1] = a.y; e.dir[2] = a.z; e.dir[3] = a.w;
    e.dir[4] = b.x; e.dir[5] = b.y; e.dir[6] = b.z; e.dir[7] = b.w; e.dir[8] = cc.x;
    return e;
}

__device__ __forceinline__ void eval_obs(const Views<float>& v, const EvalCam& e, const float4* sXo,
                                         const float4* sHp, uint32_t j, uint32_t slot, float eps, int loss, float& js_,
                                         float& jc_) {
    const float4 xo = sXo[slot], hp = sHp[slot];
    const Geo g = project_geo(e.co, xo.x, xo.y, xo.z, eps);
    float t0, t1;
    jdir(g, e.co, e.dir, hp.x, hp.y, hp.z, t0, t1);
    // |J h|^2 weighted at x
    kahan_add(js_, jc_, (loss ? __ldg(v.obs_w + j) : 1.0f) * fmaf(t0, t0, t1 * t1));
}

// Six CTAs per SM (at most 85 registers per thread; 240 -> 220 us on the large workload
// against four).
template <int TB>
__global__ void __launch_bounds__(TB, 6) k_tile_eval(Views<float> v, CondHandle lm_cond, int use_cond, Caps cap) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ float4 sXo[TILE_PTS], sHp[TILE_PTS];                // x and h of the tile's points
    __shared__ unsigned int s_next;
    DevState* st = v.st;
    const int active = st->lm_active;
    const float eps = (float)st->opt.eps;
    const int loss = st->opt.loss;
    const int lane = threadIdx.x & 31;
    float js_ = 0.0f, jc_ = 0.0f;   // compensated |J h|^2
    for (int tile = blockIdx.x; active && tile < v.n_tiles; tile += gridDim.x) {
        const TileRange T = tile_range(v, tile);
        for (int i = threadIdx.x; i < T.npt; i += TB) {
            const size_t e = T.base + 3 * i;
            sXo[i] = make_float4(v.x[e], v.x[e + 1], v.x[e + 2], 0.0f);
            sHp[i] = make_float4(v.h[e], v.h[e + 1], v.h[e + 2], 0.0f);
        }
        uint32_t *sRun, *sShort;
        uint8_t* sSlot;
        stage_compact<TB>(v, T, cap, dsm, sRun, sShort, sSlot);
        if (threadIdx.x == 0) s_next = 0u;
        __syncthreads();
        for (;;) {
            unsigned int r = 0;
            if (lane == 0) r = atomicAdd(&s_next, 1u);
            r = __shfl_sync(FULL, r, 0);
            if (r >= T.nl) break;
            const uint32_t start = sRun[3 * r] - T.lo, len = sRun[3 * r + 1];
            const EvalCam e = load_eval_cam(v, sRun[3 * r + 2]);
            for (uint32_t off = lane; off < len; off += 32) {
                const uint32_t i = start + off;
                eval_obs(v, e, sXo, sHp, T.lo + i, sSlot[i], eps, loss, js_, jc_);
            }
        }
        {
            const uint32_t n = T.hi - T.ss;
            const uint32_t chunk = odd_chunk<uint32_t>(n, TB);
            const uint32_t a = T.ss + min(threadIdx.x * chunk, n), b = T.ss + min(threadIdx.x * chunk + chunk, n);
            uint32_t cur = NO_CAM;
            EvalCam e;
            for (uint32_t j = a; j < b; ++j) {
                const uint32_t key = sShort[j - T.ss];
                const uint32_t c = key >> 8;
                if (c != cur) {
                    cur = c;
                    e = load_eval_cam(v, c);
                }
                eval_obs(v, e, sXo, sHp, j, key & 0xffu, eps, loss, js_, jc_);
            }
        }
        __syncthreads();   // the next tile's staging overwrites the points
    }
    double in[1] = {(double)js_ - (double)jc_}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_COST], out) && threadIdx.x == 0) {
        // pose factors: k_factor_eval ran just before
        const bool fac = v.n_fac > 0;
        lm_decide(st, active, st->F_res + (fac ? st->fac_cost_new : 0.0), out[0] + (fac ? st->fac_jh2 : 0.0));
        if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
    }
}

template <typename K>
int prepare(K kernel, int tb, size_t dyn) {
    if (ensure_dynamic_smem((const void*)kernel, (int)dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, tb, dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

// The tile kernels stage a whole tile's observation table (compact form); a problem
// whose largest tile does not fit in shared memory keeps the per-thread-chunk kernels
// (all grids 0).
void plan_tile_kernels(LaunchCfg& L, int n_tiles, int sms, int max_long_obs, int max_short_obs, int max_long_runs) {
    L.tn_grid = L.tl_grid = L.te_grid = 0;
    L.tk_run_cap = std::max(1, max_long_runs);
    L.tk_short_cap = std::max(1, max_short_obs);
    L.tk_long_cap = (std::max(1, max_long_obs) + 15) / 16 * 16;
    const Caps cap{L.tk_run_cap, L.tk_short_cap, L.tk_long_cap};
    if (compact_bytes(cap) > 160 * 1024) return;
    L.tn_smem = L.tl_smem = L.te_smem = (int)compact_bytes(cap);
    const int bn = std::min(prepare(k_tile_normal<TN_TB, true>, TN_TB, L.tn_smem),
                            prepare(k_tile_normal<TN_TB, false>, TN_TB, L.tn_smem));
    const int bc = prepare(k_tile_cg<TN_TB>, TN_TB, L.tn_smem);
    const int bl = std::min(prepare(k_tile_linearize<TL_TB, true>, TL_TB, L.tl_smem),
                            prepare(k_tile_linearize<TL_TB, false>, TL_TB, L.tl_smem));
    const int be = prepare(k_tile_eval<TE_TB>, TE_TB, L.te_smem);
    if (bn < 1 || bl < 1 || be < 1 || bc < 1) return;
    const int nt = std::max(1, n_tiles);
    L.tn_grid = nt;   // one CTA per tile
    L.tl_grid = std::max(1, std::min({nt, sms * bl, MAX_GRID}));
    L.te_grid = std::max(1, std::min({nt, sms * be, MAX_GRID}));
}

void launch_tile_normal(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate,
                        const float* zs, int use_beta) {
    const Caps cap{L.tk_run_cap, L.tk_short_cap, L.tk_long_cap};
    if (L.tn_plain_q) k_tile_normal<TN_TB, true><<<L.tn_grid, TN_TB, L.tn_smem, s>>>(v, gate, zs, use_beta, cap);
    else k_tile_normal<TN_TB, false><<<L.tn_grid, TN_TB, L.tn_smem, s>>>(v, gate, zs, use_beta, cap);
}

void launch_cg_round(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate, CondHandle c,
                     int use) {
    k_cg_cameras<<<std::max(1, (v.n_cams + CGC_CAMS - 1) / CGC_CAMS), CGC_TB, 0, s>>>(v, gate);
    launch_factor_matvec(v, L, s, gate, v.z, 0);   // pose factors: |J_f u|^2 before the round's reduction
    k_tile_cg<TN_TB><<<L.tn_grid, TN_TB, L.tn_smem, s>>>(v, gate, Caps{L.tk_run_cap, L.tk_short_cap, L.tk_long_cap},
                                                         c, use);
}

void launch_tile_linearize(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, int mode, float* res_out,
                           float* jac_out, CondHandle lm_cond, int use_cond) {
    const Caps cap{L.tk_run_cap, L.tk_short_cap, L.tk_long_cap};
    if (L.tn_plain_q)
        k_tile_linearize<TL_TB, true><<<L.tl_grid, TL_TB, L.tl_smem, s>>>(v, mode, res_out, jac_out, lm_cond, use_cond,
                                                                        cap);
    else
        k_tile_linearize<TL_TB, false><<<L.tl_grid, TL_TB, L.tl_smem, s>>>(v, mode, res_out, jac_out, lm_cond,
                                                                         use_cond, cap);
}

void launch_tile_eval(const Views<float>& v, const LaunchCfg& L, cudaStream_t s, CondHandle lm_cond, int use_cond) {
    k_tile_eval<TE_TB><<<L.te_grid, TE_TB, L.te_smem, s>>>(v, lm_cond, use_cond,
                                                           Caps{L.tk_run_cap, L.tk_short_cap, L.tk_long_cap});
}

}  // namespace gbba
