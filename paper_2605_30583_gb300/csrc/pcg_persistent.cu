// Persistent PCGNR (Sec. V-A of arXiv 2605.30583) for problems whose tiles fit in the
// GPU's aggregate shared memory.
//
// One cooperative launch runs every PCG iteration of one LM step.  The grid is one
// CTA per SM; CTA b owns a contiguous run of tiles (balanced by observation count)
// and keeps, for the whole solve, its observation keys and its points' X, D, M^-1
// and PCG vectors in shared memory.  Grid-wide sums travel through an exchange:
// slot-spread atomic sums followed by a grid barrier, after which every CTA reads the
// same totals and so takes the same stop decision.  Every wait is time-bounded: on a
// time-out the CTA sets an error flag, every CTA leaves, and the solve reports
// BA_ERR_TIMEOUT.
//
// Two forms of the same Krylov iteration:
//
// k_pcg_persistent (the default form): the textbook recurrences, two
// exchanges per iteration:
//   A  p = z + beta p (points in smem; cameras double-buffered in global), then
//      q = J^T J p + mu D p with |J p|^2 and p^T D p;            -> exchange
//   B  alpha = r^T z / (|J p|^2 + mu p^T D p); h += alpha p; r -= alpha q; z = M^-1 r;
//      r^T z, |r|^2                                              -> exchange
//   C  stop test (|r| <= tol |r_0| or the iteration cap), beta.
//
// k_pcg_persistent_1x: one exchange per iteration.  The recurrences are arranged as in
// the CG of Chronopoulos and Gear (J. Comput. Appl. Math. 25, 1989): with u = M^-1 r,
// w = A u and s = A p carried by s = w + beta s,
//   gamma = r^T u,  delta = u^T A u = |J u|^2 + mu u^T D u,
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev),
// so both inner products of an iteration come out of the one exchange that follows
// the operator.  Each CTA keeps its own copy of the camera vectors it touches and
// updates them from the assembled camera sums of the operator, so no second exchange
// publishes them; the one CTA that owns a camera adds it to the inner products and
// writes its step.  Same iterates in exact arithmetic; in FP32 the recurrence for s
// lets the updated residual drift from the true one sooner.
//   M  w = J^T W J u: point part in shared memory, camera part into one of three
//      rotating accumulator sets; |J u|^2 with the partials of the previous update;
//   X  exchange: gamma, |r|^2, u^T D u, |J u|^2 over the grid; stop test, alpha, beta;
//   U  p = u + beta p, s = w + beta s, h += alpha p, r -= alpha s, u = M^-1 r.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"
#include "mixed_common.cuh"

namespace gbba {

namespace {

// Grid-wide barrier number `epoch` (1, 2, ... within a launch) for a co-resident
// (cooperative) grid.  Each CTA adds one to a counter, cleared before the launch, with
// release semantics, and waits until it reaches epoch * nblocks: the count can only
// get there once every CTA has arrived, and a CTA that has already moved on to the
// next barrier only raises it further.  False on time-out or when another CTA has
// already reported one.  Limits below 1 ms are checked at every poll (0: give up at the
// first poll that finds the barrier incomplete), longer ones every 16th poll.
__device__ __forceinline__ bool grid_sync_on(unsigned long long* cnt, int* err, unsigned int nblocks,
                                             unsigned long long epoch, long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(cnt), "l"(1ull) : "memory");
        const unsigned long long target = epoch * nblocks;
        const long long t0 = global_ns();
        unsigned spins = 0;
        for (;;) {
            unsigned long long c;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(cnt) : "memory");
            if (c >= target) break;
            if (timeout_ns < 1000000LL || (++spins & 15u) == 0u) {
                if (*reinterpret_cast<volatile int*>(err)) { ok = 0; break; }
                if (global_ns() - t0 >= timeout_ns) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(DevState* st, unsigned int nblocks, unsigned long long epoch) {
    return grid_sync_on(&st->bar_count, &st->bar_err, nblocks, epoch, st->opt.wait_ns);
}

// Grid-wide sums of XCH_NV per-CTA values, then the grid barrier.  Exchange e adds
// into slot set e % 3 (CTA b into slot b % NSLOT, so concurrent atomics spread over
// NSLOT lines); every CTA then reads the same totals.  Block 0 clears set (e + 1) % 3
// before it arrives: that set was last read right after exchange e - 2, which every
// CTA has left, and is next filled after exchange e.  `mine` is read in thread 0;
// `sh` holds XCH_NV doubles.  False on time-out.
__device__ bool exchange(DevState* st, double* pslots, unsigned long long epoch, const double (&mine)[XCH_NV],
                         double (&tot)[XCH_NV], double* sh) {
    double* cur = pslots + (size_t)(epoch % 3ull) * NSLOT * SLOT_STRIDE;
    if (blockIdx.x == 0) {
        double* nx = pslots + (size_t)((epoch + 1ull) % 3ull) * NSLOT * SLOT_STRIDE;
        for (int i = threadIdx.x; i < NSLOT * SLOT_STRIDE; i += blockDim.x) nx[i] = 0.0;
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < XCH_NV; ++k)
            if (mine[k] != 0.0) slot_add(cur, k, mine[k]);
    }
    if (!grid_sync(st, gridDim.x, epoch)) return false;
    if (threadIdx.x < 32) {
        double x[XCH_NV];
#pragma unroll
        for (int k = 0; k < XCH_NV; ++k) x[k] = slot_sum_warp(cur, k);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < XCH_NV; ++k) sh[k] = x[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < XCH_NV; ++k) tot[k] = sh[k];
    return true;
}

// Local index of camera c in the CTA's sorted camera list (c must be listed).
__device__ __forceinline__ uint32_t local_cam(const uint32_t* sCid, uint32_t ncb, uint32_t c) {
    uint32_t lo = 0, hi = ncb;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sCid[mid] <= c) lo = mid; else hi = mid;
    }
    return lo;
}

// Pose factors k = b, b + G, ... of CTA b through the operator (both cameras of each
// are in the CTA's list): returns this thread's part of |J_f d|^2.
__device__ __forceinline__ float factor_pass(const Views<float>& v, const uint32_t* sCid, uint32_t ncb,
                                          const float* sDir, float* acc, int stride) {
    float jj = 0.0f;
    for (int k = blockIdx.x + (int)gridDim.x * (int)threadIdx.x; k < v.n_fac; k += stride) {
        const uint32_t ca = v.fac_cam[2 * (size_t)k], cb = v.fac_cam[2 * (size_t)k + 1];
        jj += factor_normal(v.fac_J + 72 * (size_t)k, sDir + 12 * local_cam(sCid, ncb, ca),
                            sDir + 12 * local_cam(sCid, ncb, cb), acc + (size_t)ca * CA_STRIDE,
                            acc + (size_t)cb * CA_STRIDE);
    }
    return jj;
}

}  // namespace

template <int TB>
__global__ void __launch_bounds__(TB, 1) k_pcg_persistent(Views<float> v, const uint32_t* __restrict__ blk_tile,
                                                         const uint32_t* __restrict__ blk_cam_off,
                                                         const uint32_t* __restrict__ blk_cams,
                                                         double* __restrict__ pslots) {
    DevState* st = v.st;
    if (st->pcg_active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CAMS_PER_PASS = TB / 9;
    __shared__ double red[64];
    __shared__ double shx[XCH_NV + 1];
    __shared__ float s_cam_r[9 * CAMS_PER_PASS];
    const int tid = threadIdx.x;
    // cameras owned by this CTA: blockIdx.x + gridDim.x * j, j < n_own
    const int n_own = v.n_cams > (int)blockIdx.x ? (v.n_cams - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const uint32_t t0 = blk_tile[blockIdx.x], t1 = blk_tile[blockIdx.x + 1];
    const uint32_t ob = v.tile_off[t0], oe = v.tile_off[t1];
    const uint32_t no = oe - ob;
    const int pb = (int)(t0 * TILE_PTS);
    const int pe = min((int)(t1 * TILE_PTS), v.n_pts);
    const int np = pe > pb ? pe - pb : 0;
    const int n3 = 3 * np;
    const int n3p = (n3 + 3) & ~3;
    uint32_t* skey = reinterpret_cast<uint32_t*>(smem);
    // X and p of the CTA's points as (x, y, z, 0) quadruples: one 128-bit load each
    float4* sX4 = reinterpret_cast<float4*>(smem + (((size_t)no * 4 + 15) & ~(size_t)15));
    float4* sP4 = sX4 + np;
    float* sD = reinterpret_cast<float*>(sP4 + np);
    float* sR = sD + n3p;
    float* sZ = sR + n3p;
    float* sH = sZ + n3p;
    float* sQ = sH + n3p;
    float* sM = sQ + n3p;   // 6 per point
    // cameras seen by this CTA (sorted): records (R, t, f, k1, k2) and direction records
    const uint32_t cb = blk_cam_off[blockIdx.x], ncb = blk_cam_off[blockIdx.x + 1] - cb;
    uint32_t* sCid = reinterpret_cast<uint32_t*>(sM + ((6 * np + 3) & ~3));
    float* sCam = reinterpret_cast<float*>(sCid + ((ncb + 3) & ~3u));   // 16 per camera
    float* sDir = sCam + 16 * (size_t)ncb;                              // 12 per camera
    const size_t g0 = v.pt_off + 3 * (size_t)pb;
    for (uint32_t i = tid; i < ncb; i += TB) sCid[i] = __ldg(blk_cams + cb + i) & ~BLK_CAM_OWNER;
    for (uint32_t i = tid; i < 16 * ncb; i += TB)
        sCam[i] = __ldg(v.cam_pre + (size_t)(__ldg(blk_cams + cb + i / 16) & ~BLK_CAM_OWNER) * CP_STRIDE + i % 16);
    for (uint32_t i = tid; i < no; i += TB) skey[i] = __ldg(v.obs_key + ob + i);
    for (int i = tid; i < n3; i += TB) {
        sD[i] = v.D[g0 + i];
        sR[i] = v.r[g0 + i];
        sZ[i] = v.z[g0 + i];
        sH[i] = 0.0f;
    }
    for (int i = tid; i < np; i += TB) {
        sX4[i] = make_float4(v.x[g0 + 3 * i], v.x[g0 + 3 * i + 1], v.x[g0 + 3 * i + 2], 0.0f);
        sP4[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    for (int i = tid; i < 6 * np; i += TB) sM[i] = v.Minv_p[6 * (size_t)pb + i];
    __syncthreads();
    // keys carry the CTA-local camera index from here on (no search in the loop)
    for (uint32_t i = tid; i < no; i += TB) {
        const uint32_t key = skey[i];
        skey[i] = (local_cam(sCid, ncb, key >> 8) << 8) | (key & 0xffu);
    }
    __syncthreads();

    const double mu = st->mu;
    const float muf = (float)mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;   // robust loss: IRLS weights per observation
    const double tol2 = st->opt.tol * st->opt.tol;
    const double rr0 = st->rr0;
    const int max_pcg = st->opt.max_pcg;
    double rz = st->rz, rr = rr0, alpha = 0.0;
    float beta = 0.0f;
    unsigned long long epoch = 0ull;
    int k = 0;
    bool ok = true, numeric_fail = false;
    // this thread's observation chunk (block-local indices) and its first tile
    const uint32_t chunk = odd_chunk<uint32_t>(no, TB);
    const uint32_t ja = min(tid * chunk, no), jb = min(ja + chunk, no);
    uint32_t tfirst = t0;
    {
        uint32_t lo = t0, hi = t1;   // largest t in [t0, t1) with tile_off[t] - ob <= ja
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(v.tile_off + mid) - ob <= ja) lo = mid; else hi = mid;
        }
        tfirst = lo;
    }

    while (k < max_pcg) {
        const float* pc_old = v.pc + (size_t)(k & 1) * v.pc_stride;
        float* pc_new = v.pc + (size_t)((k & 1) ^ 1) * v.pc_stride;
        // ------------------------------------------------------------ phase A
        float pdp = 0.0f, pdpc = 0.0f, jp2 = 0.0f, jp2c = 0.0f;   // Kahan pairs
        // direction records of this CTA's cameras: p_c = z_c + beta p_prev_c, phi = J_l p_w
        // (global loads first, so their latency overlaps the point loop below)
        for (uint32_t i = tid; i < ncb; i += TB) {
            float dir[9];
            camera_dir(v, sCid[i], v.z, pc_old, beta, dir);
#pragma unroll
            for (int q = 0; q < 9; ++q) sDir[12 * i + q] = dir[q];
        }
        // owned cameras (b, b + G, ...): one thread per vector entry, all in parallel
        for (int idx = tid; idx < 9 * n_own; idx += TB) {
            const int c = blockIdx.x + (int)gridDim.x * (idx / 9);
            const size_t e = 9 * (size_t)c + idx % 9;
            const float zc = __ldcg(v.z + e);
            const float pk = beta != 0.0f ? fmaf(beta, __ldcg(pc_old + e), zc) : zc;
            pc_new[e] = pk;
            kahan_add(pdp, pdpc, __ldg(v.D + e) * pk * pk);
        }
        for (int i = tid; i < np; i += TB) {
            const float4 po = sP4[i];
            const float p0 = fmaf(beta, po.x, sZ[3 * i]);
            const float p1 = fmaf(beta, po.y, sZ[3 * i + 1]);
            const float p2 = fmaf(beta, po.z, sZ[3 * i + 2]);
            sP4[i] = make_float4(p0, p1, p2, 0.0f);
            sQ[3 * i] = 0.0f;
            sQ[3 * i + 1] = 0.0f;
            sQ[3 * i + 2] = 0.0f;
            kahan_add(pdp, pdpc, fmaf(sD[3 * i] * p0, p0, fmaf(sD[3 * i + 1] * p1, p1, sD[3 * i + 2] * p2 * p2)));
        }
        __syncthreads();
        {
            uint32_t cur = NO_CAM;
            float acc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
            if (ja < jb) {
                uint32_t tcur = tfirst;
                uint32_t tend = __ldg(v.tile_off + tcur + 1) - ob;
                int tpt = (int)(tcur * TILE_PTS) - pb;
                Cam cam;
                float dir[9];
                for (uint32_t j = ja; j < jb; ++j) {
                    while (j >= tend) {
                        ++tcur;
                        tend = __ldg(v.tile_off + tcur + 1) - ob;
                        tpt = (int)(tcur * TILE_PTS) - pb;
                    }
                    const uint32_t key = skey[j];
                    const uint32_t lc = key >> 8;   // the CTA's local camera index
                    const int lp = tpt + (int)(key & 0xffu);
                    if (lc != cur) {
                        if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)sCid[cur] * CA_STRIDE, acc);
                        cur = lc;
                        // records as 128-bit shared loads (both arrays are 16-byte aligned)
                        const float4* r4 = reinterpret_cast<const float4*>(sCam + 16 * lc);
                        const float4 ra = r4[0], rb = r4[1], rc = r4[2], rd = r4[3];
                        cam.R[0] = ra.x; cam.R[1] = ra.y; cam.R[2] = ra.z; cam.R[3] = ra.w;
                        cam.R[4] = rb.x; cam.R[5] = rb.y; cam.R[6] = rb.z; cam.R[7] = rb.w;
                        cam.R[8] = rc.x; cam.t[0] = rc.y; cam.t[1] = rc.z; cam.t[2] = rc.w;
                        cam.f = rd.x; cam.k1 = rd.y; cam.k2 = rd.z;
                        const float4* d4 = reinterpret_cast<const float4*>(sDir + 12 * lc);
                        const float4 da = d4[0], db = d4[1], dc = d4[2];
                        dir[0] = da.x; dir[1] = da.y; dir[2] = da.z; dir[3] = da.w;
                        dir[4] = db.x; dir[5] = db.y; dir[6] = db.z; dir[7] = db.w; dir[8] = dc.x;
                    }
                    const float4 xp = sX4[lp], pp = sP4[lp];
                    const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
                    kahan_add(jp2, jp2c, weighted ? obs_normal<true>(cam, dir, xs, ds, eps, acc, sQ + 3 * lp,
                                                                     __ldg(v.obs_w + ob + j))
                                                  : obs_normal(cam, dir, xs, ds, eps, acc, sQ + 3 * lp));
                }
            }
            // every lane of the warp reaches this one collective
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)sCid[cur] * CA_STRIDE, acc);
        }
        if (v.n_fac > 0) kahan_add(jp2, jp2c, factor_pass(v, sCid, ncb, sDir, v.cam_acc, (int)gridDim.x * TB));
        double sj, sp;
        {
            double mine[XCH_NV] = {0.0, 0.0, 0.0, 0.0}, tot[XCH_NV];
            block_sum2c(jp2, jp2c, pdp, pdpc, red, mine[0], mine[1]);
            if (!exchange(st, pslots, ++epoch, mine, tot, shx)) { ok = false; break; }
            sj = tot[0];
            sp = tot[1];
        }
        // ------------------------------------------------------------ phase B
        const double denom = sj + mu * sp;
        if (!(denom > 0.0) || !isfinite(denom)) {
            numeric_fail = !isfinite(denom);
            break;   // every CTA sees the same sums and leaves here
        }
        alpha = rz / denom;
        const float af = (float)alpha;
        float lrz = 0.0f, lrzc = 0.0f, lrr = 0.0f, lrrc = 0.0f;   // Kahan pairs
        // points: all of it in shared memory
        auto update_points = [&]() {
            for (int i = tid; i < np; i += TB) {
                const int e = 3 * i;
                const float4 p4 = sP4[i];
                const float pq[3] = {p4.x, p4.y, p4.z};
                float r3[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float pk = pq[q];
                    sH[e + q] = fmaf(af, pk, sH[e + q]);
                    r3[q] = fmaf(-af, fmaf(muf, sD[e + q] * pk, sQ[e + q]), sR[e + q]);
                    sR[e + q] = r3[q];
                }
                const float* m = sM + 6 * i;
                const float z0 = fmaf(m[0], r3[0], fmaf(m[1], r3[1], m[2] * r3[2]));
                const float z1 = fmaf(m[1], r3[0], fmaf(m[3], r3[1], m[4] * r3[2]));
                const float z2 = fmaf(m[2], r3[0], fmaf(m[4], r3[1], m[5] * r3[2]));
                sZ[e] = z0; sZ[e + 1] = z1; sZ[e + 2] = z2;
                kahan_add(lrz, lrzc, fmaf(r3[0], z0, fmaf(r3[1], z1, r3[2] * z2)));
                kahan_add(lrr, lrrc, fmaf(r3[0], r3[0], fmaf(r3[1], r3[1], r3[2] * r3[2])));
            }
        };
        if (n_own <= CAMS_PER_PASS) {
            // owned cameras in one pass, nine threads per camera (one per row); their
            // global loads go out before the point update, which hides their latency
            const int j = tid / 9, i = tid - 9 * j;
            const bool mine = j < n_own;
            const int c = blockIdx.x + (int)gridDim.x * j;
            const size_t e = 9 * (size_t)c + i;
            float qi = 0.0f, pk = 0.0f, hk = 0.0f, rk = 0.0f, dk = 0.0f;
            if (mine) {
                const float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
                if (i < 3) {
                    const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
                    qi = fmaf(__ldg(JL + i), __ldcg(ca + 0), fmaf(__ldg(JL + 3 + i), __ldcg(ca + 1),
                                                              __ldg(JL + 6 + i) * __ldcg(ca + 2)));
                } else {
                    qi = __ldcg(ca + i);
                }
                pk = pc_new[e];
                hk = v.h[e];
                rk = v.r[e];
                dk = __ldg(v.D + e);
            }
            update_points();
            float ri = 0.0f;
            if (mine) {
                v.p[e] = pk;
                v.h[e] = fmaf(af, pk, hk);
                ri = fmaf(-af, fmaf(muf, dk * pk, qi), rk);
                v.r[e] = ri;
                s_cam_r[tid] = ri;
            }
            __syncthreads();
            if (mine) {
                const float* M = v.Minv_c + (size_t)c * MC_STRIDE + 9 * i;
                const float* rr9 = s_cam_r + 9 * j;
                float z = 0.0f;
#pragma unroll
                for (int q = 0; q < 9; ++q) z = fmaf(__ldg(M + q), rr9[q], z);
                v.z[e] = z;
                kahan_add(lrz, lrzc, ri * z);
                kahan_add(lrr, lrrc, ri * ri);
                v.cam_acc[(size_t)c * CA_STRIDE + i] = 0.0f;
            }
        } else {
            // owned cameras: nine threads per camera (one per row), CAMS_PER_PASS per pass
            for (int j0 = 0; j0 < n_own; j0 += CAMS_PER_PASS) {
                const int idx = tid;
                const int j = j0 + idx / 9, i = idx % 9;
                const bool mine = idx < 9 * CAMS_PER_PASS && j < n_own;
                const int c = blockIdx.x + (int)gridDim.x * j;
                const size_t e = 9 * (size_t)c + i;
                float ri = 0.0f;
                if (mine) {
                    const float* ca = v.cam_acc + (size_t)c * CA_STRIDE;
                    float qi;
                    if (i < 3) {
                        const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
                        qi = fmaf(__ldg(JL + i), __ldcg(ca + 0), fmaf(__ldg(JL + 3 + i), __ldcg(ca + 1),
                                                                  __ldg(JL + 6 + i) * __ldcg(ca + 2)));
                    } else {
                        qi = __ldcg(ca + i);
                    }
                    const float pk = pc_new[e];
                    v.p[e] = pk;
                    v.h[e] = fmaf(af, pk, v.h[e]);
                    ri = fmaf(-af, fmaf(muf, __ldg(v.D + e) * pk, qi), v.r[e]);
                    v.r[e] = ri;
                    s_cam_r[idx] = ri;
                }
                __syncthreads();
                if (mine) {
                    const float* M = v.Minv_c + (size_t)c * MC_STRIDE + 9 * i;
                    const float* rr9 = s_cam_r + 9 * (idx / 9);
                    float z = 0.0f;
#pragma unroll
                    for (int q = 0; q < 9; ++q) z = fmaf(__ldg(M + q), rr9[q], z);
                    v.z[e] = z;
                    kahan_add(lrz, lrzc, ri * z);
                    kahan_add(lrr, lrrc, ri * ri);
                    v.cam_acc[(size_t)c * CA_STRIDE + i] = 0.0f;
                }
                __syncthreads();
            }
            update_points();
        }
        double rzn, rrn;
        {
            double mine[XCH_NV] = {0.0, 0.0, 0.0, 0.0}, tot[XCH_NV];
            block_sum2c(lrz, lrzc, lrr, lrrc, red, mine[0], mine[1]);
            if (!exchange(st, pslots, ++epoch, mine, tot, shx)) { ok = false; break; }
            rzn = tot[0];
            rrn = tot[1];
        }
        // ------------------------------------------------------------ phase C
        ++k;
        rr = rrn;
        if (!isfinite(rzn) || !isfinite(rrn)) { numeric_fail = true; break; }
        if (rrn <= tol2 * rr0) break;
        beta = (float)(rzn / rz);
        rz = rzn;
    }
    // points' h back to global for the candidate step
    for (int i = tid; i < n3; i += TB) v.h[g0 + i] = sH[i];
    if (blockIdx.x == 0 && tid == 0) {
        st->pcg_iter = k;
        st->pcg_total += k;
        st->rz = rz;
        st->rr = rr;
        st->alpha = alpha;
        st->beta = beta;
        st->pcg_active = 0;
        if (!ok) st->status = 5;
        else if (numeric_fail) st->status = 4;
    }
}


// ------------------------------------------------------------ one-exchange form ---

namespace {


__device__ __forceinline__ bool owns(const uint32_t* sOwn, int lc) { return (sOwn[lc >> 5] >> (lc & 31)) & 1u; }

// Camera direction records (phi = J_l u_w, u_t, u_intr) of the CTA's cameras from u.
template <int TB>
__device__ __forceinline__ void camera_dirs(const Views<float>& v, const uint32_t* sCid, const float* sCu,
                                            float* sDir, int ne) {
    for (int e = threadIdx.x; e < ne; e += TB) {
        const int lc = e / 9, i = e - 9 * lc;
        float d;
        if (i < 3) {
            const float* JL = v.cam_pre + (size_t)sCid[lc] * CP_STRIDE + CP_JL + 3 * i;
            const float* u = sCu + 9 * lc;
            d = fmaf(__ldg(JL), u[0], fmaf(__ldg(JL + 1), u[1], __ldg(JL + 2) * u[2]));
        } else {
            d = sCu[e];
        }
        sDir[12 * lc + i] = d;
    }
}

// Warp sums of the update's three compensated partials (Kahan pairs s - c) into
// red[3 * warp + k]: compensated FP32 pairs inside the warp (warp_sum_pair).
__device__ __forceinline__ void warp_partials3(float a, float ac, float b, float bc, float c, float cc,
                                               double* red) {
    const double sa = warp_sum_pair(a, -ac), sb = warp_sum_pair(b, -bc), sc = warp_sum_pair(c, -cc);
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        red[3 * w] = sa;
        red[3 * w + 1] = sb;
        red[3 * w + 2] = sc;
    }
}

// Residual replacement of the one-exchange form: with A h assembled (points in sQ,
// cameras in the accumulator set `cacc`), r = b - A h with b = -g and u = M^-1 r (p and
// s are kept); the partials of r^T u, |r|^2 and u^T D u go to red_u as the update phase
// leaves them, and the owners clear the accumulator set `clear` as it does.
template <int TB>
__device__ void replace_residual(const Views<float>& v, const float* cacc, const uint32_t* sCid, const uint32_t* sOwn,
                                 int ne, int np, size_t g0, float muf, const float4* sX4, float4* sU4,
                                 const float* sD2, float* sR, const float* sH, float* sQ, const float* sM, float* sCu,
                                 float* sCr, const float* sCh, float* clear, double* red_u) {
    const int tid = threadIdx.x;
    float lg = 0.0f, lr = 0.0f, lu = 0.0f, lgc = 0.0f, lrc = 0.0f, luc = 0.0f;   // Kahan pairs
    // cameras, step 1: r = -g - (J^T J h + mu D h)
    for (int e = tid; e < ne; e += TB) {
        const int lc = e / 9, i = e - 9 * lc;
        const uint32_t c = sCid[lc];
        const float* ca = cacc + (size_t)c * CA_STRIDE;
        float q;
        if (i < 3) {
            const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
            q = fmaf(__ldg(JL + i), __ldcg(ca + 0), fmaf(__ldg(JL + 3 + i), __ldcg(ca + 1),
                                                       __ldg(JL + 6 + i) * __ldcg(ca + 2)));
        } else {
            q = __ldcg(ca + i);
        }
        const float ah = fmaf(muf, __ldg(v.D + 9 * (size_t)c + i) * sCh[e], q);
        sCr[e] = (float)(-v.cam_lin[(size_t)c * CL_STRIDE + CL_G + i]) - ah;
    }
    // points
    for (int i = tid; i < np; i += TB) {
        const float Dq[3] = {sX4[i].w, sU4[i].w, sD2[i]};
        float r3[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int e = 3 * i + q;
            const float ah = fmaf(muf, Dq[q] * sH[e], sQ[e]);
            r3[q] = -v.g[g0 + e] - ah;
            sR[e] = r3[q];
            sQ[e] = 0.0f;
        }
        const float* m = sM + 6 * i;
        const float z0 = fmaf(m[0], r3[0], fmaf(m[1], r3[1], m[2] * r3[2]));
        const float z1 = fmaf(m[1], r3[0], fmaf(m[3], r3[1], m[4] * r3[2]));
        const float z2 = fmaf(m[2], r3[0], fmaf(m[4], r3[1], m[5] * r3[2]));
        sU4[i] = make_float4(z0, z1, z2, Dq[1]);
        kahan_add(lg, lgc, fmaf(r3[0], z0, fmaf(r3[1], z1, r3[2] * z2)));
        kahan_add(lr, lrc, fmaf(r3[0], r3[0], fmaf(r3[1], r3[1], r3[2] * r3[2])));
        kahan_add(lu, luc, fmaf(Dq[0] * z0, z0, fmaf(Dq[1] * z1, z1, Dq[2] * z2 * z2)));
    }
    __syncthreads();   // camera r
    // cameras, step 2: u = M^-1 r
    for (int e = tid; e < ne; e += TB) {
        const int lc = e / 9, i = e - 9 * lc;
        const uint32_t c = sCid[lc];
        const float* M = v.Minv_c + (size_t)c * MC_STRIDE + 9 * i;
        const float* r9 = sCr + 9 * lc;
        float z = 0.0f;
#pragma unroll
        for (int q = 0; q < 9; ++q) z = fmaf(__ldg(M + q), r9[q], z);
        sCu[e] = z;
        if (owns(sOwn, lc)) {
            const float ri = r9[i];
            kahan_add(lg, lgc, ri * z);
            kahan_add(lr, lrc, ri * ri);
            kahan_add(lu, luc, __ldg(v.D + 9 * (size_t)c + i) * z * z);
            clear[(size_t)c * CA_STRIDE + i] = 0.0f;
        }
    }
    warp_partials3(lg, lgc, lr, lrc, lu, luc, red_u);
}

}  // namespace

template <int TB>
__global__ void __launch_bounds__(TB, 1) k_pcg_persistent_1x(Views<float> v, const uint32_t* __restrict__ blk_tile,
                                                         const uint32_t* __restrict__ blk_cam_off,
                                                         const uint32_t* __restrict__ blk_cams,
                                                         double* __restrict__ pslots) {
    DevState* st = v.st;
    if (st->pcg_active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NW = TB / 32;
    __shared__ double red_u[3 * NW], red_m[NW], shx[XCH_NV + 1];
    const int tid = threadIdx.x;
    const uint32_t t0 = blk_tile[blockIdx.x], t1 = blk_tile[blockIdx.x + 1];
    const uint32_t ob = v.tile_off[t0], oe = v.tile_off[t1];
    const uint32_t no = oe - ob;
    const int pb = (int)(t0 * TILE_PTS);
    const int pe = min((int)(t1 * TILE_PTS), v.n_pts);
    const int np = pe > pb ? pe - pb : 0;
    const int n3p = (3 * np + 3) & ~3;
    const uint32_t cb = blk_cam_off[blockIdx.x], ncb = blk_cam_off[blockIdx.x + 1] - cb;
    const int ne = 9 * (int)ncb;   // camera vector entries of this CTA
    // shared memory, carved in the order pcg1_smem_bytes counts it
    uint32_t* skey = reinterpret_cast<uint32_t*>(smem);
    float4* sX4 = reinterpret_cast<float4*>(smem + (((size_t)no * 4 + 15) & ~(size_t)15));   // (X, D_0)
    float4* sU4 = sX4 + np;                                                                  // (u, D_1)
    float* sD2 = reinterpret_cast<float*>(sU4 + np);
    float* sP = sD2 + ((np + 3) & ~3);
    float* sS = sP + n3p;
    float* sR = sS + n3p;
    float* sH = sR + n3p;
    float* sQ = sH + n3p;
    float* sM = sQ + n3p;
    uint32_t* sCid = reinterpret_cast<uint32_t*>(sM + ((6 * np + 3) & ~3));
    uint32_t* sOwn = sCid + ((ncb + 3) & ~3u);
    float* sCam = reinterpret_cast<float*>(sOwn + ((((ncb + 31) >> 5) + 3) & ~3u));
    float* sDir = sCam + 16 * (size_t)ncb;
    float* sCu = sDir + 12 * (size_t)ncb;
    float* sCp = sCu + ne;
    float* sCs = sCp + ne;
    float* sCr = sCs + ne;
    float* sCh = sCr + ne;
    const size_t g0 = v.pt_off + 3 * (size_t)pb;
    const size_t cas = (size_t)CA_STRIDE * v.n_cams;   // floats between accumulator sets

    for (uint32_t i = tid; i < ncb; i += TB) sCid[i] = __ldg(blk_cams + cb + i) & ~BLK_CAM_OWNER;
    for (uint32_t w = tid; w < (ncb + 31) / 32; w += TB) {
        uint32_t m = 0u;
        for (uint32_t j = 0; j < 32u && 32u * w + j < ncb; ++j)
            if (__ldg(blk_cams + cb + 32u * w + j) & BLK_CAM_OWNER) m |= 1u << j;
        sOwn[w] = m;
    }
    for (uint32_t i = tid; i < no; i += TB) skey[i] = __ldg(v.obs_key + ob + i);
    // partials of r^T u, |r|^2, u^T D u (Kahan pairs)
    float lg = 0.0f, lr = 0.0f, lu = 0.0f, lgc = 0.0f, lrc = 0.0f, luc = 0.0f;
    for (int i = tid; i < np; i += TB) {
        const size_t e = g0 + 3 * (size_t)i;
        const float D0 = v.D[e], D1 = v.D[e + 1], D2 = v.D[e + 2];
        const float u0 = v.z[e], u1 = v.z[e + 1], u2 = v.z[e + 2];
        const float r0 = v.r[e], r1 = v.r[e + 1], r2 = v.r[e + 2];
        sX4[i] = make_float4(v.x[e], v.x[e + 1], v.x[e + 2], D0);
        sU4[i] = make_float4(u0, u1, u2, D1);
        sD2[i] = D2;
        sR[3 * i] = r0; sR[3 * i + 1] = r1; sR[3 * i + 2] = r2;
        kahan_add(lg, lgc, fmaf(r0, u0, fmaf(r1, u1, r2 * u2)));
        kahan_add(lr, lrc, fmaf(r0, r0, fmaf(r1, r1, r2 * r2)));
        kahan_add(lu, luc, fmaf(D0 * u0, u0, fmaf(D1 * u1, u1, D2 * u2 * u2)));
    }
    for (int i = tid; i < n3p; i += TB) {
        sP[i] = 0.0f;
        sS[i] = 0.0f;
        sH[i] = 0.0f;
        sQ[i] = 0.0f;
    }
    for (int i = tid; i < 6 * np; i += TB) sM[i] = v.Minv_p[6 * (size_t)pb + i];
    __syncthreads();   // camera ids and owner bits
    // keys carry the CTA-local camera index from here on (no search in the loop)
    for (uint32_t i = tid; i < no; i += TB) {
        const uint32_t key = skey[i];
        skey[i] = (local_cam(sCid, ncb, key >> 8) << 8) | (key & 0xffu);
    }
    for (uint32_t i = tid; i < 16 * ncb; i += TB)
        sCam[i] = __ldg(v.cam_pre + (size_t)sCid[i / 16] * CP_STRIDE + i % 16);
    for (int e = tid; e < ne; e += TB) {
        const int lc = e / 9, i = e - 9 * lc;
        const size_t ge = 9 * (size_t)sCid[lc] + i;
        const float u = v.z[ge], r = v.r[ge];
        sCu[e] = u;
        sCr[e] = r;
        sCp[e] = 0.0f;
        sCs[e] = 0.0f;
        sCh[e] = 0.0f;
        if (owns(sOwn, lc)) {
            kahan_add(lg, lgc, r * u);
            kahan_add(lr, lrc, r * r);
            kahan_add(lu, luc, __ldg(v.D + ge) * u * u);
        }
    }
    warp_partials3(lg, lgc, lr, lrc, lu, luc, red_u);
    __syncthreads();   // camera u
    camera_dirs<TB>(v, sCid, sCu, sDir, ne);
    __syncthreads();

    const double mu = st->mu;
    const float muf = (float)mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;   // robust loss: IRLS weights per observation
    const double tol2 = st->opt.tol * st->opt.tol;
    const double rr0 = st->rr0;
    const int max_pcg = st->opt.max_pcg;
    double gam = st->rz, gam_prev = 1.0, alpha = 0.0, alpha_prev = 1.0, rr = rr0;
    float beta = 0.0f;
    unsigned long long epoch = 0ull;
    int k = 0;    // PCG updates
    int it = 0;   // operator passes (they rotate the camera accumulator sets)
    // Residual replacement (van der Vorst and Ye, SIAM J. Sci. Comput. 22, 2000): when the
    // recursively updated residual meets the tolerance, one operator pass on h gives the
    // true residual r = b - A h (b = -g), which replaces r (and u = M^-1 r) while the
    // search directions p, s are kept; the solve stops only on a true residual that
    // meets the tolerance.  At most MAX_CHECKS such checks per solve; past them the
    // recursive residual decides.
    constexpr int MAX_CHECKS = 4;
    int checks = 0;
    bool verify = false;   // the coming operator pass applies A to h
    bool true_r = false;   // r was just replaced by the true residual
    bool ok = true, numeric_fail = false;
    // this thread's observation chunk (block-local indices) and its first tile
    const uint32_t chunk = odd_chunk<uint32_t>(no, TB);
    const uint32_t ja = min(tid * chunk, no), jb = min(ja + chunk, no);
    uint32_t tfirst = t0;
    {
        uint32_t lo = t0, hi = t1;   // largest t in [t0, t1) with tile_off[t] - ob <= ja
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(v.tile_off + mid) - ob <= ja) lo = mid; else hi = mid;
        }
        tfirst = lo;
    }

    while (k < max_pcg) {
        float* cacc = v.cam_acc + (size_t)(it % CA_SETS) * cas;
        // ------------------------------------------------------------ M: w = A u (A h when verifying)
        float jj = 0.0f, jjc = 0.0f;   // Kahan pair
        {
            uint32_t cur = NO_CAM;
            float acc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
            if (ja < jb) {
                uint32_t tcur = tfirst;
                uint32_t tend = __ldg(v.tile_off + tcur + 1) - ob;
                int tpt = (int)(tcur * TILE_PTS) - pb;
                Cam cam;
                float dir[9];
                for (uint32_t j = ja; j < jb; ++j) {
                    while (j >= tend) {
                        ++tcur;
                        tend = __ldg(v.tile_off + tcur + 1) - ob;
                        tpt = (int)(tcur * TILE_PTS) - pb;
                    }
                    const uint32_t key = skey[j];
                    const uint32_t lc = key >> 8;   // the CTA's local camera index
                    const int lp = tpt + (int)(key & 0xffu);
                    if (lc != cur) {
                        if (cur != NO_CAM) flush_matvec(cacc + (size_t)sCid[cur] * CA_STRIDE, acc);
                        cur = lc;
                        // records as 128-bit shared loads (both arrays are 16-byte aligned)
                        const float4* r4 = reinterpret_cast<const float4*>(sCam + 16 * lc);
                        const float4 ra = r4[0], rb = r4[1], rc = r4[2], rd = r4[3];
                        cam.R[0] = ra.x; cam.R[1] = ra.y; cam.R[2] = ra.z; cam.R[3] = ra.w;
                        cam.R[4] = rb.x; cam.R[5] = rb.y; cam.R[6] = rb.z; cam.R[7] = rb.w;
                        cam.R[8] = rc.x; cam.t[0] = rc.y; cam.t[1] = rc.z; cam.t[2] = rc.w;
                        cam.f = rd.x; cam.k1 = rd.y; cam.k2 = rd.z;
                        const float4* d4 = reinterpret_cast<const float4*>(sDir + 12 * lc);
                        const float4 da = d4[0], db = d4[1], dc = d4[2];
                        dir[0] = da.x; dir[1] = da.y; dir[2] = da.z; dir[3] = da.w;
                        dir[4] = db.x; dir[5] = db.y; dir[6] = db.z; dir[7] = db.w; dir[8] = dc.x;
                    }
                    const float4 xp = sX4[lp], up = sU4[lp];
                    const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {up.x, up.y, up.z};
                    kahan_add(jj, jjc, weighted ? obs_normal<true>(cam, dir, xs, ds, eps, acc, sQ + 3 * lp,
                                                                   __ldg(v.obs_w + ob + j))
                                                : obs_normal(cam, dir, xs, ds, eps, acc, sQ + 3 * lp));
                }
            }
            // every lane of the warp reaches this one collective
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM) flush_matvec(cacc + (size_t)sCid[cur] * CA_STRIDE, acc);
        }
        if (v.n_fac > 0) kahan_add(jj, jjc, factor_pass(v, sCid, ncb, sDir, cacc, (int)gridDim.x * TB));
        const double jw = warp_sum_pair(jj, -jjc);
        if ((tid & 31) == 0) red_m[tid >> 5] = jw;
        __syncthreads();
        // ------------------------------------------------------------ X: exchange
        double mine[XCH_NV] = {0.0, 0.0, 0.0, 0.0}, tot[XCH_NV];
        if (tid == 0) {
            for (int w = 0; w < NW; ++w) {
                if (!verify) {   // a verification pass carries only its operator sums
                    mine[0] += red_u[3 * w];
                    mine[1] += red_u[3 * w + 1];
                    mine[2] += red_u[3 * w + 2];
                }
                mine[3] += red_m[w];
            }
        }
        if (!exchange(st, pslots, ++epoch, mine, tot, shx)) { ok = false; break; }
        if (verify) {
            // ---------------------------------------------------- R: r = b - A h, restart
            replace_residual<TB>(v, cacc, sCid, sOwn, ne, np, g0, muf, sX4, sU4, sD2, sR, sH, sQ, sM, sCu, sCr, sCh,
                                 v.cam_acc + (size_t)((it + 2) % CA_SETS) * cas, red_u);
            __syncthreads();   // camera u
            camera_dirs<TB>(v, sCid, sCu, sDir, ne);
            __syncthreads();
            verify = false;
            true_r = true;
            ++it;
            continue;
        }
        const double g_k = tot[0], rr_k = tot[1], udu = tot[2], jju = tot[3];
        if (!isfinite(g_k) || !isfinite(rr_k)) { numeric_fail = true; break; }
        rr = rr_k;
        if (k > 0 && rr_k <= tol2 * rr0) {
            if (true_r || checks >= MAX_CHECKS) break;   // a true residual (or no checks left)
            // check the recursive residual against the true one: the next pass applies A to h
            ++checks;
            verify = true;
            for (int i = tid; i < np; i += TB)
                sU4[i] = make_float4(sH[3 * i], sH[3 * i + 1], sH[3 * i + 2], sU4[i].w);
            for (int e = tid; e < ne; e += TB) sCu[e] = sCh[e];
            __syncthreads();
            camera_dirs<TB>(v, sCid, sCu, sDir, ne);
            __syncthreads();
            ++it;
            continue;
        }
        const double b_k = k > 0 ? g_k / gam_prev : 0.0;
        const double delta = jju + mu * udu;                                  // u^T A u
        const double denom = k > 0 ? delta - b_k * g_k / alpha_prev : delta;   // p^T A p
        if (!(denom > 0.0) || !isfinite(denom)) {
            numeric_fail = !isfinite(denom);
            break;   // every CTA sees the same sums and leaves here
        }
        gam = g_k;
        alpha = g_k / denom;
        beta = (float)b_k;
        const float af = (float)alpha;
        // ------------------------------------------------------------ U: update
        lg = lr = lu = lgc = lrc = luc = 0.0f;
        // cameras, step 1: w from the assembled sums, then p, s, h, r
        for (int e = tid; e < ne; e += TB) {
            const int lc = e / 9, i = e - 9 * lc;
            const uint32_t c = sCid[lc];
            const float* ca = cacc + (size_t)c * CA_STRIDE;
            float q;
            if (i < 3) {
                const float* JL = v.cam_pre + (size_t)c * CP_STRIDE + CP_JL;
                q = fmaf(__ldg(JL + i), __ldcg(ca + 0), fmaf(__ldg(JL + 3 + i), __ldcg(ca + 1),
                                                           __ldg(JL + 6 + i) * __ldcg(ca + 2)));
            } else {
                q = __ldcg(ca + i);
            }
            const float u = sCu[e];
            const float w = fmaf(muf, __ldg(v.D + 9 * (size_t)c + i) * u, q);
            const float pk = fmaf(beta, sCp[e], u);
            const float sk = fmaf(beta, sCs[e], w);
            sCp[e] = pk;
            sCs[e] = sk;
            sCh[e] = fmaf(af, pk, sCh[e]);
            sCr[e] = fmaf(-af, sk, sCr[e]);
        }
        // points: all of it in shared memory
        for (int i = tid; i < np; i += TB) {
            const float4 x4 = sX4[i], u4 = sU4[i];
            const float Dq[3] = {x4.w, u4.w, sD2[i]};
            const float uq[3] = {u4.x, u4.y, u4.z};
            float r3[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int e = 3 * i + q;
                const float w = fmaf(muf, Dq[q] * uq[q], sQ[e]);
                const float pk = fmaf(beta, sP[e], uq[q]);
                const float sk = fmaf(beta, sS[e], w);
                sP[e] = pk;
                sS[e] = sk;
                sQ[e] = 0.0f;
                sH[e] = fmaf(af, pk, sH[e]);
                r3[q] = fmaf(-af, sk, sR[e]);
                sR[e] = r3[q];
            }
            const float* m = sM + 6 * i;
            const float z0 = fmaf(m[0], r3[0], fmaf(m[1], r3[1], m[2] * r3[2]));
            const float z1 = fmaf(m[1], r3[0], fmaf(m[3], r3[1], m[4] * r3[2]));
            const float z2 = fmaf(m[2], r3[0], fmaf(m[4], r3[1], m[5] * r3[2]));
            sU4[i] = make_float4(z0, z1, z2, u4.w);
            kahan_add(lg, lgc, fmaf(r3[0], z0, fmaf(r3[1], z1, r3[2] * z2)));
            kahan_add(lr, lrc, fmaf(r3[0], r3[0], fmaf(r3[1], r3[1], r3[2] * r3[2])));
            kahan_add(lu, luc, fmaf(Dq[0] * z0, z0, fmaf(Dq[1] * z1, z1, Dq[2] * z2 * z2)));
        }
        __syncthreads();   // camera r
        // cameras, step 2: u = M^-1 r; the owner adds the partials and clears the
        // accumulator set that the iteration after next fills (its last readers are
        // past the exchange above)
        {
            float* clear = v.cam_acc + (size_t)((it + 2) % CA_SETS) * cas;
            for (int e = tid; e < ne; e += TB) {
                const int lc = e / 9, i = e - 9 * lc;
                const uint32_t c = sCid[lc];
                const float* M = v.Minv_c + (size_t)c * MC_STRIDE + 9 * i;
                const float* r9 = sCr + 9 * lc;
                float z = 0.0f;
#pragma unroll
                for (int q = 0; q < 9; ++q) z = fmaf(__ldg(M + q), r9[q], z);
                sCu[e] = z;
                if (owns(sOwn, lc)) {
                    const float ri = r9[i];
                    kahan_add(lg, lgc, ri * z);
                    kahan_add(lr, lrc, ri * ri);
                    kahan_add(lu, luc, __ldg(v.D + 9 * (size_t)c + i) * z * z);
                    clear[(size_t)c * CA_STRIDE + i] = 0.0f;
                }
            }
        }
        warp_partials3(lg, lgc, lr, lrc, lu, luc, red_u);
        __syncthreads();   // camera u
        camera_dirs<TB>(v, sCid, sCu, sDir, ne);
        __syncthreads();
        gam_prev = g_k;
        alpha_prev = alpha;
        true_r = false;
        ++k;
        ++it;
    }
    // closing exchange: past it no CTA reads an accumulator set any more, so the
    // owners leave all of them cleared
    if (ok) {
        double z4[XCH_NV] = {0.0, 0.0, 0.0, 0.0}, t4[XCH_NV];
        __syncthreads();
        ok = exchange(st, pslots, ++epoch, z4, t4, shx);
    }
    for (int e = tid; e < ne; e += TB) {
        const int lc = e / 9, i = e - 9 * lc;
        if (!owns(sOwn, lc)) continue;
        const uint32_t c = sCid[lc];
        v.h[9 * (size_t)c + i] = sCh[e];
        if (ok)
            for (int set = 0; set < CA_SETS; ++set) v.cam_acc[set * cas + (size_t)c * CA_STRIDE + i] = 0.0f;
    }
    for (int i = tid; i < 3 * np; i += TB) v.h[g0 + i] = sH[i];
    if (blockIdx.x == 0 && tid == 0) {
        st->pcg_iter = k;
        st->pcg_total += k;
        st->rz = gam;
        st->rr = rr;
        st->alpha = alpha;
        st->beta = beta;
        st->pcg_active = 0;
        if (!ok) st->status = 5;
        else if (numeric_fail) st->status = 4;
    }
}

// ------------------------------------------------------------------ host ----------

int persistent_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

cudaError_t persistent_prepare(int form, int smem_bytes, int* blocks_per_sm) {
    const void* f = form == PCG_TWO_EXCHANGE ? (const void*)k_pcg_persistent<PCG_TB>
                                            : (const void*)k_pcg_persistent_1x<PCG_TB>;
    cudaError_t e = ensure_dynamic_smem(f, smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, PCG_TB, smem_bytes);
}

cudaError_t launch_pcg_persistent(const Views<float>& v, const uint32_t* blk_tile, const uint32_t* blk_cam_off,
                                  const uint32_t* blk_cams, double* pslots, int grid, int smem_bytes, int form,
                                  cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PCG_TB);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (form == PCG_TWO_EXCHANGE)
        return cudaLaunchKernelEx(&cfg, k_pcg_persistent<PCG_TB>, v, blk_tile, blk_cam_off, blk_cams, pslots);
    return cudaLaunchKernelEx(&cfg, k_pcg_persistent_1x<PCG_TB>, v, blk_tile, blk_cam_off, blk_cams, pslots);
}

// Self-test of the bounded grid wait: a cooperative grid of `grid` CTAs waits at a
// barrier that counts one CTA more than it has, which nothing will ever complete.
// Every CTA must give up after `timeout_ns`, set the shared error word and return;
// scratch = {arrival count (u64), error word (i32), CTAs that gave up (u32)}.
__global__ void k_selftest_wait(unsigned long long* scratch, long long timeout_ns) {
    int* err = reinterpret_cast<int*>(scratch + 1);
    unsigned int* gave_up = reinterpret_cast<unsigned int*>(scratch + 1) + 1;
    const bool ok = grid_sync_on(scratch, err, gridDim.x + 1, 1ull, timeout_ns);
    if (!ok && threadIdx.x == 0) atomicAdd(gave_up, 1u);
}

__global__ void k_selftest_rcp64(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = rcp64(x[i]);
}

void launch_selftest_rcp64(const double* x, double* y, int64_t n, cudaStream_t s) {
    const int64_t b = (n + 255) / 256;
    k_selftest_rcp64<<<(unsigned int)(b < 1024 ? b : 1024), 256, 0, s>>>(x, y, n);
}

cudaError_t launch_selftest_wait(void* scratch, int grid, long long timeout_ns, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(64);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_selftest_wait, (unsigned long long*)scratch, timeout_ns);
}

}  // namespace gbba
