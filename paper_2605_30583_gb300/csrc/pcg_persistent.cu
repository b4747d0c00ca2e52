// Persistent PCGNR (Sec. V-A of arXiv 2605.30583) for problems whose tiles fit in the
// GPU's aggregate shared memory.
//
// One cooperative launch runs every PCG iteration of one LM step.  The grid is one
// CTA per SM; CTA b owns a contiguous run of tiles (balanced by observation count)
// and keeps, for the whole solve, its observation keys and its points' X, D, M^-1,
// r, z, h, p and q in shared memory.  Per iteration only the camera-side data
// (directions, accumulators, the camera part of the vectors) goes through global
// memory.  Two grid-wide barriers separate the phases:
//   A  p = z + beta p (points in smem; cameras double-buffered in global), then
//      q = J^T J p + mu D p with |J p|^2 and p^T D p;
//   B  alpha = r^T z / (|J p|^2 + mu p^T D p); h += alpha p; r -= alpha q; z = M^-1 r;
//   C  r^T z, |r|^2 -> stop test (|r| <= tol |r_0| or the iteration cap), beta.
// Every CTA takes the stop decision from the same global sums, so all leave the
// loop together.  The barrier spins are time-bounded: on a time-out the CTA sets an
// error flag, every CTA leaves, and the solve reports BA_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"
#include "mixed_common.cuh"

namespace gbba {

namespace {

constexpr long long BARRIER_TIMEOUT_NS = 2000000000LL;   // 2 s

// Grid-wide barrier for a co-resident (cooperative) grid; false on time-out or when
// another CTA has already reported one.
__device__ __forceinline__ bool grid_sync(DevState* st, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* gen = &st->bar_gen;
        volatile int* err = &st->bar_err;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == nblocks - 1) {
            st->bar_count = 0u;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const long long t0 = global_ns();
            while (*gen == g) {
                if (*err) { ok = 0; break; }
                if (global_ns() - t0 > BARRIER_TIMEOUT_NS) {
                    atomicExch(&st->bar_err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum over slots of component k of one slot set, broadcast to the whole CTA.
__device__ __forceinline__ void slot_pair(const double* set, double* sh, double& a, double& b) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const double x = slot_sum_warp(set, 0), y = slot_sum_warp(set, 1);
        if (threadIdx.x == 0) { sh[0] = x; sh[1] = y; }
    }
    __syncthreads();
    a = sh[0];
    b = sh[1];
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
    __shared__ double sh2[2];
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
    for (uint32_t i = tid; i < ncb; i += TB) sCid[i] = __ldg(blk_cams + cb + i);
    for (uint32_t i = tid; i < 16 * ncb; i += TB)
        sCam[i] = __ldg(v.cam_pre + (size_t)__ldg(blk_cams + cb + i / 16) * CP_STRIDE + i % 16);
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

    const double mu = st->mu;
    const float muf = (float)mu;
    const float eps = (float)st->opt.eps;
    const bool weighted = st->opt.loss != 0;   // robust loss: IRLS weights per observation
    const double tol2 = st->opt.tol * st->opt.tol;
    const double rr0 = st->rr0;
    const int max_pcg = st->opt.max_pcg;
    double rz = st->rz, rr = rr0, alpha = 0.0;
    float beta = 0.0f;
    int k = 0;
    bool ok = true, numeric_fail = false;
    // this thread's observation chunk (block-local indices) and its first tile
    const uint32_t chunk = (no + TB - 1) / TB;
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
        const int set = k % 3;
        double* mv = pslots + (size_t)set * NSLOT * SLOT_STRIDE;
        double* up = pslots + (size_t)(3 + set) * NSLOT * SLOT_STRIDE;
        const float* pc_old = v.pc + (size_t)(k & 1) * v.pc_stride;
        float* pc_new = v.pc + (size_t)((k & 1) ^ 1) * v.pc_stride;
        // ------------------------------------------------------------ phase A
        float pdp = 0.0f, jp2 = 0.0f;
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
            pdp = fmaf(__ldg(v.D + e) * pk, pk, pdp);
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
            pdp = fmaf(sD[3 * i] * p0, p0, fmaf(sD[3 * i + 1] * p1, p1, fmaf(sD[3 * i + 2] * p2, p2, pdp)));
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
                    const uint32_t c = key >> 8;
                    const int lp = tpt + (int)(key & 0xffu);
                    if (c != cur) {
                        if (cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
                        cur = c;
                        uint32_t lo = 0, hi = ncb;   // local index of camera c
                        while (hi - lo > 1) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (sCid[mid] <= c) lo = mid; else hi = mid;
                        }
                        const float* rec = sCam + 16 * lo;
#pragma unroll
                        for (int q = 0; q < 9; ++q) cam.R[q] = rec[q];
                        cam.t[0] = rec[9]; cam.t[1] = rec[10]; cam.t[2] = rec[11];
                        cam.f = rec[12]; cam.k1 = rec[13]; cam.k2 = rec[14];
                        const float* dr = sDir + 12 * lo;
#pragma unroll
                        for (int q = 0; q < 9; ++q) dir[q] = dr[q];
                    }
                    const float4 xp = sX4[lp], pp = sP4[lp];
                    const float xs[3] = {xp.x, xp.y, xp.z}, ds[3] = {pp.x, pp.y, pp.z};
                    if (weighted) jp2 += obs_normal<true>(cam, dir, xs, ds, eps, acc, sQ + 3 * lp, __ldg(v.obs_w + ob + j));
                    else jp2 += obs_normal(cam, dir, xs, ds, eps, acc, sQ + 3 * lp);
                }
            }
            // every lane of the warp reaches this one collective
            const bool head = seg_reduce<9>(cur, acc);
            if (head && cur != NO_CAM) flush_matvec(v.cam_acc + (size_t)cur * CA_STRIDE, acc);
        }
        {
            double bj, bp;
            block_sum2(jp2, pdp, red, bj, bp);
            if (tid == 0) {
                slot_add(mv, 0, bj);
                slot_add(mv, 1, bp);
            }
        }
        if (!grid_sync(st, gridDim.x)) { ok = false; break; }
        // ------------------------------------------------------------ phase B
        double sj, sp;
        slot_pair(mv, sh2, sj, sp);
        const double denom = sj + mu * sp;
        if (!(denom > 0.0) || !isfinite(denom)) {
            numeric_fail = !isfinite(denom);
            break;   // every CTA sees the same sums and leaves here
        }
        alpha = rz / denom;
        const float af = (float)alpha;
        float lrz = 0.0f, lrr = 0.0f;
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
                ri = fmaf(-af, fmaf(muf * __ldg(v.D + e), pk, qi), v.r[e]);
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
                lrz = fmaf(ri, z, lrz);
                lrr = fmaf(ri, ri, lrr);
                v.cam_acc[(size_t)c * CA_STRIDE + i] = 0.0f;
            }
            __syncthreads();
        }
        for (int i = tid; i < np; i += TB) {
            const int e = 3 * i;
            const float4 p4 = sP4[i];
            const float pq[3] = {p4.x, p4.y, p4.z};
            float r3[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float pk = pq[q];
                sH[e + q] = fmaf(af, pk, sH[e + q]);
                r3[q] = fmaf(-af, fmaf(muf * sD[e + q], pk, sQ[e + q]), sR[e + q]);
                sR[e + q] = r3[q];
            }
            const float* m = sM + 6 * i;
            const float z0 = fmaf(m[0], r3[0], fmaf(m[1], r3[1], m[2] * r3[2]));
            const float z1 = fmaf(m[1], r3[0], fmaf(m[3], r3[1], m[4] * r3[2]));
            const float z2 = fmaf(m[2], r3[0], fmaf(m[4], r3[1], m[5] * r3[2]));
            sZ[e] = z0; sZ[e + 1] = z1; sZ[e + 2] = z2;
            lrz = fmaf(r3[0], z0, fmaf(r3[1], z1, fmaf(r3[2], z2, lrz)));
            lrr = fmaf(r3[0], r3[0], fmaf(r3[1], r3[1], fmaf(r3[2], r3[2], lrr)));
        }
        if (blockIdx.x == 0) {   // the slot sets of the next iteration start from zero
            const int nx = (k + 1) % 3;
            double* a0 = pslots + (size_t)nx * NSLOT * SLOT_STRIDE;
            double* a1 = pslots + (size_t)(3 + nx) * NSLOT * SLOT_STRIDE;
            for (int i = tid; i < NSLOT * SLOT_STRIDE; i += TB) { a0[i] = 0.0; a1[i] = 0.0; }
        }
        {
            double brz, brr;
            block_sum2(lrz, lrr, red, brz, brr);
            if (tid == 0) {
                slot_add(up, 0, brz);
                slot_add(up, 1, brr);
            }
        }
        if (!grid_sync(st, gridDim.x)) { ok = false; break; }
        // ------------------------------------------------------------ phase C
        double rzn, rrn;
        slot_pair(up, sh2, rzn, rrn);
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

// ------------------------------------------------------------------ host ----------

int persistent_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

cudaError_t persistent_prepare(int smem_bytes, int* blocks_per_sm) {
    cudaError_t e = ensure_dynamic_smem((const void*)k_pcg_persistent<PCG_TB>, smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pcg_persistent<PCG_TB>, PCG_TB,
                                                         smem_bytes);
}

cudaError_t launch_pcg_persistent(const Views<float>& v, const uint32_t* blk_tile, const uint32_t* blk_cam_off,
                                  const uint32_t* blk_cams, double* pslots, int grid, int smem_bytes,
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
    return cudaLaunchKernelEx(&cfg, k_pcg_persistent<PCG_TB>, v, blk_tile, blk_cam_off, blk_cams, pslots);
}

}  // namespace gbba
