// Locality ordering built once per bound problem (our counterpart of the
// shared-index build of Sec. IV-A, "Shared Read/Add", of arXiv 2605.30583):
//
//  1. each point's key is the smallest camera index observing it; points are
//     sorted by (key, caller index), giving the internal point order;
//  2. tiles are TILE_PTS consecutive internal points;
//  3. observations are sorted by (tile, camera, tile slot, caller index), so a
//     tile's observations are contiguous and grouped into camera runs;
//  4. inside each tile the runs of at least LONG_RUN observations move to the front.
//
// Sorting is a bitonic network on (64-bit key, 32-bit value) pairs: shared-memory
// passes for distances below 2048 elements and global passes above.  Deterministic
// (ties broken by the value), so the same input always gives the same order.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "kernels.h"

namespace gbba {

namespace {

// Odd, so camera-dependent starting slots spread over all TILE_PTS (a power of two).
constexpr uint64_t SLOT_ROTATION = 89;

constexpr int LOCAL_ELEMS = 2048;
// Largest tile (observations) sorted in shared memory: 16,384 64-bit keys, 128 KB.
constexpr int TILE_SORT_MAX = 16384;
constexpr int LOCAL_THREADS = LOCAL_ELEMS / 2;

__device__ __forceinline__ bool pair_less(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

__global__ void k_fill_u32(uint32_t* a, size_t n, uint32_t v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_point_min_camera(const uint32_t* cam_idx, const uint32_t* pt_idx, int64_t n_obs,
                                   uint32_t* pt_key) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x)
        atomicMin(&pt_key[pt_idx[o]], cam_idx[o]);
}

__global__ void k_point_sort_keys(const uint32_t* pt_key, int n_pts, size_t sort_n, uint64_t* keys,
                                  uint32_t* vals) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sort_n; i += (size_t)gridDim.x * blockDim.x) {
        if (i < (size_t)n_pts) {
            keys[i] = ((uint64_t)pt_key[i] << 32) | (uint64_t)i;
            vals[i] = (uint32_t)i;
        } else {
            keys[i] = ~0ull;
            vals[i] = 0xffffffffu;
        }
    }
}

__global__ void k_point_perm(const uint32_t* vals, int n_pts, uint32_t* pt_user, uint32_t* pt_internal) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pts; j += gridDim.x * blockDim.x) {
        const uint32_t u = vals[j];
        pt_user[j] = u;
        pt_internal[u] = (uint32_t)j;
    }
}

__global__ void k_tile_count(const uint32_t* pt_idx, const uint32_t* pt_internal, int64_t n_obs,
                             uint32_t* tile_cnt) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&tile_cnt[pt_internal[pt_idx[o]] / TILE_PTS], 1u);
}

// Exclusive scan of cnt[0..n) into off[0..n] with one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_single(const uint32_t* cnt, int n, uint32_t* off) {
    __shared__ uint32_t part[1024];
    const int per = (n + 1023) / 1024;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < 1024; ++i) {
            const uint32_t t = part[i];
            part[i] = run;
            run += t;
        }
        off[n] = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int i = lo; i < hi; ++i) {
        off[i] = run;
        run += cnt[i];
    }
}

__global__ void k_obs_sort_keys(const uint32_t* cam_idx, const uint32_t* pt_idx, const uint32_t* pt_internal,
                                int64_t n_obs, size_t sort_n, uint64_t* keys, uint32_t* vals) {
    for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < sort_n; o += (size_t)gridDim.x * blockDim.x) {
        if (o < (size_t)n_obs) {
            const uint32_t ip = pt_internal[pt_idx[o]];
            const uint64_t tile = ip / TILE_PTS, slot = ip % TILE_PTS;
            // within a camera's run the points are ordered from a camera-dependent
            // starting slot: threads that walk different cameras' runs of one tile in
            // step then touch different points (no same-address shared atomics)
            const uint64_t rslot = (slot + SLOT_ROTATION * (uint64_t)cam_idx[o]) % TILE_PTS;
            keys[o] = (tile << 40) | ((uint64_t)cam_idx[o] << 16) | (rslot << 8);
            vals[o] = (uint32_t)o;
        } else {
            keys[o] = ~0ull;
            vals[o] = 0xffffffffu;
        }
    }
}

// Tile-bucketed observation sort: each observation goes to a free place in its tile's
// range (any order: the sort below orders it fully), keyed (camera, rotated slot, caller
// index); then one CTA per tile sorts the bucket in shared memory (bitonic network on the
// bucket padded to a power of two) and writes the keys and values k_obs_gather reads.
__global__ void k_obs_bucket(const uint32_t* cam_idx, const uint32_t* pt_idx, const uint32_t* pt_internal,
                             int64_t n_obs, const uint32_t* tile_off, uint32_t* cursor, uint64_t* keys) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ip = pt_internal[pt_idx[o]];
        const uint32_t tile = ip / TILE_PTS, slot = ip % TILE_PTS, cam = cam_idx[o];
        const uint64_t rslot = (slot + SLOT_ROTATION * (uint64_t)cam) % TILE_PTS;
        const uint32_t at = tile_off[tile] + atomicAdd(&cursor[tile], 1u);
        keys[at] = ((uint64_t)cam << 40) | (rslot << 32) | (uint64_t)o;
    }
}

__global__ void k_tile_sort(const uint32_t* tile_off, int n_tiles, uint64_t* keys, uint32_t* vals) {
    extern __shared__ uint64_t sk[];
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint32_t lo = tile_off[t], n = tile_off[t + 1] - lo;
        uint32_t pn = 2;
        while (pn < n) pn <<= 1;
        for (uint32_t i = threadIdx.x; i < pn; i += blockDim.x) sk[i] = i < n ? keys[lo + i] : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= pn; k <<= 1)
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t q = threadIdx.x; q < pn / 2; q += blockDim.x) {
                    const uint32_t i = 2 * j * (q / j) + (q % j), l = i + j;
                    const uint64_t a = sk[i], b = sk[l];
                    if ((b < a) == ((i & k) == 0)) {
                        sk[i] = b;
                        sk[l] = a;
                    }
                }
                __syncthreads();
            }
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t key = sk[i];
            const uint64_t cam = key >> 40, rslot = (key >> 32) & 0xffu;
            keys[lo + i] = ((uint64_t)t << 40) | (cam << 16) | (rslot << 8);
            vals[lo + i] = (uint32_t)(key & 0xffffffffu);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void k_obs_gather(const uint64_t* keys, const uint32_t* vals, const double* pixels, int64_t n_obs,
                             uint32_t* obs_key, T* obs_uv, uint32_t* obs_user) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_obs; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[j];
        const uint32_t o = vals[j];
        const uint32_t cam = (uint32_t)((k >> 16) & 0xffffffu);
        const uint32_t rslot = (uint32_t)((k >> 8) & 0xffu);
        const uint32_t slot = (uint32_t)((rslot + TILE_PTS - (SLOT_ROTATION * (uint64_t)cam) % TILE_PTS) % TILE_PTS);
        obs_key[j] = (cam << 8) | slot;
        obs_uv[2 * j] = (T)pixels[2 * (size_t)o];
        obs_uv[2 * j + 1] = (T)pixels[2 * (size_t)o + 1];
        obs_user[j] = o;
    }
}

// --- long runs first ------------------------------------------------------------------
// Inside each tile the camera runs of length >= LONG_RUN move to the front (camera order
// kept), the short runs follow.  The tile kernels walk the long runs in camera-uniform
// steps of 32 observations and the short tail thread by thread; every other kernel only
// needs each camera's observations of a tile to be contiguous, which stays true.  One
// warp per tile walks the runs, 32 observations at a time (ballot of run heads).

// Calls visit(start, len) for every run of tile [lo, hi) in order (uniform in the warp).
template <typename F>
__device__ __forceinline__ void for_each_run(const uint32_t* __restrict__ obs_key, uint32_t lo, uint32_t hi, F&& visit) {
    const int lane = threadIdx.x & 31;
    uint32_t cur = lo;
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t j = base + lane;
        const bool head = j < hi && j > lo && (obs_key[j - 1] >> 8) != (obs_key[j] >> 8);
        uint32_t hm = __ballot_sync(0xffffffffu, head);
        while (hm) {
            const uint32_t h = base + (uint32_t)(__ffs(hm) - 1);
            visit(cur, h - cur);
            cur = h;
            hm &= hm - 1u;
        }
    }
    if (hi > lo) visit(cur, hi - cur);
}

__global__ void k_long_count(const uint32_t* __restrict__ obs_key, const uint32_t* __restrict__ tile_off, int n_tiles,
                             uint32_t* n_long, uint32_t* long_obs) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tiles; t += warps) {
        uint32_t nl = 0, no = 0;
        for_each_run(obs_key, tile_off[t], tile_off[t + 1], [&](uint32_t, uint32_t len) {
            if (len >= (uint32_t)LONG_RUN) { ++nl; no += len; }
        });
        if ((threadIdx.x & 31) == 0) {
            n_long[t] = nl;
            long_obs[t] = no;
        }
    }
}

// Copies each run to its place (long runs from the tile's start, short runs after them)
// and writes the long-run table {start, length, camera} and the short tail's start.
template <typename T>
__global__ void k_long_place(const uint32_t* __restrict__ obs_key, const T* __restrict__ obs_uv,
                             const uint32_t* __restrict__ obs_user, const uint32_t* __restrict__ tile_off,
                             const uint32_t* __restrict__ long_off, const uint32_t* __restrict__ long_obs, int n_tiles,
                             uint32_t* tmp_key, T* tmp_uv, uint32_t* tmp_user, uint32_t* long_run,
                             uint32_t* short_start) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_tiles; t += warps) {
        const uint32_t lo = tile_off[t], hi = tile_off[t + 1];
        uint32_t next_long = lo, next_short = lo + long_obs[t], e = long_off[t];
        for_each_run(obs_key, lo, hi, [&](uint32_t start, uint32_t len) {
            uint32_t dest;
            if (len >= (uint32_t)LONG_RUN) {
                dest = next_long;
                next_long += len;
                if (lane == 0) {
                    long_run[3 * (size_t)e] = dest;
                    long_run[3 * (size_t)e + 1] = len;
                    long_run[3 * (size_t)e + 2] = obs_key[start] >> 8;
                }
                ++e;
            } else {
                dest = next_short;
                next_short += len;
            }
            for (uint32_t i = lane; i < len; i += 32) {
                tmp_key[dest + i] = obs_key[start + i];
                tmp_user[dest + i] = obs_user[start + i];
                tmp_uv[2 * (size_t)(dest + i)] = obs_uv[2 * (size_t)(start + i)];
                tmp_uv[2 * (size_t)(dest + i) + 1] = obs_uv[2 * (size_t)(start + i) + 1];
            }
        });
        if (lane == 0) short_start[t] = lo + long_obs[t];
    }
}

template <typename T>
__global__ void k_copy_back(const uint32_t* tmp_key, const T* tmp_uv, const uint32_t* tmp_user, int64_t n_obs,
                            uint32_t* obs_key, T* obs_uv, uint32_t* obs_user) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_obs; j += (int64_t)gridDim.x * blockDim.x) {
        obs_key[j] = tmp_key[j];
        obs_user[j] = tmp_user[j];
        obs_uv[2 * j] = tmp_uv[2 * j];
        obs_uv[2 * j + 1] = tmp_uv[2 * j + 1];
    }
}

// Point-major index by a counting sort inside each tile: a tile's observation range
// holds exactly the observations of its TILE_PTS points, so the point offsets are the
// tile's first observation plus an exclusive scan of per-slot counts, and each point's
// observations are placed in increasing position j (lanes of a 32-observation step
// ranked among equal slots, steps in order): the same index as sorting (point, j).
// One warp per tile; `cnt` holds the warp's 256 slot counters in shared memory.
constexpr int PM_WARPS = 4;

__global__ void __launch_bounds__(32 * PM_WARPS) k_pm_tiles(const uint32_t* __restrict__ obs_key,
                                                            const uint32_t* __restrict__ tile_off, int n_tiles,
                                                            int n_pts, int64_t n_obs, uint32_t* obs_pm,
                                                            uint32_t* pt_obs_off) {
    static_assert(TILE_PTS == 256, "one-byte point slots");
    __shared__ uint32_t cnt_all[PM_WARPS][TILE_PTS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* cnt = cnt_all[wid];
    const uint32_t lower = (1u << lane) - 1u;
    for (int t = blockIdx.x * PM_WARPS + wid; t < n_tiles; t += gridDim.x * PM_WARPS) {
        const uint32_t lo = tile_off[t], hi = tile_off[t + 1];
        for (int s = lane; s < TILE_PTS; s += 32) cnt[s] = 0u;
        __syncwarp();
        for (uint32_t j = lo + lane; j < hi; j += 32) atomicAdd(&cnt[obs_key[j] & 0xffu], 1u);
        __syncwarp();
        // exclusive scan of the 256 counters: 8 per lane, then across lanes
        uint32_t c[TILE_PTS / 32], run = 0u;
#pragma unroll
        for (int k = 0; k < TILE_PTS / 32; ++k) {
            c[k] = cnt[lane * (TILE_PTS / 32) + k];
            run += c[k];
        }
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        uint32_t base = incl - run;
        const int pt0 = t * TILE_PTS;
#pragma unroll
        for (int k = 0; k < TILE_PTS / 32; ++k) {
            const int s2 = lane * (TILE_PTS / 32) + k;
            cnt[s2] = base;
            if (pt0 + s2 < n_pts) pt_obs_off[pt0 + s2] = lo + base;
            base += c[k];
        }
        __syncwarp();
        // stable placement, 32 observations a step
        for (uint32_t j0 = lo; j0 < hi; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool ok = j < hi;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const uint32_t slot = obs_key[j] & 0xffu;
                const unsigned same = __match_any_sync(act, slot);
                const uint32_t at = cnt[slot] + (uint32_t)__popc(same & lower);
                obs_pm[lo + at] = j;
                __syncwarp(act);
                if ((same >> lane) >> 1 == 0u) cnt[slot] += (uint32_t)__popc(same);   // highest lane of the group
            }
            __syncwarp();
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) pt_obs_off[n_pts] = (uint32_t)n_obs;
}

// --- bitonic network --------------------------------------------------------------

// Compare-exchange of positions i < l = i + j; ascending iff (i & k) == 0.
__device__ __forceinline__ void cx_global(uint64_t* keys, uint32_t* vals, size_t i, size_t l, size_t k) {
    const uint64_t ka = keys[i], kb = keys[l];
    const uint32_t va = vals[i], vb = vals[l];
    const bool asc = (i & k) == 0;
    if (pair_less(kb, vb, ka, va) == asc) {
        keys[i] = kb; keys[l] = ka;
        vals[i] = vb; vals[l] = va;
    }
}

__global__ void k_bitonic_global(uint64_t* keys, uint32_t* vals, size_t n, size_t k, size_t j) {
    const size_t pairs = n / 2;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < pairs; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = 2 * j * (t / j) + (t % j);
        cx_global(keys, vals, i, i + j, k);
    }
}

// Runs stages (k, j) for j = j0, j0/2, ..., 1 inside blocks of `elems` elements;
// if full_sort, first runs every k = 2 .. elems (sorting each block bitonically).
__global__ void __launch_bounds__(LOCAL_THREADS) k_bitonic_local(uint64_t* keys, uint32_t* vals, size_t elems,
                                                                 size_t k_outer, int full_sort) {
    __shared__ uint64_t sk[LOCAL_ELEMS];
    __shared__ uint32_t sv[LOCAL_ELEMS];
    const size_t base = (size_t)blockIdx.x * elems;
    for (size_t i = threadIdx.x; i < elems; i += blockDim.x) {
        sk[i] = keys[base + i];
        sv[i] = vals[base + i];
    }
    __syncthreads();
    const size_t pairs = elems / 2;
    auto stage = [&](size_t k, size_t j) {
        for (size_t t = threadIdx.x; t < pairs; t += blockDim.x) {
            const size_t i = 2 * j * (t / j) + (t % j), l = i + j;
            const bool asc = ((base + i) & k) == 0;
            const uint64_t ka = sk[i], kb = sk[l];
            const uint32_t va = sv[i], vb = sv[l];
            if (pair_less(kb, vb, ka, va) == asc) {
                sk[i] = kb; sk[l] = ka;
                sv[i] = vb; sv[l] = va;
            }
        }
        __syncthreads();
    };
    if (full_sort) {
        for (size_t k = 2; k <= elems; k <<= 1)
            for (size_t j = k >> 1; j > 0; j >>= 1) stage(k, j);
    } else {
        for (size_t j = elems >> 1; j > 0; j >>= 1) stage(k_outer, j);
    }
    for (size_t i = threadIdx.x; i < elems; i += blockDim.x) {
        keys[base + i] = sk[i];
        vals[base + i] = sv[i];
    }
}

void bitonic_sort(uint64_t* keys, uint32_t* vals, size_t n, cudaStream_t s) {
    // n is a power of two >= 2
    const size_t elems = n < (size_t)LOCAL_ELEMS ? n : (size_t)LOCAL_ELEMS;
    const int lblocks = (int)(n / elems);
    const int lthreads = (int)(elems / 2 < (size_t)LOCAL_THREADS ? elems / 2 : (size_t)LOCAL_THREADS);
    k_bitonic_local<<<lblocks, lthreads, 0, s>>>(keys, vals, elems, 0, 1);
    const int gthreads = 256;
    const size_t gblocks_need = (n / 2 + gthreads - 1) / gthreads;
    const int gblocks = (int)(gblocks_need > 65535 ? 65535 : gblocks_need);
    for (size_t k = 2 * elems; k <= n; k <<= 1) {
        for (size_t j = k >> 1; j >= elems; j >>= 1) k_bitonic_global<<<gblocks, gthreads, 0, s>>>(keys, vals, n, k, j);
        k_bitonic_local<<<lblocks, lthreads, 0, s>>>(keys, vals, elems, k, 0);
    }
}

inline size_t pow2_at_least(size_t n) {
    size_t p = 2;
    while (p < n) p <<= 1;
    return p;
}

inline int blocks_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b > 8192 ? 8192 : b);
}

}  // namespace

template <typename T>
void build_order(const Views<T>& v, const OrderBuffers& b, cudaStream_t s) {
    const int TB = 256;
    uint32_t* pt_user = const_cast<uint32_t*>(v.pt_user);
    uint32_t* pt_internal = const_cast<uint32_t*>(v.pt_internal);
    uint32_t* tile_off = const_cast<uint32_t*>(v.tile_off);
    // 1. point keys and point order
    k_fill_u32<<<blocks_for(v.n_pts, TB), TB, 0, s>>>(b.pt_key, (size_t)v.n_pts, 0xffffffffu);
    k_point_min_camera<<<blocks_for(v.n_obs, TB), TB, 0, s>>>(b.cam_idx, b.pt_idx, v.n_obs, b.pt_key);
    const size_t np2 = pow2_at_least((size_t)v.n_pts);
    k_point_sort_keys<<<blocks_for(np2, TB), TB, 0, s>>>(b.pt_key, v.n_pts, np2, b.keys, b.vals);
    bitonic_sort(b.keys, b.vals, np2, s);
    k_point_perm<<<blocks_for(v.n_pts, TB), TB, 0, s>>>(b.vals, v.n_pts, pt_user, pt_internal);
    // 2. tiles
    k_fill_u32<<<blocks_for(v.n_tiles, TB), TB, 0, s>>>(b.tile_cnt, (size_t)v.n_tiles, 0u);
    k_tile_count<<<blocks_for(v.n_obs, TB), TB, 0, s>>>(b.pt_idx, pt_internal, v.n_obs, b.tile_cnt);
    k_scan_single<<<1, 1024, 0, s>>>(b.tile_cnt, v.n_tiles, tile_off);
    // 3. observation order: sorted inside each tile's bucket in shared memory when the
    //    largest tile fits TILE_SORT_MAX observations, else one global sort
    uint32_t most = 0;
    {
        std::vector<uint32_t> toff((size_t)v.n_tiles + 1);
        if (cudaMemcpyAsync(toff.data(), tile_off, 4 * toff.size(), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess) {
            for (int t = 0; t < v.n_tiles; ++t) most = std::max(most, toff[t + 1] - toff[t]);
        } else {
            most = ~0u;   // the error surfaces at the caller's next check; take the general path
        }
    }
    if (most <= (uint32_t)TILE_SORT_MAX) {
        uint32_t pn = 2;
        while (pn < most) pn <<= 1;
        k_fill_u32<<<blocks_for(v.n_tiles, TB), TB, 0, s>>>(b.tile_cnt, (size_t)v.n_tiles, 0u);
        k_obs_bucket<<<blocks_for(v.n_obs, TB), TB, 0, s>>>(b.cam_idx, b.pt_idx, pt_internal, v.n_obs, tile_off,
                                                             b.tile_cnt, b.keys);
        const size_t smem = 8 * (size_t)pn;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tile_sort<<<std::max(1, std::min(v.n_tiles, 65535)), 512, smem, s>>>(tile_off, v.n_tiles, b.keys, b.vals);
    } else {
        const size_t no2 = pow2_at_least((size_t)v.n_obs);
        k_obs_sort_keys<<<blocks_for(no2, TB), TB, 0, s>>>(b.cam_idx, b.pt_idx, pt_internal, v.n_obs, no2, b.keys,
                                                           b.vals);
        bitonic_sort(b.keys, b.vals, no2, s);
    }
    k_obs_gather<T><<<blocks_for(v.n_obs, TB), TB, 0, s>>>(b.keys, b.vals, b.pixels, v.n_obs,
                                                           const_cast<uint32_t*>(v.obs_key),
                                                           const_cast<T*>(v.obs_uv),
                                                           const_cast<uint32_t*>(v.obs_user));
    // 4. long runs first inside every tile, and the long-run table
    {
        uint32_t* n_long = b.tile_cnt;            // [n_tiles + 1] scratch (the tile counts are done)
        uint32_t* long_obs = b.vals;               // [n_tiles] scratch (the sort values are consumed)
        uint32_t* tmp_key = reinterpret_cast<uint32_t*>(b.keys);     // the sort scratch is free here
        uint32_t* tmp_user = tmp_key + v.n_obs;
        T* tmp_uv = reinterpret_cast<T*>(const_cast<double*>(b.pixels));   // the uploaded pixels are consumed
        k_long_count<<<blocks_for(32 * (size_t)v.n_tiles, TB), TB, 0, s>>>(v.obs_key, tile_off, v.n_tiles, n_long,
                                                                            long_obs);
        k_scan_single<<<1, 1024, 0, s>>>(n_long, v.n_tiles, const_cast<uint32_t*>(v.long_off));
        k_long_place<T><<<blocks_for(32 * (size_t)v.n_tiles, TB), TB, 0, s>>>(
            v.obs_key, v.obs_uv, v.obs_user, tile_off, v.long_off, long_obs, v.n_tiles, tmp_key, tmp_uv, tmp_user,
            const_cast<uint32_t*>(v.long_run), const_cast<uint32_t*>(v.short_start));
        k_copy_back<T><<<blocks_for(v.n_obs, TB), TB, 0, s>>>(tmp_key, tmp_uv, tmp_user, v.n_obs,
                                                              const_cast<uint32_t*>(v.obs_key), const_cast<T*>(v.obs_uv),
                                                              const_cast<uint32_t*>(v.obs_user));
    }
    // 5. point-major index over the tile-major order (every point has >= 2 observations,
    //    so every internal point owns a non-empty run), one counting sort per tile
    {
        const int grid = (int)std::min<int64_t>(8192, ((int64_t)v.n_tiles + PM_WARPS - 1) / PM_WARPS);
        k_pm_tiles<<<std::max(1, grid), 32 * PM_WARPS, 0, s>>>(v.obs_key, tile_off, v.n_tiles, v.n_pts, v.n_obs,
                                                               const_cast<uint32_t*>(v.obs_pm),
                                                               const_cast<uint32_t*>(v.pt_obs_off));
    }
}

void sort_pairs(uint64_t* keys, uint32_t* vals, size_t n, cudaStream_t s) { bitonic_sort(keys, vals, n, s); }

namespace {
// Within a tile the observations are ordered by (camera, point slot), and moving the
// long runs to the front keeps each run's order, so two observations of one point by
// one camera end up next to each other.
__global__ void k_repeated_keys(const uint32_t* __restrict__ obs_key, int64_t n_obs, uint32_t* flag) {
    for (int64_t j = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_obs; j += (int64_t)gridDim.x * blockDim.x)
        if (obs_key[j] == obs_key[j - 1]) atomicOr(flag, 1u);
}
}  // namespace

void flag_repeated_keys(const uint32_t* obs_key, int64_t n_obs, uint32_t* flag, cudaStream_t s) {
    if (n_obs < 2) return;
    k_repeated_keys<<<blocks_for((size_t)n_obs, 256), 256, 0, s>>>(obs_key, n_obs, flag);
}

template void build_order<float>(const Views<float>&, const OrderBuffers&, cudaStream_t);
template void build_order<double>(const Views<double>&, const OrderBuffers&, cudaStream_t);

}  // namespace gbba
