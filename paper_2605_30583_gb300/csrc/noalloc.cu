// Allocation-free reprojection cost: F = 1/2 sum |r|^2 over caller-provided device
// arrays, for callers that cannot allocate device memory at all.
//
// Some callers may not call cudaMalloc, or may not hand this library a workspace:
// code running while a stream is being captured into a graph, hosts whose device
// memory is entirely owned by another allocator, or real-time loops where any
// allocation is forbidden.  This entry point computes the same cost as ba_evaluate
// (mixed precision: FP32 residuals, FP64 sum) but keeps its scratch -- camera records
// and per-block partial sums -- in one statically sized array that lives in the
// library's module for as long as the library is loaded (on every device that loads
// it, until process exit).  It never allocates.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "device_common.cuh"
#include "gbba.h"
#include "problem.h"

namespace gbba {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_OBS_PER_BLOCK = 4 * NA_THREADS;   // observations per block, 4 per thread

// Scratch layout (bytes): [camera records: NOALLOC_MAX_CAMS x 16 floats]
//                         [block partial sums: NOALLOC_MAX_BLOCKS doubles]
//                         [ticket: one unsigned int, 256 bytes reserved]
constexpr size_t NA_CAM_BYTES = (size_t)BA_NOALLOC_MAX_CAMS * 16 * sizeof(float);
constexpr size_t NA_PART_BYTES = (size_t)BA_NOALLOC_MAX_BLOCKS * sizeof(double);
constexpr size_t NA_SCRATCH_BYTES = NA_CAM_BYTES + NA_PART_BYTES + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

struct NaScratch {
    float* cams;
    double* partials;
    unsigned int* ticket;
};

__global__ void k_na_cameras(const float* __restrict__ cams, int n_cams, NaScratch sc) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cams; c += gridDim.x * blockDim.x) {
        double p[9];
        for (int k = 0; k < 9; ++k) p[k] = (double)cams[9 * (size_t)c + k];
        float rec[CP_STRIDE];
        camera_record(p, rec);
        for (int k = 0; k < 16; ++k) sc.cams[16 * (size_t)c + k] = rec[k];
    }
}

// One block per NA_OBS_PER_BLOCK observations; the last block to finish sums the
// block partials in block order.  An index out of range is never followed: that
// observation contributes NaN, so the returned cost is NaN.
__global__ void __launch_bounds__(NA_THREADS) k_na_cost(const float* __restrict__ pts, const uint32_t* __restrict__ cam_idx,
                                                        const uint32_t* __restrict__ pt_idx,
                                                        const float* __restrict__ pixels, int64_t n_obs, int n_cams,
                                                        int n_pts, float eps, NaScratch sc,
                                                        double* __restrict__ cost_out) {
    __shared__ double sh[32];
    __shared__ bool is_last;
    double acc = 0.0;
    const int64_t base = (int64_t)blockIdx.x * NA_OBS_PER_BLOCK;
    for (int k = 0; k < NA_OBS_PER_BLOCK / NA_THREADS; ++k) {
        const int64_t o = base + (int64_t)k * NA_THREADS + threadIdx.x;
        if (o < n_obs) {
            const uint32_t c = cam_idx[o], i = pt_idx[o];
            if (c >= (uint32_t)n_cams || i >= (uint32_t)n_pts) {
                acc = __longlong_as_double(0x7ff8000000000000LL);   // quiet NaN
                continue;
            }
            const Cam cam = load_cam(sc.cams + 16 * (size_t)c);
            const float* X = pts + 3 * (size_t)i;
            float r0, r1;
            project_residual(cam, X[0], X[1], X[2], eps, pixels[2 * o], pixels[2 * o + 1], r0, r1);
            acc += (double)r0 * r0 + (double)r1 * r1;
        }
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        sc.partials[blockIdx.x] = s;
        __threadfence();
        is_last = atomicAdd(sc.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(&sc.partials[b]);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        *cost_out = 0.5 * t;
        *sc.ticket = 0u;
    }
}

// Device address of the scratch array per device, looked up with that device current
// (the host-side symbol is only a stand-in, never a device address).  It is looked up
// again on every call made outside stream capture, so a device reset (which may load
// the module at another address) is followed; under capture the address cached by the
// last uncaptured call on that device is used.
std::mutex g_na_mutex;
void* g_na_addr[64] = {nullptr};

}  // namespace

}  // namespace gbba

using namespace gbba;

extern "C" ba_status ba_cost_noalloc(int32_t n_cams, int32_t n_pts, int64_t n_obs, const float* cams,
                                     const float* pts, const uint32_t* cam_idx, const uint32_t* pt_idx,
                                     const float* pixels, double eps_depth, double* cost_dev, void* stream) {
    if (n_cams < 1 || n_pts < 1 || n_obs < 1) {
        set_error("ba_cost_noalloc: sizes must be positive (n_cams=%d n_pts=%d n_obs=%lld)", n_cams, n_pts,
                  (long long)n_obs);
        return BA_ERR_INVALID_ARG;
    }
    if (n_cams > BA_NOALLOC_MAX_CAMS) {
        set_error("ba_cost_noalloc: %d cameras exceed the fixed scratch capacity of %d cameras", n_cams,
                  BA_NOALLOC_MAX_CAMS);
        return BA_ERR_INVALID_ARG;
    }
    const int64_t blocks = (n_obs + NA_OBS_PER_BLOCK - 1) / NA_OBS_PER_BLOCK;
    if (blocks > BA_NOALLOC_MAX_BLOCKS) {
        set_error("ba_cost_noalloc: %lld observations exceed the fixed scratch capacity of %lld observations",
                  (long long)n_obs, (long long)BA_NOALLOC_MAX_BLOCKS * NA_OBS_PER_BLOCK);
        return BA_ERR_INVALID_ARG;
    }
    if (!cams || !pts || !cam_idx || !pt_idx || !pixels || !cost_dev || !(eps_depth >= 0)) {
        set_error("ba_cost_noalloc: null pointer or negative eps_depth");
        return BA_ERR_INVALID_ARG;
    }
    int dev = 0;
    GBBA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("ba_cost_noalloc: device ordinal %d out of the supported range", dev);
        return BA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GBBA_CUDA(cudaStreamIsCapturing(s, &cap));
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* a = nullptr;
            GBBA_CUDA(cudaGetSymbolAddress(&a, g_noalloc_scratch));
            g_na_addr[dev] = a;
        } else if (!g_na_addr[dev]) {
            set_error("ba_cost_noalloc: the first call on device %d must come before any stream capture", dev);
            return BA_ERR_STATE;
        }
        base = g_na_addr[dev];
    }
    NaScratch sc;
    sc.cams = reinterpret_cast<float*>(base);
    sc.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + NA_CAM_BYTES);
    sc.ticket = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(base) + NA_CAM_BYTES + NA_PART_BYTES);
    // the ticket must start at zero on every call (an earlier failed call may have left it set)
    GBBA_CUDA(cudaMemsetAsync(sc.ticket, 0, sizeof(unsigned int), s));
    const int cgrid = (n_cams + 255) / 256;
    k_na_cameras<<<cgrid, 256, 0, s>>>(cams, n_cams, sc);
    k_na_cost<<<(unsigned int)blocks, NA_THREADS, 0, s>>>(pts, cam_idx, pt_idx, pixels, n_obs, n_cams, n_pts,
                                                          (float)eps_depth, sc, cost_dev);
    GBBA_CUDA(cudaGetLastError());
    return BA_OK;
}
