// C ABI of libgbba (include/gbba.h): validation, the single workspace, the
// locality ordering, parameter transfer, evaluation and the LM + PCGNR solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "gbba.h"
#include "kernels.h"
#include "problem.h"

namespace gbba {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

ba_status cuda_status(cudaError_t e, const char* what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    cudaGetLastError();   // clear a non-sticky error so later calls do not report it again
    return BA_ERR_CUDA;
}

namespace {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Bump {
    size_t off = 0;
    size_t take(size_t bytes) {
        off = align_up(off, 256);
        size_t o = off;
        off += bytes;
        return o;
    }
};

inline size_t pow2_at_least(size_t n) {
    size_t p = 2;
    while (p < n) p <<= 1;
    return p;
}

}  // namespace

Layout compute_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, int32_t precision, int32_t n_fac) {
    Layout l{};
    const size_t T = precision == BA_PREC_FP64 ? 8 : 4;
    const size_t nc = (size_t)n_cams, np = (size_t)n_pts, no = (size_t)n_obs;
    const size_t n_tiles = (np + TILE_PTS - 1) / TILE_PTS;
    const size_t n_quads = (np + 3) / 4;
    const size_t pt_off = align_up(9 * nc, 4);
    const size_t n_vec = pt_off + 12 * n_quads;
    const size_t pc_stride = align_up(9 * nc, 64);
    Bump b;
    l.state = b.take(sizeof(DevState));
    l.partials = b.take(sizeof(double) * MAX_GRID * NPART);
    l.obs_key = b.take(4 * no);
    l.obs_uv = b.take(T * 2 * no);
    l.obs_user = b.take(4 * no);
    l.tile_off = b.take(4 * (n_tiles + 1));
    l.pt_user = b.take(4 * np);
    l.pt_internal = b.take(4 * np);
    l.obs_pm = b.take(4 * no);
    l.pt_obs_off = b.take(4 * (np + 1));
    l.staging = b.take(8 * (9 * nc + 3 * np));
    l.blk_tile = b.take(4 * (MAX_PBLOCKS + 1));
    l.blk_cam_off = b.take(4 * (MAX_PBLOCKS + 1));
    // per-CTA camera lists of the persistent PCG kernel: each CTA lists the cameras of
    // its observations and pose factors, and every other camera is listed once, so
    // n_obs + 2 n_fac + n_cams + MAX_PBLOCKS entries always suffice; the plan is only
    // used when they fit in shared memory, so cap the region
    const size_t nfc = 2 * (size_t)std::max(0, n_fac);
    l.blk_cams = b.take(4 * std::min(no + nfc + nc + MAX_PBLOCKS, (size_t)(MAX_PBLOCKS * 4096)));
    l.pslots = b.take(8 * PSLOT_TOTAL);
    // long-run tables: a tile holds at most (its observations / LONG_RUN) long runs
    l.long_off = b.take(4 * (n_tiles + 1));
    l.long_run = b.take(12 * (no / LONG_RUN + n_tiles));
    l.short_start = b.take(4 * n_tiles);
    const size_t union_base = align_up(b.off, 256);
    // solver arrays
    Bump s;
    s.off = union_base;
    for (int i = 0; i < 10; ++i) l.vec[i] = s.take(T * n_vec);
    l.cam_pre = s.take(4 * CP_STRIDE * nc);
    l.cam_pre_new = s.take(4 * CP_STRIDE * nc);
    l.cam_dir = s.take(4 * CD_STRIDE * nc);
    l.cam_acc = s.take(4 * CA_STRIDE * nc * CA_SETS);
    l.pc = s.take(4 * 2 * pc_stride);
    l.cam_lin = s.take(8 * CL_STRIDE * nc);
    l.cam_H = s.take(4 * CH_STRIDE * nc);
    l.pt_H = s.take(T * PH_STRIDE * 4 * n_quads);
    l.Minv_c = s.take(T * MC_STRIDE * nc);
    l.Minv_p = s.take(T * MP_STRIDE * 4 * n_quads);
    l.obs_w = s.take(4 * no);
    const size_t nf = (size_t)std::max(0, n_fac);
    l.fac_cam = s.take(4 * 2 * nf);
    l.fac_meas = s.take(8 * 6 * nf);
    l.fac_sqrt = s.take(8 * 6 * nf);
    l.fac_J = s.take(4 * 72 * nf);
    if (precision == BA_PREC_FP64) {
        l.jac = s.take(T * 24 * no);
        l.res = s.take(T * 2 * no);
        l.cam64 = s.take(8 * CP_STRIDE * nc);
        l.cam64_new = s.take(8 * CP_STRIDE * nc);
        l.cam_H64 = s.take(8 * CH_STRIDE * nc);
        l.xm = l.xm_new = l.cam_lo = l.cam_lo_new = l.rbuf = 0;
    } else {
        l.jac = l.res = l.cam64 = l.cam64_new = l.cam_H64 = 0;
        l.xm = s.take(8 * n_vec);
        l.xm_new = s.take(8 * n_vec);
        l.cam_lo = s.take(4 * CLO_STRIDE * nc);
        l.cam_lo_new = s.take(4 * CLO_STRIDE * nc);
        l.rbuf = s.take(4 * 2 * no);
    }
    // ordering scratch (only live during ba_bind_workspace), overlaps the solver arrays
    Bump o;
    o.off = union_base;
    l.sort_cap = pow2_at_least(std::max(no, np));
    l.s_cam_idx = o.take(4 * no);
    l.s_pt_idx = o.take(4 * no);
    l.s_pixels = o.take(8 * 2 * no);
    l.s_pt_key = o.take(4 * np);
    l.s_tile_cnt = o.take(4 * (n_tiles + 1));
    l.s_keys = o.take(8 * l.sort_cap);
    l.s_vals = o.take(4 * l.sort_cap);
    l.total = align_up(std::max(s.off, o.off), 256);
    return l;
}

template <typename T>
Views<T> make_views(ba_problem* p) {
    Views<T> v{};
    const Layout& l = p->lay;
    char* w = p->ws;
    v.n_cams = p->n_cams;
    v.n_pts = p->n_pts;
    v.n_tiles = p->n_tiles;
    v.n_quads = (p->n_pts + 3) / 4;
    v.n_obs = p->n_obs;
    v.pc_stride = (int64_t)((9 * (size_t)p->n_cams + 63) / 64 * 64);
    v.pt_off = p->pt_off;
    v.n_vec = p->n_vec;
    v.obs_key = (const uint32_t*)(w + l.obs_key);
    v.obs_uv = (const T*)(w + l.obs_uv);
    v.obs_user = (const uint32_t*)(w + l.obs_user);
    v.tile_off = (const uint32_t*)(w + l.tile_off);
    v.pt_user = (const uint32_t*)(w + l.pt_user);
    v.pt_internal = (const uint32_t*)(w + l.pt_internal);
    v.obs_pm = (const uint32_t*)(w + l.obs_pm);
    v.pt_obs_off = (const uint32_t*)(w + l.pt_obs_off);
    v.long_off = (const uint32_t*)(w + l.long_off);
    v.long_run = (const uint32_t*)(w + l.long_run);
    v.short_start = (const uint32_t*)(w + l.short_start);
    T** vecs[10] = {&v.x, &v.x_new, &v.h, &v.r, &v.z, &v.p, &v.q, &v.g, &v.D, &v.s};
    for (int i = 0; i < 10; ++i) *vecs[i] = (T*)(w + l.vec[i]);
    v.cam_pre = (float*)(w + l.cam_pre);
    v.cam_pre_new = (float*)(w + l.cam_pre_new);
    v.cam_dir = (float*)(w + l.cam_dir);
    v.cam_acc = (float*)(w + l.cam_acc);
    v.pc = (float*)(w + l.pc);
    v.cam_lin = (double*)(w + l.cam_lin);
    v.cam_H = (float*)(w + l.cam_H);
    v.pt_H = (T*)(w + l.pt_H);
    v.Minv_c = (T*)(w + l.Minv_c);
    v.Minv_p = (T*)(w + l.Minv_p);
    v.cam64 = l.cam64 ? (double*)(w + l.cam64) : nullptr;
    v.cam64_new = l.cam64_new ? (double*)(w + l.cam64_new) : nullptr;
    v.cam_H64 = l.cam_H64 ? (double*)(w + l.cam_H64) : nullptr;
    v.xm = l.xm ? (double*)(w + l.xm) : nullptr;
    v.xm_new = l.xm_new ? (double*)(w + l.xm_new) : nullptr;
    v.cam_lo = l.cam_lo ? (float*)(w + l.cam_lo) : nullptr;
    v.cam_lo_new = l.cam_lo_new ? (float*)(w + l.cam_lo_new) : nullptr;
    v.rbuf = l.rbuf ? (float*)(w + l.rbuf) : nullptr;
    v.jac = l.jac ? (T*)(w + l.jac) : nullptr;
    v.res = l.res ? (T*)(w + l.res) : nullptr;
    v.obs_w = (float*)(w + l.obs_w);
    v.n_fac = p->n_fac;
    v.fac_cam = (const uint32_t*)(w + l.fac_cam);
    v.fac_meas = (const double*)(w + l.fac_meas);
    v.fac_sqrt = (const double*)(w + l.fac_sqrt);
    v.fac_J = (float*)(w + l.fac_J);
    v.st = (DevState*)(w + l.state);
    v.partials = (double*)(w + l.partials);
    v.staging = w + l.staging;
    return v;
}

template Views<float> make_views<float>(ba_problem*);
template Views<double> make_views<double>(ba_problem*);

// ------------------------------------------------------------------ solve ------
// The solve is four kinds of steps, for either precision:
//   init      first linearisation of the solve;
//   lm_head   block-Jacobi preconditioner (and, with the persistent plan, the whole PCG);
//   pcg_iter  one PCG iteration (multi-kernel PCG only);
//   lm_tail   candidate step, its evaluation and the LM decision, commit, relinearise.

static bool inner_pcg(const ba_problem* p) {
    return !(p->precision == BA_PREC_MIXED && p->use_persistent) || p->use_schur;
}

static void step_init(ba_problem* p, cudaStream_t s, CondHandle lm_c, int use) {
    if (p->precision == BA_PREC_MIXED) {
        launch_init_state(p->vf.st, s);
        launch_camera_precompute(p->vf, p->L, s);
        launch_residual(p->vf, p->L, s, 0);
        launch_linearize(p->vf, p->L, s, 0, nullptr, nullptr, lm_c, use);
    } else {
        launch_init_state(p->vd.st, s);
        launch64_camera_precompute(p->vd, p->L, s);
        launch64_linearize(p->vd, p->L, s, 0, nullptr, nullptr, lm_c, use);
    }
}

static void step_pcg_iter(ba_problem* p, cudaStream_t s, CondHandle pcg_c, int use) {
    if (p->precision == BA_PREC_MIXED && p->use_schur) {   // reduced camera system
        const Views<float>& v = p->vf;
        launch_schur(v, s, 1, &v.st->pcg_active);
        launch_update(v, p->L, s, pcg_c, use, 1);
    } else if (p->precision == BA_PREC_MIXED && p->use_cg) {
        const Views<float>& v = p->vf;
        launch_cg_round(v, p->L, s, &v.st->pcg_active, pcg_c, use);
    } else if (p->precision == BA_PREC_MIXED) {
        const Views<float>& v = p->vf;
        launch_matvec(v, p->L, s, &v.st->pcg_active, v.z, 1);
        launch_update(v, p->L, s, pcg_c, use);
    } else {
        const Views<double>& v = p->vd;
        launch64_direction(v, p->L, s, v.z, 1, &v.st->pcg_active);
        launch64_matvec(v, p->L, s, &v.st->pcg_active);
        launch64_update(v, p->L, s, pcg_c, use);
    }
}

static void step_lm_head(ba_problem* p, cudaStream_t s, CondHandle pcg_c, int use, bool inline_pcg, int max_pcg) {
    if (p->precision == BA_PREC_MIXED && p->use_schur) {
        // blocks of H' (camera and point inverses, D), then the reduced right-hand side
        const Views<float>& v = p->vf;
        launch_precond(v, p->L, s, pcg_c, 0, nullptr);
        launch_schur(v, s, 0, &v.st->lm_active);
        launch_schur_start(v, p->L, s, pcg_c, use);
    } else if (p->precision == BA_PREC_MIXED) {
        const Views<float>& v = p->vf;
        launch_precond(v, p->L, s, pcg_c, use, p->use_persistent ? p->pslots : nullptr);
        if (p->use_persistent)
            launch_pcg_persistent(v, p->blk_tile, p->blk_cam_off, p->blk_cams, p->pslots, p->p_grid,
                                  p->p_form == PCG_TWO_EXCHANGE ? p->p_smem_two : p->p_smem_one, p->p_form, s);
    } else {
        launch64_precond(p->vd, p->L, s, pcg_c, use);
    }
    // the one-reduction rounds take one more launch than updates: round 0 only stages
    if (inline_pcg && inner_pcg(p))
        for (int k = 0; k < max_pcg + (p->use_cg ? 1 : 0); ++k) step_pcg_iter(p, s, pcg_c, use);
}

static void step_lm_tail(ba_problem* p, cudaStream_t s, CondHandle lm_c, int use) {
    if (p->precision == BA_PREC_MIXED) {
        const Views<float>& v = p->vf;
        if (p->use_schur) launch_schur(v, s, 2, &v.st->lm_active);   // points back-substituted
        launch_candidate(v, p->L, s);
        launch_residual(v, p->L, s, 1);   // r(x') and F'; the relinearisation reuses r
        launch_eval_candidate(v, p->L, s, lm_c, use);
        launch_commit(v, p->L, s);
        launch_linearize(v, p->L, s, 1, nullptr, nullptr, lm_c, 0);
    } else {
        const Views<double>& v = p->vd;
        launch64_candidate(v, p->L, s);
        launch64_eval_candidate(v, p->L, s, lm_c, use);
        launch64_commit(v, p->L, s);
        launch64_linearize(v, p->L, s, 1, nullptr, nullptr, lm_c, 0);
    }
}

static DevState* dev_state(ba_problem* p) { return p->precision == BA_PREC_MIXED ? p->vf.st : p->vd.st; }

// Adds a WHILE conditional node at the current capture position of `s`; returns its
// body graph.  The handle must already exist on the capturing graph.
static cudaError_t add_while_node(cudaStream_t s, CondHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = (cudaGraphConditionalHandle)h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np);
    if (e != cudaSuccess) return e;
    *body = np.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// One CUDA graph for a whole solve: init, then WHILE(lm) { lm_head; WHILE(pcg)
// { pcg_iter }; lm_tail }, finish.  Loop flags are set on the device by the kernels
// that decide them; both loops are bounded by the iteration caps in the device state.
static ba_status build_graph_loops(ba_problem* p) {
    cudaStream_t s0 = p->cap[0], s1 = p->cap[1], s2 = p->cap[2];
    cudaGraph_t top;
    GBBA_CUDA(cudaGraphCreate(&top, 0));
    cudaGraphConditionalHandle lm_h, pcg_h;
    GBBA_CUDA(cudaGraphConditionalHandleCreate(&lm_h, top, 0, cudaGraphCondAssignDefault));
    GBBA_CUDA(cudaStreamBeginCaptureToGraph(s0, top, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    step_init(p, s0, (CondHandle)lm_h, 1);
    cudaGraph_t lm_body;
    cudaError_t e = add_while_node(s0, (CondHandle)lm_h, &lm_body);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&pcg_h, lm_body, 0, 0);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s1, lm_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        const bool inner = inner_pcg(p);
        step_lm_head(p, s1, (CondHandle)pcg_h, inner ? 1 : 0, false, 0);
        if (inner) {
            cudaGraph_t pcg_body;
            e = add_while_node(s1, (CondHandle)pcg_h, &pcg_body);
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(s2, pcg_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                step_pcg_iter(p, s2, (CondHandle)pcg_h, 1);
                cudaGraph_t tmp;
                e = cudaStreamEndCapture(s2, &tmp);
            }
        }
        if (e == cudaSuccess) step_lm_tail(p, s1, (CondHandle)lm_h, 1);
        cudaGraph_t tmp1;
        cudaError_t e1 = cudaStreamEndCapture(s1, &tmp1);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) launch_finish_state(dev_state(p), s0);
    cudaGraph_t tmp0;
    cudaError_t e0 = cudaStreamEndCapture(s0, &tmp0);
    if (e == cudaSuccess) e = e0;
    if (e != cudaSuccess) {
        cudaGraphDestroy(top);
        return cuda_status(e, "building the solve graph");
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, top, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(top);
        return cuda_status(e, "cudaGraphInstantiate");
    }
    p->graph.graph = top;
    p->graph.exec = exec;
    return BA_OK;
}

// The fixed predicated sequence: max_lm_iters LM slots of max_pcg_iters PCG slots;
// kernels of idle slots return at once.
static void enqueue_solve_predicated(ba_problem* p, const ba_options& o, cudaStream_t s) {
    step_init(p, s, 0, 0);
    for (int it = 0; it < o.max_lm_iters; ++it) {
        step_lm_head(p, s, 0, 0, true, o.max_pcg_iters);
        step_lm_tail(p, s, 0, 0);
    }
    launch_finish_state(dev_state(p), s);
}

}  // namespace gbba

using namespace gbba;

// ------------------------------------------------------------------ C ABI ------

extern "C" {

const char* ba_last_error(void) { return g_err; }

const char* ba_status_string(int32_t s) {
    switch (s) {
        case BA_OK: return "ok";
        case BA_ERR_INVALID_ARG: return "invalid argument";
        case BA_ERR_CUDA: return "CUDA error";
        case BA_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case BA_ERR_NUMERIC: return "numeric failure (NaN/Inf or non-SPD block)";
        case BA_ERR_TIMEOUT: return "device wait timed out";
        case BA_ERR_NOT_IMPLEMENTED: return "not implemented";
        case BA_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

int32_t ba_abi_version(void) { return 2; }

ba_status ba_selftest_wait_timeout(void* scratch, int32_t grid, int32_t timeout_ms, void* stream, int32_t* gave_up,
                                   int32_t* error_word) {
    if (!scratch || !gave_up || !error_word || ((uintptr_t)scratch & 15u) != 0) {
        set_error("ba_selftest_wait_timeout: null or misaligned pointer");
        return BA_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    GBBA_CUDA(cudaGetDevice(&dev));
    GBBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (grid < 1 || grid > sms || timeout_ms < 1 || timeout_ms > 2000) {
        set_error("ba_selftest_wait_timeout: grid must be in [1, %d] and timeout in [1, 2000] ms", sms);
        return BA_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    GBBA_CUDA(cudaMemsetAsync(scratch, 0, 16, s));
    GBBA_CUDA(launch_selftest_wait(scratch, grid, 1000000LL * timeout_ms, s));
    int32_t words[4];
    GBBA_CUDA(cudaMemcpyAsync(words, scratch, 16, cudaMemcpyDeviceToHost, s));
    GBBA_CUDA(cudaStreamSynchronize(s));
    *error_word = words[2];
    *gave_up = words[3];
    return BA_OK;
}

ba_status ba_selftest_rcp64(const double* x, double* y, int64_t n, void* stream) {
    if (!x || !y || n < 1) {
        set_error("ba_selftest_rcp64: null pointer or n < 1");
        return BA_ERR_INVALID_ARG;
    }
    launch_selftest_rcp64(x, y, n, (cudaStream_t)stream);
    GBBA_CUDA(cudaGetLastError());
    return BA_OK;
}

ba_status ba_options_default(ba_options* o) {
    if (!o) {
        set_error("ba_options_default: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    o->max_lm_iters = 20;
    o->max_pcg_iters = 50;
    o->pcg_rel_tol = 1e-3;
    o->initial_trust_region = 100.0;
    o->min_diag = 1e-6;
    o->max_diag = 1e32;
    o->max_mu = 1e16;
    o->eps_depth = 0.0;
    o->use_graph = 1;
    o->pcg_kernel = 2;
    o->rotation_update = 0;
    o->loss = 0;
    o->loss_scale = 1.0;
    o->solver = 0;
    o->wait_timeout_ms = 2000;
    o->residual_precision = 1;
    return BA_OK;
}

namespace {

// Validation of the observation arrays and their copy into the problem, split over the
// host's cores for large problems (one pass over 28.8M observations on one core takes
// ~0.2 s).  Each thread takes a contiguous range of observations: it checks the indices
// and pixels up to its first bad observation, copies its range, and marks the points it
// sees in two bitmaps of its own (seen once, seen at least twice).  The bitmaps are then
// merged word by word over the threads, and the first bad observation or the first point
// seen fewer than twice is reported, as a sequential pass would report it.
struct ObsCheck {
    int64_t bad_obs = -1;   // first bad observation
    bool range = false;     // ... because of an index (else a pixel)
    int32_t bad_pt = -1;    // first point observed fewer than twice
    uint32_t bad_deg = 0;
};

ObsCheck check_and_copy_observations(int32_t n_cams, int32_t n_pts, int64_t n_obs, const uint32_t* cam_idx,
                                     const uint32_t* pt_idx, const double* pixels, uint32_t* cam_out,
                                     uint32_t* pt_out, double* px_out) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, 16, n_obs >> 20}));
    const size_t words = ((size_t)n_pts + 63) / 64;
    std::vector<uint64_t> once((size_t)nt * words, 0ull), twice((size_t)nt * words, 0ull);
    std::vector<int64_t> first_bad(nt, -1);
    std::vector<char> bad_range(nt, 0);
    auto work = [&](int t) {
        const int64_t a = n_obs * t / nt, b = n_obs * (t + 1) / nt;
        uint64_t* o1 = once.data() + (size_t)t * words;
        uint64_t* o2 = twice.data() + (size_t)t * words;
        for (int64_t o = a; o < b; ++o) {
            const uint32_t c = cam_idx[o], i = pt_idx[o];
            if (c >= (uint32_t)n_cams || i >= (uint32_t)n_pts) {
                first_bad[t] = o;
                bad_range[t] = 1;
                return;
            }
            if (!std::isfinite(pixels[2 * o]) || !std::isfinite(pixels[2 * o + 1])) {
                first_bad[t] = o;
                return;
            }
            const uint64_t bit = 1ull << (i & 63u);
            uint64_t& w1 = o1[i >> 6];
            o2[i >> 6] |= w1 & bit;
            w1 |= bit;
        }
        std::memcpy(cam_out + a, cam_idx + a, 4 * (size_t)(b - a));
        std::memcpy(pt_out + a, pt_idx + a, 4 * (size_t)(b - a));
        std::memcpy(px_out + 2 * a, pixels + 2 * a, 16 * (size_t)(b - a));
    };
    // merge: a point is seen twice if one thread saw it twice or two threads saw it
    std::vector<uint64_t> seen1(words, 0ull), seen2(words, 0ull);
    auto merge = [&](int t) {
        const size_t w0 = words * t / nt, w1 = words * (t + 1) / nt;
        for (size_t w = w0; w < w1; ++w) {
            uint64_t s1 = 0ull, s2 = 0ull;
            for (int u = 0; u < nt; ++u) {
                const uint64_t a1 = once[(size_t)u * words + w];
                s2 |= twice[(size_t)u * words + w] | (s1 & a1);
                s1 |= a1;
            }
            seen1[w] = s1;
            seen2[w] = s2;
        }
    };
    auto run = [&](auto&& f) {
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(f, t);
        f(0);
        for (auto& x : th) x.join();
    };
    run(work);
    ObsCheck r;
    for (int t = 0; t < nt; ++t)
        if (first_bad[t] >= 0) {
            r.bad_obs = first_bad[t];
            r.range = bad_range[t] != 0;
            return r;
        }
    run(merge);
    for (size_t w = 0; w < words; ++w) {
        const uint64_t valid = (w + 1 < words || (n_pts & 63) == 0) ? ~0ull : ((1ull << (n_pts & 63)) - 1ull);
        const uint64_t short_pts = ~seen2[w] & valid;
        if (short_pts) {
            const int b = __builtin_ctzll(short_pts);
            r.bad_pt = (int32_t)(64 * w + b);
            r.bad_deg = ((seen1[w] >> b) & 1ull) ? 1u : 0u;
            return r;
        }
    }
    return r;
}

}  // namespace

ba_status ba_problem_create(int32_t n_cams, int32_t n_pts, int64_t n_obs, const uint32_t* cam_idx,
                            const uint32_t* pt_idx, const double* pixels, int32_t precision, ba_problem** out) {
    if (!out) {
        set_error("ba_problem_create: out is null");
        return BA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n_cams < 1 || n_cams >= (1 << 24) || n_pts < 1 || n_obs < 1 || n_obs >= (int64_t)0xffffffffLL) {
        set_error("ba_problem_create: sizes out of range (n_cams=%d n_pts=%d n_obs=%lld)", n_cams, n_pts,
                  (long long)n_obs);
        return BA_ERR_INVALID_ARG;
    }
    if (!cam_idx || !pt_idx || !pixels) {
        set_error("ba_problem_create: null input array");
        return BA_ERR_INVALID_ARG;
    }
    if (precision != BA_PREC_MIXED && precision != BA_PREC_FP64) {
        set_error("ba_problem_create: unknown precision %d", precision);
        return BA_ERR_INVALID_ARG;
    }
    ba_problem* p = new (std::nothrow) ba_problem();
    if (!p) {
        set_error("ba_problem_create: out of host memory");
        return BA_ERR_INVALID_ARG;
    }
    try {
        p->cam_idx.resize((size_t)n_obs);
        p->pt_idx.resize((size_t)n_obs);
        p->pixels.resize(2 * (size_t)n_obs);
    } catch (...) {
        delete p;
        set_error("ba_problem_create: out of host memory");
        return BA_ERR_INVALID_ARG;
    }
    const ObsCheck chk = check_and_copy_observations(n_cams, n_pts, n_obs, cam_idx, pt_idx, pixels, p->cam_idx.data(),
                                                     p->pt_idx.data(), p->pixels.data());
    if (chk.bad_obs >= 0 || chk.bad_pt >= 0) {
        if (chk.bad_obs >= 0 && chk.range)
            set_error("ba_problem_create: observation %lld has camera %u / point %u out of range",
                      (long long)chk.bad_obs, cam_idx[chk.bad_obs], pt_idx[chk.bad_obs]);
        else if (chk.bad_obs >= 0)
            set_error("ba_problem_create: observation %lld has a non-finite pixel", (long long)chk.bad_obs);
        else
            set_error("ba_problem_create: point %d is observed %u time(s); at least 2 are required", chk.bad_pt,
                      chk.bad_deg);
        delete p;
        return BA_ERR_INVALID_ARG;
    }
    p->n_cams = n_cams;
    p->n_pts = n_pts;
    p->n_obs = n_obs;
    p->n_tiles = (n_pts + TILE_PTS - 1) / TILE_PTS;
    p->precision = precision;
    p->pt_off = (int64_t)((9 * (size_t)n_cams + 3) / 4 * 4);
    p->n_vec = p->pt_off + 12 * (int64_t)(((size_t)n_pts + 3) / 4);
    p->lay = compute_layout(n_cams, n_pts, n_obs, precision);
    *out = p;
    return BA_OK;
}

static void release_graph(ba_problem* p) {
    for (GraphCache* g : {&p->graph, &p->graph_unrolled}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        *g = GraphCache{};
    }
    p->unrolled_lm = p->unrolled_pcg = -1;
}

void ba_problem_destroy(ba_problem* p) {
    if (!p) return;
    release_graph(p);
    for (auto& s : p->cap)
        if (s) cudaStreamDestroy(s);
    delete p;
}

ba_status ba_workspace_size(const ba_problem* p, size_t* bytes) {
    if (!p || !bytes) {
        set_error("ba_workspace_size: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    *bytes = p->lay.total;
    return BA_OK;
}

ba_status ba_set_pose_factors(ba_problem* p, int32_t n, const uint32_t* cam_a, const uint32_t* cam_b,
                              const double* meas, const double* sqrt_info) {
    if (!p) {
        set_error("ba_set_pose_factors: null problem");
        return BA_ERR_INVALID_ARG;
    }
    if (p->bound) {
        set_error("ba_set_pose_factors: the problem is bound; set factors before ba_bind_workspace");
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision != BA_PREC_MIXED) {
        set_error("ba_set_pose_factors: pose factors are available for the mixed-precision form only");
        return BA_ERR_NOT_IMPLEMENTED;
    }
    if (n < 0 || (n > 0 && (!cam_a || !cam_b || !meas))) {
        set_error("ba_set_pose_factors: bad count or null array");
        return BA_ERR_INVALID_ARG;
    }
    for (int32_t k = 0; k < n; ++k) {
        if (cam_a[k] >= (uint32_t)p->n_cams || cam_b[k] >= (uint32_t)p->n_cams || cam_a[k] == cam_b[k]) {
            set_error("ba_set_pose_factors: factor %d ties cameras %u and %u", k, cam_a[k], cam_b[k]);
            return BA_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 6; ++i) {
            const double m = meas[6 * (size_t)k + i];
            const double w = sqrt_info ? sqrt_info[6 * (size_t)k + i] : 1.0;
            if (!std::isfinite(m) || !std::isfinite(w) || w < 0.0) {
                set_error("ba_set_pose_factors: factor %d has a non-finite value or a negative weight", k);
                return BA_ERR_INVALID_ARG;
            }
        }
    }
    p->n_fac = n;
    p->fac_cam.resize(2 * (size_t)n);
    p->fac_meas.assign(meas, meas + 6 * (size_t)n);
    p->fac_sqrt.assign(6 * (size_t)n, 1.0);
    for (int32_t k = 0; k < n; ++k) {
        p->fac_cam[2 * (size_t)k] = cam_a[k];
        p->fac_cam[2 * (size_t)k + 1] = cam_b[k];
    }
    if (sqrt_info) p->fac_sqrt.assign(sqrt_info, sqrt_info + 6 * (size_t)n);
    p->lay = compute_layout(p->n_cams, p->n_pts, p->n_obs, p->precision, n);
    return BA_OK;
}

static ba_status check_bound(const ba_problem* p, const char* who) {
    if (!p) {
        set_error("%s: null problem", who);
        return BA_ERR_INVALID_ARG;
    }
    if (!p->bound) {
        set_error("%s: no workspace bound (call ba_bind_workspace first)", who);
        return BA_ERR_STATE;
    }
    return BA_OK;
}

static ba_status write_options(ba_problem* p, const ba_options* o);

// Persistent PCG plan: one CTA per SM, contiguous tile runs balanced by observation
// count; a form is used only when every CTA's keys and point state fit in its shared
// memory.  Each CTA lists the cameras of its observations and of its pose factors
// (factor k runs in CTA k % G); a camera that neither sees is listed by CTA c % G, and
// the first list holding a camera owns it.
static ba_status plan_persistent(ba_problem* p, int sms) {
    const int nt = p->n_tiles;
    std::vector<uint32_t> off((size_t)nt + 1);
    GBBA_CUDA(cudaMemcpy(off.data(), p->vf.tile_off, 4 * off.size(), cudaMemcpyDeviceToHost));
    const int G = std::min(std::min(sms, MAX_PBLOCKS), nt);
    if (G < 1) return BA_OK;
    std::vector<uint32_t> bt((size_t)G + 1, 0);
    const double total = (double)off[nt];
    int t = 0;
    for (int b = 1; b < G; ++b) {
        const double target = total * b / G;
        while (t < nt && (double)off[t] < target) ++t;
        bt[b] = (uint32_t)std::max(t, (int)bt[b - 1]);
    }
    bt[G] = (uint32_t)nt;
    const size_t limit = (size_t)std::max(0, persistent_max_smem() - 4096);
    auto point_bytes = [&](int b) {
        const size_t no = off[bt[b + 1]] - off[bt[b]];
        const long pb = (long)bt[b] * TILE_PTS, pe = std::min((long)bt[b + 1] * TILE_PTS, (long)p->n_pts);
        const size_t np = pe > pb ? (size_t)(pe - pb) : 0;
        const size_t n3p = (3 * np + 3) & ~(size_t)3;
        // keys, X and p as float4, D r z h q as 3-float arrays, M^-1 (6 per point)
        return ((4 * no + 15) & ~(size_t)15) + 32 * np + 4 * (5 * n3p + ((6 * np + 3) & ~(size_t)3));
    };
    size_t worst = 0;
    for (int b = 0; b < G; ++b) worst = std::max(worst, point_bytes(b));
    if (worst > limit) return BA_OK;   // too large: the multi-kernel PCG path is used
    // distinct cameras of each CTA's observations (sorted), then the unseen ones
    std::vector<uint32_t> keys((size_t)p->n_obs);
    GBBA_CUDA(cudaMemcpy(keys.data(), p->vf.obs_key, 4 * keys.size(), cudaMemcpyDeviceToHost));
    std::vector<std::vector<uint32_t>> lists((size_t)G);
    std::vector<char> seen((size_t)p->n_cams, 0);
    for (int b = 0; b < G; ++b) {
        std::vector<uint32_t>& cb = lists[b];
        for (uint32_t j = off[bt[b]]; j < off[bt[b + 1]]; ++j) cb.push_back(keys[j] >> 8);
        std::sort(cb.begin(), cb.end());
        cb.erase(std::unique(cb.begin(), cb.end()), cb.end());
        for (uint32_t c : cb) seen[c] = 1;
    }
    // pose factor k runs in CTA k % G, which lists both of its cameras
    for (int32_t k = 0; k < p->n_fac; ++k)
        for (int e = 0; e < 2; ++e) {
            const uint32_t c = p->fac_cam[2 * (size_t)k + e];
            std::vector<uint32_t>& cb = lists[k % G];
            auto it = std::lower_bound(cb.begin(), cb.end(), c);
            if (it == cb.end() || *it != c) cb.insert(it, c);
            seen[c] = 1;
        }
    for (int c = 0; c < p->n_cams; ++c)
        if (!seen[c]) {
            std::vector<uint32_t>& cb = lists[c % G];
            cb.insert(std::upper_bound(cb.begin(), cb.end(), (uint32_t)c), (uint32_t)c);
        }
    std::fill(seen.begin(), seen.end(), 0);
    std::vector<uint32_t> coff((size_t)G + 1, 0), cams;
    size_t worst_one = 0, worst_two = 0;
    for (int b = 0; b < G; ++b) {
        for (uint32_t c : lists[b]) {
            cams.push_back(seen[c] ? c : (c | BLK_CAM_OWNER));
            seen[c] = 1;
        }
        coff[b + 1] = (uint32_t)cams.size();
        const size_t ncb = lists[b].size();
        const size_t no = off[bt[b + 1]] - off[bt[b]];
        const long pb = (long)bt[b] * TILE_PTS, pe = std::min((long)bt[b + 1] * TILE_PTS, (long)p->n_pts);
        const size_t np = pe > pb ? (size_t)(pe - pb) : 0;
        worst_two = std::max(worst_two, point_bytes(b) + 4 * ((ncb + 3) & ~(size_t)3) + 4 * 28 * ncb);
        worst_one = std::max(worst_one, pcg1_smem_bytes(no, np, ncb));
    }
    const size_t cap = (p->lay.pslots - p->lay.blk_cams) / 4;
    if (cams.size() > cap) return BA_OK;
    auto fits = [&](int form, size_t bytes) {
        int bps = 0;
        if (bytes > limit) return false;
        if (persistent_prepare(form, (int)bytes, &bps) != cudaSuccess || bps < 1) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    p->fits_one = fits(PCG_ONE_EXCHANGE, worst_one);
    p->fits_two = fits(PCG_TWO_EXCHANGE, worst_two);
    if (!p->fits_one && !p->fits_two) return BA_OK;
    GBBA_CUDA(cudaMemcpy(p->blk_tile, bt.data(), 4 * bt.size(), cudaMemcpyHostToDevice));
    GBBA_CUDA(cudaMemcpy(p->blk_cam_off, coff.data(), 4 * coff.size(), cudaMemcpyHostToDevice));
    GBBA_CUDA(cudaMemcpy(p->blk_cams, cams.data(), 4 * cams.size(), cudaMemcpyHostToDevice));
    p->persistent = true;
    p->p_grid = G;
    p->p_smem_one = (int)worst_one;
    p->p_smem_two = (int)worst_two;
    p->p_form = p->fits_one ? PCG_ONE_EXCHANGE : PCG_TWO_EXCHANGE;   // the default form first
    return BA_OK;
}

ba_status ba_bind_workspace(ba_problem* p, void* ws, size_t bytes, void* stream) {
    if (!p || !ws) {
        set_error("ba_bind_workspace: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    if (((uintptr_t)ws & 255u) != 0) {
        set_error("ba_bind_workspace: workspace must be 256-byte aligned");
        return BA_ERR_INVALID_ARG;
    }
    if (bytes < p->lay.total) {
        set_error("ba_bind_workspace: workspace has %zu bytes, needs %zu", bytes, p->lay.total);
        return BA_ERR_WORKSPACE_TOO_SMALL;
    }
    release_graph(p);
    p->bound = false;
    p->linearized = false;
    p->ws = (char*)ws;
    p->ws_bytes = bytes;
    p->stream = (cudaStream_t)stream;
    GBBA_CUDA(cudaGetDevice(&p->device));
    for (auto& s : p->cap)
        if (!s) GBBA_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int sms = 0;
    GBBA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    p->L.item_block = 256;
    p->L.item_grid = std::min(MAX_GRID, sms * 8);
    if (p->precision == BA_PREC_MIXED) {
        p->L.lin_grid = std::min(MAX_GRID, sms * std::max(1, occupancy_blocks_linearize()));
        p->L.mv_grid = std::min(MAX_GRID, sms * std::max(1, occupancy_blocks_matvec()));
        p->L.ev_grid = std::min(MAX_GRID, sms * std::max(1, occupancy_blocks_eval()));
        p->L.res_grid = std::min(MAX_GRID, sms * occupancy_blocks_residual());
    }
    const Layout& l = p->lay;
    char* w = p->ws;
    cudaStream_t s = p->stream;
    GBBA_CUDA(cudaMemsetAsync(w + l.state, 0, sizeof(DevState), s));
    GBBA_CUDA(cudaMemsetAsync(w + l.partials, 0, sizeof(double) * MAX_GRID * NPART, s));
    {
        // evaluation and operator calls made before any solve use the default options
        ba_options d;
        ba_options_default(&d);
        ba_status ost = write_options(p, &d);
        if (ost) return ost;
    }
    GBBA_CUDA(cudaMemcpyAsync(w + l.s_cam_idx, p->cam_idx.data(), 4 * (size_t)p->n_obs, cudaMemcpyHostToDevice, s));
    GBBA_CUDA(cudaMemcpyAsync(w + l.s_pt_idx, p->pt_idx.data(), 4 * (size_t)p->n_obs, cudaMemcpyHostToDevice, s));
    GBBA_CUDA(cudaMemcpyAsync(w + l.s_pixels, p->pixels.data(), 16 * (size_t)p->n_obs, cudaMemcpyHostToDevice, s));
    OrderBuffers b{};
    b.cam_idx = (const uint32_t*)(w + l.s_cam_idx);
    b.pt_idx = (const uint32_t*)(w + l.s_pt_idx);
    b.pixels = (const double*)(w + l.s_pixels);
    b.pt_key = (uint32_t*)(w + l.s_pt_key);
    b.tile_cnt = (uint32_t*)(w + l.s_tile_cnt);
    b.keys = (uint64_t*)(w + l.s_keys);
    b.vals = (uint32_t*)(w + l.s_vals);
    b.sort_cap = l.sort_cap;
    p->vf = make_views<float>(p);
    p->vd = make_views<double>(p);
    if (p->precision == BA_PREC_MIXED) build_order<float>(p->vf, b, s);
    else build_order<double>(p->vd, b, s);
    GBBA_CUDA(cudaGetLastError());
    // repeated (camera, point) observations decide how the tile operator sums points;
    // the point-key scratch is free once the order is built
    uint32_t repeated = 1u;
    if (p->precision == BA_PREC_MIXED) {
        GBBA_CUDA(cudaMemsetAsync(b.pt_key, 0, sizeof(uint32_t), s));
        flag_repeated_keys(p->vf.obs_key, p->n_obs, b.pt_key, s);
        GBBA_CUDA(cudaGetLastError());
        GBBA_CUDA(cudaMemcpyAsync(&repeated, b.pt_key, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    // the scratch overlapped the solver arrays: clear them before first use
    const size_t ub = l.vec[0];
    GBBA_CUDA(cudaMemsetAsync(w + ub, 0, l.total - ub, s));
    if (p->n_fac > 0) {   // pose factors live among the solver arrays
        GBBA_CUDA(cudaMemcpyAsync(w + l.fac_cam, p->fac_cam.data(), 4 * p->fac_cam.size(), cudaMemcpyHostToDevice, s));
        GBBA_CUDA(cudaMemcpyAsync(w + l.fac_meas, p->fac_meas.data(), 8 * p->fac_meas.size(), cudaMemcpyHostToDevice, s));
        GBBA_CUDA(cudaMemcpyAsync(w + l.fac_sqrt, p->fac_sqrt.data(), 8 * p->fac_sqrt.size(), cudaMemcpyHostToDevice, s));
    }
    GBBA_CUDA(cudaStreamSynchronize(s));
    p->blk_tile = (uint32_t*)(w + l.blk_tile);
    p->blk_cam_off = (uint32_t*)(w + l.blk_cam_off);
    p->blk_cams = (uint32_t*)(w + l.blk_cams);
    p->pslots = (double*)(w + l.pslots);
    p->persistent = p->fits_one = p->fits_two = false;
    if (p->precision == BA_PREC_MIXED) {
        ba_status pst = plan_persistent(p, sms);
        if (pst) return pst;
        const size_t nt = (size_t)p->n_tiles;
        std::vector<uint32_t> toff(nt + 1), loff(nt + 1), sst(nt);
        GBBA_CUDA(cudaMemcpy(toff.data(), p->vf.tile_off, 4 * toff.size(), cudaMemcpyDeviceToHost));
        GBBA_CUDA(cudaMemcpy(loff.data(), p->vf.long_off, 4 * loff.size(), cudaMemcpyDeviceToHost));
        GBBA_CUDA(cudaMemcpy(sst.data(), p->vf.short_start, 4 * sst.size(), cudaMemcpyDeviceToHost));
        uint32_t most_long = 1, most_short = 1, most_runs = 1;
        for (size_t t = 0; t < nt; ++t) {
            most_long = std::max(most_long, sst[t] - toff[t]);
            most_short = std::max(most_short, toff[t + 1] - sst[t]);
            most_runs = std::max(most_runs, loff[t + 1] - loff[t]);
        }
        plan_tile_kernels(p->L, p->n_tiles, sms, (int)most_long, (int)most_short, (int)most_runs);
        p->L.tn_plain_q = repeated == 0u;
        GBBA_CUDA(cudaGetLastError());
    }
    p->bound = true;
    return BA_OK;
}

ba_status ba_set_params(ba_problem* p, const double* cams, const double* pts) {
    ba_status st = check_bound(p, "ba_set_params");
    if (st) return st;
    if (!cams || !pts) {
        set_error("ba_set_params: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    double* stg = (double*)(p->ws + p->lay.staging);
    GBBA_CUDA(cudaMemcpyAsync(stg, cams, 72 * (size_t)p->n_cams, cudaMemcpyHostToDevice, p->stream));
    GBBA_CUDA(cudaMemcpyAsync(stg + 9 * (size_t)p->n_cams, pts, 24 * (size_t)p->n_pts, cudaMemcpyHostToDevice, p->stream));
    return ba_set_params_device(p, stg, stg + 9 * (size_t)p->n_cams, 1);
}

ba_status ba_get_params(ba_problem* p, double* cams, double* pts) {
    ba_status st = check_bound(p, "ba_get_params");
    if (st) return st;
    if (!cams || !pts) {
        set_error("ba_get_params: null pointer");
        return BA_ERR_INVALID_ARG;
    }
    double* stg = (double*)(p->ws + p->lay.staging);
    st = ba_get_params_device(p, stg, stg + 9 * (size_t)p->n_cams, 1);
    if (st) return st;
    GBBA_CUDA(cudaMemcpyAsync(cams, stg, 72 * (size_t)p->n_cams, cudaMemcpyDeviceToHost, p->stream));
    GBBA_CUDA(cudaMemcpyAsync(pts, stg + 9 * (size_t)p->n_cams, 24 * (size_t)p->n_pts, cudaMemcpyDeviceToHost, p->stream));
    GBBA_CUDA(cudaStreamSynchronize(p->stream));
    return BA_OK;
}

ba_status ba_set_params_device(ba_problem* p, const void* cams, const void* pts, int32_t dtype) {
    ba_status st = check_bound(p, "ba_set_params_device");
    if (st) return st;
    if (!cams || !pts || (dtype != 0 && dtype != 1)) {
        set_error("ba_set_params_device: null pointer or bad dtype %d", dtype);
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision == BA_PREC_MIXED) launch_pack(p->vf, p->L, p->stream, cams, pts, dtype);
    else launch64_pack(p->vd, p->L, p->stream, cams, pts, dtype);
    GBBA_CUDA(cudaGetLastError());
    p->linearized = false;
    return BA_OK;
}

ba_status ba_get_params_device(ba_problem* p, void* cams, void* pts, int32_t dtype) {
    ba_status st = check_bound(p, "ba_get_params_device");
    if (st) return st;
    if (!cams || !pts || (dtype != 0 && dtype != 1)) {
        set_error("ba_get_params_device: null pointer or bad dtype %d", dtype);
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision == BA_PREC_MIXED) launch_unpack(p->vf, p->L, p->stream, p->vf.xm, cams, pts, dtype);
    else launch64_unpack(p->vd, p->L, p->stream, cams, pts, dtype);
    GBBA_CUDA(cudaGetLastError());
    return BA_OK;
}

static ba_status read_state(ba_problem* p, DevState* host) {
    GBBA_CUDA(cudaMemcpyAsync(host, p->ws + p->lay.state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
    GBBA_CUDA(cudaStreamSynchronize(p->stream));
    return BA_OK;
}

ba_status ba_evaluate(ba_problem* p, double* cost_out, void* residuals, void* jacobian) {
    ba_status st = check_bound(p, "ba_evaluate");
    if (st) return st;
    DevState* dst = dev_state(p);
    // evaluation (and ba_apply_normal after it) is always w.r.t. the angle-axis
    // parameters and the squared loss
    static_assert(offsetof(DevOptions, loss) == offsetof(DevOptions, retract) + sizeof(int32_t), "adjacent");
    const int32_t plain[2] = {0, 0};   // retract, loss
    GBBA_CUDA(cudaMemcpyAsync(&dst->opt.retract, plain, sizeof(plain), cudaMemcpyHostToDevice, p->stream));
    if (p->precision == BA_PREC_MIXED) {
        launch_camera_precompute(p->vf, p->L, p->stream);
        launch_residual(p->vf, p->L, p->stream, 0, 1);   // evaluation: the squared loss
        launch_linearize(p->vf, p->L, p->stream, 2, (float*)residuals, (float*)jacobian, 0, 0);
    } else {
        launch64_camera_precompute(p->vd, p->L, p->stream);
        launch64_linearize(p->vd, p->L, p->stream, 2, (double*)residuals, (double*)jacobian, 0, 0);
    }
    GBBA_CUDA(cudaGetLastError());
    p->linearized = true;
    if (cost_out) {
        double c = 0;
        GBBA_CUDA(cudaMemcpyAsync(&c, &dst->cost_out, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
        GBBA_CUDA(cudaStreamSynchronize(p->stream));
        *cost_out = c;
    }
    return BA_OK;
}

static ba_status check_options(const ba_options* o) {
    if (!o) {
        set_error("null options");
        return BA_ERR_INVALID_ARG;
    }
    if (o->max_lm_iters < 0 || o->max_pcg_iters < 0 || !(o->pcg_rel_tol >= 0) || !(o->initial_trust_region > 0) ||
        !(o->min_diag > 0) || !(o->max_diag >= o->min_diag) || !(o->eps_depth >= 0) || !(o->max_mu > 0) ||
        (o->pcg_kernel < 0 || o->pcg_kernel > 3) || o->use_graph < 0 || o->use_graph > 2 ||
        (o->rotation_update != 0 && o->rotation_update != 1) || o->loss < 0 || o->loss > 2 ||
        !(o->loss_scale > 0) || (o->solver != 0 && o->solver != 1) || o->wait_timeout_ms < 0 ||
        o->wait_timeout_ms > 60000 || (o->residual_precision != 0 && o->residual_precision != 1)) {
        set_error("invalid options (iterations must be >= 0, tolerances/diagonal bounds positive, "
                  "wait_timeout_ms in [0, 60000], residual_precision 0 or 1)");
        return BA_ERR_INVALID_ARG;
    }
    return BA_OK;
}

static ba_status write_options(ba_problem* p, const ba_options* o) {
    DevOptions d{};
    d.max_lm = o->max_lm_iters;
    d.max_pcg = o->max_pcg_iters;
    d.tol = o->pcg_rel_tol;
    d.mu0 = 1.0 / o->initial_trust_region;
    d.min_diag = o->min_diag;
    d.max_diag = o->max_diag;
    // the mixed form's PCG vectors scale like g / (mu D): past mu ~ 1e19 their FP32
    // squares underflow, so its LM stops at 1e16 at the latest
    d.max_mu = p->precision == BA_PREC_MIXED ? std::min(o->max_mu, 1e16) : o->max_mu;
    d.eps = o->eps_depth;
    d.retract = o->rotation_update;
    d.loss = o->loss;
    d.loss_scale = o->loss_scale;
    d.wait_ns = 1000000LL * (int64_t)o->wait_timeout_ms;
    d.res_df = o->residual_precision;
    static_assert(offsetof(DevState, opt) == 0, "options first");
    GBBA_CUDA(cudaMemcpyAsync(p->ws + p->lay.state, &d, sizeof(d), cudaMemcpyHostToDevice, p->stream));
    return BA_OK;
}

ba_status ba_get_stats(ba_problem* p, ba_stats* stats, ba_iter_stat* hist, int32_t cap) {
    ba_status st = check_bound(p, "ba_get_stats");
    if (st) return st;
    if (!stats) {
        set_error("ba_get_stats: null stats");
        return BA_ERR_INVALID_ARG;
    }
    DevState* h = new DevState;
    st = read_state(p, h);
    if (st) {
        delete h;
        return st;
    }
    stats->initial_cost = h->F0;
    stats->final_cost = h->F;
    stats->lm_iters = h->lm_iter;
    stats->accepted = h->n_accepted;
    stats->pcg_iters_total = h->pcg_total;
    stats->status = h->status;
    stats->solve_ns = h->t_end - h->t_start;
    if (hist && cap > 0) {
        const int n = std::min(std::min(cap, h->lm_iter), HIST_CAP);
        static_assert(sizeof(IterRec) == sizeof(ba_iter_stat), "history record layout");
        memcpy(hist, h->hist, sizeof(IterRec) * (size_t)n);
    }
    delete h;
    return BA_OK;
}

ba_status ba_solve(ba_problem* p, const ba_options* o, ba_stats* stats, ba_iter_stat* hist, int32_t cap) {
    ba_status st = check_bound(p, "ba_solve");
    if (st) return st;
    if ((st = check_options(o))) return st;
    if (o->solver == 1 && p->precision != BA_PREC_MIXED) {
        set_error("ba_solve: the Schur-complement solver is available for the mixed-precision form only");
        return BA_ERR_NOT_IMPLEMENTED;
    }
    if (o->solver == 1 && p->n_fac > 0) {
        set_error("ba_solve: the Schur-complement solver does not take pose factors");
        return BA_ERR_NOT_IMPLEMENTED;
    }
    if ((st = write_options(p, o))) return st;
    const bool want_schur = o->solver == 1;
    // pcg_kernel 2: the persistent kernel's one-exchange form when its plan fits, else its
    // two-exchange form; 0: the two-exchange form; otherwise (or when neither plan fits)
    // separate kernels
    const int want_form = (o->pcg_kernel == 2 && p->fits_one) ? PCG_ONE_EXCHANGE : PCG_TWO_EXCHANGE;
    const bool want_persistent = !want_schur && o->pcg_kernel != 1 && o->pcg_kernel != 3 &&
                                 (want_form == PCG_ONE_EXCHANGE ? p->fits_one : p->fits_two);
    // pcg_kernel 3: separate kernels with the one-reduction recurrences (tile kernels)
    const bool want_cg = p->precision == BA_PREC_MIXED && !want_schur && o->pcg_kernel == 3 && p->L.tn_grid > 0;
    if (want_persistent != p->use_persistent || want_schur != p->use_schur || want_cg != p->use_cg ||
        (want_persistent && want_form != p->p_form)) {
        release_graph(p);   // cached graphs were built for the other PCG form
        p->use_persistent = want_persistent;
        p->use_schur = want_schur;
        p->use_cg = want_cg;
        if (want_persistent) p->p_form = want_form;
    }
    // A cooperative kernel cannot sit inside a conditional node, so with the persistent
    // PCG kernel the default graph is the fixed LM sequence (six kernels per LM step).
    const int graph_mode = (o->use_graph == 1 && p->use_persistent) ? 2 : o->use_graph;
    if (graph_mode == 2) {
        // the predicated sequence (every PCG and LM slot launched, idle ones return
        // at once) captured into one plain graph; rebuilt when the caps change
        if (!p->graph_unrolled.exec || p->unrolled_lm != o->max_lm_iters || p->unrolled_pcg != o->max_pcg_iters) {
            if (p->graph_unrolled.exec) cudaGraphExecDestroy(p->graph_unrolled.exec);
            if (p->graph_unrolled.graph) cudaGraphDestroy(p->graph_unrolled.graph);
            p->graph_unrolled = GraphCache{};
            cudaStream_t cs = p->cap[0];
            GBBA_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
            enqueue_solve_predicated(p, *o, cs);
            cudaGraph_t g;
            GBBA_CUDA(cudaStreamEndCapture(cs, &g));
            cudaGraphExec_t ex;
            cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_status(e, "cudaGraphInstantiate (unrolled)");
            }
            p->graph_unrolled.graph = g;
            p->graph_unrolled.exec = ex;
            p->unrolled_lm = o->max_lm_iters;
            p->unrolled_pcg = o->max_pcg_iters;
        }
        GBBA_CUDA(cudaGraphLaunch(p->graph_unrolled.exec, p->stream));
    } else if (graph_mode == 1) {
        if (!p->graph.exec && (st = build_graph_loops(p))) return st;
        GBBA_CUDA(cudaGraphLaunch(p->graph.exec, p->stream));
    } else {
        enqueue_solve_predicated(p, *o, p->stream);
        GBBA_CUDA(cudaGetLastError());
    }
    p->linearized = true;
    if (!stats) return BA_OK;
    return ba_get_stats(p, stats, hist, cap);
}

ba_status ba_apply_normal(ba_problem* p, double mu, const void* vin, void* out, double* vAv) {
    ba_status st = check_bound(p, "ba_apply_normal");
    if (st) return st;
    if (!vin || !out || !(mu >= 0)) {
        set_error("ba_apply_normal: null vector or negative mu");
        return BA_ERR_INVALID_ARG;
    }
    if (!p->linearized) {
        set_error("ba_apply_normal: call ba_evaluate first");
        return BA_ERR_STATE;
    }
    cudaStream_t s = p->stream;
    // state: mu, an active LM iteration so the preconditioner kernel runs
    DevState* dst = dev_state(p);
    GBBA_CUDA(cudaMemcpyAsync(&dst->mu, &mu, sizeof(double), cudaMemcpyHostToDevice, s));
    int32_t one = 1;
    GBBA_CUDA(cudaMemcpyAsync(&dst->lm_active, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (p->precision == BA_PREC_MIXED) {
        const Views<float>& v = p->vf;
        launch_precond(v, p->L, s, 0, 0, nullptr);
        launch_set_direction(v, p->L, s, (const float*)vin);
        launch_matvec(v, p->L, s, nullptr, v.p, 0);
        launch_normal_out(v, p->L, s, (float*)out);
        GBBA_CUDA(cudaGetLastError());
        double acc[NSLOT * SLOT_STRIDE];
        GBBA_CUDA(cudaMemcpyAsync(acc, dst->acc_mv, sizeof(acc), cudaMemcpyDeviceToHost, s));
        GBBA_CUDA(cudaMemsetAsync(dst->acc_mv, 0, sizeof(acc), s));
        GBBA_CUDA(cudaStreamSynchronize(s));
        double jp2 = 0, pdp = 0;
        for (int k = 0; k < NSLOT; ++k) {
            jp2 += acc[k * SLOT_STRIDE];
            pdp += acc[k * SLOT_STRIDE + 1];
        }
        if (vAv) *vAv = jp2 + mu * pdp;
    } else {
        const Views<double>& v = p->vd;
        launch64_precond(v, p->L, s, 0, 0);
        launch64_set_vec(v, p->L, s, (const double*)vin, v.z);   // the given vector as zs
        launch64_direction(v, p->L, s, v.z, 0, nullptr);          // p = v, q = mu D p
        launch64_matvec(v, p->L, s, nullptr);                     // q += J^T J p
        launch64_get_vec(v, p->L, s, v.q, (double*)out);
        GBBA_CUDA(cudaGetLastError());
        double jp2 = 0, pdp = 0;
        GBBA_CUDA(cudaMemcpyAsync(&jp2, &dst->jp2, sizeof(double), cudaMemcpyDeviceToHost, s));
        GBBA_CUDA(cudaMemcpyAsync(&pdp, &dst->pDp, sizeof(double), cudaMemcpyDeviceToHost, s));
        GBBA_CUDA(cudaStreamSynchronize(s));
        if (vAv) *vAv = jp2 + mu * pdp;
    }
    return BA_OK;
}

ba_status ba_repeat_normal(ba_problem* p, int32_t launches) {
    ba_status st = check_bound(p, "ba_repeat_normal");
    if (st) return st;
    if (launches < 0) {
        set_error("ba_repeat_normal: negative count");
        return BA_ERR_INVALID_ARG;
    }
    if (!p->linearized) {
        set_error("ba_repeat_normal: call ba_apply_normal first");
        return BA_ERR_STATE;
    }
    if (p->precision == BA_PREC_MIXED) {
        for (int i = 0; i < launches; ++i) launch_matvec(p->vf, p->L, p->stream, nullptr, p->vf.p, 0);
        GBBA_CUDA(cudaMemsetAsync(p->vf.st->acc_mv, 0, NSLOT * SLOT_STRIDE * sizeof(double), p->stream));
    } else {
        for (int i = 0; i < launches; ++i) launch64_matvec(p->vd, p->L, p->stream, nullptr);
    }
    GBBA_CUDA(cudaGetLastError());
    return BA_OK;
}

ba_status ba_profile_kernels(ba_problem* p, int32_t reps, double* us, int32_t n) {
    ba_status st = check_bound(p, "ba_profile_kernels");
    if (st) return st;
    if (reps < 1 || !us || n < 1) {
        set_error("ba_profile_kernels: reps >= 1 and an output array are required");
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision != BA_PREC_MIXED) {
        set_error("ba_profile_kernels: FP64 form not built yet");
        return BA_ERR_NOT_IMPLEMENTED;
    }
    if (!p->linearized) {
        set_error("ba_profile_kernels: call ba_evaluate or ba_solve first");
        return BA_ERR_STATE;
    }
    const Views<float>& v = p->vf;
    cudaStream_t s = p->stream;
    // keep every gate open: huge PCG cap, zero tolerance, active flags set
    DevOptions o{};
    o.max_lm = 1 << 30;
    o.max_pcg = 1 << 30;
    o.tol = 0.0;
    o.mu0 = 0.01;
    o.min_diag = 1e-6;
    o.max_diag = 1e32;
    o.max_mu = 1e300;
    o.eps = 0.0;
    o.wait_ns = 2000000000LL;
    o.res_df = 1;
    GBBA_CUDA(cudaMemcpyAsync(p->ws + p->lay.state, &o, sizeof(o), cudaMemcpyHostToDevice, s));
    const int32_t flags[4] = {1, 1, 1, 1};
    auto open_gates = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(&v.st->lm_active, &flags[0], 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&v.st->accepted, &flags[1], 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&v.st->relin, &flags[2], 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&v.st->pcg_active, &flags[3], 4, cudaMemcpyHostToDevice, s);
        return e;
    };
    cudaEvent_t e0, e1;
    GBBA_CUDA(cudaEventCreate(&e0));
    GBBA_CUDA(cudaEventCreate(&e1));
    // each launch timed alone, its gates opened just before it (a kernel that closes a
    // gate, e.g. the LM decision, would otherwise leave the next launches idle); the
    // first launch warms up
    auto timeit = [&](auto&& launch) -> double {
        double total = 0.0;
        for (int i = 0; i <= reps; ++i) {
            open_gates();
            cudaEventRecord(e0, s);
            launch();
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) total += ms;
        }
        return 1e3 * total / reps;
    };
    // the persistent PCG kernel first, while the state is the caller's linearisation:
    // one launch = one PCG solve (50 iterations, zero tolerance), timed alone after a
    // preconditioner launch that resets its state
    double out_pcg[2] = {-1.0, 0.0};
    if (p->persistent) {
        o.max_pcg = 50;
        GBBA_CUDA(cudaMemcpyAsync(p->ws + p->lay.state, &o, sizeof(o), cudaMemcpyHostToDevice, s));
        launch_init_state(v.st, s);
        open_gates();
        launch_camera_precompute(v, p->L, s);
        launch_residual(v, p->L, s, 0);
        launch_linearize(v, p->L, s, 0, nullptr, nullptr, 0, 0);
        double total_ms = 0.0;
        for (int i = 0; i <= reps; ++i) {
            open_gates();
            launch_precond(v, p->L, s, 0, 0, p->pslots);
            cudaEventRecord(e0, s);
            GBBA_CUDA(launch_pcg_persistent(v, p->blk_tile, p->blk_cam_off, p->blk_cams, p->pslots, p->p_grid,
                                            p->p_form == PCG_TWO_EXCHANGE ? p->p_smem_two : p->p_smem_one,
                                            p->p_form, s));
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) total_ms += ms;   // the first launch warms up
        }
        int32_t iters = 0;
        GBBA_CUDA(cudaMemcpy(&iters, &v.st->pcg_iter, 4, cudaMemcpyDeviceToHost));
        out_pcg[0] = 1e3 * total_ms / reps;
        out_pcg[1] = iters;
        o.max_pcg = 1 << 30;
        GBBA_CUDA(cudaMemcpyAsync(p->ws + p->lay.state, &o, sizeof(o), cudaMemcpyHostToDevice, s));
    }
    double out[8];
    out[0] = timeit([&] { launch_camera_precompute(v, p->L, s); });
    out[1] = timeit([&] { launch_linearize(v, p->L, s, 1, nullptr, nullptr, 0, 0); });
    out[2] = timeit([&] { launch_precond(v, p->L, s, 0, 0, nullptr); });
    out[3] = timeit([&] { launch_matvec(v, p->L, s, nullptr, v.z, 1); });
    {
        // the update skips its work once the operator sums it consumes are cleared, so
        // each timed launch follows a re-armed |J p|^2 slot and is timed alone
        const double one = 1.0;
        double total = 0.0;
        for (int i = 0; i <= reps; ++i) {
            open_gates();
            GBBA_CUDA(cudaMemcpyAsync(&v.st->acc_mv[0], &one, sizeof(double), cudaMemcpyHostToDevice, s));
            cudaEventRecord(e0, s);
            launch_update(v, p->L, s, 0, 0);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) total += ms;
        }
        out[4] = 1e3 * total / reps;
    }
    // one round of the one-reduction PCG past its first (so the update is applied),
    // before the candidate kernels overwrite the direction records it reads
    double out_cg = -1.0;
    if (p->L.tn_grid > 0) {
        const int32_t it1 = 1;
        const double ab[2] = {1e-6, 0.5};   // alpha, beta (adjacent in the state)
        double total = 0.0;
        for (int i = 0; i <= reps; ++i) {
            open_gates();
            GBBA_CUDA(cudaMemcpyAsync(&v.st->pcg_iter, &it1, 4, cudaMemcpyHostToDevice, s));
            GBBA_CUDA(cudaMemcpyAsync(&v.st->alpha, ab, sizeof(ab), cudaMemcpyHostToDevice, s));
            cudaEventRecord(e0, s);
            launch_cg_round(v, p->L, s, nullptr, 0, 0);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (i > 0) total += ms;
        }
        out_cg = 1e3 * total / reps;
    }
    const double out_res = timeit([&] { launch_residual(v, p->L, s, 0); });
    out[5] = timeit([&] { launch_candidate(v, p->L, s); });
    out[6] = timeit([&] { launch_eval_candidate(v, p->L, s, 0, 0); });
    out[7] = timeit([&] { launch_commit(v, p->L, s); });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GBBA_CUDA(cudaGetLastError());
    for (int i = 0; i < n && i < 8; ++i) us[i] = out[i];
    for (int i = 8; i < n && i < 10; ++i) us[i] = out_pcg[i - 8];
    if (n > 10) us[10] = out_cg;
    if (n > 11) us[11] = out_res;
    // restore the default options; the solver state is re-initialised by the next solve
    ba_options d;
    ba_options_default(&d);
    p->linearized = false;
    return write_options(p, &d);
}

// ---- autograd entries: the cost and its adjoint J^T r at caller-given parameters ---

ba_status ba_cost_forward(ba_problem* p, const void* cams, const void* pts, int32_t dtype, double* cost_dev) {
    ba_status st = check_bound(p, "ba_cost_forward");
    if (st) return st;
    if (!cams || !pts || !cost_dev || (dtype != 0 && dtype != 1)) {
        set_error("ba_cost_forward: null pointer or bad dtype %d", dtype);
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision == BA_PREC_MIXED) launch_cost_grad(p->vf, p->L, p->stream, cams, pts, dtype, 0, cost_dev);
    else launch64_cost_grad(p->vd, p->L, p->stream, cams, pts, dtype, 0, cost_dev);
    GBBA_CUDA(cudaGetLastError());
    p->linearized = false;   // the camera gradient buffer was cleared as scratch
    return BA_OK;
}

ba_status ba_cost_backward(ba_problem* p, const void* cams, const void* pts, int32_t dtype, const double* grad_out,
                           void* grad_cams, void* grad_pts) {
    ba_status st = check_bound(p, "ba_cost_backward");
    if (st) return st;
    if (!cams || !pts || !grad_out || !grad_cams || !grad_pts || (dtype != 0 && dtype != 1)) {
        set_error("ba_cost_backward: null pointer or bad dtype %d", dtype);
        return BA_ERR_INVALID_ARG;
    }
    if (p->precision == BA_PREC_MIXED) {
        launch_cost_grad(p->vf, p->L, p->stream, cams, pts, dtype, 1, nullptr);
        launch_grad_out(p->vf, p->L, p->stream, grad_out, grad_cams, grad_pts, dtype);
    } else {
        launch64_cost_grad(p->vd, p->L, p->stream, cams, pts, dtype, 1, nullptr);
        launch64_grad_out(p->vd, p->L, p->stream, grad_out, grad_cams, grad_pts, dtype);
    }
    GBBA_CUDA(cudaGetLastError());
    p->linearized = false;   // the gradient buffers of the linearisation were used as scratch
    return BA_OK;
}

}  // extern "C"
