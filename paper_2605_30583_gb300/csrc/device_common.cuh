// Device-side building blocks shared by the kernels of libgbba.
//
// Camera model: Snavely reprojection factor, Sec. VI-A of arXiv 2605.30583.
// Jacobian: closed form derived by hand (Sec. V asks for the Jacobian of each
// factor with respect to its tunable nodes); the derivation is in the comments of
// proj_jacobian below.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace gbba {

// ------------------------------------------------------------------ reductions ---

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, in a fixed order; valid in thread 0.  `sh` holds at
// least blockDim.x / 32 doubles.  Contains __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += sh[i];
    }
    return s;
}

// Grid-wide reduction of NV doubles with a deterministic result: every block writes
// its partial sums to partials[block * NV + k]; the last block to finish sums the
// partials in block order and returns true (the totals are then in out[0..NV) of
// thread 0).  ticket is reset by the last block so the next launch can reuse it.
template <int NV>
__device__ __forceinline__ bool grid_reduce(const double (&v)[NV], double* partials,
                                            unsigned int* ticket, double (&out)[NV]) {
    __shared__ double sh[32];
    __shared__ bool is_last;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = block_sum(v[k], sh);
        if (threadIdx.x == 0) partials[blockIdx.x * NV + k] = s;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            s += __ldcg(&partials[b * NV + k]);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) out[k] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// Slot-spread accumulation: block b adds into slot b % NSLOT.
__device__ __forceinline__ void slot_add(double* base, int k, double v) {
    atomicAdd(&base[(blockIdx.x % NSLOT) * SLOT_STRIDE + k], v);
}

// Sum over the NSLOT slots of component k; call with a full warp, result in every lane.
__device__ __forceinline__ double slot_sum_warp(const double* base, int k) {
    double v = __ldcg(&base[(threadIdx.x & 31) * SLOT_STRIDE + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1/x in FP64: hardware approximation refined by two Newton-Raphson steps
// y <- y + y (1 - x y), each roughly doubling the correct bits.  Zero, non-finite and
// |x| outside [1e-300, 1e300] (where x y or the approximation could leave the normal
// range, flushing or overflowing before the refinement) take the IEEE quotient.
__device__ __forceinline__ double rcp64(double x) {
    const double ax = fabs(x);
    if (!(ax >= 1e-300 && ax <= 1e300)) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    y = fma(y, fma(-x, y, 1.0), y);
    return y;
}

// Kahan's compensated summation (W. Kahan, "Further remarks on reducing truncation
// errors", CACM 8(1), 1965) of FP32 terms: s - c is the running sum, c the negated
// low-order part lost so far.  Per-thread partials of the FP64 reductions use it, so a
// thread's FP32 sum over many terms keeps the accuracy of its largest term's rounding.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Knuth's TwoSum: s + e == a + b exactly (s = fl(a + b)).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp sum of per-lane compensated values hi + lo in FP32 pairs: every level adds the
// partner's high parts with TwoSum and carries the rounding error into the low parts,
// so the result has about twice FP32's precision (FP64 shuffles cost ~67x more on this
// GPU).  Result valid in lane 0 as a double.
__device__ __forceinline__ double warp_sum_pair(float hi, float lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo = lo + l2 + e;
    }
    return (double)hi + (double)lo;
}

// Block sums of two compensated per-thread partials (Kahan pairs s - c): compensated
// FP32 pairs inside each warp, FP64 across warps.  Results valid in thread 0.  `sh`
// holds 2 * (blockDim.x / 32) doubles.  Contains __syncthreads.
__device__ __forceinline__ void block_sum2c(float sa, float ca, float sb, float cb, double* sh, double& ra,
                                            double& rb) {
    const double a = warp_sum_pair(sa, -ca), b = warp_sum_pair(sb, -cb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[w] = a;
        sh[nw + w] = b;
    }
    __syncthreads();
    ra = rb = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < nw; ++i) {
            ra += sh[i];
            rb += sh[nw + i];
        }
    }
}

// Block sums of two FP32 per-thread partials: FP32 inside each warp (32 terms), FP64
// across warps.  Results valid in thread 0.  `sh` holds 2 * (blockDim.x / 32) doubles.
__device__ __forceinline__ void block_sum2(float a, float b, double* sh, double& ra, double& rb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[w] = (double)a;
        sh[nw + w] = (double)b;
    }
    __syncthreads();
    ra = rb = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < nw; ++i) {
            ra += sh[i];
            rb += sh[nw + i];
        }
    }
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ camera precompute ---

// Rodrigues coefficients A = sin(th)/th, B = (1 - cos th)/th^2 and the left-Jacobian
// coefficient C = (th - sin th)/th^3, evaluated in FP64.  For th^2 < 1e-4 the Taylor
// series to th^6 are used (no cancellation; truncation below 1e-16 there).
__device__ __forceinline__ void rodrigues_coeffs(double th2, double& A, double& B, double& C) {
    if (th2 < 1e-4) {
        A = 1.0 + th2 * (-1.0 / 6.0 + th2 * (1.0 / 120.0 + th2 * (-1.0 / 5040.0)));
        B = 0.5 + th2 * (-1.0 / 24.0 + th2 * (1.0 / 720.0 + th2 * (-1.0 / 40320.0)));
        C = 1.0 / 6.0 + th2 * (-1.0 / 120.0 + th2 * (1.0 / 5040.0 + th2 * (-1.0 / 362880.0)));
    } else {
        const double th = sqrt(th2);
        double s, c, sh, ch;
        sincos(th, &s, &c);
        sincos(0.5 * th, &sh, &ch);
        A = s / th;
        B = 2.0 * sh * sh / th2;
        C = (th - s) / (th2 * th);
    }
}

// Writes one camera record (layout.h, CamPre) from 9 parameters (w, t, f, k1, k2):
// R(w) = I + A [w]x + B [w]x^2 and J_l(w) = I + B [w]x + C [w]x^2, where J_l is the
// left Jacobian of the rotation exponential: R(w + d) = Exp(J_l(w) d) R(w) + O(|d|^2),
// so d(R(w) X)/dw . d = (J_l d) x (R X).
// With `retract` the record is for the tangent-space update R <- Exp(d) R(w): the
// rotation Jacobian is then taken w.r.t. d at d = 0, i.e. J_l is replaced by I.
// `lo` (optional, CLO_STRIDE floats): the FP32 rounding error of R, t, f, k1, k2 at the
// same offsets as in `out`, so out + lo carries them to ~2^-48 (double-float values).
__device__ __forceinline__ void camera_record(const double* c, float* out, bool retract = false,
                                              float* lo = nullptr) {
    const double w0 = c[0], w1 = c[1], w2 = c[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, C;
    rodrigues_coeffs(th2, A, B, C);
    // [w]x and [w]x^2 = w w^T - th2 I
    const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    const double K2[9] = {w0 * w0 - th2, w0 * w1, w0 * w2,
                          w1 * w0, w1 * w1 - th2, w1 * w2,
                          w2 * w0, w2 * w1, w2 * w2 - th2};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        out[CP_R + i] = (float)(I + A * K[i] + B * K2[i]);
        out[CP_JL + i] = retract ? (float)I : (float)(I + B * K[i] + C * K2[i]);
    }
    out[CP_T + 0] = (float)c[3];
    out[CP_T + 1] = (float)c[4];
    out[CP_T + 2] = (float)c[5];
    out[CP_F] = (float)c[6];
    out[CP_K1] = (float)c[7];
    out[CP_K2] = (float)c[8];
    out[CP_PAD] = 0.0f;
    if (lo) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double I = (i % 4 == 0) ? 1.0 : 0.0;
            const double r = I + A * K[i] + B * K2[i];
            lo[CP_R + i] = (float)(r - (double)(float)r);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) lo[CP_T + i] = (float)(c[3 + i] - (double)(float)c[3 + i]);
        lo[CP_PAD] = 0.0f;
    }
}

// Unit quaternion (q0; q1 q2 q3) of the rotation vector v: (cos(t/2); sin(t/2) v / t),
// t = |v|, with the Taylor series of both factors for t^2 < 1e-12.
__device__ __forceinline__ void rotvec_quat(const double* v, double* q) {
    const double t2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double c, s_over_t;
    if (t2 < 1e-12) {
        c = 1.0 - t2 / 8.0 + t2 * t2 / 384.0;
        s_over_t = 0.5 - t2 / 48.0 + t2 * t2 / 3840.0;
    } else {
        const double t = sqrt(t2);
        double sn;
        sincos(0.5 * t, &sn, &c);
        s_over_t = sn / t;
    }
    q[0] = c;
    q[1] = s_over_t * v[0];
    q[2] = s_over_t * v[1];
    q[3] = s_over_t * v[2];
}

// Rotation vector of Exp(h) Exp(w) (the retraction of a tangent step h at w), through
// the Hamilton product of unit quaternions q(h) q(w), taken with q0 >= 0, and
// w' = 2 atan2(|q_v|, q0) q_v / |q_v| (series 2 / q0 (1 - |q_v|^2 / (3 q0^2)) when
// |q_v| < 1e-7).  FP64.
__device__ __forceinline__ void compose_rotvec(const double* h, const double* w, double* out) {
    double a[4], b[4];
    rotvec_quat(h, a);
    rotvec_quat(w, b);
    double q0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double q1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double q2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double q3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    if (q0 < 0.0) {
        q0 = -q0; q1 = -q1; q2 = -q2; q3 = -q3;
    }
    const double n = sqrt(q1 * q1 + q2 * q2 + q3 * q3);
    const double scale = n > 1e-7 ? 2.0 * atan2(n, q0) / n : (2.0 / q0) * (1.0 - n * n / (3.0 * q0 * q0));
    out[0] = scale * q1;
    out[1] = scale * q2;
    out[2] = scale * q3;
}

// Robust loss on s = |r|^2 of one observation (0 squared, 1 Huber, 2 Cauchy; scale d):
// rho(s) and the IRLS weight rho'(s).
//   Huber:  rho = s (s <= d^2), 2 d sqrt(s) - d^2;   rho' = 1, d / sqrt(s)
//   Cauchy: rho = d^2 log(1 + s / d^2);              rho' = 1 / (1 + s / d^2)
__device__ __forceinline__ float loss_weight(float s, int loss, float d) {
    if (loss == 1) return s <= d * d ? 1.0f : d * rsqrtf(s);
    if (loss == 2) return 1.0f / (1.0f + s / (d * d));
    return 1.0f;
}

__device__ __forceinline__ float loss_rho(float s, int loss, float d) {
    if (loss == 1) return s <= d * d ? s : 2.0f * d * sqrtf(s) - d * d;
    if (loss == 2) return d * d * log1pf(s / (d * d));
    return s;
}

__device__ __forceinline__ double loss_weight64(double s, int loss, double d) {
    if (loss == 1) return s <= d * d ? 1.0 : d / sqrt(s);
    if (loss == 2) return 1.0 / (1.0 + s / (d * d));
    return 1.0;
}

__device__ __forceinline__ double loss_rho64(double s, int loss, double d) {
    if (loss == 1) return s <= d * d ? s : 2.0 * d * sqrt(s) - d * d;
    if (loss == 2) return d * d * log1p(s / (d * d));
    return s;
}

// ------------------------------------------------------------- projection core ---

struct Cam {
    float R[9], t[3], f, k1, k2;
};

__device__ __forceinline__ Cam load_cam(const float* __restrict__ rec) {
    const float4* r4 = reinterpret_cast<const float4*>(rec);
    const float4 a = __ldg(r4 + 0), b = __ldg(r4 + 1), c = __ldg(r4 + 2), d = __ldg(r4 + 3);
    Cam m;
    m.R[0] = a.x; m.R[1] = a.y; m.R[2] = a.z; m.R[3] = a.w;
    m.R[4] = b.x; m.R[5] = b.y; m.R[6] = b.z; m.R[7] = b.w;
    m.R[8] = c.x; m.t[0] = c.y; m.t[1] = c.z; m.t[2] = c.w;
    m.f = d.x; m.k1 = d.y; m.k2 = d.z;
    return m;
}

// Geometry of one observation: RX = R X, P = RX + t, iz = 1/d_safe, normalised point
// p, |p|^2, radial scale s = 1 + k1 |p|^2 + k2 |p|^4, and A = d(pixel)/dP (2x3).
//
// pixel = f s(n2) p with p = -P.xy / d_safe, n2 = |p|^2.
//   d(pixel)/dp = f (s I + 2 s' p p^T),  s' = k1 + 2 k2 n2            (2x2, symmetric M)
//   dp/dP       = -iz [[1, 0, px], [0, 1, py]]   (d_safe shifts P.z by a constant)
//   A = M dp/dP = -iz [M col0, M col1, px M col0 + py M col1]
struct Geo {
    float RX[3];
    float p[2];
    float n2, s;
    float A[6];   // row-major 2x3
};

__device__ __forceinline__ Geo project_geo(const Cam& c, float X0, float X1, float X2, float eps) {
    Geo g;
    g.RX[0] = fmaf(c.R[0], X0, fmaf(c.R[1], X1, c.R[2] * X2));
    g.RX[1] = fmaf(c.R[3], X0, fmaf(c.R[4], X1, c.R[5] * X2));
    g.RX[2] = fmaf(c.R[6], X0, fmaf(c.R[7], X1, c.R[8] * X2));
    const float P0 = g.RX[0] + c.t[0];
    const float P1 = g.RX[1] + c.t[1];
    const float P2 = g.RX[2] + c.t[2];
    const float d = P2 + (P2 >= 0.0f ? eps : -eps);
    const float iz = __frcp_rn(d);
    g.p[0] = -P0 * iz;
    g.p[1] = -P1 * iz;
    g.n2 = fmaf(g.p[0], g.p[0], g.p[1] * g.p[1]);
    const float sp = fmaf(2.0f * c.k2, g.n2, c.k1);         // s'
    g.s = fmaf(g.n2, fmaf(c.k2, g.n2, c.k1), 1.0f);
    const float a = c.f * g.s;
    const float b = 2.0f * c.f * sp;
    const float m00 = fmaf(b * g.p[0], g.p[0], a);
    const float m01 = b * g.p[0] * g.p[1];
    const float m11 = fmaf(b * g.p[1], g.p[1], a);
    const float niz = -iz;
    g.A[0] = niz * m00;
    g.A[1] = niz * m01;
    g.A[2] = niz * fmaf(m00, g.p[0], m01 * g.p[1]);
    g.A[3] = niz * m01;
    g.A[4] = niz * m11;
    g.A[5] = niz * fmaf(m01, g.p[0], m11 * g.p[1]);
    return g;
}

// Inverse of one camera block, one warp per camera: lane j < 18 holds column j of
// the augmented matrix [A | I] (A = H + mu D, 9 x 9, SPD) and Gauss-Jordan elimination
// without pivoting runs over the 9 pivots in FP64.  Lanes 9..17 end with the columns
// of A^-1.  Returns false (in every lane) if a pivot is not positive.
__device__ __forceinline__ bool warp_block_inverse9(double (&col)[9], int lane) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double piv = __shfl_sync(0xffffffffu, col[k], k);
        ok = ok && (piv > 0.0) && isfinite(piv);
        const double ip = rcp64(piv > 0.0 ? piv : 1.0);
        const double rk = col[k] * ip;   // row k of the updated matrix, this lane's column
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double aik = __shfl_sync(0xffffffffu, col[i], k);
            if (i != k) col[i] = fma(-aik, rk, col[i]);
        }
        col[k] = rk;
    }
    (void)lane;
    return ok;
}

// Levenberg-Marquardt decision after a candidate evaluation (Sec. V, Madsen's
// quality-based damping).  Fn = F(x + h), jh2 = |J h|^2, st->gh = g^T h.
// L = -g^T h - 1/2 |J h|^2, rho = (F - Fn) / L; the step is accepted iff Fn is finite,
// L > 0 and rho > 0; then mu <- mu max(1/3, 1 - (2 rho - 1)^3), nu <- 2, else
// mu <- mu nu, nu <- 2 nu.  Records the iteration and sets the loop flags.  One thread.
__device__ __forceinline__ void lm_decide(DevState* st, int active, double Fn, double jh2) {
    if (!active) {
        st->accepted = 0;
        st->relin = 0;
        return;
    }
    const double L = -st->gh - 0.5 * jh2;
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
    st->jh2 = jh2;
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
    const bool more = st->lm_iter < st->opt.max_lm && st->mu <= st->opt.max_mu && st->F > 0.0 && st->status == 0;
    st->lm_active = more ? 1 : 0;
    st->relin = (acc && more) ? 1 : 0;
}

// 1/x to within 1 ulp (the hardware reciprocal approximation, denormals flushed).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Geometry of one observation without the explicit 2x3 A: J d and J^T t are applied
// in factored form (see apply_A / apply_At).
struct GeoLite {
    float RX[3];
    float p[2];
    float n2, s, iz, a, b;   // a = f s, b = 2 f s'
};

__device__ __forceinline__ GeoLite project_lite(const Cam& c, float X0, float X1, float X2, float eps) {
    GeoLite g;
    g.RX[0] = fmaf(c.R[0], X0, fmaf(c.R[1], X1, c.R[2] * X2));
    g.RX[1] = fmaf(c.R[3], X0, fmaf(c.R[4], X1, c.R[5] * X2));
    g.RX[2] = fmaf(c.R[6], X0, fmaf(c.R[7], X1, c.R[8] * X2));
    const float P2 = g.RX[2] + c.t[2];
    const float d = P2 + (P2 >= 0.0f ? eps : -eps);
    g.iz = rcp_approx(d);
    g.p[0] = -(g.RX[0] + c.t[0]) * g.iz;
    g.p[1] = -(g.RX[1] + c.t[1]) * g.iz;
    g.n2 = fmaf(g.p[0], g.p[0], g.p[1] * g.p[1]);
    g.s = fmaf(g.n2, fmaf(c.k2, g.n2, c.k1), 1.0f);
    g.a = c.f * g.s;
    g.b = 2.0f * c.f * fmaf(2.0f * c.k2, g.n2, c.k1);
    return g;
}

// A dP with A = M dp/dP, M = a I + b p p^T, dp/dP = -iz [[1, 0, px], [0, 1, py]].
__device__ __forceinline__ void apply_A(const GeoLite& g, float d0, float d1, float d2, float& t0, float& t1) {
    const float e0 = -g.iz * fmaf(g.p[0], d2, d0);
    const float e1 = -g.iz * fmaf(g.p[1], d2, d1);
    const float pe = g.b * fmaf(g.p[0], e0, g.p[1] * e1);
    t0 = fmaf(g.a, e0, pe * g.p[0]);
    t1 = fmaf(g.a, e1, pe * g.p[1]);
}

// A^T t (M symmetric).
__device__ __forceinline__ void apply_At(const GeoLite& g, float t0, float t1, float& u0, float& u1, float& u2) {
    const float pt = g.b * fmaf(g.p[0], t0, g.p[1] * t1);
    const float w0 = -g.iz * fmaf(g.a, t0, pt * g.p[0]);
    const float w1 = -g.iz * fmaf(g.a, t1, pt * g.p[1]);
    u0 = w0;
    u1 = w1;
    u2 = fmaf(g.p[0], w0, g.p[1] * w1);
}

// Residual only (no Jacobian): f s p - u.
__device__ __forceinline__ void project_residual(const Cam& c, float X0, float X1, float X2, float eps,
                                                 float u0, float u1, float& r0, float& r1) {
    const float P0 = fmaf(c.R[0], X0, fmaf(c.R[1], X1, c.R[2] * X2)) + c.t[0];
    const float P1 = fmaf(c.R[3], X0, fmaf(c.R[4], X1, c.R[5] * X2)) + c.t[1];
    const float P2 = fmaf(c.R[6], X0, fmaf(c.R[7], X1, c.R[8] * X2)) + c.t[2];
    const float d = P2 + (P2 >= 0.0f ? eps : -eps);
    const float iz = __frcp_rn(d);
    const float p0 = -P0 * iz, p1 = -P1 * iz;
    const float n2 = fmaf(p0, p0, p1 * p1);
    const float s = fmaf(n2, fmaf(c.k2, n2, c.k1), 1.0f);
    const float fs = c.f * s;
    r0 = fmaf(fs, p0, -u0);
    r1 = fmaf(fs, p1, -u1);
}

}  // namespace gbba
