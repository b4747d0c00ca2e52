// Plain all-FP64 form of the LM + PCGNR solver (the comparison baseline): the same
// algorithm as the mixed-precision path (Sec. V of arXiv 2605.30583) written the
// straightforward way -- FP64 everywhere, the Jacobian computed once per
// linearisation and stored (24 doubles per observation), and one FP64 global atomic
// per camera entry and observation for every camera-side sum.  Points are owned by
// one thread each (the point-major index), so point sums need no atomics.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"

namespace gbba {

using V64 = Views<double>;

namespace {

// Camera record in FP64, same field order as the FP32 record (CP_*).
// With `retract` the rotation Jacobian is taken w.r.t. the tangent step d of
// R <- Exp(d) R(w) at d = 0: J_l is replaced by I.
__device__ void camera_record64(const double* c, double* out, bool retract = false) {
    const double w0 = c[0], w1 = c[1], w2 = c[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, C;
    rodrigues_coeffs(th2, A, B, C);
    const double K[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    const double K2[9] = {w0 * w0 - th2, w0 * w1, w0 * w2, w1 * w0, w1 * w1 - th2, w1 * w2,
                          w2 * w0, w2 * w1, w2 * w2 - th2};
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        out[CP_R + i] = I + A * K[i] + B * K2[i];
        out[CP_JL + i] = retract ? I : I + B * K[i] + C * K2[i];
    }
    for (int k = 0; k < 3; ++k) out[CP_T + k] = c[3 + k];
    out[CP_F] = c[6];
    out[CP_K1] = c[7];
    out[CP_K2] = c[8];
    out[CP_PAD] = 0.0;
}

// Residual and the 2x12 Jacobian (camera 9 columns, point 3) of one observation.
__device__ void obs_jacobian64(const double* cam, double X0, double X1, double X2, double eps, double u0,
                               double u1, double& r0, double& r1, double* J /* [2][12] */) {
    const double* R = cam + CP_R;
    const double* JL = cam + CP_JL;
    const double RX0 = R[0] * X0 + R[1] * X1 + R[2] * X2;
    const double RX1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
    const double RX2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
    const double P0 = RX0 + cam[CP_T], P1 = RX1 + cam[CP_T + 1], P2 = RX2 + cam[CP_T + 2];
    const double d = P2 + (P2 >= 0.0 ? eps : -eps);
    const double iz = 1.0 / d;
    const double p0 = -P0 * iz, p1 = -P1 * iz;
    const double n2 = p0 * p0 + p1 * p1;
    const double f = cam[CP_F], k1 = cam[CP_K1], k2 = cam[CP_K2];
    const double s = 1.0 + n2 * (k1 + k2 * n2);
    const double sp = k1 + 2.0 * k2 * n2;
    r0 = f * s * p0 - u0;
    r1 = f * s * p1 - u1;
    if (!J) return;
    // A = d(pixel)/dP = M dp/dP, M = f (s I + 2 s' p p^T), dp/dP = -iz [[1,0,p0],[0,1,p1]]
    const double a = f * s, b = 2.0 * f * sp;
    const double m00 = a + b * p0 * p0, m01 = b * p0 * p1, m11 = a + b * p1 * p1;
    const double A0 = -iz * m00, A1 = -iz * m01, A2 = -iz * (m00 * p0 + m01 * p1);
    const double A3 = -iz * m01, A4 = -iz * m11, A5 = -iz * (m01 * p0 + m11 * p1);
    for (int k = 0; k < 3; ++k) {
        const double wa = JL[k], wb = JL[3 + k], wc = JL[6 + k];   // column k of J_l
        const double c0 = wb * RX2 - wc * RX1, c1 = wc * RX0 - wa * RX2, c2 = wa * RX1 - wb * RX0;
        J[k] = A0 * c0 + A1 * c1 + A2 * c2;
        J[12 + k] = A3 * c0 + A4 * c1 + A5 * c2;
    }
    J[3] = A0; J[4] = A1; J[5] = A2;
    J[15] = A3; J[16] = A4; J[17] = A5;
    J[6] = s * p0; J[7] = f * n2 * p0; J[8] = f * n2 * n2 * p0;
    J[18] = s * p1; J[19] = f * n2 * p1; J[20] = f * n2 * n2 * p1;
    for (int k = 0; k < 3; ++k) {
        J[9 + k] = A0 * R[k] + A1 * R[3 + k] + A2 * R[6 + k];
        J[21 + k] = A3 * R[k] + A4 * R[3 + k] + A5 * R[6 + k];
    }
}

__device__ __forceinline__ int grid_threads() { return gridDim.x * blockDim.x; }
__device__ __forceinline__ int gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }

}  // namespace

__global__ void k64_camera_precompute(V64 v) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads()) {
        camera_record64(v.x + 9 * (size_t)c, v.cam64 + (size_t)c * CP_STRIDE, v.st->opt.retract != 0);
        for (int k = 0; k < CL_STRIDE; ++k) v.cam_lin[(size_t)c * CL_STRIDE + k] = 0.0;
        for (int k = 0; k < CH_STRIDE; ++k) v.cam_H64[(size_t)c * CH_STRIDE + k] = 0.0;
    }
}

// Linearisation: thread per point over its observations; stores r and J per
// observation, point sums in registers, camera sums by FP64 atomics.
__global__ void k64_linearize(V64 v, int mode, double* res_out, double* jac_out, CondHandle lm_cond, int use_cond) {
    if (mode == 1 && v.st->relin == 0) return;
    const double eps = v.st->opt.eps;
    // robust loss (evaluation, mode 2, is always the squared loss)
    const int loss = mode == 2 ? 0 : v.st->opt.loss;
    const double lscale = v.st->opt.loss_scale;
    double cost = 0.0;
    for (int ip = gtid(); ip < v.n_pts; ip += grid_threads()) {
        const double* X = v.x + v.pt_off + 3 * (size_t)ip;
        double gp[3] = {0, 0, 0}, hp[6] = {0, 0, 0, 0, 0, 0};
        for (uint32_t k = v.pt_obs_off[ip]; k < v.pt_obs_off[ip + 1]; ++k) {
            const uint32_t j = v.obs_pm[k];
            const uint32_t c = v.obs_key[j] >> 8;
            double J[24], r0, r1;
            obs_jacobian64(v.cam64 + (size_t)c * CP_STRIDE, X[0], X[1], X[2], eps, v.obs_uv[2 * (size_t)j],
                           v.obs_uv[2 * (size_t)j + 1], r0, r1, J);
            if (mode == 2) {   // evaluation output: the unweighted residual and Jacobian
                const uint32_t o = v.obs_user[j];
                if (res_out) { res_out[2 * (size_t)o] = r0; res_out[2 * (size_t)o + 1] = r1; }
                if (jac_out) for (int q = 0; q < 24; ++q) jac_out[24 * (size_t)o + q] = J[q];
            }
            if (loss) {   // IRLS: the stored rows are scaled by sqrt(rho'(|r|^2))
                const double s2 = r0 * r0 + r1 * r1;
                cost += loss_rho64(s2, loss, lscale);
                const double sw = sqrt(loss_weight64(s2, loss, lscale));
                r0 *= sw;
                r1 *= sw;
                for (int q = 0; q < 24; ++q) J[q] *= sw;
            } else {
                cost += r0 * r0 + r1 * r1;
            }
            for (int q = 0; q < 24; ++q) v.jac[24 * (size_t)j + q] = J[q];
            v.res[2 * (size_t)j] = r0;
            v.res[2 * (size_t)j + 1] = r1;
            double* gc = v.cam_lin + (size_t)c * CL_STRIDE;
            double* hc = v.cam_H64 + (size_t)c * CH_STRIDE;
            for (int a = 0; a < 9; ++a) {
                atomicAdd(gc + a, J[a] * r0 + J[12 + a] * r1);
                for (int b = a; b < 9; ++b) atomicAdd(hc + tri_index(9, a, b), J[a] * J[b] + J[12 + a] * J[12 + b]);
            }
            for (int a = 0; a < 3; ++a) {
                gp[a] += J[9 + a] * r0 + J[21 + a] * r1;
                for (int b = a; b < 3; ++b) hp[tri_index(3, a, b)] += J[9 + a] * J[9 + b] + J[21 + a] * J[21 + b];
            }
        }
        for (int a = 0; a < 3; ++a) v.g[v.pt_off + 3 * (size_t)ip + a] = gp[a];
        for (int a = 0; a < 6; ++a) v.pt_H[(size_t)ip * PH_STRIDE + a] = hp[a];
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

// Block-Jacobi inverses (FP64, camera blocks by warp Gauss-Jordan, points by adjugate)
// and the PCGNR start: r = -g, z = M^-1 r, p = 0, h = 0.
__global__ void k64_precond(V64 v, CondHandle pcg_cond, int use_cond) {
    DevState* st = v.st;
    if (st->lm_active == 0) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(pcg_cond, 0u);
        return;
    }
    const double mu = st->mu, lo = st->opt.min_diag, hi = st->opt.max_diag;
    double rz = 0.0, rr = 0.0;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = gtid() >> 5; c < v.n_cams; c += warps) {
        const double* H = v.cam_H64 + (size_t)c * CH_STRIDE;
        double col[9];
        const int j = lane < 18 ? lane : 17;
        for (int i = 0; i < 9; ++i) {
            if (j < 9) {
                double h = H[tri_index(9, i < j ? i : j, i < j ? j : i)];
                if (i == j) h += mu * fmin(fmax(h, lo), hi);
                col[i] = h;
            } else {
                col[i] = (i == j - 9) ? 1.0 : 0.0;
            }
        }
        const double hdiag = lane < 9 ? H[tri_index(9, lane, lane)] : 0.0;
        const bool ok = warp_block_inverse9(col, lane);
        double* Mo = v.Minv_c + (size_t)c * MC_STRIDE;
        if (lane >= 9 && lane < 18)
            for (int i = 0; i < 9; ++i) Mo[i * 9 + (lane - 9)] = col[i];
        if (!ok && lane < 9) {
            const double dd = hdiag + mu * fmin(fmax(hdiag, lo), hi);
            for (int i = 0; i < 9; ++i) Mo[i * 9 + lane] = (i == lane && dd > 0.0) ? 1.0 / dd : 0.0;
        }
        __syncwarp();
        if (lane < 9) {
            const size_t e = 9 * (size_t)c + lane;
            v.D[e] = fmin(fmax(hdiag, lo), hi);
            const double* gc = v.cam_lin + (size_t)c * CL_STRIDE;
            const double ri = -gc[lane];
            double z = 0.0;
            for (int k = 0; k < 9; ++k) z += Mo[lane * 9 + k] * (-gc[k]);
            v.r[e] = ri;
            v.z[e] = z;
            v.p[e] = 0.0;
            v.h[e] = 0.0;
            rz += ri * z;
            rr += ri * ri;
        }
    }
    for (int i = gtid(); i < v.n_pts; i += grid_threads()) {
        const double* H = v.pt_H + (size_t)i * PH_STRIDE;
        const size_t e = v.pt_off + 3 * (size_t)i;
        double a00 = H[0], a01 = H[1], a02 = H[2], a11 = H[3], a12 = H[4], a22 = H[5];
        const double d0 = fmin(fmax(a00, lo), hi), d1 = fmin(fmax(a11, lo), hi), d2 = fmin(fmax(a22, lo), hi);
        a00 += mu * d0; a11 += mu * d1; a22 += mu * d2;
        const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
        const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
        const double det = a00 * c00 + a01 * c01 + a02 * c02;
        double m[6];
        if (det > 0.0 && isfinite(det) && a00 > 0.0 && c22 > 0.0) {
            const double id = 1.0 / det;
            m[0] = c00 * id; m[1] = c01 * id; m[2] = c02 * id; m[3] = c11 * id; m[4] = c12 * id; m[5] = c22 * id;
        } else {
            m[0] = a00 > 0 ? 1.0 / a00 : 0.0; m[1] = 0.0; m[2] = 0.0;
            m[3] = a11 > 0 ? 1.0 / a11 : 0.0; m[4] = 0.0; m[5] = a22 > 0 ? 1.0 / a22 : 0.0;
        }
        for (int k = 0; k < 6; ++k) v.Minv_p[(size_t)i * MP_STRIDE + k] = m[k];
        v.D[e] = d0; v.D[e + 1] = d1; v.D[e + 2] = d2;
        const double r0 = -v.g[e], r1 = -v.g[e + 1], r2 = -v.g[e + 2];
        const double z0 = m[0] * r0 + m[1] * r1 + m[2] * r2;
        const double z1 = m[1] * r0 + m[3] * r1 + m[4] * r2;
        const double z2 = m[2] * r0 + m[4] * r1 + m[5] * r2;
        v.r[e] = r0; v.r[e + 1] = r1; v.r[e + 2] = r2;
        v.z[e] = z0; v.z[e + 1] = z1; v.z[e + 2] = z2;
        v.p[e] = v.p[e + 1] = v.p[e + 2] = 0.0;
        v.h[e] = v.h[e + 1] = v.h[e + 2] = 0.0;
        rz += r0 * z0 + r1 * z1 + r2 * z2;
        rr += r0 * r0 + r1 * r1 + r2 * r2;
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_PRE], out) && threadIdx.x == 0) {
        st->rz = out[0];
        st->rr0 = out[1];
        st->rr = out[1];
        st->beta = 0.0;
        st->pcg_iter = 0;
        // a non-finite r^T z means a non-finite gradient or block (a Jacobian that
        // overflowed, e.g. a point at a camera centre): a numeric failure, not a stall
        if (!isfinite(out[0]) || !isfinite(out[1])) st->status = 4;
        st->pcg_active = (out[1] > 0.0 && isfinite(out[0]) && st->opt.max_pcg > 0) ? 1 : 0;
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// p = zs + beta p (beta = 0 for a given direction zs = p); q = mu D p, the start of
// the atomically accumulated normal product; p^T D p.
__global__ void k64_direction(V64 v, const double* zs, int use_beta, const int32_t* gate) {
    if (gate && *gate == 0) return;
    DevState* st = v.st;
    const double beta = use_beta ? st->beta : 0.0, mu = st->mu;
    double pdp = 0.0;
    for (size_t e = gtid(); e < (size_t)v.n_vec; e += grid_threads()) {
        const double pk = beta != 0.0 ? zs[e] + beta * v.p[e] : zs[e];
        v.p[e] = pk;
        v.q[e] = mu * v.D[e] * pk;
        pdp += v.D[e] * pk * pk;
    }
    double in[1] = {pdp}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_DIR], out) && threadIdx.x == 0) st->pDp = out[0];
}

// q += J^T J p with the stored Jacobian: thread per point, t = J_o p per observation,
// camera part by FP64 atomics, point part in registers.
__global__ void k64_matvec(V64 v, const int32_t* gate) {
    if (gate && *gate == 0) return;
    DevState* st = v.st;
    double jp2 = 0.0;
    for (int ip = gtid(); ip < v.n_pts; ip += grid_threads()) {
        const size_t ep = v.pt_off + 3 * (size_t)ip;
        const double pp0 = v.p[ep], pp1 = v.p[ep + 1], pp2 = v.p[ep + 2];
        double qp0 = 0.0, qp1 = 0.0, qp2 = 0.0;
        for (uint32_t k = v.pt_obs_off[ip]; k < v.pt_obs_off[ip + 1]; ++k) {
            const uint32_t j = v.obs_pm[k];
            const uint32_t c = v.obs_key[j] >> 8;
            const double* J = v.jac + 24 * (size_t)j;
            const double* pc = v.p + 9 * (size_t)c;
            double t0 = J[9] * pp0 + J[10] * pp1 + J[11] * pp2;
            double t1 = J[21] * pp0 + J[22] * pp1 + J[23] * pp2;
            for (int a = 0; a < 9; ++a) {
                t0 += J[a] * pc[a];
                t1 += J[12 + a] * pc[a];
            }
            jp2 += t0 * t0 + t1 * t1;
            double* qc = v.q + 9 * (size_t)c;
            for (int a = 0; a < 9; ++a) atomicAdd(qc + a, J[a] * t0 + J[12 + a] * t1);
            qp0 += J[9] * t0 + J[21] * t1;
            qp1 += J[10] * t0 + J[22] * t1;
            qp2 += J[11] * t0 + J[23] * t1;
        }
        v.q[ep] += qp0;
        v.q[ep + 1] += qp1;
        v.q[ep + 2] += qp2;
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

// h += alpha p; r -= alpha q; z = M^-1 r; r^T z, |r|^2; the last block takes the PCG
// stop decision and sets the loop flag.  Never gated.
__global__ void k64_update(V64 v, CondHandle pcg_cond, int use_cond) {
    DevState* st = v.st;
    const int active = st->pcg_active;
    double rz = 0.0, rr = 0.0;
    if (active) {
        const double alpha = st->alpha;
        for (int c = gtid(); c < v.n_cams; c += grid_threads()) {
            const size_t e = 9 * (size_t)c;
            double rn[9];
            for (int k = 0; k < 9; ++k) {
                v.h[e + k] += alpha * v.p[e + k];
                rn[k] = v.r[e + k] - alpha * v.q[e + k];
                v.r[e + k] = rn[k];
            }
            const double* M = v.Minv_c + (size_t)c * MC_STRIDE;
            for (int i = 0; i < 9; ++i) {
                double z = 0.0;
                for (int k = 0; k < 9; ++k) z += M[9 * i + k] * rn[k];
                v.z[e + i] = z;
                rz += rn[i] * z;
                rr += rn[i] * rn[i];
            }
        }
        for (int i = gtid(); i < v.n_pts; i += grid_threads()) {
            const size_t e = v.pt_off + 3 * (size_t)i;
            double rn[3];
            for (int k = 0; k < 3; ++k) {
                v.h[e + k] += alpha * v.p[e + k];
                rn[k] = v.r[e + k] - alpha * v.q[e + k];
                v.r[e + k] = rn[k];
            }
            const double* m = v.Minv_p + (size_t)i * MP_STRIDE;
            const double z0 = m[0] * rn[0] + m[1] * rn[1] + m[2] * rn[2];
            const double z1 = m[1] * rn[0] + m[3] * rn[1] + m[4] * rn[2];
            const double z2 = m[2] * rn[0] + m[4] * rn[1] + m[5] * rn[2];
            v.z[e] = z0; v.z[e + 1] = z1; v.z[e + 2] = z2;
            rz += rn[0] * z0 + rn[1] * z1 + rn[2] * z2;
            rr += rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
        }
    }
    double in[2] = {rz, rr}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_UPD], out) && threadIdx.x == 0) {
        if (active) {
            st->pcg_iter += 1;
            st->pcg_total += 1;
            st->rr = out[1];
            const double tol = st->opt.tol;
            if (!isfinite(out[0]) || !isfinite(out[1])) {
                st->status = 4;
                st->pcg_active = 0;
            } else if (out[1] <= tol * tol * st->rr0 || st->pcg_iter >= st->opt.max_pcg) {
                st->pcg_active = 0;
            } else {
                st->beta = out[0] / st->rz;
                st->rz = out[0];
            }
        }
        if (use_cond) cudaGraphSetConditional(pcg_cond, st->pcg_active ? 1u : 0u);
    }
}

// Candidate x' = x + h, g^T h, camera records at x'.
__global__ void k64_candidate(V64 v) {
    DevState* st = v.st;
    if (st->lm_active == 0) return;
    const bool retract = st->opt.retract != 0;
    double gh = 0.0;
    for (size_t e = gtid(); e < (size_t)v.n_vec; e += grid_threads()) {
        const bool cam = e < 9 * (size_t)v.n_cams;
        if (!(retract && cam && e % 9 < 3)) v.x_new[e] = v.x[e] + v.h[e];   // rotations: below
        const double ge = cam ? v.cam_lin[(e / 9) * CL_STRIDE + e % 9] : (e >= (size_t)v.pt_off ? v.g[e] : 0.0);
        gh += ge * v.h[e];
    }
    for (int c = gtid(); c < v.n_cams; c += grid_threads()) {
        double xn[9];
        for (int k = 0; k < 9; ++k) xn[k] = v.x[9 * (size_t)c + k] + v.h[9 * (size_t)c + k];
        if (retract) {   // R' = Exp(h_w) R(w)
            compose_rotvec(v.h + 9 * (size_t)c, v.x + 9 * (size_t)c, xn);
            for (int k = 0; k < 3; ++k) v.x_new[9 * (size_t)c + k] = xn[k];
        }
        camera_record64(xn, v.cam64_new + (size_t)c * CP_STRIDE, retract);
    }
    double in[1] = {gh}, out[1];
    if (grid_reduce<1>(in, v.partials, &st->tickets[TK_CAND], out) && threadIdx.x == 0) st->gh = out[0];
}

// F(x') and |J h|^2 with the stored Jacobian; the last block applies the LM rule.
__global__ void k64_eval_candidate(V64 v, CondHandle lm_cond, int use_cond) {
    DevState* st = v.st;
    const int active = st->lm_active;
    const double eps = st->opt.eps;
    const int loss = st->opt.loss;
    const double lscale = st->opt.loss_scale;
    double fnew = 0.0, jh2 = 0.0;
    if (active) {
        for (int ip = gtid(); ip < v.n_pts; ip += grid_threads()) {
            const double* Xn = v.x_new + v.pt_off + 3 * (size_t)ip;
            const double* hp = v.h + v.pt_off + 3 * (size_t)ip;
            for (uint32_t k = v.pt_obs_off[ip]; k < v.pt_obs_off[ip + 1]; ++k) {
                const uint32_t j = v.obs_pm[k];
                const uint32_t c = v.obs_key[j] >> 8;
                double r0, r1;
                obs_jacobian64(v.cam64_new + (size_t)c * CP_STRIDE, Xn[0], Xn[1], Xn[2], eps, v.obs_uv[2 * (size_t)j],
                               v.obs_uv[2 * (size_t)j + 1], r0, r1, nullptr);
                fnew += loss ? loss_rho64(r0 * r0 + r1 * r1, loss, lscale) : r0 * r0 + r1 * r1;
                const double* J = v.jac + 24 * (size_t)j;   // sqrt(w)-scaled: |J h|^2 is weighted
                const double* hc = v.h + 9 * (size_t)c;
                double t0 = J[9] * hp[0] + J[10] * hp[1] + J[11] * hp[2];
                double t1 = J[21] * hp[0] + J[22] * hp[1] + J[23] * hp[2];
                for (int a = 0; a < 9; ++a) {
                    t0 += J[a] * hc[a];
                    t1 += J[12 + a] * hc[a];
                }
                jh2 += t0 * t0 + t1 * t1;
            }
        }
    }
    double in[2] = {fnew, jh2}, out[2];
    if (grid_reduce<2>(in, v.partials, &st->tickets[TK_COST], out) && threadIdx.x == 0) {
        lm_decide(st, active, 0.5 * out[0], out[1]);
        if (use_cond) cudaGraphSetConditional(lm_cond, st->lm_active ? 1u : 0u);
    }
}

__global__ void k64_commit(V64 v) {
    if (v.st->accepted == 0) return;
    for (size_t e = gtid(); e < (size_t)v.n_vec; e += grid_threads()) v.x[e] = v.x_new[e];
    for (int c = gtid(); c < v.n_cams; c += grid_threads()) {
        for (int k = 0; k < CP_STRIDE; ++k) v.cam64[(size_t)c * CP_STRIDE + k] = v.cam64_new[(size_t)c * CP_STRIDE + k];
        for (int k = 0; k < CL_STRIDE; ++k) v.cam_lin[(size_t)c * CL_STRIDE + k] = 0.0;
        for (int k = 0; k < CH_STRIDE; ++k) v.cam_H64[(size_t)c * CH_STRIDE + k] = 0.0;
    }
}

template <typename S>
__global__ void k64_pack(V64 v, const S* cams, const S* pts) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) v.x[9 * (size_t)c + k] = (double)cams[9 * (size_t)c + k];
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) v.x[e + k] = (double)pts[3 * (size_t)u + k];
    }
}

template <typename S>
__global__ void k64_unpack(V64 v, S* cams, S* pts) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) cams[9 * (size_t)c + k] = (S)v.x[9 * (size_t)c + k];
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) pts[3 * (size_t)u + k] = (S)v.x[e + k];
    }
}

// user-layout vector <-> internal p / q
__global__ void k64_set_vec(V64 v, const double* src, double* dst) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) dst[9 * (size_t)c + k] = src[9 * (size_t)c + k];
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) dst[e + k] = src[9 * (size_t)v.n_cams + 3 * (size_t)u + k];
    }
}

__global__ void k64_get_vec(V64 v, const double* src, double* dst) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) dst[9 * (size_t)c + k] = src[9 * (size_t)c + k];
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) dst[9 * (size_t)v.n_cams + 3 * (size_t)u + k] = src[e + k];
    }
}

// ------------------------------------------------------------- autograd ------
template <typename S>
__global__ void k64_pack_to(V64 v, const S* cams, const S* pts, double* dst) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) dst[9 * (size_t)c + k] = (double)cams[9 * (size_t)c + k];
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) dst[e + k] = (double)pts[3 * (size_t)u + k];
    }
}

__global__ void k64_records_from(V64 v, const double* src, double* dst) {
    for (int c = gtid(); c < v.n_cams; c += grid_threads()) {
        camera_record64(src + 9 * (size_t)c, dst + (size_t)c * CP_STRIDE);
        for (int k = 0; k < CL_STRIDE; ++k) v.cam_lin[(size_t)c * CL_STRIDE + k] = 0.0;
    }
}

// F = 1/2 |r|^2 and, if want_grad, J^T r (cameras by FP64 atomics, points in registers).
__global__ void k64_cost_grad(V64 v, const double* xs, const double* crec, int want_grad, double* cost_dev) {
    const double eps = v.st->opt.eps;
    double cost = 0.0;
    for (int ip = gtid(); ip < v.n_pts; ip += grid_threads()) {
        const double* X = xs + v.pt_off + 3 * (size_t)ip;
        double gp[3] = {0, 0, 0};
        for (uint32_t k = v.pt_obs_off[ip]; k < v.pt_obs_off[ip + 1]; ++k) {
            const uint32_t j = v.obs_pm[k];
            const uint32_t c = v.obs_key[j] >> 8;
            double J[24], r0, r1;
            obs_jacobian64(crec + (size_t)c * CP_STRIDE, X[0], X[1], X[2], eps, v.obs_uv[2 * (size_t)j],
                           v.obs_uv[2 * (size_t)j + 1], r0, r1, want_grad ? J : nullptr);
            cost += r0 * r0 + r1 * r1;
            if (want_grad) {
                for (int a = 0; a < 9; ++a) atomicAdd(v.cam_lin + (size_t)c * CL_STRIDE + a, J[a] * r0 + J[12 + a] * r1);
                for (int a = 0; a < 3; ++a) gp[a] += J[9 + a] * r0 + J[21 + a] * r1;
            }
        }
        if (want_grad)
            for (int a = 0; a < 3; ++a) v.g[v.pt_off + 3 * (size_t)ip + a] = gp[a];
    }
    double in[1] = {cost}, out[1];
    if (grid_reduce<1>(in, v.partials, &v.st->tickets[TK_MISC], out) && threadIdx.x == 0) {
        v.st->cost_out = 0.5 * out[0];
        if (cost_dev) *cost_dev = 0.5 * out[0];
    }
}

template <typename S>
__global__ void k64_grad_out(V64 v, const double* grad_out, S* gc, S* gp) {
    const double s = *grad_out;
    for (int c = gtid(); c < v.n_cams; c += grid_threads())
        for (int k = 0; k < 9; ++k) gc[9 * (size_t)c + k] = (S)(s * v.cam_lin[(size_t)c * CL_STRIDE + k]);
    for (int u = gtid(); u < v.n_pts; u += grid_threads()) {
        const size_t e = v.pt_off + 3 * (size_t)v.pt_internal[u];
        for (int k = 0; k < 3; ++k) gp[3 * (size_t)u + k] = (S)(s * v.g[e + k]);
    }
}

// ------------------------------------------------------------------ launchers --

namespace {
inline int g64(const LaunchCfg& L, size_t items) {
    size_t g = (items + L.item_block - 1) / L.item_block;
    return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)L.item_grid));
}
}  // namespace

void launch64_camera_precompute(const V64& v, const LaunchCfg& L, cudaStream_t s) {
    k64_camera_precompute<<<g64(L, v.n_cams), L.item_block, 0, s>>>(v);
}
void launch64_linearize(const V64& v, const LaunchCfg& L, cudaStream_t s, int mode, double* r, double* J,
                        CondHandle c, int use) {
    k64_linearize<<<g64(L, v.n_pts), L.item_block, 0, s>>>(v, mode, r, J, c, use);
}
void launch64_precond(const V64& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k64_precond<<<g64(L, std::max((size_t)v.n_pts, 32 * (size_t)v.n_cams)), L.item_block, 0, s>>>(v, c, use);
}
void launch64_direction(const V64& v, const LaunchCfg& L, cudaStream_t s, const double* zs, int use_beta,
                        const int32_t* gate) {
    k64_direction<<<g64(L, v.n_vec), L.item_block, 0, s>>>(v, zs, use_beta, gate);
}
void launch64_matvec(const V64& v, const LaunchCfg& L, cudaStream_t s, const int32_t* gate) {
    k64_matvec<<<g64(L, v.n_pts), L.item_block, 0, s>>>(v, gate);
}
void launch64_update(const V64& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k64_update<<<g64(L, std::max(v.n_pts, v.n_cams)), L.item_block, 0, s>>>(v, c, use);
}
void launch64_candidate(const V64& v, const LaunchCfg& L, cudaStream_t s) {
    k64_candidate<<<g64(L, v.n_vec), L.item_block, 0, s>>>(v);
}
void launch64_eval_candidate(const V64& v, const LaunchCfg& L, cudaStream_t s, CondHandle c, int use) {
    k64_eval_candidate<<<g64(L, v.n_pts), L.item_block, 0, s>>>(v, c, use);
}
void launch64_commit(const V64& v, const LaunchCfg& L, cudaStream_t s) {
    k64_commit<<<g64(L, v.n_vec), L.item_block, 0, s>>>(v);
}
void launch64_pack(const V64& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts, int dtype) {
    const int g = g64(L, std::max(v.n_cams, v.n_pts));
    if (dtype == 1) k64_pack<double><<<g, L.item_block, 0, s>>>(v, (const double*)cams, (const double*)pts);
    else k64_pack<float><<<g, L.item_block, 0, s>>>(v, (const float*)cams, (const float*)pts);
}
void launch64_unpack(const V64& v, const LaunchCfg& L, cudaStream_t s, void* cams, void* pts, int dtype) {
    const int g = g64(L, std::max(v.n_cams, v.n_pts));
    if (dtype == 1) k64_unpack<double><<<g, L.item_block, 0, s>>>(v, (double*)cams, (double*)pts);
    else k64_unpack<float><<<g, L.item_block, 0, s>>>(v, (float*)cams, (float*)pts);
}
void launch64_set_vec(const V64& v, const LaunchCfg& L, cudaStream_t s, const double* src, double* dst) {
    k64_set_vec<<<g64(L, std::max(v.n_cams, v.n_pts)), L.item_block, 0, s>>>(v, src, dst);
}
void launch64_cost_grad(const V64& v, const LaunchCfg& L, cudaStream_t s, const void* cams, const void* pts, int dtype,
                        int want_grad, double* cost_dev) {
    const int g = g64(L, std::max(v.n_cams, v.n_pts));
    if (dtype == 1) k64_pack_to<double><<<g, L.item_block, 0, s>>>(v, (const double*)cams, (const double*)pts, v.x_new);
    else k64_pack_to<float><<<g, L.item_block, 0, s>>>(v, (const float*)cams, (const float*)pts, v.x_new);
    k64_records_from<<<g64(L, v.n_cams), L.item_block, 0, s>>>(v, v.x_new, v.cam64_new);
    k64_cost_grad<<<g64(L, v.n_pts), L.item_block, 0, s>>>(v, v.x_new, v.cam64_new, want_grad, cost_dev);
}
void launch64_grad_out(const V64& v, const LaunchCfg& L, cudaStream_t s, const double* grad_out, void* gc, void* gp,
                       int dtype) {
    const int g = g64(L, std::max(v.n_cams, v.n_pts));
    if (dtype == 1) k64_grad_out<double><<<g, L.item_block, 0, s>>>(v, grad_out, (double*)gc, (double*)gp);
    else k64_grad_out<float><<<g, L.item_block, 0, s>>>(v, grad_out, (float*)gc, (float*)gp);
}
void launch64_get_vec(const V64& v, const LaunchCfg& L, cudaStream_t s, const double* src, double* dst) {
    k64_get_vec<<<g64(L, std::max(v.n_cams, v.n_pts)), L.item_block, 0, s>>>(v, src, dst);
}

}  // namespace gbba
